// schedule.h -- task orders of the persistent multi-pass kernels (host and device).
//
// A persistent kernel runs a fixed list of tasks; CTA b takes tasks b, b + grid, ...  A task
// that reads a ring slot waits on a per-slot counter that the producing pass increments once
// per finished task.  The orders below keep every wait on tasks that come earlier in the list,
// so the CTA holding the earliest unfinished task is running it and a fully resident grid
// cannot deadlock.  tests/test_schedule_host.py compiles this header for the host and checks
// that property, and that every (batch, pass, index) appears exactly once, for many shapes.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define HM_HD __host__ __device__ __forceinline__
#else
#define HM_HD inline
#endif

namespace hm {

// Two-pass order (Algorithm 2's transform split into a pass over the low bits and one over the
// high bits) with lag D: the first Dh = min(D, n_batches) stages run pass 1 of batches
// 0 .. Dh-1; middle stage s (0 <= s < n_batches - Dh) runs pass 1 of batch s + Dh, then pass 2
// of batch s; the tail runs pass 2 of the last Dh batches.  n_batches (p1 + p2) tasks.
HM_HD void twopass_decode(int64_t task, int p1, int p2, int64_t n_batches, int lag, int64_t& g, int& kind,
                          int& r) {
    const int64_t Dh = lag < n_batches ? lag : n_batches;
    const int64_t nm = n_batches - Dh;
    const int64_t per_stage = (int64_t)p1 + p2;
    if (task < Dh * p1) { g = task / p1; kind = 1; r = (int)(task % p1); return; }
    int64_t tt = task - Dh * p1;
    if (tt < nm * per_stage) {
        const int64_t s = tt / per_stage;
        const int rr = (int)(tt % per_stage);
        if (rr < p1) { g = s + Dh; kind = 1; r = rr; }
        else { g = s; kind = 2; r = rr - p1; }
        return;
    }
    tt -= nm * per_stage;
    g = nm + tt / p2;
    kind = 2;
    r = (int)(tt % p2);
}

// What a two-pass task waits for, R ring slots: pass 1 of batch g on pass 2 of batch g - R
// (the slot's previous user; nothing for g < R), pass 2 of g on pass 1 of g.  Returns the
// counter (0: none, 1: pass-1 completions, 2: pass-2 completions) of slot g mod R and the
// count it must reach (before any bias).
HM_HD int twopass_dependency(int64_t g, int kind, int R, int p1, int p2, int& slot, unsigned& need) {
    slot = (int)(g % R);
    if (kind == 1) {
        need = (unsigned)((g / R) * p2);
        return g >= R ? 2 : 0;
    }
    need = (unsigned)((g / R + 1) * p1);
    return 1;
}

// Three-pass order (the adjoint) with lag D, R >= 2D + 1 ring slots: stage s runs pass 1 of
// batch s, pass 2 of batch s - D and pass 3 of batch s - 2D (n_batches + 2D stages of
// p1 + p2 + p3 tasks; g outside [0, n_batches): nothing to do).  Every pass reads what the
// previous one wrote D stages (D (p1 + p2 + p3) tasks) earlier.
HM_HD void g3_decode(int64_t task, int p1, int p2, int p3, int D, int& kind, int64_t& g, int& r) {
    const int64_t per = (int64_t)p1 + p2 + p3;
    const int64_t st = task / per;
    r = (int)(task % per);
    if (r < p1) { kind = 1; g = st; }
    else if (r < p1 + p2) { kind = 2; g = st - D; r -= p1; }
    else { kind = 3; g = st - 2 * D; r -= p1 + p2; }
}

// What a three-pass task waits for: pass 1 of g on pass 3 of g - R (nothing for g < R), pass 2
// of g on pass 1 of g, pass 3 of g on pass 2 of g.  Returns the pass whose per-slot counter
// (slot g mod R) must reach `need` (0: none).
HM_HD int g3_dependency(int64_t g, int kind, int R, int p1, int p2, int p3, int& slot, unsigned& need) {
    slot = (int)(g % R);
    if (kind == 1) {
        need = (unsigned)((g / R) * p3);
        return g >= R ? 3 : 0;
    }
    if (kind == 2) {
        need = (unsigned)((g / R + 1) * p1);
        return 1;
    }
    need = (unsigned)((g / R + 1) * p2);
    return 2;
}

}  // namespace hm
