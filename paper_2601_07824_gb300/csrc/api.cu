// api.cu -- C ABI of libhadamag (declared in include/hadamag.h): argument checks, context
// buffers, planning of the launches, result read-back and the final FP64 logarithms.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/hadamag.h"
#include "ctx.h"
#include "sre_fwd.h"
#include "extra.h"

using namespace hm;

extern "C" const char* hadamag_status_string(hadamag_status s) {
    switch (s) {
        case HADAMAG_OK: return "ok";
        case HADAMAG_ERR_INVALID_ARG: return "invalid argument";
        case HADAMAG_ERR_UNSUPPORTED: return "unsupported";
        case HADAMAG_ERR_OOM: return "out of memory";
        case HADAMAG_ERR_CUDA: return "CUDA error";
        case HADAMAG_ERR_TIMEOUT: return "device wait timed out";
        case HADAMAG_ERR_NONFINITE: return "non-finite result";
    }
    return "unknown status";
}

namespace hm {

hadamag_status fail(hadamag_ctx_t c, hadamag_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->last_error, sizeof(c->last_error), fmt, ap);
        va_end(ap);
    }
    return s;
}

hadamag_status cuda_fail(hadamag_ctx_t c, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, HADAMAG_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    }
    return fail(c, HADAMAG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

hadamag_status ensure_buf(hadamag_ctx_t c, DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes && b.ptr) return HADAMAG_OK;
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaFree");
    }
    size_t sz = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&b.ptr, sz);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        return cuda_fail(c, e, "cudaMalloc");
    }
    b.bytes = sz;
    return HADAMAG_OK;
}

bool aligned16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

// complex128 input -> complex64 copy in the context (the kernels compute in FP32).
hadamag_status as_c64(hadamag_ctx_t c, const void* psi, int64_t n, hadamag_dtype dt, cudaStream_t st,
                      const float2** out) {
    if (dt == HADAMAG_C64) {
        *out = reinterpret_cast<const float2*>(psi);
        return HADAMAG_OK;
    }
    if (dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype %d", (int)dt);
    hadamag_status s = ensure_buf(c, c->conv, (size_t)n * sizeof(float2));
    if (s) return s;
    cudaError_t e = launch_c128_to_c64(psi, reinterpret_cast<float2*>(c->conv.ptr), n, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "c128_to_c64");
    *out = reinterpret_cast<const float2*>(c->conv.ptr);
    return HADAMAG_OK;
}

// X-string counts up to this use the small-task two-pass shape instead of the tuned one.
constexpr int64_t kFewXstrings = 64;

int sre_mode(double n) { return n == 1.0 ? 1 : n == 2.0 ? 2 : n == 3.0 ? 3 : 0; }

// Two-pass launch shape for N: X-strings per batch A, ring slots R (0: the default), units per
// pass-1 warp UPW (K1 = 10), column tiles per pass-2 task TPT, and the lag (stages) between a
// batch's pass 1 and its pass 2 (1 <= lag < R).
TwoPlan plan_twopass(int N, int UPW, int TPT, int R, int lag) {
    TwoPlan p{};
    const int L = N - 1, K1 = twopass_k1(N), M = L - K1;
    const size_t per_a = ((size_t)1 << L) * sizeof(float2);
    int A = 1;
    if (K1 == 10) {
        A = 8;  // X-strings per batch: the 8 pass-1 warps share the state rows of two units
        p.U = 1;
        // ring slots: 4 while they total <= 64 MiB, else 3 (N = 20: 3 x 32 MiB, inside L2)
        p.R = ((size_t)4 * A * per_a <= ((size_t)64 << 20)) ? 4 : 3;
    } else {
        p.U = 1;
        p.R = (N <= 22) ? 4 : 2;
    }
    p.A = A;
    if (R > 0) p.R = R;
    p.tiles = twopass_tiles_per_a(N);
    p.triples = twopass_triples_per_a(N);
    p.UPW = (K1 == 10) ? UPW : 1;
    p.TPT = TPT;
    p.lag = lag < p.R ? lag : p.R - 1;
    // a pass-1 task covers A X-strings x (U or 1) warps x UPW units per warp (K1 = 10), or one
    // unit (K1 = 13); a pass-2 task covers TPT adjacent column tiles
    p.p1 = (K1 == 10) ? (1 << M) / (p.U * p.UPW) : (1 << M);
    p.p2 = A * p.tiles / p.TPT;
    p.scratch_bytes = (size_t)p.R * A * per_a;
    return p;
}

// Runs Algorithm 2 over `count` X-strings (all of them when a_list is null).  per_a = 0:
// per-CTA partial triples go to c->part and *nparts receives their number.  per_a = 1:
// per-X-string triples are written to terms (device).
hadamag_status run_sre(hadamag_ctx_t c, const float2* psi, int N, double n, int64_t count,
                       const int64_t* a_list, int per_a, double* terms, cudaStream_t st, int64_t* nparts) {
    int mode = sre_mode(n);
    if (mode == 0 && c->fp32_powers && n <= 4.0 && n * (N + 2) <= 100.0) mode = 4;
    hadamag_status s;
    cudaError_t e;
    if (N == 15 && count > kFewXstrings && (s = tune_twopass(c, psi, N, n, mode, st))) return s;
    if (N < 15 || (N == 15 && !c->twopass_shape[N][mode].UPW)) {
        OnepassArgs A{};
        A.psi = psi; A.N = N; A.nq = n; A.count = count; A.a_list = a_list;
        A.per_a = per_a; A.status = (int*)c->status.ptr; A.grid = 0;
        if (!per_a) {
            int64_t maxgrid = (int64_t)c->sm_count * 64;
            if ((s = ensure_buf(c, c->part, (size_t)maxgrid * 3 * sizeof(double)))) return s;
            A.out = (double*)c->part.ptr;
            A.grid = (int)maxgrid;
        } else {
            A.out = terms;
        }
        e = launch_onepass(A, mode, c->sm_count, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "sre_onepass");
        if (nparts) *nparts = A.grid;
        return HADAMAG_OK;
    }
    if (N > 24) return fail(c, HADAMAG_ERR_UNSUPPORTED, "exact SRE supports N <= 24 (got %d)", N);
    if (count <= kFewXstrings) {
        // a few X-strings (Algorithm 3's per-step evaluations): a pinned shape, else the shape
        // with the most, smallest tasks, so that they spread over the grid (the tuned shapes
        // are for full sums)
        const TwoShape& ps = c->twopass_shape[N][mode];
        const TwoPlan pl = (ps.pinned && ps.UPW) ? plan_twopass(N, ps.UPW, ps.TPT, ps.R, ps.lag) : plan_twopass(N, 2, 1);
        return launch_twopass_plan(c, psi, N, n, mode, pl, count, a_list, 0, per_a, terms, st, nparts);
    }
    if ((s = tune_twopass(c, psi, N, n, mode, st))) return s;
    const TwoShape& sh = c->twopass_shape[N][mode];
    TwoPlan pl = sh.UPW ? plan_twopass(N, sh.UPW, sh.TPT, sh.R, sh.lag) : plan_twopass(N);
    return launch_twopass_plan(c, psi, N, n, mode, pl, count, a_list, 0, per_a, terms, st, nparts);
}

// One two-pass launch with plan `pl` (X-strings a_list[i], or a_base + i without a list).
hadamag_status launch_twopass_plan(hadamag_ctx_t c, const float2* psi, int N, double n, int mode, const TwoPlan& pl,
                                   int64_t count, const int64_t* a_list, int64_t a_base, int per_a, double* terms,
                                   cudaStream_t st, int64_t* nparts) {
    hadamag_status s;
    cudaError_t e;
    int& grid_max = c->twopass_grid[N][mode];  // queried once per context (a host round trip)
    if (!grid_max && (e = twopass_max_grid(N, mode, c->sm_count, &grid_max)) != cudaSuccess)
        return cuda_fail(c, e, "occupancy");
    int grid = grid_max;
    if ((s = ensure_buf(c, c->scratch, pl.scratch_bytes))) return s;
    if ((s = ensure_buf(c, c->counters, 2 * 64 * sizeof(unsigned)))) return s;
    TwoPassParams P{};
    P.psi = psi; P.N = N; P.nq = n; P.count = count; P.a_list = a_list; P.a_base = a_base;
    P.scratch = (float2*)c->scratch.ptr; P.R = pl.R; P.A = pl.A; P.U = pl.U;
    P.UPW = pl.UPW; P.TPT = pl.TPT; P.lag = pl.lag;
    P.n_batches = (count + pl.A - 1) / pl.A;
    P.p1 = pl.p1; P.p2 = pl.p2;
    P.done1 = (unsigned*)c->counters.ptr; P.done2 = P.done1 + 64;
    P.status = (int*)c->status.ptr; P.spin_limit = c->spin_limit; P.wait_bias = c->wait_bias;
    P.per_a = per_a;
    const int64_t total_tasks = P.n_batches * ((int64_t)pl.p1 + pl.p2);
    if (grid > total_tasks) grid = (int)total_tasks;
    if (grid < 1) grid = 1;
    if (per_a) {
        if ((s = ensure_buf(c, c->tiles, (size_t)count * pl.triples * 3 * sizeof(double)))) return s;
        P.out = (double*)c->tiles.ptr;
    } else {
        if ((s = ensure_buf(c, c->part, (size_t)grid * 3 * sizeof(double)))) return s;
        P.out = (double*)c->part.ptr;
    }
    if ((e = cudaMemsetAsync(c->counters.ptr, 0, 2 * 64 * sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(c, e, "memset counters");
    e = launch_twopass(P, mode, grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sre_twopass");
    if (per_a) {
        e = launch_sum_tiles((double*)c->tiles.ptr, count, pl.triples, terms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "sum_tiles");
    }
    if (nparts) *nparts = grid;
    return HADAMAG_OK;
}

// The two-pass autotuner: on the first uncaptured call for (N, mode) it times each candidate
// task shape on a bounded range of X-strings (a >= 2^(N-1), the common kind; two launches each,
// the second timed with CUDA events on the call's stream) and keeps the fastest for the context.
// Candidates: units per pass-1 warp {2, 4} (K1 = 10) x tiles per pass-2 task {2, 4} x a pass-2
// lag of 1 or 2 stages (for N = 20 also 2, 3 or 4 ring slots) or, where a stage holds few tasks,
// the lag that puts 1.5 grid rounds of tasks between a batch's two passes.  At N = 15 the split itself is tuned: the one-pass kernel (the
// whole 2^14-value transform in one CTA's shared memory) against two passes through L2 (10 + 4
// bits; tiles per pass-2 task {1, 2}).  Under stream capture, or with autotuning off, the
// defaults run (one pass at N = 15).
hadamag_status tune_twopass(hadamag_ctx_t c, const float2* psi, int N, double n, int mode, cudaStream_t st) {
    TwoShape& sh = c->twopass_shape[N][mode];
    if (sh.UPW || sh.onepass || !c->autotune) return HADAMAG_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(c, e, "capture query");
    if (cap != cudaStreamCaptureStatusNone) return HADAMAG_OK;
    struct Cand { int UPW, TPT, R, lag; };  // UPW 0: the one-pass kernel (N = 15)
    Cand cands[32];
    int nc = 0;
    const bool k10 = twopass_k1(N) == 10;
    int grid = 0;
    if ((e = twopass_max_grid(N, mode, c->sm_count, &grid)) != cudaSuccess) return cuda_fail(c, e, "occupancy");
    if (N == 15) cands[nc++] = {0, 0, 0, 1};
    for (int upw : {2, 4}) {
        if (!k10 && upw != 2) continue;
        for (int tpt : {1, 2, 4}) {
            if (tpt > twopass_tiles_per_a(N) || (tpt == 1 && N != 15)) continue;
            for (int lag : {1, 2}) {
                if (N == 20) {
                    cands[nc++] = {upw, tpt, 3, lag};
                    if (lag == 1) {
                        cands[nc++] = {upw, tpt, 4, lag};
                        cands[nc++] = {upw, tpt, 2, lag};  // 64 MiB ring: no scratch write-back
                    }
                } else {
                    cands[nc++] = {upw, tpt, 0, lag};
                }
            }
            // and the lag that spaces a batch's two passes 1.5 grid rounds apart (few tasks per
            // stage at N <= 18), with lag + 1 ring slots within 64 MiB
            if (k10 && grid > 0) {
                const TwoPlan q = plan_twopass(N, upw, tpt);
                const int deep = pipeline_lag((int64_t)q.p1 + q.p2, grid, 1, (size_t)q.A << (N - 1) << 3,
                                              (size_t)64 << 20);
                if (deep > 2) cands[nc++] = {upw, tpt, deep + 1, deep};
            }
        }
    }
    const int64_t cnt = int64_t(1) << (N <= 20 ? 13 : 10);
    const int64_t base = int64_t(1) << (N - 1);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(c, HADAMAG_ERR_CUDA, "events");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(c, HADAMAG_ERR_CUDA, "events"); }
    float best = 1e30f;
    Cand win = cands[0];
    hadamag_status s = HADAMAG_OK;
    for (int k = 0; k < nc && !s; ++k) {
        const TwoPlan pl = cands[k].UPW ? plan_twopass(N, cands[k].UPW, cands[k].TPT, cands[k].R, cands[k].lag)
                                        : TwoPlan{};
        for (int rep = 0; rep < 2 && !s; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            int64_t np = 0;
            if (cands[k].UPW) {
                s = launch_twopass_plan(c, psi, N, n, mode, pl, cnt, nullptr, base, 0, nullptr, st, &np);
            } else {
                OnepassArgs A{};
                A.psi = psi; A.N = N; A.nq = n; A.count = cnt; A.a_list = nullptr; A.a_base = base;
                A.per_a = 0; A.status = (int*)c->status.ptr;
                const int64_t maxgrid = (int64_t)c->sm_count * 64;
                if ((s = ensure_buf(c, c->part, (size_t)maxgrid * 3 * sizeof(double)))) break;
                A.out = (double*)c->part.ptr;
                A.grid = (int)maxgrid;
                if ((e = launch_onepass(A, mode, c->sm_count, st)) != cudaSuccess) s = cuda_fail(c, e, "sre_onepass");
                c->launches++;
            }
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (s) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { s = cuda_fail(c, e, "tune sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; win = cands[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if ((s = status_word_now(c, st))) return s;
    sh.UPW = win.UPW;
    sh.TPT = win.TPT;
    sh.R = win.R;
    sh.lag = win.lag;
    sh.onepass = win.UPW == 0;
    return HADAMAG_OK;
}

// Reads the device status word (synchronising `st`) without clearing it.
hadamag_status status_word_now(hadamag_ctx_t c, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->host_status, c->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy status");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "stream sync");
    return status_word(c);
}

hadamag_status begin(hadamag_ctx_t c, cudaStream_t st) {
    c->last_error[0] = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    e = cudaMemsetAsync(c->status.ptr, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset status");
    return HADAMAG_OK;
}

// Copy `n` result doubles and the status word to pinned host memory and wait for the stream.
hadamag_status finish(hadamag_ctx_t c, const double* res_dev, int n, cudaStream_t st) {
    cudaError_t e;
    if (n > 0 && (e = cudaMemcpyAsync(c->host_res, res_dev, n * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy result");
    if ((e = cudaMemcpyAsync(c->host_status, c->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy status");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "stream sync");
    return status_word(c);
}

hadamag_status status_word(hadamag_ctx_t c) {
    int w = *c->host_status;
    if (w & ST_TIMEOUT) return fail(c, HADAMAG_ERR_TIMEOUT, "an inter-CTA wait ran out of iterations");
    if (w & ST_BADARG) return fail(c, HADAMAG_ERR_INVALID_ARG, "an X-string list entry is outside [0, dim)");
    if (w & ST_NONPOS)
        return fail(c, HADAMAG_ERR_NONFINITE, "S(a) + eps <= 0 at an evaluated X-string (use eps > 0)");
    return HADAMAG_OK;
}

}  // namespace hm

// ---------------------------------------------------------------------------------------
extern "C" hadamag_status hadamag_create(hadamag_ctx_t* out, int device) {
    if (!out) return HADAMAG_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HADAMAG_ERR_INVALID_ARG;
    }
    hadamag_ctx_t c = new (std::nothrow) hadamag_ctx_s();
    if (!c) return HADAMAG_ERR_OOM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->host_res, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->host_status, sizeof(int));
    if (e != cudaSuccess) {
        hadamag_destroy(c);
        cudaGetLastError();
        return HADAMAG_ERR_CUDA;
    }
    if (ensure_buf(c, c->status, sizeof(int)) || ensure_buf(c, c->res, 64 * sizeof(double))) {
        hadamag_destroy(c);
        return HADAMAG_ERR_OOM;
    }
    *out = c;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_destroy(hadamag_ctx_t c) {
    if (!c) return HADAMAG_OK;
    cudaSetDevice(c->device);
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    for (DevBuf* b : c->all_bufs())
        if (b->ptr) cudaFree(b->ptr);
    if (c->host_res) cudaFreeHost(c->host_res);
    if (c->host_table) cudaFreeHost(c->host_table);
    if (c->host_status) cudaFreeHost(c->host_status);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_path(hadamag_ctx_t c, hadamag_path p) {
    if (!c || (p != HADAMAG_PATH_AUTO && p != HADAMAG_PATH_CUDACORE && p != HADAMAG_PATH_TENSOR))
        return HADAMAG_ERR_INVALID_ARG;
    c->path = p;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_fp32_powers(hadamag_ctx_t c, int on) {
    if (!c || (on != 0 && on != 1)) return HADAMAG_ERR_INVALID_ARG;
    c->fp32_powers = on;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_wait_limit(hadamag_ctx_t c, long long spins, unsigned bias) {
    if (!c || spins < 1) return HADAMAG_ERR_INVALID_ARG;
    c->spin_limit = spins;
    c->wait_bias = bias;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_autotune(hadamag_ctx_t c, int on) {
    if (!c || (on != 0 && on != 1)) return HADAMAG_ERR_INVALID_ARG;
    c->autotune = on;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_twopass_shape(hadamag_ctx_t c, int N, double n, int* out5) {
    if (!c || !out5 || N < 15 || N > 24 || !(n > 0.0)) return HADAMAG_ERR_INVALID_ARG;
    int mode = sre_mode(n);
    if (mode == 0 && c->fp32_powers && n <= 4.0 && n * (N + 2) <= 100.0) mode = 4;
    const TwoShape& sh = c->twopass_shape[N][mode];
    if (sh.onepass) {
        for (int k = 0; k < 5; ++k) out5[k] = -1;
        return HADAMAG_OK;
    }
    const TwoPlan pl = sh.UPW ? plan_twopass(N, sh.UPW, sh.TPT, sh.R, sh.lag) : plan_twopass(N);
    out5[0] = sh.UPW ? pl.UPW : 0;
    out5[1] = sh.UPW ? pl.TPT : 0;
    out5[2] = sh.UPW ? pl.R : 0;
    out5[3] = sh.UPW ? pl.A : 0;
    out5[4] = sh.UPW ? pl.lag : 0;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_twopass_shape(hadamag_ctx_t c, int N, double n, int upw, int tpt, int R,
                                                    int lag) {
    if (!c || N < 15 || N > 24 || !(n > 0.0)) return HADAMAG_ERR_INVALID_ARG;
    int mode = sre_mode(n);
    if (mode == 0 && c->fp32_powers && n <= 4.0 && n * (N + 2) <= 100.0) mode = 4;
    TwoShape& sh = c->twopass_shape[N][mode];
    if (upw == -1 && N == 15) {  // the one-pass kernel
        sh = TwoShape{};
        sh.onepass = 1;
        return HADAMAG_OK;
    }
    const bool k10 = twopass_k1(N) == 10;
    if ((k10 ? (upw != 2 && upw != 4) : upw != 2) || tpt < 1 || tpt > twopass_tiles_per_a(N) ||
        (twopass_tiles_per_a(N) % tpt) || !(R == 0 || (R >= 2 && R <= 63)) || lag < 1 ||
        lag >= plan_twopass(N, upw, tpt, R).R)
        return HADAMAG_ERR_INVALID_ARG;
    sh.UPW = upw;
    sh.TPT = tpt;
    sh.R = R;
    sh.lag = lag;
    sh.onepass = 0;
    sh.pinned = 1;
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_launch_count(hadamag_ctx_t c, uint64_t* n) {
    if (!c || !n) return HADAMAG_ERR_INVALID_ARG;
    *n = c->launches;
    return HADAMAG_OK;
}

extern "C" const char* hadamag_last_error(hadamag_ctx_t c) { return c ? c->last_error : ""; }

extern "C" hadamag_status hadamag_sre(hadamag_ctx_t c, const void* psi, int N, double n,
                                      hadamag_dtype dt, double* M_out, double* lost_out,
                                      hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !M_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 24) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 24] (got %d)", N);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(c, HADAMAG_ERR_INVALID_ARG, "n must be > 0");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    const int64_t dim = int64_t(1) << N;
    const float2* p;
    if ((s = as_c64(c, psi, dim, dt, st, &p))) return s;
    double sums[3];
    if ((s = sre_sums(c, p, N, n, st, sums))) return s;
    return sre_from_sums(c, N, n, sums, M_out, lost_out);
}

namespace hm {

// Exact per-call sums [S_n, S_1, T_1] over all X-strings, picking the transform path.
hadamag_status sre_sums(hadamag_ctx_t c, const float2* p, int N, double n, cudaStream_t st, double sums[3]) {
    hadamag_status s;
    cudaError_t e;
    int64_t nparts = 0;
    const int64_t dim = int64_t(1) << N;
    bool tensor = use_tensor_path(c, N, n);
    if (tensor) {
        if ((s = run_sre_tensor(c, p, N, n, dim, nullptr, 0, nullptr, st, &nparts))) return s;
    } else {
        if ((s = run_sre(c, p, N, n, dim, nullptr, 0, nullptr, st, &nparts))) return s;
    }
    e = launch_sum_triples((const double*)c->part.ptr, nparts, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    sums[0] = c->host_res[0]; sums[1] = c->host_res[1]; sums[2] = c->host_res[2];
    return HADAMAG_OK;
}

// Eq. (sre) with the n -> 1 Shannon limit, and lost_norm (Sec. 4.1), in FP64.
hadamag_status sre_from_sums(hadamag_ctx_t c, int N, double n, const double sums[3], double* M_out,
                             double* lost_out) {
    const double two_n = std::ldexp(1.0, N);
    double M;
    if (n == 1.0) M = -sums[2] / sums[1] + std::log2(sums[1]) - (double)N;
    else M = std::log2(sums[0] / two_n) / (1.0 - n);
    if (M == 0.0) M = 0.0;  // no negative zero
    *M_out = M;
    if (lost_out) *lost_out = 1.0 - sums[1] / two_n;
    if (!std::isfinite(M) || !std::isfinite(sums[1]))
        return fail(c, HADAMAG_ERR_NONFINITE, "non-finite sums (S_n=%g, S_1=%g)", sums[0], sums[1]);
    return HADAMAG_OK;
}

}  // namespace hm

extern "C" hadamag_status hadamag_sre_even_sector(hadamag_ctx_t c, const void* psi, int N, double n,
                                                  hadamag_dtype dt, double* M_out, double* lost_out,
                                                  hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !M_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 24) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 24] (got %d)", N);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(c, HADAMAG_ERR_INVALID_ARG, "n must be > 0");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    const float2* p;
    if ((s = as_c64(c, psi, int64_t(1) << N, dt, st, &p))) return s;
    const int64_t count = int64_t(1) << (N - 1);
    if ((s = ensure_buf(c, c->alist, (size_t)count * sizeof(int64_t)))) return s;
    int64_t* al = (int64_t*)c->alist.ptr;
    e = launch_even_xstrings(count, al, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "even_xstrings");
    int64_t nparts = 0;
    if (use_tensor_path(c, N, n)) s = run_sre_tensor(c, p, N, n, count, al, 0, nullptr, st, &nparts);
    else s = run_sre(c, p, N, n, count, al, 0, nullptr, st, &nparts);
    if (s) return s;
    e = launch_sum_triples((const double*)c->part.ptr, nparts, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    const double sums[3] = {c->host_res[0], c->host_res[1], c->host_res[2]};
    return sre_from_sums(c, N, n, sums, M_out, lost_out);
}

extern "C" hadamag_status hadamag_sre_host(hadamag_ctx_t c, const void* psi_host, int N, double n,
                                           hadamag_dtype dt, double* M_out, double* lost_out) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!psi_host || !M_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null pointer");
    if (N < 1 || N > 24) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 24] (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    cudaStream_t st = c->own_stream;
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    const size_t bytes = ((size_t)1 << N) * (dt == HADAMAG_C64 ? 8 : 16);
    if ((s = ensure_buf(c, c->staging, bytes))) return s;
    cudaError_t e = cudaMemcpyAsync(c->staging.ptr, psi_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy psi to device");
    return hadamag_sre(c, c->staging.ptr, N, n, dt, M_out, lost_out, reinterpret_cast<hadamag_stream_t>(st));
}

extern "C" hadamag_status hadamag_sre_terms(hadamag_ctx_t c, const void* psi, int N, double n,
                                            hadamag_dtype dt, const int64_t* a_list, int64_t count,
                                            double* terms, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !a_list || !terms) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 28) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 28] (got %d)", N);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(c, HADAMAG_ERR_INVALID_ARG, "n must be > 0");
    if (N > 24 && n != 2.0) return fail(c, HADAMAG_ERR_UNSUPPORTED, "N > 24 supports n = 2 only");
    if (count < 0) return fail(c, HADAMAG_ERR_INVALID_ARG, "count < 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    if (count == 0) return finish(c, nullptr, 0, st);
    const float2* p;
    if ((s = as_c64(c, psi, int64_t(1) << N, dt, st, &p))) return s;
    if (use_tensor_path(c, N, n)) s = run_sre_tensor(c, p, N, n, count, a_list, 1, terms, st, nullptr);
    else if (N <= 24) s = run_sre(c, p, N, n, count, a_list, 1, terms, st, nullptr);
    else s = run_sre_hbm_terms(c, p, N, count, a_list, terms, st);
    if (s) return s;
    return finish(c, nullptr, 0, st);
}

extern "C" hadamag_status hadamag_mc_xstrings(hadamag_ctx_t c, uint64_t seed, int64_t count, int N,
                                              int64_t* a_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!a_out || count < 0 || N < 1 || N > 30) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    if (count == 0) return HADAMAG_OK;
    cudaError_t e = launch_mc_xstrings(seed, count, N, a_out, reinterpret_cast<cudaStream_t>(stream));
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mc_xstrings");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_sre_mc(hadamag_ctx_t c, const void* psi, int N, int64_t samples,
                                         uint64_t seed, hadamag_dtype dt, double* M2_out,
                                         double* stderr_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !M2_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 28) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 28] (got %d)", N);
    if (samples < 1 || samples > (int64_t(1) << 30)) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad sample count");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    const float2* p;
    if ((s = as_c64(c, psi, int64_t(1) << N, dt, st, &p))) return s;
    // samples, then the exactly evaluated X-string a = 0 (the row holding the identity string)
    if ((s = ensure_buf(c, c->alist, (size_t)(samples + 1) * sizeof(int64_t)))) return s;
    if ((s = ensure_buf(c, c->terms, (size_t)(samples + 1) * 3 * sizeof(double)))) return s;
    int64_t* al = (int64_t*)c->alist.ptr;
    double* tm = (double*)c->terms.ptr;
    cudaError_t e = launch_mc_xstrings(seed, samples, N, al, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mc_xstrings");
    if ((e = cudaMemsetAsync(al + samples, 0, sizeof(int64_t), st)) != cudaSuccess) return cuda_fail(c, e, "memset");
    if (use_tensor_path(c, N, 2.0)) s = run_sre_tensor(c, p, N, 2.0, samples + 1, al, 1, tm, st, nullptr);
    else if (N <= 24) s = run_sre(c, p, N, 2.0, samples + 1, al, 1, tm, st, nullptr);
    else s = run_sre_hbm_terms(c, p, N, samples + 1, al, tm, st);
    if (s) return s;
    e = launch_mc_stats(tm, al, samples, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mc_stats");
    if ((s = finish(c, (const double*)c->res.ptr, 4, st))) return s;
    const double mean = c->host_res[0], var = c->host_res[1], n_nz = c->host_res[2], S0 = c->host_res[3];
    const double two_n = std::ldexp(1.0, N), w = (two_n - 1.0) / two_n;
    const double Shat = S0 / two_n + w * mean;
    *M2_out = -std::log2(Shat);
    if (stderr_out) *stderr_out = n_nz > 0.0 ? w * std::sqrt(var / n_nz) / (Shat * std::log(2.0)) : 0.0;
    if (!std::isfinite(*M2_out)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite estimate");
    return HADAMAG_OK;
}
