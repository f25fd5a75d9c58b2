// batched.cu -- M_2 and dM_2/dpsi* of many states of uneven N in ONE persistent launch.
//
// The state table (built on the host) lists the large states first, then the small ones, each
// group largest first.  Every CTA of the (fully resident) grid runs two phases:
//   1. large states (15 <= N <= 18), in table order, with the static schedule of the
//      single-state adjoint: the tasks of all large states form one list (per state: the stage
//      tasks of the three passes in g3_decode order, then its finalize tasks), and CTA b runs
//      tasks b, b + grid, b + 2 grid, ...  The task code is inlined (per N), so this phase makes
//      no function calls.  Passes 1-3 scatter into per-CTA partial gradients; the finalize tasks
//      reduce those partials (FP64, fixed CTA order), write the gradient and zero the partials.
//      Each large state has its own set of partials (a buffer slot) unless the states would
//      need more memory than the host's budget allows; then states take turns on the slots, a
//      state's pass 3 waiting for the finalize of the previous state on its slot.
//   2. small states (N <= 14), through a dynamic ticket counter: the X-strings in n_chunks equal
//      chunks, one item each, done by one CTA with the one-pass adjoint (grad_phases.cuh) into
//      private partial gradients (one per thread group); with one chunk the item itself reduces
//      the partials in a fixed order and writes dM_2/dpsi* and M_2, otherwise a finalize item
//      after the chunks does.  CTAs enter this phase as they run out of large-state tasks.
// Forward only (no gradient requested, the FWD kernel): small states skip the cube, the back
// transform and the scatter; large states run passes 1 and 2 only, and one finalize task per
// state turns the pass-2 sums into M_2 once every pass-2 task has counted in.
// In phase 1 every task waits only on tasks earlier in the list, so the CTA holding the earliest
// unfinished task is running it (the single-state argument); in phase 2 only a finalize item
// waits, on chunk items with smaller tickets that running CTAs hold.  So the launch cannot
// deadlock; waits are bounded and report a timeout through the status word.  The pass-2 sums
// reach S_2 through atomics, so M_2 may differ between runs in the last bits.
#include "batched.h"
#include "grad_phases.cuh"

namespace hm {

// dM_2/dpsi* and M_2 of a small state from S_2 and its nparts partial gradients (fixed order).
__device__ __forceinline__ void small_finish(const BatchState& s, double S2, int nparts, double* m2_out) {
    const int64_t dim = int64_t(1) << s.N;
    const double scale = -1.0 / (0.69314718055994530942 * S2);
    if (!s.fwd) for (int64_t z = threadIdx.x; z < dim; z += blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int k = 0; k < nparts; ++k) {
            const float2 v = __ldcg(s.gsmall + (size_t)k * dim + z);
            gx += v.x;
            gy += v.y;
        }
        if (s.grad) s.grad[z] = make_float2((float)(gx * scale), (float)(gy * scale));
    }
    if (threadIdx.x == 0) m2_out[s.out_idx] = -log2(S2 / (double)dim);
    __syncthreads();
}

// Chunk c of a small state: X-strings [c 2^N / n_chunks, (c + 1) 2^N / n_chunks).  Not inlined:
// the small-state items get their own register allocation.
template <int L, bool FWD>
__device__ __noinline__ void small_item(const BatchState& s, float2* smem, double* m2_out, int c) {
    constexpr int G = OnepassShape<L>::G, GPC = 256 / G;  // groups of one 256-thread CTA
    static_assert(L >= 9 && L <= 13, "small items cover N = 10..14");
    __shared__ double sums[GPC][2];
    const uint32_t tid = threadIdx.x, gi = tid / G, t = tid % G;
    const int64_t dim = int64_t(1) << L << 1, per = dim / s.n_chunks;
    float2* sm = smem + (size_t)gi * tile_slots(L);
    double acc = 0.0, acc1 = 0.0;
    grad_onepass_group<L, FWD>(s.psi, L + 1, FWD ? nullptr : s.gsmall + ((size_t)c * GPC + gi) * dim, gi, GPC, sm,
                               acc, acc1, (int64_t)c * per, per);
    if (t == 0) { sums[gi][0] = acc; sums[gi][1] = acc1; }
    __syncthreads();
    double S2 = 0.0;
    for (int k = 0; k < GPC; ++k) S2 += sums[k][0];
    if (s.n_chunks > 1) {
        // the finalize item combines the chunks: publish this chunk's S_2 and partials
        if (tid == 0) {
            s.s2[c] = S2;
            __threadfence();
            red_release_add(s.ctr, 1u);
        }
        __syncthreads();
        return;
    }
    small_finish(s, S2, GPC, m2_out);
}

// Finalize item of a small state split into n_chunks > 1 chunks.
__device__ __noinline__ bool small_finalize(const BatchedParams& B, const BatchState& s, double* m2_out) {
    if (!cta_wait_geq(s.ctr, (unsigned)s.n_chunks + B.ctl.wait_bias, B.ctl.status, B.ctl.spin_limit)) return false;
    double S2 = 0.0;
    for (int c = 0; c < s.n_chunks; ++c) S2 += reinterpret_cast<volatile double*>(s.s2)[c];
    small_finish(s, S2, s.n_chunks * (256 >> (s.N - 6)), m2_out);
    return true;
}

// One stage task (local index `local` in the state's list) of a large state.  prev_ok: this CTA
// has already seen the previous user of the state's partial-gradient slot finish (its pass-3
// tasks then skip that wait).
template <int M, bool FWD>
__device__ __forceinline__ bool large_task(const BatchedParams& B, const BatchState& s, int64_t local, float2* smem,
                                           bool& prev_ok) {
    if constexpr (FWD) {
        // forward only: stage st = pass 1 of batch st, pass 2 of batch st - lag; a slot is reused
        // once its pass 2 is done (the done3 / p3 fields of the state view point at done2 / p2)
        const G3State S{s.psi, s.N, s.scratch, s.R, s.A, s.U, s.n_batches, s.p1, s.p2, s.p2,
                        s.ctr, s.ctr + 64, s.ctr + 64, 0, s.UPW, s.TPT};
        const int64_t per_stage = (int64_t)s.p1 + s.p2;
        const int64_t st = local / per_stage;
        int r = (int)(local % per_stage);
        if (r < s.p1) {
            if (st >= s.n_batches) return true;
            return g3_pass1<M>(S, B.ctl, st, r, smem);
        }
        r -= s.p1;
        if (st - s.lag < 0 || st - s.lag >= s.n_batches) return true;
        double acc = 0.0, acc1 = 0.0;
        return g3_pass2<M, true>(S, B.ctl, st - s.lag, r, smem, acc, acc1, s.s2);
    } else {
        const G3State S{s.psi, s.N, s.scratch, s.R, s.A, s.U, s.n_batches, s.p1, s.p2, s.p3,
                        s.ctr, s.ctr + 64, s.ctr + 128, 0, s.UPW, s.TPT};
        int kind, r;
        int64_t g;
        g3_decode(local, s.p1, s.p2, s.p3, s.lag, kind, g, r);
        if (g < 0 || g >= s.n_batches) return true;
        if (kind == 1) return g3_pass1<M>(S, B.ctl, g, r, smem);
        if (kind == 2) {
            double acc = 0.0, acc1 = 0.0;
            return g3_pass2<M>(S, B.ctl, g, r, smem, acc, acc1, s.s2);
        }
        // pass 3 writes the shared partials: the previous large state on the slot must have
        // released them (waited for once per CTA and state)
        const unsigned* prev = prev_ok ? nullptr : s.prev_fin;
        prev_ok = true;
        return g3_pass3<M>(S, B.ctl, g, r, smem, s.gpart + ((size_t)blockIdx.x << s.N), prev,
                           prev ? s.prev_nfin : 0u);
    }
}

// Finalize task f of a large state (forward: the only one; else one slice of the gradient).
__device__ __forceinline__ bool finalize_task(const BatchedParams& B, const BatchState& s, int f, double* m2_out) {
    if (s.fwd) {
        // forward only: every pass-2 task has added its sums into s2
        for (int k = 0; k < s.R; ++k) {
            const int64_t nb = (s.n_batches > k) ? (s.n_batches - k + s.R - 1) / s.R : 0;
            if (!cta_wait_geq(s.ctr + 64 + k, (unsigned)(nb * s.p2) + B.ctl.wait_bias, B.ctl.status, B.ctl.spin_limit))
                return false;
        }
        if (threadIdx.x == 0) {
            double S2 = 0.0;
            for (int l = 0; l < kS2Lanes; ++l) S2 += reinterpret_cast<volatile double*>(s.s2)[2 * l];
            m2_out[s.out_idx] = -log2(S2 / (double)(int64_t(1) << s.N));
        }
        __syncthreads();
        return true;
    }
    // all pass-3 tasks of this state are done: every slot's counter reached its final value
    for (int k = 0; k < s.R; ++k) {
        const int64_t nb = (s.n_batches > k) ? (s.n_batches - k + s.R - 1) / s.R : 0;
        if (!cta_wait_geq(s.ctr + 128 + k, (unsigned)(nb * s.p3) + B.ctl.wait_bias, B.ctl.status, B.ctl.spin_limit))
            return false;
    }
    const int64_t dim = int64_t(1) << s.N;
    const int64_t chunk = (dim + s.n_fin - 1) / s.n_fin;
    const int64_t z0 = (int64_t)f * chunk, z1 = (z0 + chunk < dim) ? z0 + chunk : dim;
    double S2 = 0.0;
    for (int l = 0; l < kS2Lanes; ++l) S2 += reinterpret_cast<volatile double*>(s.s2)[2 * l];
    const double scale = -1.0 / (0.69314718055994530942 * S2);
    for (int64_t z = z0 + threadIdx.x; z < z1; z += blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int k = 0; k < B.nparts; ++k) {
            float2* p = s.gpart + ((size_t)k << s.N) + z;
            const float2 v = __ldcg(p);
            gx += v.x;
            gy += v.y;
            __stcg(p, make_float2(0.f, 0.f));
        }
        if (s.grad) s.grad[z] = make_float2((float)(gx * scale), (float)(gy * scale));
    }
    if (threadIdx.x == 0 && f == 0) m2_out[s.out_idx] = -log2(S2 / (double)dim);
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(s.fin, 1u);
    return true;
}

// This CTA's tasks of one large state: local indices first, first + grid, ... below the
// state's stage tasks plus finalize tasks.
template <int M, bool FWD>
__device__ __forceinline__ bool run_large(const BatchedParams& B, const BatchState& s, int64_t first, float2* smem) {
    bool prev_ok = s.prev_fin == nullptr;
    for (int64_t t = first; t < s.n_stage_tasks + s.n_fin; t += gridDim.x) {
        const bool ok = t < s.n_stage_tasks ? large_task<M, FWD>(B, s, t, smem, prev_ok)
                                            : finalize_task(B, s, (int)(t - s.n_stage_tasks), B.m2_out);
        if (!ok) return false;
    }
    return true;
}

template <bool FWD>
__global__ void __launch_bounds__(256, 2) batched_kernel(BatchedParams B) {
    extern __shared__ float2 smem[];
    __shared__ long long s_ticket;
    const uint32_t tid = threadIdx.x;
    // ---- phase 1: large states, static round-robin over their task list ----
    int64_t base = 0;  // list index of the current state's first task
    for (int k = 0; k < B.n_large; ++k) {
        const BatchState& s = B.states[k];
        // this CTA's first task of the state: the first list index >= base that is = blockIdx
        // modulo the grid
        const int64_t first = (((int64_t)blockIdx.x - base) % gridDim.x + gridDim.x) % gridDim.x;
        bool ok = true;
        switch (s.N) {
            case 15: ok = run_large<4, FWD>(B, s, first, smem); break;
            case 16: ok = run_large<5, FWD>(B, s, first, smem); break;
            case 17: ok = run_large<6, FWD>(B, s, first, smem); break;
            case 18: ok = run_large<7, FWD>(B, s, first, smem); break;
            default: break;
        }
        if (!ok) return;
        base += s.n_stage_tasks + s.n_fin;
    }
    // ---- phase 2: small states, dynamic tickets ----
    for (;;) {
        if (tid == 0) s_ticket = (long long)atomicAdd(B.ticket, 1ull);
        __syncthreads();
        const int64_t tau = s_ticket;
        __syncthreads();
        if (tau >= B.total) break;
        // the small state whose ticket segment holds tau (segments are contiguous, in order)
        int lo = B.n_large, hi = B.n_states - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.states[mid].task_begin <= tau) lo = mid;
            else hi = mid - 1;
        }
        const BatchState& s = B.states[lo];
        const int64_t local = tau - s.task_begin;
        if (local >= s.n_chunks) {
            if (!small_finalize(B, s, B.m2_out)) break;
            continue;
        }
        const int c = (int)local;
        switch (s.N) {
            case 10: small_item<9, FWD>(s, smem, B.m2_out, c); break;
            case 11: small_item<10, FWD>(s, smem, B.m2_out, c); break;
            case 12: small_item<11, FWD>(s, smem, B.m2_out, c); break;
            case 13: small_item<12, FWD>(s, smem, B.m2_out, c); break;
            case 14: small_item<13, FWD>(s, smem, B.m2_out, c); break;
            default: break;
        }
    }
}

size_t batched_smem_bytes() { return (size_t)(tile_slots(13) + kStageSlots) * sizeof(float2); }

// Resident CTAs of both kernels (the smaller, so either grid is fully resident).
cudaError_t batched_max_grid(int sm_count, int* grid) {
    int occ_min = 1 << 30;
    for (auto k : {batched_kernel<false>, batched_kernel<true>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batched_smem_bytes());
        if (e != cudaSuccess) return e;
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, batched_smem_bytes())) != cudaSuccess)
            return e;
        occ_min = occ < occ_min ? occ : occ_min;
    }
    *grid = (occ_min < 1 ? 1 : occ_min) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_batched(const BatchedParams& B, bool fwd, int grid, cudaStream_t st) {
    if (fwd) batched_kernel<true><<<grid, 256, batched_smem_bytes(), st>>>(B);
    else batched_kernel<false><<<grid, 256, batched_smem_bytes(), st>>>(B);
    return cudaGetLastError();
}

}  // namespace hm
