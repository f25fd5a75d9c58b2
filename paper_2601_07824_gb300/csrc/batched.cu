// batched.cu -- M_2 and dM_2/dpsi* of many states of uneven N in ONE persistent launch.
//
// Work list (built on the host, largest first), taken through a dynamic ticket counter:
//   * small states (N <= 14): one self-contained item per state, done by one CTA: every X-string
//     with the one-pass adjoint (grad_phases.cuh), a private partial gradient per thread group,
//     then the CTA reduces the partials in a fixed order and writes dM_2/dpsi* and M_2;
//   * large states (15 <= N <= 18): the three passes of the adjoint (pass 1/2/3 tasks in stage
//     order, runtime dispatch on M = N - 11), scattering into per-CTA partial gradients, followed
//     by finalize tasks that reduce those partials (FP64, fixed CTA order), write the gradient
//     and zero the partials.  Each large state has its own set of partials (a buffer slot) unless
//     the states would need more memory than the host's budget allows; then states take turns on
//     the slots, a state's pass 3 waiting for the finalize of the previous state on its slot.
// Forward only (no gradient requested): small states skip the cube, the back transform and the
// scatter; large states run passes 1 and 2 only, and one finalize task per state turns the
// pass-2 sums into M_2 once every pass-2 task has counted in.  No partial-gradient buffers.
// Every wait is on a task with a smaller ticket, which a running CTA already holds, so the
// launch cannot deadlock (waits are bounded and report a timeout through the status word).
// Assignment of tasks to CTAs is dynamic, so sums may differ between runs in the last bits.
#include "batched.h"
#include "grad_phases.cuh"

namespace hm {

// The task functions are not inlined: each gets its own register allocation under the
// kernel's 128-register cap (inlined into one loop they needed ~245 and spilled ~1.2 KB).
template <int L, bool FWD>
__device__ __noinline__ void small_item(const BatchState& s, float2* smem, double* m2_out, int idx) {
    constexpr int G = OnepassShape<L>::G, GPC = 256 / G;  // groups of one 256-thread CTA
    static_assert(L >= 9 && L <= 13, "small items cover N = 10..14");
    __shared__ double sums[GPC][2];
    const uint32_t tid = threadIdx.x, gi = tid / G, t = tid % G;
    const int64_t dim = int64_t(1) << L << 1;
    float2* sm = smem + (size_t)gi * tile_slots(L);
    double acc = 0.0, acc1 = 0.0;
    grad_onepass_group<L, FWD>(s.psi, L + 1, FWD ? nullptr : s.gsmall + (size_t)gi * dim, gi, GPC, sm, acc, acc1);
    if (t == 0) { sums[gi][0] = acc; sums[gi][1] = acc1; }
    __syncthreads();
    double S2 = 0.0;
    for (int k = 0; k < GPC; ++k) S2 += sums[k][0];
    const double scale = -1.0 / (0.69314718055994530942 * S2);
    if (!FWD) for (int64_t z = tid; z < dim; z += blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int k = 0; k < GPC; ++k) {
            const float2 v = s.gsmall[(size_t)k * dim + z];
            gx += v.x;
            gy += v.y;
        }
        if (s.grad) s.grad[z] = make_float2((float)(gx * scale), (float)(gy * scale));
    }
    if (tid == 0) m2_out[s.out_idx] = -log2(S2 / (double)dim);
    __syncthreads();
}

template <int M>
__device__ __forceinline__ bool large_task_fwd(const BatchState& s, const G3Ctl& ctl, int64_t local, float2* smem) {
    // forward only: stage st = pass 1 of batch st, pass 2 of batch st - 1; a slot is reused once
    // its pass 2 is done (the done3 / p3 fields of the state view point at done2 / p2)
    const G3State S{s.psi, s.N, s.scratch, s.R, s.A, s.U, s.n_batches, s.p1, s.p2, s.p2,
                    s.ctr, s.ctr + 64, s.ctr + 64, 0, s.UPW, s.TPT};
    const int64_t per_stage = (int64_t)s.p1 + s.p2;
    const int64_t st = local / per_stage;
    int r = (int)(local % per_stage);
    if (r < s.p1) {
        if (st >= s.n_batches) return true;
        return g3_pass1<M>(S, ctl, st, r, smem);
    }
    r -= s.p1;
    if (st - 1 < 0 || st - 1 >= s.n_batches) return true;
    double acc = 0.0, acc1 = 0.0;
    return g3_pass2<M, true>(S, ctl, st - 1, r, smem, acc, acc1, s.s2);
}

template <int M>
__device__ __noinline__ bool large_task(const BatchedParams& B, const BatchState& s, int64_t local, float2* smem) {
    if (s.fwd) return large_task_fwd<M>(s, B.ctl, local, smem);
    const G3State S{s.psi, s.N, s.scratch, s.R, s.A, s.U, s.n_batches, s.p1, s.p2, s.p3,
                    s.ctr, s.ctr + 64, s.ctr + 128, 0, s.UPW, s.TPT};
    const int64_t per_stage = (int64_t)s.p1 + s.p2 + s.p3;
    const int64_t st = local / per_stage;
    int r = (int)(local % per_stage);
    int kind;
    int64_t g;
    if (r < s.p1) { kind = 1; g = st; }
    else if (r < s.p1 + s.p2) { kind = 2; g = st - 1; r -= s.p1; }
    else { kind = 3; g = st - 2; r -= s.p1 + s.p2; }
    if (g < 0 || g >= s.n_batches) return true;
    if (kind == 1) return g3_pass1<M>(S, B.ctl, g, r, smem);
    if (kind == 2) {
        double acc = 0.0, acc1 = 0.0;
        return g3_pass2<M>(S, B.ctl, g, r, smem, acc, acc1, s.s2);
    }
    // pass 3 writes the shared partials: the previous large state must have released them
    const unsigned* prev = s.prev_fin;
    return g3_pass3<M>(S, B.ctl, g, r, smem, s.gpart + ((size_t)blockIdx.x << s.N), prev, prev ? s.prev_nfin : 0u);
}

__device__ __noinline__ bool finalize_task(const BatchedParams& B, const BatchState& s, int f, double* m2_out,
                                              int idx) {
    if (s.fwd) {
        // forward only: every pass-2 task has added its sums into s2
        for (int k = 0; k < s.R; ++k) {
            const int64_t nb = (s.n_batches > k) ? (s.n_batches - k + s.R - 1) / s.R : 0;
            if (!cta_wait_geq(s.ctr + 64 + k, (unsigned)(nb * s.p2) + B.ctl.wait_bias, B.ctl.status, B.ctl.spin_limit))
                return false;
        }
        if (threadIdx.x == 0) {
            const double S2 = *reinterpret_cast<volatile double*>(s.s2);
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
    const double S2 = *reinterpret_cast<volatile double*>(s.s2);
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
    if (threadIdx.x == 0) { __threadfence(); red_release_add(s.fin, 1u); }
    return true;
}

__global__ void __launch_bounds__(256, 2) batched_kernel(BatchedParams B) {
    extern __shared__ float2 smem[];
    __shared__ long long s_ticket;
    const uint32_t tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_ticket = (long long)atomicAdd(B.ticket, 1ull);
        __syncthreads();
        const int64_t tau = s_ticket;
        __syncthreads();
        if (tau >= B.total) break;
        // the state whose ticket segment holds tau (segments are contiguous, in state order)
        int lo = 0, hi = B.n_states - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.states[mid].task_begin <= tau) lo = mid;
            else hi = mid - 1;
        }
        const int idx = lo;
        const BatchState& s = B.states[idx];
        const int64_t local = tau - s.task_begin;
        bool ok = true;
        if (s.kind == 0) {
            switch (s.N * 2 + s.fwd) {
                case 20: small_item<9, false>(s, smem, B.m2_out, idx); break;
                case 22: small_item<10, false>(s, smem, B.m2_out, idx); break;
                case 24: small_item<11, false>(s, smem, B.m2_out, idx); break;
                case 26: small_item<12, false>(s, smem, B.m2_out, idx); break;
                case 28: small_item<13, false>(s, smem, B.m2_out, idx); break;
                case 21: small_item<9, true>(s, smem, B.m2_out, idx); break;
                case 23: small_item<10, true>(s, smem, B.m2_out, idx); break;
                case 25: small_item<11, true>(s, smem, B.m2_out, idx); break;
                case 27: small_item<12, true>(s, smem, B.m2_out, idx); break;
                case 29: small_item<13, true>(s, smem, B.m2_out, idx); break;
                default: break;
            }
        } else if (local < s.n_stage_tasks) {
            switch (s.N) {
                case 15: ok = large_task<4>(B, s, local, smem); break;
                case 16: ok = large_task<5>(B, s, local, smem); break;
                case 17: ok = large_task<6>(B, s, local, smem); break;
                case 18: ok = large_task<7>(B, s, local, smem); break;
                default: break;
            }
        } else {
            ok = finalize_task(B, s, (int)(local - s.n_stage_tasks), B.m2_out, idx);
        }
        if (!ok) break;
    }
}

size_t batched_smem_bytes() { return (size_t)(tile_slots(13) + kStageSlots) * sizeof(float2); }

cudaError_t batched_max_grid(int sm_count, int* grid) {
    cudaError_t e = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_smem_bytes());
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel, 256, batched_smem_bytes())) != cudaSuccess)
        return e;
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_batched(const BatchedParams& B, int grid, cudaStream_t st) {
    batched_kernel<<<grid, 256, batched_smem_bytes(), st>>>(B);
    return cudaGetLastError();
}

}  // namespace hm
