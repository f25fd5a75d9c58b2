// grad_api.cu -- C ABI entry point for dM_2/dpsi* (adjoint kernels in grad.cu).
#include <algorithm>
#include <cmath>

#include "ctx.h"
#include "grad.h"
#include "sre_fwd.h"

using namespace hm;

namespace hm {

// Enqueues the adjoint kernels over the X-strings a0 .. a0 + count - 1: per-part FP32 partial
// gradients dS_2/dpsi* in c->grad_acc and per-part FP64 sums [S_2, S_1, 0] in c->part
// (*nparts parts).  For 16 <= N, a0 and count must be multiples of 8.  No host synchronisation.
hadamag_status enqueue_grad_parts(hadamag_ctx_t c, const float2* p, int N, int64_t a0, int64_t count, cudaStream_t st,
                                  int64_t* nparts_out) {
    hadamag_status s;
    cudaError_t e;
    const int64_t dim = int64_t(1) << N;
    int64_t nparts = 0;
    if (N <= 15) {
        int groups_max = c->sm_count * 8;
        const int64_t cap_bytes = (int64_t)512 << 20;  // partial gradients: at most 512 MiB
        while (groups_max > 1 && (int64_t)groups_max * dim * 8 > cap_bytes) groups_max >>= 1;
        const int gpc = grad_onepass_gpc(N);
        if (groups_max < gpc) groups_max = gpc;
        if ((s = ensure_buf(c, c->grad_acc, (size_t)groups_max * dim * sizeof(float2)))) return s;
        if ((s = ensure_buf(c, c->part, (size_t)groups_max * 3 * sizeof(double)))) return s;
        if ((e = cudaMemsetAsync(c->grad_acc.ptr, 0, (size_t)groups_max * dim * sizeof(float2), st)) != cudaSuccess)
            return cuda_fail(c, e, "memset partials");
        int ng = 0;
        e = launch_grad_onepass(p, N, (double*)c->part.ptr, (float2*)c->grad_acc.ptr, groups_max, &ng, st, a0, count);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "grad_onepass");
        nparts = ng;
    } else {
        GradParams P{};
        const int M = N - 11;
        const size_t per_a = (size_t)dim / 2 * sizeof(float2);
        // X-strings per batch: 8 (the 8 pass-1 warps share the state rows of two units, staged
        // once) unless the tuner found 2 faster for this N (more, smaller pass-1 tasks)
        const int A = c->grad_xbatch[N] ? c->grad_xbatch[N] : 8;
        P.psi = p; P.N = N; P.A = A; P.U = 8 / A;
        P.n_batches = count / A;
        P.a_base = a0;
        // 2 units per pass-1 warp, 1 column tile per pass-2 task: at these sizes (2^(N-11) units)
        // larger tasks leave too few per pipeline stage for the grid (measured slower)
        const int tiles = 1024 >> (13 - M);
        P.UPW = 2;
        P.TPT = 1;
        P.p1 = (1 << M) / (P.U * P.UPW);
        P.p2 = A * tiles / P.TPT;
        P.p3 = A * ((1 << M) / 16);
        int grid = 0;
        if ((e = grad_threepass_grid(N, c->sm_count, &grid)) != cudaSuccess) return cuda_fail(c, e, "occupancy");
        // stages between the passes of a batch, for a ring of 2 lag + 1 slots within 96 MiB of
        // L2 (N = 16: 8, 17: 4, 18: 2, 19 and 20: 1 with two CTAs per SM)
        P.lag = pipeline_lag((int64_t)P.p1 + P.p2 + P.p3, grid, 2, (size_t)A * per_a, (size_t)96 << 20);
        P.R = 2 * P.lag + 1;
        if ((s = ensure_buf(c, c->scratch, (size_t)P.R * A * per_a))) return s;
        if ((s = ensure_buf(c, c->counters, 3 * 64 * sizeof(unsigned)))) return s;
        if ((s = ensure_buf(c, c->grad_acc, (size_t)grid * dim * sizeof(float2)))) return s;
        if ((s = ensure_buf(c, c->part, (size_t)grid * 3 * sizeof(double)))) return s;
        if ((e = cudaMemsetAsync(c->grad_acc.ptr, 0, (size_t)grid * dim * sizeof(float2), st)) != cudaSuccess)
            return cuda_fail(c, e, "memset partials");
        if ((e = cudaMemsetAsync(c->counters.ptr, 0, 3 * 64 * sizeof(unsigned), st)) != cudaSuccess)
            return cuda_fail(c, e, "memset counters");
        P.scratch = (float2*)c->scratch.ptr;
        P.done1 = (unsigned*)c->counters.ptr; P.done2 = P.done1 + 64; P.done3 = P.done1 + 128;
        P.status = (int*)c->status.ptr; P.spin_limit = c->spin_limit; P.wait_bias = c->wait_bias;
        P.gpart = (float2*)c->grad_acc.ptr;
        P.sums = (double*)c->part.ptr;
        e = launch_grad_threepass(P, grid, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "grad_threepass");
        nparts = grid;
    }
    *nparts_out = nparts;
    return HADAMAG_OK;
}

// The adjoint's x-batch tuner: on the first uncaptured call for N >= 16 (autotuning on), times
// the three-pass kernel on 2^13 X-strings (a >= 2^(N-1)) with 8 and with 2 X-strings per batch
// (two launches each, the second timed with CUDA events) and keeps the faster for the context.
static hadamag_status tune_grad(hadamag_ctx_t c, const float2* p, int N, cudaStream_t st) {
    if (N < 16 || c->grad_xbatch[N] || !c->autotune) return HADAMAG_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(c, e, "capture query");
    if (cap != cudaStreamCaptureStatusNone) return HADAMAG_OK;
    const int64_t dim = int64_t(1) << N, cnt = std::min<int64_t>(dim / 2, int64_t(1) << 13);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(c, HADAMAG_ERR_CUDA, "events");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(c, HADAMAG_ERR_CUDA, "events"); }
    hadamag_status s = HADAMAG_OK;
    float best = 1e30f;
    int win = 8;
    for (int cand : {8, 2}) {
        c->grad_xbatch[N] = cand;
        for (int rep = 0; rep < 2 && !s; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            int64_t np = 0;
            s = enqueue_grad_parts(c, p, N, dim / 2, cnt, st, &np);
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (s) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { s = cuda_fail(c, e, "tune sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; win = cand; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->grad_xbatch[N] = s ? 0 : win;
    if (s) return s;
    return status_word_now(c, st);
}

// Enqueues the adjoint: gradient written to grad_out (same dtype as `dt`), and the FP64 sums
// [S_2, S_1, 0] left in c->res (device).  No host synchronisation.
hadamag_status enqueue_grad(hadamag_ctx_t c, const float2* p, int N, void* grad_out, bool c128, cudaStream_t st) {
    hadamag_status s;
    cudaError_t e;
    const int64_t dim = int64_t(1) << N;
    int64_t nparts = 0;
    if ((s = enqueue_grad_parts(c, p, N, 0, dim, st, &nparts))) return s;
    e = launch_sum_triples((const double*)c->part.ptr, nparts, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    e = launch_grad_finalize((const float2*)c->grad_acc.ptr, nparts, dim, (const double*)c->res.ptr, grad_out, c128, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "grad_finalize");
    return HADAMAG_OK;
}

}  // namespace hm

extern "C" hadamag_status hadamag_sre_grad(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt,
                                           double* M2_out, void* grad, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !aligned16(grad) || !M2_out)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 20) return fail(c, HADAMAG_ERR_INVALID_ARG, "gradient needs 1 <= N <= 20 (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    const float2* p;
    if ((s = as_c64(c, psi, int64_t(1) << N, dt, st, &p))) return s;
    if ((s = tune_grad(c, p, N, st))) return s;
    if ((s = enqueue_grad(c, p, N, grad, dt == HADAMAG_C128, st))) return s;
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    const double S2 = c->host_res[0];
    double M2 = -std::log2(S2 / std::ldexp(1.0, N));
    if (M2 == 0.0) M2 = 0.0;
    *M2_out = M2;
    if (!std::isfinite(M2)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite S_2");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_set_grad_xbatch(hadamag_ctx_t c, int N, int A) {
    if (!c || N < 16 || N > 20 || (A != 2 && A != 4 && A != 8)) return HADAMAG_ERR_INVALID_ARG;
    c->grad_xbatch[N] = A;
    return HADAMAG_OK;
}
