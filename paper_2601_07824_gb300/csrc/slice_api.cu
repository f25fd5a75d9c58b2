// slice_api.cu -- exact SRE and its adjoint over a slice [a0, a1) of the X-strings, for
// splitting one state's computation across GPUs (or across calls), and the combination of the
// slices' partial results.
//
// The a-loop of Algorithm 2 is a sum of independent per-X-string terms; Sec. 4.1 distributes it
// over threads, processes and GPUs, each contributing a partial sum, combined by one reduction.
//
// Determinism of the forward sums.  The X-strings are grouped into chunks of
// hadamag_sre_chunk(N) consecutive values.  A chunk's triple [S_n, S_1, T_1] is a fixed-order
// FP64 sum of its per-X-string triples, each a fixed-order sum of its tile partials, so it
// depends only on the chunk: not on the launch that computed it, the slice around it, the grid
// or the GPU.  hadamag_sre_combine adds chunk triples in chunk order; every chunk-aligned
// partition of [0, 2^N) -- one slice or many, on one GPU or many -- gives the same bits.
#include <cmath>

#include "../../include/hadamag.h"
#include "ctx.h"
#include "extra.h"
#include "grad.h"
#include "sre_fwd.h"
#include "sre_tc.h"

namespace hm {
namespace {

constexpr int kChunkLog2 = 12;
constexpr size_t kTileBudget = (size_t)256 << 20;  // per-(X-string, tile) partials per launch

__global__ void iota_xstrings(int64_t a0, int64_t count, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a0 + i;
}

// out[c] = sum of in[c*ch .. (c+1)*ch) (triples), one CTA per chunk: fixed per-thread strides,
// then a fixed tree.
__global__ void chunk_sums(const double* __restrict__ in, int64_t ch, double* __restrict__ out) {
    __shared__ double s[3][256];
    const double* base = in + (size_t)blockIdx.x * ch * 3;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = threadIdx.x; i < ch; i += blockDim.x) {
        a0 += base[i * 3];
        a1 += base[i * 3 + 1];
        a2 += base[i * 3 + 2];
    }
    s[0][threadIdx.x] = a0;
    s[1][threadIdx.x] = a1;
    s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[blockIdx.x * 3] = s[0][0];
        out[blockIdx.x * 3 + 1] = s[1][0];
        out[blockIdx.x * 3 + 2] = s[2][0];
    }
}

int64_t chunk_of(int N) { return int64_t(1) << (N < kChunkLog2 ? N : kChunkLog2); }

// X-strings per launch: a whole number of chunks whose per-(X-string, tile) partials fit the
// budget.
int64_t batch_of(hadamag_ctx_t c, int N, double n) {
    int64_t per_a = 1;
    if (use_tensor_path(c, N, n)) per_a = tc_triples_per_a(N);
    else if (N > 15) per_a = twopass_triples_per_a(N);
    int64_t b = chunk_of(N);
    while ((size_t)(2 * b) * per_a * 3 * sizeof(double) <= kTileBudget && 2 * b <= (int64_t(1) << N)) b *= 2;
    return b;
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" int64_t hadamag_sre_chunk(int N) { return (N < 1 || N > 24) ? 0 : chunk_of(N); }

extern "C" hadamag_status hadamag_sre_slice(hadamag_ctx_t c, const void* psi, int N, double n, hadamag_dtype dt,
                                            int64_t a0, int64_t a1, double* chunks_dev, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !chunks_dev || ((uintptr_t)chunks_dev & 7u))
        return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 24) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 24] (got %d)", N);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(c, HADAMAG_ERR_INVALID_ARG, "n must be > 0");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    const int64_t dim = int64_t(1) << N, ch = chunk_of(N);
    if (a0 < 0 || a1 < a0 || a1 > dim || a0 % ch || a1 % ch)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "slice [%lld, %lld) must lie in [0, 2^N) on multiples of %lld",
                    (long long)a0, (long long)a1, (long long)ch);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    if (a1 == a0) return finish(c, nullptr, 0, st);
    const float2* p;
    if ((s = as_c64(c, psi, dim, dt, st, &p))) return s;
    const int64_t B = batch_of(c, N, n);
    const int64_t first = (a1 - a0) < B ? (a1 - a0) : B;
    if ((s = ensure_buf(c, c->alist, (size_t)first * sizeof(int64_t)))) return s;
    if ((s = ensure_buf(c, c->terms, (size_t)first * 3 * sizeof(double)))) return s;
    int64_t* al = (int64_t*)c->alist.ptr;
    double* tm = (double*)c->terms.ptr;
    const bool tensor = use_tensor_path(c, N, n);
    for (int64_t b0 = a0; b0 < a1; b0 += B) {
        const int64_t cnt = (a1 - b0) < B ? (a1 - b0) : B;
        int64_t blocks = (cnt + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        iota_xstrings<<<(unsigned)blocks, 256, 0, st>>>(b0, cnt, al);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "iota_xstrings");
        s = tensor ? run_sre_tensor(c, p, N, n, cnt, al, 1, tm, st, nullptr)
                   : run_sre(c, p, N, n, cnt, al, 1, tm, st, nullptr);
        if (s) return s;
        chunk_sums<<<(unsigned)(cnt / ch), 256, 0, st>>>(tm, ch, chunks_dev + (size_t)((b0 - a0) / ch) * 3);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "chunk_sums");
    }
    return finish(c, nullptr, 0, st);
}

extern "C" hadamag_status hadamag_sre_combine(int N, double n, const double* chunks_host, int64_t nchunks,
                                              double* M_out, double* lost_norm_out) {
    if (N < 1 || N > 24 || !chunks_host || !M_out) return HADAMAG_ERR_INVALID_ARG;
    if (!(n > 0.0) || !std::isfinite(n)) return HADAMAG_ERR_INVALID_ARG;
    if (nchunks != (int64_t(1) << N) / chunk_of(N)) return HADAMAG_ERR_INVALID_ARG;
    double sums[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < nchunks; ++i) {
        sums[0] += chunks_host[3 * i];
        sums[1] += chunks_host[3 * i + 1];
        sums[2] += chunks_host[3 * i + 2];
    }
    return sre_from_sums(nullptr, N, n, sums, M_out, lost_norm_out);
}

extern "C" hadamag_status hadamag_sre_grad_slice(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt,
                                                 int64_t a0, int64_t a1, double* sums_out, void* dS_dev,
                                                 hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !aligned16(dS_dev) || !sums_out)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 20) return fail(c, HADAMAG_ERR_INVALID_ARG, "gradient needs 1 <= N <= 20 (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    const int64_t dim = int64_t(1) << N, ch = chunk_of(N);
    if (a0 < 0 || a1 < a0 || a1 > dim || a0 % ch || a1 % ch)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "slice [%lld, %lld) must lie in [0, 2^N) on multiples of %lld",
                    (long long)a0, (long long)a1, (long long)ch);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    if (a1 == a0) {
        if ((e = cudaMemsetAsync(dS_dev, 0, (size_t)dim * sizeof(double2), st)) != cudaSuccess)
            return cuda_fail(c, e, "memset dS");
        sums_out[0] = sums_out[1] = 0.0;
        return finish(c, nullptr, 0, st);
    }
    const float2* p;
    if ((s = as_c64(c, psi, dim, dt, st, &p))) return s;
    int64_t nparts = 0;
    if ((s = enqueue_grad_parts(c, p, N, a0, a1 - a0, st, &nparts))) return s;
    e = launch_sum_triples((const double*)c->part.ptr, nparts, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    e = launch_grad_sum_parts((const float2*)c->grad_acc.ptr, nparts, dim, (double2*)dS_dev, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "grad_sum_parts");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    sums_out[0] = c->host_res[0];
    sums_out[1] = c->host_res[1];
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_sre_grad_combine(hadamag_ctx_t c, const void* dS_dev, int N, double S2,
                                                   hadamag_dtype dt, double* M2_out, void* grad_dev,
                                                   hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(dS_dev) || !aligned16(grad_dev) || !M2_out)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 20) return fail(c, HADAMAG_ERR_INVALID_ARG, "gradient needs 1 <= N <= 20 (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    if (!(S2 > 0.0) || !std::isfinite(S2)) return fail(c, HADAMAG_ERR_NONFINITE, "S_2 must be finite and > 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    if ((s = begin(c, st))) return s;
    const int64_t dim = int64_t(1) << N;
    cudaError_t e = launch_grad_scale((const double2*)dS_dev, dim, S2, grad_dev, dt == HADAMAG_C128, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "grad_scale");
    double M2 = -std::log2(S2 / std::ldexp(1.0, N));
    *M2_out = M2 == 0.0 ? 0.0 : M2;
    return finish(c, nullptr, 0, st);
}
