// mc.cu -- uniform-X Monte-Carlo helpers: SplitMix64 X-strings and FP64 sample statistics.
//
// The estimator follows from the per-X-string decomposition of Algorithm 2 (Sec. 3.1.2):
// S_2 / 2^N = [S(0) + sum_{a != 0} S(a)] / 2^N with S(a) = sum_b |chi_b(a)|^4.  The X-string
// a = 0, which holds the identity string, is evaluated exactly (the paper likewise takes the
// identity out of its sampling, Sec. 4.2 footnote) and the others are sampled uniformly:
// S_hat = [S(0) + (2^N - 1) mean_{a_i != 0} S(a_i)] / 2^N.  X-strings come from SplitMix64
// (Steele, Lea & Flood, OOPSLA 2014): output i = mix(seed + (i+1) * gamma), a_i = its top N
// bits (samples that come out 0 are dropped), so sample i depends only on (seed, i).
#include "extra.h"
#include "rng.cuh"
#include "sre_fwd.h"

namespace hm {

__global__ void mc_xstrings_kernel(uint64_t seed, int64_t count, int N, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)(splitmix64_out(seed, (uint64_t)i) >> (64 - N));
}

// out4 = [mean, unbiased variance, count] of terms[3i] over samples with a_i != 0, and S(0)
// = terms[3n] (the exactly evaluated a = 0 entry appended after the samples).  Fixed order.
__global__ void mc_stats_kernel(const double* __restrict__ t, const int64_t* __restrict__ a, int64_t n,
                                double* __restrict__ out4) {
    __shared__ double s[256];
    __shared__ double cnt[256];
    double acc = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (a[i] != 0) { acc += t[3 * i]; c += 1.0; }
    s[threadIdx.x] = acc;
    cnt[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) { s[threadIdx.x] += s[threadIdx.x + w]; cnt[threadIdx.x] += cnt[threadIdx.x + w]; }
        __syncthreads();
    }
    const double m = cnt[0] > 0.0 ? s[0] / cnt[0] : 0.0, total = cnt[0];
    __syncthreads();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (a[i] != 0) { const double d = t[3 * i] - m; v += d * d; }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out4[0] = m;
        out4[1] = total > 1.0 ? s[0] / (total - 1.0) : 0.0;
        out4[2] = total;
        out4[3] = t[3 * n];
    }
}

// The 2^(N-1) even-weight X-strings: a_i = 2i + parity(i), a bijection from [0, 2^(N-1)) onto
// the even-weight a in [0, 2^N) (the X-sectors that survive a U(1) or prod_j Z_j symmetry).
__global__ void even_xstrings_kernel(int64_t count, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (i << 1) | (int64_t)(__popcll((unsigned long long)i) & 1);
}

cudaError_t launch_even_xstrings(int64_t count, int64_t* out, cudaStream_t st) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    even_xstrings_kernel<<<(unsigned)blocks, 256, 0, st>>>(count, out);
    return cudaGetLastError();
}

cudaError_t launch_mc_xstrings(uint64_t seed, int64_t count, int N, int64_t* out, cudaStream_t st) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    mc_xstrings_kernel<<<(unsigned)blocks, 256, 0, st>>>(seed, count, N, out);
    return cudaGetLastError();
}

cudaError_t launch_mc_stats(const double* terms, const int64_t* a_list, int64_t count, double* out4, cudaStream_t st) {
    mc_stats_kernel<<<1, 256, 0, st>>>(terms, a_list, count, out4);
    return cudaGetLastError();
}

}  // namespace hm

namespace hm {

// Per-X-string sums [S_2(a), S_1(a), 0] for 25 <= N <= 28 (three-pass kernel, HBM scratch).
hadamag_status run_sre_hbm_terms(hadamag_ctx_t c, const float2* psi, int N, int64_t count, const int64_t* a_list,
                                 double* terms, cudaStream_t st) {
    if (N < 25 || N > 28) return fail(c, HADAMAG_ERR_UNSUPPORTED, "three-pass schedule covers N = 25..28");
    hadamag_status s;
    cudaError_t e;
    const size_t per_a = ((size_t)1 << (N - 1)) * sizeof(float2);
    const int tiles = hbm_tiles_per_a(N);
    HbmParams P{};
    P.psi = psi; P.N = N; P.count = count; P.a_list = a_list; P.R = 3;
    P.n_batches = count;
    P.p1 = P.p2 = P.p3 = 1 << (N - 14);
    if ((s = ensure_buf(c, c->scratch, (size_t)P.R * per_a))) return s;
    if ((s = ensure_buf(c, c->counters, 3 * 64 * sizeof(unsigned)))) return s;
    if ((s = ensure_buf(c, c->tiles, (size_t)count * tiles * 3 * sizeof(double)))) return s;
    P.scratch = (float2*)c->scratch.ptr;
    P.done1 = (unsigned*)c->counters.ptr; P.done2 = P.done1 + 64; P.done3 = P.done1 + 128;
    P.status = (int*)c->status.ptr; P.spin_limit = c->spin_limit; P.wait_bias = c->wait_bias;
    P.out = (double*)c->tiles.ptr;
    if ((e = cudaMemsetAsync(c->counters.ptr, 0, 3 * 64 * sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(c, e, "memset counters");
    int grid = 0;
    e = launch_hbm(P, c->sm_count, &grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sre_threepass");
    e = launch_sum_tiles((double*)c->tiles.ptr, count, tiles, terms, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_tiles");
    return HADAMAG_OK;
}

}  // namespace hm
