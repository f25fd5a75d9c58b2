// mc.cu -- uniform-X Monte-Carlo helpers: SplitMix64 X-strings and FP64 sample statistics.
//
// The estimator follows from the per-X-string decomposition of Algorithm 2 (Sec. 3.1.2):
// S_2 / 2^N = E_{a ~ U}[ S(a) ] with S(a) = sum_b |chi_b(a)|^4.  X-strings come from
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output i = mix(seed + (i+1) * gamma),
// a_i = its top N bits, so sample i depends only on (seed, i) and any range can be redone.
#include "extra.h"
#include "sre_fwd.h"

namespace hm {

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void mc_xstrings_kernel(uint64_t seed, int64_t count, int N, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)(splitmix64_out(seed, (uint64_t)i) >> (64 - N));
}

// out2[0] = mean of terms[3i], out2[1] = unbiased sample variance (fixed summation order).
__global__ void mc_stats_kernel(const double* __restrict__ t, int64_t n, double* __restrict__ out2) {
    __shared__ double s[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += t[3 * i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = s[0] / (double)n;
    __syncthreads();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double d = t[3 * i] - mean;
        v += d * d;
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = mean;
        out2[1] = n > 1 ? s[0] / (double)(n - 1) : 0.0;
    }
}

cudaError_t launch_mc_xstrings(uint64_t seed, int64_t count, int N, int64_t* out, cudaStream_t st) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    mc_xstrings_kernel<<<(unsigned)blocks, 256, 0, st>>>(seed, count, N, out);
    return cudaGetLastError();
}

cudaError_t launch_mc_stats(const double* terms, int64_t count, double* out2, cudaStream_t st) {
    mc_stats_kernel<<<1, 256, 0, st>>>(terms, count, out2);
    return cudaGetLastError();
}

}  // namespace hm
