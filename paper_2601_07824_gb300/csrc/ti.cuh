// ti.cuh -- per-chain arithmetic of the thermodynamic-integration estimator (Sec. 3.2,
// Algorithm 3), host- and device-callable so that the same code drives the kernels in ti.cu.
//
// Chain l reads the SplitMix64 stream started at seed + l: output 0 gives the start pattern
// (its top N bits), output 1 + 2t the bit flipped at step t (mod N, a symmetric one-bit
// proposal) and output 2 + 2t the acceptance variate u = (top 53 bits) / 2^53 in [0, 1).
#pragma once
#include <math.h>
#include <stdint.h>

#include "rng.cuh"

namespace hm {

// beta_l = l / (L-1) on [0, 1], computed as l * (1 / (L-1)) with the last point exactly 1
__host__ __device__ __forceinline__ double ti_beta(int l, int L) {
    return l == L - 1 ? 1.0 : (double)l * (1.0 / (double)(L - 1));
}

__host__ __device__ __forceinline__ int64_t ti_start_pattern(uint64_t seed, int l, int N) {
    return (int64_t)(splitmix64_out(seed + (uint64_t)l, 0) >> (64 - N));
}

__host__ __device__ __forceinline__ int ti_flip_bit(uint64_t seed, int l, int64_t t, int N) {
    return (int)(splitmix64_out(seed + (uint64_t)l, (uint64_t)(1 + 2 * t)) % (uint64_t)N);
}

__host__ __device__ __forceinline__ double ti_uniform(uint64_t seed, int l, int64_t t) {
    return (double)(splitmix64_out(seed + (uint64_t)l, (uint64_t)(2 + 2 * t)) >> 11) * 0x1p-53;
}

// Metropolis acceptance of a move from energy fa to f2 at inverse temperature beta
__host__ __device__ __forceinline__ bool ti_accept(double u, double beta, double f2, double fa) {
    return u < exp(fmin(0.0, -beta * (f2 - fa)));
}

// Composite Simpson weight of grid point l on [0, 1] with L >= 3 points; for even L the last
// three intervals take Simpson's 3/8 rule.
__host__ __device__ __forceinline__ double ti_simpson_weight(int l, int L) {
    const double h = 1.0 / (double)(L - 1);
    const int n13 = (L & 1) ? L - 1 : L - 4;  // intervals covered by the 1/3 rule (even)
    double w = 0.0;
    if (n13 > 0 && l <= n13) w += (l == 0 || l == n13) ? h / 3.0 : ((l & 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0);
    if (!(L & 1) && l >= L - 4) {
        const int k = l - (L - 4);
        w += (k == 0 || k == 3) ? 3.0 * h / 8.0 : 9.0 * h / 8.0;
    }
    return w;
}

// M_2 from the quadrature I of the chain means: I = ln Z_0 - ln Z_1 = -ln((S_2 + 2^N eps) / 2^N)
__host__ __device__ __forceinline__ double ti_m2(double I, double eps) { return -log2(exp(-I) - eps); }

}  // namespace hm
