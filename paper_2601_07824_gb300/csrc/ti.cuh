// ti.cuh -- per-chain arithmetic of the thermodynamic-integration estimator (Sec. 3.2,
// Algorithm 3), host- and device-callable so that the same code drives the kernels in ti.cu.
//
// Chain l reads the SplitMix64 stream started at seed + l: output 0 gives the start pattern
// (its top N bits), output 1 + 2t the move of step t and output 2 + 2t the acceptance variate
// u = (top 53 bits) / 2^53 in [0, 1).  A move flips one bit (r mod N) or, in the even sector,
// two distinct bits b1 = r mod N, b2 = (r div N) mod (N-1) (+1 when b2 >= b1): a symmetric
// proposal that keeps the Hamming-weight parity (Sec. 3.2: for U(1) or prod_j Z_j symmetric
// states the odd-weight X-sectors have S(a) = 0); the even-sector start pattern has its bit 0
// flipped when its weight is odd.
#pragma once
#include <math.h>
#include <stdint.h>

#include "rng.cuh"

namespace hm {

// beta_l = l / (L-1) on [0, 1], computed as l * (1 / (L-1)) with the last point exactly 1
__host__ __device__ __forceinline__ double ti_beta(int l, int L) {
    return l == L - 1 ? 1.0 : (double)l * (1.0 / (double)(L - 1));
}

__host__ __device__ __forceinline__ int ti_parity(int64_t a) {
    uint64_t v = (uint64_t)a;
    v ^= v >> 32; v ^= v >> 16; v ^= v >> 8; v ^= v >> 4; v ^= v >> 2; v ^= v >> 1;
    return (int)(v & 1);
}

__host__ __device__ __forceinline__ int64_t ti_start_pattern(uint64_t seed, int l, int N, int even) {
    const int64_t a = (int64_t)(splitmix64_out(seed + (uint64_t)l, 0) >> (64 - N));
    return (even && ti_parity(a)) ? (a ^ 1) : a;
}

// XOR mask of the move proposed at step t
__host__ __device__ __forceinline__ int64_t ti_move(uint64_t seed, int l, int64_t t, int N, int even) {
    const uint64_t r = splitmix64_out(seed + (uint64_t)l, (uint64_t)(1 + 2 * t));
    const int b1 = (int)(r % (uint64_t)N);
    if (!even) return int64_t(1) << b1;
    int b2 = (int)((r / (uint64_t)N) % (uint64_t)(N - 1));
    if (b2 >= b1) ++b2;
    return (int64_t(1) << b1) | (int64_t(1) << b2);
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

// Statistical error (Eqs. Var_I_eps, m2error), Var[I] ~ sum_l w_l^2 2 tau_int sigma_f^2 / n_l,
// estimated by non-overlapping batch means: the n_s recorded samples of a chain are cut into
// B = min(32, n_s) batches of K = n_s div B consecutive samples (the remainder enters the mean
// only) and Var_l = sum_b (m_b - mbar)^2 / (B (B - 1)); delta M_2 = (d M_2 / d I) sqrt(Var[I]).
__host__ __device__ __forceinline__ int ti_n_batches(int64_t n_s) { return n_s < 32 ? (int)n_s : 32; }

__host__ __device__ inline double ti_chain_var(const double* bsum, int B, int64_t K) {
    if (B < 2) return 0.0;
    double mbar = 0.0;
    for (int b = 0; b < B; ++b) mbar += bsum[b] / (double)K;
    mbar /= (double)B;
    double v = 0.0;
    for (int b = 0; b < B; ++b) {
        const double d = bsum[b] / (double)K - mbar;
        v += d * d;
    }
    return v / ((double)B * (double)(B - 1));
}

// d M_2 / d I for M_2 = -log2(exp(-I) - eps) (+ const)
__host__ __device__ __forceinline__ double ti_m2_slope(double I, double eps) {
    return exp(-I) / ((exp(-I) - eps) * 0.693147180559945309417);
}

// M_2 from the quadrature I of the chain means, I = ln Z_0 - ln Z_1 with Z_1 = S_2 + Z_0 eps:
// Z_0 = 2^N gives -log2(exp(-I) - eps); the even sector (Z_0 = 2^(N-1)) adds 1
__host__ __device__ __forceinline__ double ti_m2(double I, double eps, int even) {
    return -log2(exp(-I) - eps) + (even ? 1.0 : 0.0);
}

}  // namespace hm
