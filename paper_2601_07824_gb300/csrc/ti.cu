// ti.cu -- thermodynamic-integration estimate of M_2 (Sec. 3.2, Eqs. Boltz to M2_TI,
// Algorithm 3).
//
// L Metropolis chains at beta_l = l / (L-1) sample X-strings a from Pi_beta(a) ~ exp(-beta f(a))
// with the energy f(a) = -ln(S(a) + eps), S(a) = sum_b |chi_b(a)|^4 the per-X-string sum of
// Algorithm 2.  Since <f>_beta = -d ln Z_beta / d beta, Z_0 = 2^N and Z_1 = S_2 + 2^N eps,
//     I = int_0^1 <f>_beta d beta = -ln((S_2 + 2^N eps) / 2^N),   M_2 = -log2(exp(-I) - eps),
// and I is taken by composite Simpson quadrature of the chain means over the beta grid (the
// last three intervals by the 3/8 rule when L is even, so any L >= 3 works).  The sign is the
// one the identity fixes: the printed return value carries the opposite sign.
//
// The chains are independent, so one step of all L chains is one batch of L per-X-string
// evaluations: the per-X kernels of Algorithm 2 (run_sre with per_a = 1, CUDA-core path) on the
// L proposals, then ti_step, one thread per chain, which decides, records and proposes the next
// move.  Random numbers are counter-based (the draws and moves are defined in ti.cuh); with
// sector = 1 the chains stay on even-weight X-strings (two-bit moves) and Z_0 = 2^(N-1).  The
// decision u < exp(min(0, -beta (f' - f))) is taken in FP64.
#include <cmath>
#include <vector>

#include "ctx.h"
#include "ti.cuh"

namespace hm {

struct TiChains {
    int64_t* a;           // [L] current X-string of each chain
    int64_t* prop;        // [L] proposals: the X-string list handed to the per-X kernels
    double* f;            // [L] energy of the current X-string
    double* acc;          // [L] sum of the energies recorded after burn-in
    double* out;          // [L + 3] chain means, I, M_2, delta M_2
    double* bsum;         // [L][B] batch sums of the recorded energies (error estimate)
    const double* terms;  // [3L] per-X sums of the listed X-strings; S(a) at 3l
    int64_t* traj;        // [L][T] chain state after each step, or null
    int* status;
    uint64_t seed;
    double eps;
    int64_t T, burn_in, n_s;
    int L, N;
    int even;  // 1: chains restricted to even-weight X-strings
    int B;     // batches per chain, K recorded steps each
    int64_t K;
};

__device__ __forceinline__ double ti_energy(const TiChains& c, double S) {
    const double x = S + c.eps;
    if (!(x > 0.0)) atomicOr(c.status, ST_NONPOS);
    return -log(x);
}

// start patterns, listed for the evaluation of their energies
__global__ void ti_start(TiChains c) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= c.L) return;
    const int64_t a = ti_start_pattern(c.seed, l, c.N, c.even);
    c.a[l] = a;
    c.prop[l] = a;
}

// energies of the start patterns, then the proposals of step 0
__global__ void ti_init(TiChains c) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= c.L) return;
    c.f[l] = ti_energy(c, c.terms[3 * l]);
    c.acc[l] = 0.0;
    for (int b = 0; b < c.B; ++b) c.bsum[(int64_t)l * c.B + b] = 0.0;
    c.prop[l] = c.a[l] ^ ti_move(c.seed, l, 0, c.N, c.even);
}

// step t: accept or reject the evaluated proposal, record, propose step t + 1
__global__ void ti_step(TiChains c, int64_t t) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= c.L) return;
    const double f2 = ti_energy(c, c.terms[3 * l]);
    double fa = c.f[l];
    int64_t a = c.a[l];
    if (ti_accept(ti_uniform(c.seed, l, t), ti_beta(l, c.L), f2, fa)) {
        a = c.prop[l];
        fa = f2;
        c.a[l] = a;
        c.f[l] = fa;
    }
    if (t >= c.burn_in) {
        c.acc[l] += fa;
        const int64_t b = (t - c.burn_in) / c.K;
        if (b < c.B) c.bsum[(int64_t)l * c.B + b] += fa;
    }
    if (c.traj) c.traj[(int64_t)l * c.T + t] = a;
    if (t + 1 < c.T) c.prop[l] = a ^ ti_move(c.seed, l, t + 1, c.N, c.even);
}

// chain means, the quadrature I, M_2 and its statistical error (fixed order)
__global__ void ti_finish(TiChains c) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double I = 0.0, var_I = 0.0;
    for (int l = 0; l < c.L; ++l) {
        const double m = c.acc[l] / (double)c.n_s, w = ti_simpson_weight(l, c.L);
        c.out[l] = m;
        I += w * m;
        var_I += w * w * ti_chain_var(c.bsum + (int64_t)l * c.B, c.B, c.K);
    }
    c.out[c.L] = I;
    c.out[c.L + 1] = ti_m2(I, c.eps, c.even);
    c.out[c.L + 2] = c.B < 2 ? 0.0 : ti_m2_slope(I, c.eps) * sqrt(var_I);
}

}  // namespace hm

using namespace hm;

extern "C" hadamag_status hadamag_sre_ti(hadamag_ctx_t c, const void* psi, int N, int L, int64_t n_s,
                                         int64_t burn_in, uint64_t seed, double eps, int sector,
                                         hadamag_dtype dt, double* M2_out, double* stderr_out,
                                         double* means_out, int64_t* traj_dev, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !M2_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (traj_dev && (reinterpret_cast<uintptr_t>(traj_dev) & 7))
        return fail(c, HADAMAG_ERR_INVALID_ARG, "misaligned trajectory buffer");
    if (N < 1 || N > 24) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, 24] (got %d)", N);
    if (L < 3 || L > 4096) return fail(c, HADAMAG_ERR_INVALID_ARG, "L must be in [3, 4096] (got %d)", L);
    if (n_s < 1 || burn_in < 0 || n_s > (int64_t(1) << 31) - 1 - burn_in)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "need n_s >= 1, burn_in >= 0, n_s + burn_in < 2^31");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(c, HADAMAG_ERR_INVALID_ARG, "eps must be finite and >= 0");
    if (sector != 0 && sector != 1) return fail(c, HADAMAG_ERR_INVALID_ARG, "sector must be 0 (all) or 1 (even)");
    if (sector == 1 && N < 2) return fail(c, HADAMAG_ERR_INVALID_ARG, "the even sector needs N >= 2");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    const float2* p;
    if ((s = as_c64(c, psi, int64_t(1) << N, dt, st, &p))) return s;
    const int B = ti_n_batches(n_s);
    if ((s = ensure_buf(c, c->ti_state, (size_t)(5 * L + 3 + (size_t)L * B) * 8))) return s;
    if ((s = ensure_buf(c, c->terms, (size_t)L * 3 * sizeof(double)))) return s;
    char* base = (char*)c->ti_state.ptr;
    TiChains ch{};
    ch.a = (int64_t*)base;
    ch.prop = (int64_t*)(base + (size_t)8 * L);
    ch.f = (double*)(base + (size_t)16 * L);
    ch.acc = (double*)(base + (size_t)24 * L);
    ch.out = (double*)(base + (size_t)32 * L);
    ch.bsum = (double*)(base + (size_t)8 * (5 * L + 3));
    ch.terms = (const double*)c->terms.ptr;
    ch.traj = traj_dev;
    ch.status = (int*)c->status.ptr;
    ch.seed = seed;
    ch.eps = eps;
    ch.T = burn_in + n_s;
    ch.burn_in = burn_in;
    ch.n_s = n_s;
    ch.L = L;
    ch.N = N;
    ch.even = sector;
    ch.B = B;
    ch.K = n_s / B;
    double* terms = (double*)c->terms.ptr;
    const unsigned grid = (unsigned)((L + 127) / 128);
    ti_start<<<grid, 128, 0, st>>>(ch);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ti_start");
    if ((s = run_sre(c, p, N, 2.0, L, ch.prop, 1, terms, st, nullptr))) return s;
    ti_init<<<grid, 128, 0, st>>>(ch);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ti_init");
    for (int64_t t = 0; t < ch.T; ++t) {
        if ((s = run_sre(c, p, N, 2.0, L, ch.prop, 1, terms, st, nullptr))) return s;
        ti_step<<<grid, 128, 0, st>>>(ch, t);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ti_step");
    }
    ti_finish<<<1, 32, 0, st>>>(ch);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ti_finish");
    std::vector<double> host((size_t)L + 3);
    if ((e = cudaMemcpyAsync(host.data(), ch.out, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(c, e, "copy chain means");
    if ((s = finish(c, nullptr, 0, st))) return s;
    if (means_out)
        for (int l = 0; l < L; ++l) means_out[l] = host[l];
    *M2_out = host[(size_t)L + 1];
    if (stderr_out) *stderr_out = host[(size_t)L + 2];
    if (!std::isfinite(*M2_out)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite estimate (I = %g)", host[L]);
    return HADAMAG_OK;
}
