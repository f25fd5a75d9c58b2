// grad.cu -- adjoint of M_2: dM_2/dpsi* (Wirtinger), recomputing c_a instead of storing 4^N values.
//
// Derivation (not in the paper; M_2 from Eq. sre, c_a = H^{(x)N} v_a from Algorithm 2):
//   dS_2/dpsi*_w = sum_a psi_{w^a} [G_a(w) + conj(G_a(w^a))],  G_a = H^{(x)N}(2 |c_a|^2 c_a).
// In the half-length form of common.cuh (W = R + iI = H^{(x)(N-1)} w, each W entry carrying the
// two Pauli strings c = 2R and c = 2iI), with Q = H^{(x)(N-1)}(R^3 + i I^3):
//   a != 0, pairs (z, z^a) with bit p = msb(a) of z clear, z' = z without bit p:
//       dS/dpsi*_z     += 32 psi_{z^a} Q(z'),      dS/dpsi*_{z^a} += 32 psi_z conj(Q(z')),
//   a == 0, pairs (2z', 2z'+1):
//       dS/dpsi*_{2z'} += 32 psi_{2z'} (Re Q + Im Q)(z'),  dS/dpsi*_{2z'+1} += 32 psi_{2z'+1} (Re Q - Im Q)(z').
// Then dM_2/dpsi* = -dS_2/dpsi* / (ln 2 S_2).
//
// Shapes: N <= 15: one group of threads per X-string (as sre_onepass), contributions summed into
// a per-group FP32 partial gradient.  N = 16..20: persistent three-pass kernel (pass 1 as the
// forward kernel; pass 2 finishes W, accumulates S_2, forms R^3 + iI^3 and transforms it back
// over the high bits in place; pass 3 transforms the low bits and scatters into a per-CTA FP32
// partial).  A pass-3 task covers one X-string, whose pairs touch each entry once, so CTAs
// update their own partial without atomics.  Partials are summed in a fixed order in FP64.
#include "common.cuh"
#include "grad.h"
#include "pairs.cuh"

namespace hm {

__device__ __forceinline__ float2 cube_parts(float2 w) {
    return make_float2(w.x * w.x * w.x, w.y * w.y * w.y);
}

// Adds the pair contributions of Q(j) for tile index z' = j to the partial gradient gp.
__device__ __forceinline__ void scatter_pair(float2* __restrict__ gp, const float2* __restrict__ psi, int64_t z,
                                             int64_t zb, float2 q) {
    // gp[z] += 32 psi[zb] Q,  gp[zb] += 32 psi[z] conj(Q)
    const float2 pz = ld_amp(psi, z), pb = ld_amp(psi, zb);
    float2 g0 = gp[z], g1 = gp[zb];
    g0.x += 32.f * (pb.x * q.x - pb.y * q.y);
    g0.y += 32.f * (pb.x * q.y + pb.y * q.x);
    g1.x += 32.f * (pz.x * q.x + pz.y * q.y);
    g1.y += 32.f * (pz.y * q.x - pz.x * q.y);
    gp[z] = g0;
    gp[zb] = g1;
}
__device__ __forceinline__ void scatter_zero(float2* __restrict__ gp, const float2* __restrict__ psi, int64_t z,
                                             float2 q) {
    const float2 p0 = ld_amp(psi, z), p1 = ld_amp(psi, z + 1);
    const float e = 32.f * (q.x + q.y), o = 32.f * (q.x - q.y);
    float2 g0 = gp[z], g1 = gp[z + 1];
    g0.x += e * p0.x; g0.y += e * p0.y;
    g1.x += o * p1.x; g1.y += o * p1.y;
    gp[z] = g0;
    gp[z + 1] = g1;
}

// ------------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(OnepassShape<L>::NT)
grad_onepass(const float2* __restrict__ psi, int N, double* __restrict__ sums, float2* __restrict__ gpart) {
    using Sh = OnepassShape<L>;
    constexpr int E = Sh::E, G = Sh::G, GPC = Sh::GPC;
    using S = TileSched<L, 0, E>;
    constexpr int SL = S::last_shift();
    extern __shared__ float2 smem[];
    __shared__ float red[16][2];
    const uint32_t tid = threadIdx.x, gi = tid / G, t = tid % G;
    float2* sm = smem + (size_t)gi * (L >= 5 ? tile_slots(L) : (1u << L));
    const int64_t ngroups = (int64_t)gridDim.x * GPC;
    const int64_t gg = (int64_t)blockIdx.x * GPC + gi;
    const int64_t dim = int64_t(1) << N;
    const int64_t iters = (dim + ngroups - 1) / ngroups;
    float2* gp = gpart + (size_t)gg * dim;
    double acc = 0.0, acc1 = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t a = gg + it * ngroups;
        const bool valid = a < dim;
        const int64_t av = valid ? a : 0;
        const int p = av ? msb64(av) : 0;
        float2 x[1 << E];
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) x[i] = pair_product(psi, deposit<E>(t, i, S::S0), av, p);
        reg_fwht<E, 0, E>(x);
        if constexpr (G <= 32) tile_rounds<L, 0, E, 1>(x, sm, t, SyncWarp());
        else tile_rounds<L, 0, E, 1>(x, sm, t, SyncCta());
        // S_2 and S_1 terms, then Y = R^3 + i I^3 back to the round-0 layout
        float q = 0.f, s1 = 0.f;
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) {
            const float2 sq = mul2(x[i], x[i]);
            s1 += sq.x + sq.y;
            q = fmaf(sq.x, sq.x, fmaf(sq.y, sq.y, q));
            x[i] = cube_parts(x[i]);
        }
        if constexpr (L >= 5) {
            if constexpr (G <= 32) __syncwarp(); else __syncthreads();
#pragma unroll
            for (int i = 0; i < (1 << E); ++i) sm[swz(deposit<E>(t, i, SL))] = x[i];
            if constexpr (G <= 32) __syncwarp(); else __syncthreads();
#pragma unroll
            for (int i = 0; i < (1 << E); ++i) x[i] = sm[swz(deposit<E>(t, i, S::S0))];
        }
        reg_fwht<E, 0, E>(x);
        if constexpr (G <= 32) tile_rounds<L, 0, E, 1>(x, sm, t, SyncWarp());
        else tile_rounds<L, 0, E, 1>(x, sm, t, SyncCta());
        if (valid) {
#pragma unroll
            for (int i = 0; i < (1 << E); ++i) {
                const int64_t zp = deposit<E>(t, i, SL);
                if (av != 0) {
                    const int64_t z = insert0(zp, p);
                    scatter_pair(gp, psi, z, z ^ av, x[i]);
                } else {
                    scatter_zero(gp, psi, zp << 1, x[i]);
                }
            }
        }
        // group sums of |c|^4 = 16 (R^4 + I^4) and |c|^2 = 4 (R^2 + I^2)
        if constexpr (G <= 32) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1)
                if (o < G) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
        } else {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
            if ((tid & 31) == 0) { red[tid >> 5][0] = q; red[tid >> 5][1] = s1; }
            __syncthreads();
            if (tid == 0) {
                float a0 = 0.f, a1 = 0.f;
                for (int w = 0; w < (G >> 5); ++w) { a0 += red[w][0]; a1 += red[w][1]; }
                q = a0; s1 = a1;
            }
            __syncthreads();
        }
        if (t == 0 && valid) { acc += 16.0 * (double)q; acc1 += 4.0 * (double)s1; }
    }
    if (t == 0) {
        sums[gg * 3 + 0] = acc;
        sums[gg * 3 + 1] = acc1;
        sums[gg * 3 + 2] = 0.0;
    }
}

// ------------------------------------------------------------------------------------------
// Three-pass persistent kernel (K1 = 10, M = N - 11), 256 threads, two CTAs per SM.
template <int M>
__global__ void __launch_bounds__(256, 2) grad_threepass(GradParams P) {
    using Sh = TwoPassShape<10, M>;
    constexpr int K1 = 10, L = Sh::L, LOGT = Sh::LOGT, T = Sh::T, TILES = Sh::TILES;
    using S2 = TileSched<13, LOGT, 5>;
    constexpr int SL2 = S2::last_shift();
    extern __shared__ float2 smem[];
    __shared__ float red[8][2];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2* __restrict__ psi = P.psi;
    const int64_t dim = int64_t(1) << P.N;
    const int64_t per_stage = (int64_t)P.p1 + P.p2 + P.p3;
    const int64_t total = (P.n_batches + 2) * per_stage;
    float2* gp = P.gpart + (size_t)blockIdx.x * dim;
    double acc = 0.0, acc1 = 0.0;

    for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
        // stage s: pass 1 of batch s, pass 2 of batch s-1, pass 3 of batch s-2
        const int64_t s = task / per_stage;
        int r = (int)(task % per_stage);
        int kind;
        int64_t g;
        if (r < P.p1) { kind = 1; g = s; }
        else if (r < P.p1 + P.p2) { kind = 2; g = s - 1; r -= P.p1; }
        else { kind = 3; g = s - 2; r -= P.p1 + P.p2; }
        if (g < 0 || g >= P.n_batches) continue;  // CTA-uniform
        const int slot = (int)(g % P.R);
        float2* sbase = P.scratch + (size_t)slot * P.A * ((size_t)1 << L);

        if (kind == 1) {
            if (g >= P.R && !cta_wait_geq(P.done3 + slot, (unsigned)((g / P.R) * P.p3) + P.wait_bias, P.status, P.spin_limit))
                return;
            const int a_idx = warp % P.A;
            const int64_t unit = ((int64_t)r * P.U + warp / P.A) * 2;
            const int64_t a = g * P.A + a_idx;
            if (a < dim) {
                float2* sm = smem + warp * tile_slots(10);
                float2 x[32];
                for (int uu = 0; uu < 2; ++uu) {
                    const PairRows<K1, M> pr(a, unit + uu);
                    float2* dst = sbase + (size_t)a_idx * ((size_t)1 << L) + ((size_t)(unit + uu) << K1);
#pragma unroll
                    for (int k = 0; k < 32; ++k) x[k] = pr.value(psi, a, lane | (k << 5));
                    reg_fwht<5, 0, 5>(x);
                    tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
#pragma unroll
                    for (int k = 0; k < 32; ++k) __stcg(dst + lane + (k << 5), x[k]);
                }
            }
            __syncthreads();
            if (tid == 0) { __threadfence(); red_release_add(P.done1 + slot, 1u); }
        } else if (kind == 2) {
            if (!cta_wait_geq(P.done1 + slot, (unsigned)((g / P.R + 1) * P.p1) + P.wait_bias, P.status, P.spin_limit))
                return;
            const int a_idx = r / TILES, tile = r % TILES;
            const int64_t a = g * P.A + a_idx;
            if (a < dim) {
                float2* src = sbase + (size_t)a_idx * ((size_t)1 << L) + (size_t)tile * T;
                float2 x[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, 8);
                    x[k] = __ldcg(src + ((size_t)(j >> LOGT) << K1) + (j & (T - 1)));
                }
                reg_fwht<5, 0, 5>(x);
                tile_rounds<13, LOGT, 5, 1>(x, smem, tid, SyncCta());
                float q = 0.f, s1 = 0.f;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const float2 sq = mul2(x[k], x[k]);
                    s1 += sq.x + sq.y;
                    q = fmaf(sq.x, sq.x, fmaf(sq.y, sq.y, q));
                    x[k] = cube_parts(x[k]);
                }
                // back to the round-0 layout, transform the high bits again, store in place
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 32; ++k) smem[swz(deposit<5>(tid, k, SL2))] = x[k];
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 32; ++k) x[k] = smem[swz(deposit<5>(tid, k, 8))];
                reg_fwht<5, 0, 5>(x);
                tile_rounds<13, LOGT, 5, 1>(x, smem, tid, SyncCta());
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, SL2);
                    __stcg(src + ((size_t)(j >> LOGT) << K1) + (j & (T - 1)), x[k]);
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
                if (lane == 0) { red[warp][0] = q; red[warp][1] = s1; }
                __syncthreads();
                if (tid == 0)
                    for (int w = 0; w < 8; ++w) { acc += 16.0 * (double)red[w][0]; acc1 += 4.0 * (double)red[w][1]; }
            }
            __syncthreads();
            if (tid == 0) { __threadfence(); red_release_add(P.done2 + slot, 1u); }
        } else {
            if (!cta_wait_geq(P.done2 + slot, (unsigned)((g / P.R + 1) * P.p2) + P.wait_bias, P.status, P.spin_limit))
                return;
            // one X-string, 16 units (two per warp): its pairs touch every entry at most once
            const int per_a = (1 << M) / 16;
            const int a_idx = r / per_a;
            const int64_t unit0 = (int64_t)(r % per_a) * 16 + warp * 2;
            const int64_t a = g * P.A + a_idx;
            if (a < dim) {
                float2* sm = smem + warp * tile_slots(10);
                float2 x[32];
                for (int uu = 0; uu < 2; ++uu) {
                    const int64_t unit = unit0 + uu;
                    const float2* src = sbase + (size_t)a_idx * ((size_t)1 << L) + ((size_t)unit << K1);
                    // column (k<<5)|lane holds tile index j = k | (lane<<5); with j' = swap of the
                    // two 5-bit halves this is the round-0 layout of the 10-bit schedule
#pragma unroll
                    for (int k = 0; k < 32; ++k) x[k] = __ldcg(src + lane + (k << 5));
                    reg_fwht<5, 0, 5>(x);
                    tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
                    // now register k holds Q at j = lane | (k << 5) (the pair-product layout)
                    const PairRows<K1, M> pr(a, unit);
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const uint32_t j = lane | (k << 5);
                        if (a >> K1) {
                            scatter_pair(gp, psi, pr.rowA + j, pr.rowB + (int64_t)(j ^ (uint32_t)pr.al), x[k]);
                        } else {
                            const int64_t row = (j >> (K1 - 1)) ? pr.rowB : pr.rowA;
                            const int64_t lp = j & ((1u << (K1 - 1)) - 1u);
                            if (a != 0) {
                                const int64_t z = row + insert0(lp, pr.p);
                                scatter_pair(gp, psi, z, z ^ a, x[k]);
                            } else {
                                scatter_zero(gp, psi, row + (lp << 1), x[k]);
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0) red_release_add(P.done3 + slot, 1u);
        }
    }
    if (tid == 0) {
        P.sums[blockIdx.x * 3 + 0] = acc;
        P.sums[blockIdx.x * 3 + 1] = acc1;
        P.sums[blockIdx.x * 3 + 2] = 0.0;
    }
}

// ------------------------------------------------------------------------------------------
// grad[z] = -(sum over partials of dS/dpsi*_z) / (ln 2 * S_2), partials summed in FP64 in order.
template <class TOut>
__global__ void grad_finalize(const float2* __restrict__ gpart, int64_t nparts, int64_t dim,
                              const double* __restrict__ s2, TOut* __restrict__ out) {
    const double scale = -1.0 / (0.69314718055994530942 * s2[0]);
    for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim; z += (int64_t)gridDim.x * blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int64_t k = 0; k < nparts; ++k) {
            const float2 v = gpart[(size_t)k * dim + z];
            gx += v.x;
            gy += v.y;
        }
        if constexpr (sizeof(TOut) == 8) out[z] = make_float2((float)(gx * scale), (float)(gy * scale));
        else out[z] = make_double2(gx * scale, gy * scale);
    }
}

// ------------------------------------------------------------------------------------------
template <int L>
static cudaError_t launch_grad_onepass_t(const float2* psi, int N, double* sums, float2* gpart, int groups_max,
                                         int* ngroups, cudaStream_t st) {
    using Sh = OnepassShape<L>;
    size_t smem = (size_t)Sh::GPC * (L >= 5 ? tile_slots(L) : (1u << L)) * sizeof(float2);
    auto k = grad_onepass<L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = groups_max / Sh::GPC;
    const int64_t need = ((int64_t(1) << (L + 1)) + Sh::GPC - 1) / Sh::GPC;
    if (grid > need) grid = (int)need;
    if (grid < 1) grid = 1;
    *ngroups = grid * Sh::GPC;
    k<<<grid, Sh::NT, smem, st>>>(psi, N, sums, gpart);
    return cudaGetLastError();
}

int grad_onepass_gpc(int N) {
    switch (N - 1) {
#define HM_CASE(LL) case LL: return OnepassShape<LL>::GPC;
        HM_CASE(0) HM_CASE(1) HM_CASE(2) HM_CASE(3) HM_CASE(4) HM_CASE(5) HM_CASE(6) HM_CASE(7)
        HM_CASE(8) HM_CASE(9) HM_CASE(10) HM_CASE(11) HM_CASE(12) HM_CASE(13) HM_CASE(14)
#undef HM_CASE
        default: return 1;
    }
}

cudaError_t launch_grad_onepass(const float2* psi, int N, double* sums, float2* gpart, int groups_max,
                                int* ngroups, cudaStream_t st) {
    switch (N - 1) {
#define HM_CASE(LL) case LL: return launch_grad_onepass_t<LL>(psi, N, sums, gpart, groups_max, ngroups, st);
        HM_CASE(0) HM_CASE(1) HM_CASE(2) HM_CASE(3) HM_CASE(4) HM_CASE(5) HM_CASE(6) HM_CASE(7)
        HM_CASE(8) HM_CASE(9) HM_CASE(10) HM_CASE(11) HM_CASE(12) HM_CASE(13) HM_CASE(14)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

static constexpr size_t kGradSmem = tile_slots(13) * sizeof(float2);

template <int M>
static cudaError_t grad3_prep(int* occ) {
    auto k = grad_threepass<M>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, 256, kGradSmem);
}

cudaError_t grad_threepass_grid(int N, int sm_count, int* grid) {
    int occ = 0;
    cudaError_t e;
    switch (N) {
        case 16: e = grad3_prep<5>(&occ); break;
        case 17: e = grad3_prep<6>(&occ); break;
        case 18: e = grad3_prep<7>(&occ); break;
        case 19: e = grad3_prep<8>(&occ); break;
        case 20: e = grad3_prep<9>(&occ); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_grad_threepass(const GradParams& P, int grid, cudaStream_t st) {
    switch (P.N) {
#define HM_CASE(NN)                                                                 \
    case NN:                                                                        \
        grad_threepass<NN - 11><<<grid, 256, kGradSmem, st>>>(P);                   \
        return cudaGetLastError();
        HM_CASE(16) HM_CASE(17) HM_CASE(18) HM_CASE(19) HM_CASE(20)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad_finalize(const float2* gpart, int64_t nparts, int64_t dim, const double* s2, void* out,
                                 bool c128, cudaStream_t st) {
    int64_t blocks = (dim + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (c128) grad_finalize<double2><<<(unsigned)blocks, 256, 0, st>>>(gpart, nparts, dim, s2, (double2*)out);
    else grad_finalize<float2><<<(unsigned)blocks, 256, 0, st>>>(gpart, nparts, dim, s2, (float2*)out);
    return cudaGetLastError();
}

}  // namespace hm
