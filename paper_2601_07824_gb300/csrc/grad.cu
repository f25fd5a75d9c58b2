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
#include "grad_phases.cuh"

namespace hm {

// ------------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(OnepassShape<L>::NT)
grad_onepass(const float2* __restrict__ psi, int N, double* __restrict__ sums, float2* __restrict__ gpart,
             int64_t a_base, int64_t count) {
    using Sh = OnepassShape<L>;
    constexpr int G = Sh::G, GPC = Sh::GPC;
    extern __shared__ float2 smem[];
    const uint32_t tid = threadIdx.x, gi = tid / G, t = tid % G;
    float2* sm = smem + (size_t)gi * (L >= 5 ? tile_slots(L) : (1u << L));
    const int64_t ngroups = (int64_t)gridDim.x * GPC;
    const int64_t gg = (int64_t)blockIdx.x * GPC + gi;
    const int64_t dim = int64_t(1) << N;
    double acc = 0.0, acc1 = 0.0;
    grad_onepass_group<L>(psi, N, gpart + (size_t)gg * dim, gg, ngroups, sm, acc, acc1, a_base, count);
    if (t == 0) {
        sums[gg * 3 + 0] = acc;
        sums[gg * 3 + 1] = acc1;
        sums[gg * 3 + 2] = 0.0;
    }
}

// ------------------------------------------------------------------------------------------
// Three-pass persistent kernel (K1 = 10, M = N - 11), 256 threads, two CTAs per SM; tasks in
// the stage order of g3_decode, CTA b taking tasks b, b + grid, ...
template <int M>
__global__ void __launch_bounds__(256, 2) grad_threepass(GradParams P) {
    extern __shared__ float2 smem[];
    const uint32_t tid = threadIdx.x;
    const G3State S{P.psi, P.N, P.scratch, P.R, P.A, P.U, P.n_batches, P.p1, P.p2, P.p3, P.done1, P.done2, P.done3,
                    P.a_base, P.UPW, P.TPT};
    const G3Ctl C{P.status, P.spin_limit, P.wait_bias};
    const int64_t dim = int64_t(1) << P.N;
    const int64_t per_stage = (int64_t)P.p1 + P.p2 + P.p3;
    const int64_t total = (P.n_batches + 2 * P.lag) * per_stage;
    float2* gp = P.gpart + (size_t)blockIdx.x * dim;
    double acc = 0.0, acc1 = 0.0;
    for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
        int kind, r;
        int64_t g;
        g3_decode(task, P.p1, P.p2, P.p3, P.lag, kind, g, r);
        if (g < 0 || g >= P.n_batches) continue;  // CTA-uniform
        bool ok;
        if (kind == 1) ok = g3_pass1<M>(S, C, g, r, smem);
        else if (kind == 2) ok = g3_pass2<M>(S, C, g, r, smem, acc, acc1);
        else ok = g3_pass3<M>(S, C, g, r, smem, gp);
        if (!ok) return;
    }
    // the 8 warps' sums (lane 0 of each), combined in a fixed order
    __shared__ double red[8][2];
    if ((tid & 31) == 0) { red[tid >> 5][0] = acc; red[tid >> 5][1] = acc1; }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < 8; ++w) { t0 += red[w][0]; t1 += red[w][1]; }
        P.sums[blockIdx.x * 3 + 0] = t0;
        P.sums[blockIdx.x * 3 + 1] = t1;
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

// dS[z] = sum over partials of dS/dpsi*_z (FP64, in partial order), unscaled: the part of
// the gradient contributed by one slice of X-strings.
__global__ void grad_sum_parts(const float2* __restrict__ gpart, int64_t nparts, int64_t dim,
                               double2* __restrict__ out) {
    for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim; z += (int64_t)gridDim.x * blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int64_t k = 0; k < nparts; ++k) {
            const float2 v = gpart[(size_t)k * dim + z];
            gx += v.x;
            gy += v.y;
        }
        out[z] = make_double2(gx, gy);
    }
}

// grad[z] = -dS[z] / (ln 2 * S_2) from the summed dS/dpsi* of every slice.
template <class TOut>
__global__ void grad_scale(const double2* __restrict__ dS, int64_t dim, double S2, TOut* __restrict__ out) {
    const double scale = -1.0 / (0.69314718055994530942 * S2);
    for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < dim; z += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = dS[z];
        if constexpr (sizeof(TOut) == 8) out[z] = make_float2((float)(v.x * scale), (float)(v.y * scale));
        else out[z] = make_double2(v.x * scale, v.y * scale);
    }
}

// ------------------------------------------------------------------------------------------
template <int L>
static cudaError_t launch_grad_onepass_t(const float2* psi, int N, double* sums, float2* gpart, int groups_max,
                                         int* ngroups, cudaStream_t st, int64_t a_base, int64_t count) {
    using Sh = OnepassShape<L>;
    size_t smem = (size_t)Sh::GPC * (L >= 5 ? tile_slots(L) : (1u << L)) * sizeof(float2);
    auto k = grad_onepass<L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = groups_max / Sh::GPC;
    const int64_t cnt = count < 0 ? (int64_t(1) << (L + 1)) : count;
    const int64_t need = (cnt + Sh::GPC - 1) / Sh::GPC;
    if (grid > need) grid = (int)need;
    if (grid < 1) grid = 1;
    *ngroups = grid * Sh::GPC;
    k<<<grid, Sh::NT, smem, st>>>(psi, N, sums, gpart, a_base, count);
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
                                int* ngroups, cudaStream_t st, int64_t a_base, int64_t count) {
    switch (N - 1) {
#define HM_CASE(LL) \
    case LL: return launch_grad_onepass_t<LL>(psi, N, sums, gpart, groups_max, ngroups, st, a_base, count);
        HM_CASE(0) HM_CASE(1) HM_CASE(2) HM_CASE(3) HM_CASE(4) HM_CASE(5) HM_CASE(6) HM_CASE(7)
        HM_CASE(8) HM_CASE(9) HM_CASE(10) HM_CASE(11) HM_CASE(12) HM_CASE(13) HM_CASE(14)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

// pass-2/3 exchange (one 2^13 tile; pass 1: 8 warps x 2^10) plus the pass-1 row staging
static constexpr size_t kGradSmem = (tile_slots(13) + kStageSlots) * sizeof(float2);

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

cudaError_t launch_grad_sum_parts(const float2* gpart, int64_t nparts, int64_t dim, double2* out, cudaStream_t st) {
    int64_t blocks = (dim + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    grad_sum_parts<<<(unsigned)blocks, 256, 0, st>>>(gpart, nparts, dim, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_scale(const double2* dS, int64_t dim, double S2, void* out, bool c128, cudaStream_t st) {
    int64_t blocks = (dim + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (c128) grad_scale<double2><<<(unsigned)blocks, 256, 0, st>>>(dS, dim, S2, (double2*)out);
    else grad_scale<float2><<<(unsigned)blocks, 256, 0, st>>>(dS, dim, S2, (float2*)out);
    return cudaGetLastError();
}

}  // namespace hm
