// sre_fwd_kernels.cuh -- exact SRE forward kernels (paper Sec. 3.1.2, Algorithm 2; Eq. sre),
// as templates with their per-mode host launchers.  Each sre_fwd_n*.cu instantiates one
// accumulation mode (n = 1, 2, 3 and other n) so that the modes compile in parallel;
// sre_fwd.cu dispatches on the mode.
//
// For every X-string a the kernels form the half-length pair product w_a (see common.cuh),
// apply the unnormalised Walsh-Hadamard transform over its N-1 index bits and reduce
// sum_b |c_a(b)|^{2n}, sum_b |c_a(b)|^2 (lost_norm, Sec. 4.1) and, for n = 1,
// sum_b |c|^2 log2 |c|^2.  Two shapes:
//
//   * sre_onepass<L>   (N <= 15, L = N-1 <= 14): a group of 2^(L-5) threads owns one X-string,
//     32 complex values per thread, shared-memory exchanges between 5-bit register rounds.
//   * sre_twopass<M>   (N = 16..24, L = 10 + M): a persistent kernel over a static task list.
//     Pass 1 (one warp per (a, unit)): pair product + transform over the 10 low bits of z',
//     written to a scratch slot in L2.  Pass 2 (one CTA per (a, column tile)): transform over
//     the M high bits + reduction.  Pass-2 tasks of a batch wait (bounded) on a counter of
//     finished pass-1 tasks; pass-1 tasks reusing a slot wait for that slot's pass-2 tasks.
//     Tasks are taken round-robin in a fixed global order in which every task only waits on
//     earlier tasks, so a co-resident grid cannot deadlock, and the FP64 sums are deterministic.
//     When the 8 warps of a pass-1 task work on the same two units for 8 X-strings that share
//     their state rows (8 consecutive X-strings of an aligned batch always do), the 4 rows are
//     copied once into shared memory (cp.async) and every warp forms its pair products there
//     instead of issuing its own loads of the same rows.  Pass-2 reductions are per warp (FP32
//     over the warp's values, FP64 across its tiles), with no CTA barrier per tile.
#pragma once
#include "common.cuh"
#include "pairs.cuh"
#include "schedule.h"
#include "sre_fwd.h"

namespace hm {

// ------------------------------------------------------------------------------------------
// One-pass kernel.
template <int L, int MODE>
__global__ void __launch_bounds__(OnepassShape<L>::NT)
sre_onepass(const float2* __restrict__ psi, int N, double nq, int64_t count,
            const int64_t* __restrict__ a_list, int64_t a_base, double* __restrict__ out, int per_a, int* status) {
    using Sh = OnepassShape<L>;
    constexpr int E = Sh::E, G = Sh::G, GPC = Sh::GPC;
    using S = TileSched<L, 0, E>;
    extern __shared__ float2 smem[];
    __shared__ float red[16][4];
    __shared__ double redd[16];
    const uint32_t tid = threadIdx.x, gi = tid / G, t = tid % G;
    float2* sm = smem + (size_t)gi * (L >= 5 ? tile_slots(L) : (1u << L));
    const int64_t ngroups = (int64_t)gridDim.x * GPC;
    const int64_t gg = (int64_t)blockIdx.x * GPC + gi;
    const int64_t iters = (count + ngroups - 1) / ngroups;
    const int64_t dim = int64_t(1) << N;
    double acc[3] = {0.0, 0.0, 0.0};

    for (int64_t it = 0; it < iters; ++it) {
        const int64_t idx = gg + it * ngroups;
        bool valid = idx < count;
        int64_t a = valid ? (a_list ? a_list[idx] : a_base + idx) : 0;
        if (a < 0 || a >= dim) {
            if (valid) atomicOr(status, ST_BADARG);
            valid = false;
            a = 0;
        }
        const int p = a ? msb64(a) : 0;
        float2 x[1 << E];
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) x[i] = pair_product(psi, deposit<E>(t, i, S::S0), a, p);
        reg_fwht<E, 0, E>(x);
        if constexpr (G <= 32) tile_rounds<L, 0, E, 1>(x, sm, t, SyncWarp());
        else tile_rounds<L, 0, E, 1>(x, sm, t, SyncCta());

        Acc<MODE> ac;
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) ac.add(x[i], nq);
        ac.fold();
        float q = ac.q, s1 = ac.s1, u = ac.u;
        double qd = ac.qd;
        double v[3];
        if constexpr (G <= 32) {
            warp_sum3<MODE>(q, s1, u, qd, G);
        } else {
            warp_sum3<MODE>(q, s1, u, qd, 32);
            if ((tid & 31) == 0) {
                red[tid >> 5][0] = q; red[tid >> 5][1] = s1; red[tid >> 5][2] = u;
                redd[tid >> 5] = qd;
            }
            __syncthreads();
            if (tid == 0) {
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                double ad = 0.0;
                for (int w = 0; w < (G >> 5); ++w) { a0 += red[w][0]; a1 += red[w][1]; a2 += red[w][2]; ad += redd[w]; }
                q = a0; s1 = a1; u = a2; qd = ad;
            }
            __syncthreads();
        }
        if (t == 0 && valid) {
            finish3<MODE>(q, s1, u, qd, nq, v);
            if (per_a) {
                out[idx * 3 + 0] = v[0]; out[idx * 3 + 1] = v[1]; out[idx * 3 + 2] = v[2];
            } else {
                acc[0] += v[0]; acc[1] += v[1]; acc[2] += v[2];
            }
        }
    }
    if (!per_a) {
        // fixed-order combination of the group leaders' FP64 sums
        __syncthreads();
        double* dd = reinterpret_cast<double*>(smem);
        if (t == 0) { dd[gi * 3 + 0] = acc[0]; dd[gi * 3 + 1] = acc[1]; dd[gi * 3 + 2] = acc[2]; }
        __syncthreads();
        if (tid == 0) {
            double s0 = 0.0, s1d = 0.0, s2 = 0.0;
            for (int g = 0; g < GPC; ++g) { s0 += dd[g * 3]; s1d += dd[g * 3 + 1]; s2 += dd[g * 3 + 2]; }
            out[blockIdx.x * 3 + 0] = s0; out[blockIdx.x * 3 + 1] = s1d; out[blockIdx.x * 3 + 2] = s2;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Persistent two-pass kernel, 256 threads per CTA (two CTAs per SM).
//   K1 = 10: pass 1 is warp-level (each warp one (X-string, unit) of 2^10 values);
//   K1 = 13: pass 1 is CTA-level (the CTA does one (X-string, unit) of 2^13 values).
//   The scratch of one X-string is [2^M units][2^K1 columns]; a pass-2 tile is all 2^M units
//   x 2^(13-M) consecutive columns (2^13 values).  Per-X-string output (per_a): one triple per
//   (tile, warp), [count][TILES][8][3].

template <int K1, int M, int MODE>
__global__ void __launch_bounds__(256, 2) sre_twopass(TwoPassParams P) {
    using Sh = TwoPassShape<K1, M>;
    constexpr int L = Sh::L, LOGT = Sh::LOGT, T = Sh::T, TILES = Sh::TILES;
    extern __shared__ float2 smem[];
    __shared__ double red64[8][3];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2* __restrict__ psi = P.psi;
    const int64_t dim = int64_t(1) << P.N;
    const int64_t per_stage = (int64_t)P.p1 + P.p2;
    const int64_t total = P.n_batches * per_stage;
    double accw[3] = {0.0, 0.0, 0.0};  // lane 0 of each warp: FP64 sums of the warp's tiles

    // task order and waits: schedule.h (twopass_decode, twopass_dependency)
    auto decode = [&](int64_t task, int64_t& g, int& kind, int& r) {
        twopass_decode(task, P.p1, P.p2, P.n_batches, P.lag, g, kind, r);
    };
    // counter and target a task waits on (none for pass 1 of the first R batches)
    auto dependency = [&](int64_t g, int kind, const unsigned*& ctr, unsigned& need) {
        int slot;
        const int which = twopass_dependency(g, kind, P.R, P.p1, P.p2, slot, need);
        ctr = which == 0 ? nullptr : (which == 1 ? P.done1 : P.done2) + slot;
        need += P.wait_bias;
    };

    unsigned seen = 0;  // thread 0: relaxed read of the next task's counter, one task ahead
    {
        int64_t g; int kind, r;
        const unsigned* c; unsigned need;
        if (tid == 0 && (int64_t)blockIdx.x < total) {
            decode(blockIdx.x, g, kind, r);
            dependency(g, kind, c, need);
            if (c) seen = ld_relaxed(c);
        }
    }

    for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
        int64_t g;
        int kind, r;
        decode(task, g, kind, r);
        const int slot = (int)(g % P.R);
        float2* sbase = P.scratch + (size_t)slot * P.A * ((size_t)1 << L);
        {
            const unsigned* c;
            unsigned need;
            dependency(g, kind, c, need);
            if (c && !cta_wait_geq(c, need, P.status, P.spin_limit, seen)) return;
        }
        if (tid == 0 && task + gridDim.x < total) {  // prefetch the next task's counter
            int64_t g2; int k2, r2;
            const unsigned* c2; unsigned n2;
            decode(task + gridDim.x, g2, k2, r2);
            dependency(g2, k2, c2, n2);
            seen = c2 ? ld_relaxed(c2) : 0u;
        }

        if (kind == 1) {
            // ---- pass 1: pair product + transform over the K1 low bits of z' ----------------
            int a_idx, sub;
            int64_t unit;
            if constexpr (K1 == 10) { a_idx = warp % P.A; unit = ((int64_t)r * P.U + warp / P.A) * P.UPW; sub = warp; }
            else { a_idx = 0; unit = r; sub = 0; }
            const int64_t i = g * P.A + a_idx;
            bool valid = i < P.count;
            int64_t a = valid ? (P.a_list ? P.a_list[i] : P.a_base + i) : 0;
            if (a < 0 || a >= dim) {
                if (valid && (tid & (K1 == 10 ? 31 : 255)) == 0) atomicOr(P.status, ST_BADARG);
                valid = false;
            }
            if constexpr (K1 == 10) {
                bool stage = false;  // CTA-uniform
                int64_t a0 = 0;
                if (P.U == 1) {
                    // every warp on the same units: rows shared when all X-strings of the batch
                    // agree in their bits above 5 (always so without a list: 8 consecutive,
                    // aligned X-strings)
                    const int64_t i0 = g * P.A;  // < count for every batch
                    a0 = P.a_list ? P.a_list[i0] : P.a_base + i0;
                    stage = a0 >= 0 && a0 < dim;
                    if (P.a_list) stage = __syncthreads_and(stage && (!valid || (a >> 5) == (a0 >> 5))) != 0;
                }
                // far batch (a >= 2^K1): row B staged block-permuted by the batch's bits 5..9 of a,
                // so both pair-product loads are a per-thread base plus a compile-time offset
                const bool far = stage && (a0 >> K1) != 0;
                const uint32_t perm = far ? (uint32_t)((a0 >> 5) & 31) : 0u;
                float2* sm = smem + sub * tile_slots(10);
                float2* rows = smem + 8 * tile_slots(10);
                for (int up = 0; up < P.UPW; up += 2) {  // UPW consecutive units per warp, two at a time
                    if (stage) {
                        if (up > 0) __syncthreads();  // every warp is done with the previous rows
                        stage_rows<M>(rows, psi, a0, unit + up, perm);
                    }
                    if (!valid) continue;
                    float2 x[32];
                    for (int uu = 0; uu < 2; ++uu) {
                        const int64_t un = unit + up + uu;
                        const PairRows<K1, M> pr(a, un);
                        float2* dst = sbase + (size_t)a_idx * ((size_t)1 << L) + ((size_t)un << K1);
                        if (far) {
                            const float2* own = rows + uu * 2048 + lane;
                            const float2* par = rows + uu * 2048 + 1024 + (lane ^ ((uint32_t)a & 31u));
#pragma unroll
                            for (int k = 0; k < 32; ++k) x[k] = conj_mul(par[k << 5], own[k << 5]);
                        } else if (stage) {
                            const float2* rw = rows + uu * 2048;
#pragma unroll
                            for (int k = 0; k < 32; ++k) x[k] = pr.value_rows(rw, rw + 1024, a, lane | (k << 5));
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k) x[k] = pr.value(psi, a, lane | (k << 5));
                        }
                        reg_fwht<5, 0, 5>(x);
                        tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
                        // registers hold j bits [0,5), lanes bits [5,10): store column (k<<5)|lane
#pragma unroll
                        for (int k = 0; k < 32; ++k) __stcg(dst + lane + (k << 5), x[k]);
                    }
                }
            } else if (valid) {
                float2 x[32];
                {
                    const PairRows<K1, M> pr(a, unit);
                    float2* dst = sbase + (size_t)a_idx * ((size_t)1 << L) + ((size_t)unit << K1);
#pragma unroll
                    for (int k = 0; k < 32; ++k) x[k] = pr.value(psi, a, deposit<5>(tid, k, 8));
                    reg_fwht<5, 0, 5>(x);
                    tile_rounds<13, 0, 5, 1>(x, smem, tid, SyncCta());
                    constexpr int SL = TileSched<13, 0, 5>::last_shift();
#pragma unroll
                    for (int k = 0; k < 32; ++k) __stcg(dst + deposit<5>(tid, k, SL), x[k]);
                }
            }
            __syncthreads();
            // the release orders the whole CTA's writes (after the barrier); a thread of the last
            // warp issues it, so thread 0 can poll the next task's counter without waiting behind
            // the release's ordering
            if (tid == 224) red_release_add(P.done1 + slot, 1u);
        } else {
            // ---- pass 2: transform over the M high bits of z' + reduction ------------------
            const int a_idx = r / (TILES / P.TPT);
            const int64_t i = g * P.A + a_idx;
            if (i < P.count) for (int tile = (r % (TILES / P.TPT)) * P.TPT, te = tile + P.TPT; tile < te; ++tile) {
                const float2* src = sbase + (size_t)a_idx * ((size_t)1 << L) + (size_t)tile * T;
                float2 x[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, 8);  // tile index (row << LOGT) | col
                    x[k] = __ldcg(src + ((size_t)(j >> LOGT) << K1) + (j & (T - 1)));
                }
                // register bits are tile bits [8, 13); those below LOGT are column bits (N = 15)
                constexpr int B0 = LOGT > 8 ? LOGT - 8 : 0;
                reg_fwht<5, B0, 5>(x);
                tile_rounds<13, LOGT, 5, 1>(x, smem, tid, SyncCta());
                if constexpr (Sh::DISCARD) {
                    // every value of the tile is in registers: drop its lines from L2 unwritten
                    if constexpr (TileSched<13, LOGT, 5>::NR == 1) __syncthreads();
                    constexpr int LPR = (T * 8) / 128;  // 128-byte lines per tile row
#pragma unroll
                    for (int q = tid; q < (1 << M) * LPR; q += 256)
                        discard_l2_line(src + ((size_t)(q / LPR) << K1) + (q % LPR) * 16);
                }
                Acc<MODE> ac;
#pragma unroll
                for (int k = 0; k < 32; ++k) ac.add(x[k], P.nq);
                ac.fold();
                float q = ac.q, s1 = ac.s1, u = ac.u;
                double qd = ac.qd;
                warp_sum3<MODE>(q, s1, u, qd, 32);
                if (lane == 0) {
                    double v[3];
                    finish3<MODE>(q, s1, u, qd, P.nq, v);
                    if (P.per_a) {
                        double* o = P.out + (((size_t)i * TILES + tile) * 8 + warp) * 3;
                        o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
                    } else {
                        accw[0] += v[0]; accw[1] += v[1]; accw[2] += v[2];
                    }
                }
            }
            __syncthreads();
            if (tid == 224) red_release_add(P.done2 + slot, 1u);
        }
    }
    if (!P.per_a) {
        // fixed-order combination of the 8 warps' FP64 sums
        if (lane == 0) { red64[warp][0] = accw[0]; red64[warp][1] = accw[1]; red64[warp][2] = accw[2]; }
        __syncthreads();
        if (tid == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < 8; ++w) { s0 += red64[w][0]; s1 += red64[w][1]; s2 += red64[w][2]; }
            P.out[blockIdx.x * 3 + 0] = s0;
            P.out[blockIdx.x * 3 + 1] = s1;
            P.out[blockIdx.x * 3 + 2] = s2;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Host launchers (templates; instantiated per mode by HM_SRE_FWD_MODE).

template <int L, int MODE>
static cudaError_t launch_onepass_t(OnepassArgs& A, int sm_count, cudaStream_t st) {
    using Sh = OnepassShape<L>;
    size_t smem = (size_t)Sh::GPC * (L >= 5 ? tile_slots(L) : (1u << L)) * sizeof(float2);
    const size_t comb = (size_t)Sh::GPC * 3 * sizeof(double);
    if (smem < comb) smem = comb;
    auto k = sre_onepass<L, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, Sh::NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t need = (A.count + Sh::GPC - 1) / Sh::GPC;
    int64_t cap = (int64_t)occ * sm_count;
    if (A.grid > 0 && A.grid < cap) cap = A.grid;
    A.grid = (int)(need < cap ? need : cap);
    if (A.grid < 1) A.grid = 1;
    k<<<A.grid, Sh::NT, smem, st>>>(A.psi, A.N, A.nq, A.count, A.a_list, A.a_base, A.out, A.per_a, A.status);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_onepass_m(OnepassArgs& A, int sm_count, cudaStream_t st) {
    switch (A.N - 1) {
#define HM_CASE(LL) case LL: return launch_onepass_t<LL, MODE>(A, sm_count, st);
        HM_CASE(0) HM_CASE(1) HM_CASE(2) HM_CASE(3) HM_CASE(4) HM_CASE(5) HM_CASE(6) HM_CASE(7)
        HM_CASE(8) HM_CASE(9) HM_CASE(10) HM_CASE(11) HM_CASE(12) HM_CASE(13) HM_CASE(14)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

// exchange buffers (pass 1: 8 warps x 2^10 values; pass 2: one 2^13 tile), plus the pass-1
// row staging for K1 = 10
template <int K1, int M>
static constexpr size_t twopass_smem() {
    return ((K1 == 10 ? 8 * tile_slots(10) : tile_slots(13)) > tile_slots(13) ? 8 * tile_slots(10) : tile_slots(13)) *
               sizeof(float2) +
           (K1 == 10 ? kStageSlots * sizeof(float2) : 0);
}

template <int K1, int M, int MODE>
static cudaError_t twopass_prepare(int* occ) {
    auto k = sre_twopass<K1, M, MODE>;
    constexpr size_t smem = twopass_smem<K1, M>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, 256, smem);
}

// The caller has run twopass_max_grid for (N, mode) on this device, which raised the
// kernel's shared-memory limit (a function attribute that persists on the device).
template <int K1, int M, int MODE>
static cudaError_t launch_twopass_t(const TwoPassParams& P, int grid, cudaStream_t st) {
    sre_twopass<K1, M, MODE><<<grid, 256, twopass_smem<K1, M>(), st>>>(P);
    return cudaGetLastError();
}

// N -> (K1, M): N = 15..20 -> (10, N-11); N = 21..24 -> (13, N-14).  (N = 15 runs two passes
// only when the autotuner picks them over the one-pass kernel.)
#define HM_TWOPASS_SWITCH(N_, EXPR)                                              \
    switch (N_) {                                                                \
        case 15: { constexpr int KK = 10, MM = 4; EXPR; }                        \
        case 16: { constexpr int KK = 10, MM = 5; EXPR; }                        \
        case 17: { constexpr int KK = 10, MM = 6; EXPR; }                        \
        case 18: { constexpr int KK = 10, MM = 7; EXPR; }                        \
        case 19: { constexpr int KK = 10, MM = 8; EXPR; }                        \
        case 20: { constexpr int KK = 10, MM = 9; EXPR; }                        \
        case 21: { constexpr int KK = 13, MM = 7; EXPR; }                        \
        case 22: { constexpr int KK = 13, MM = 8; EXPR; }                        \
        case 23: { constexpr int KK = 13, MM = 9; EXPR; }                        \
        case 24: { constexpr int KK = 13, MM = 10; EXPR; }                       \
        default: return cudaErrorInvalidValue;                                   \
    }

template <int MODE>
static cudaError_t launch_twopass_m(const TwoPassParams& P, int grid, cudaStream_t st) {
    HM_TWOPASS_SWITCH(P.N, return (launch_twopass_t<KK, MM, MODE>(P, grid, st)))
}

template <int MODE>
static cudaError_t twopass_occ_m(int N, int* occ) {
    HM_TWOPASS_SWITCH(N, return (twopass_prepare<KK, MM, MODE>(occ)))
}

// Per-mode entry points (MODE 0: any n with FP64 powers, 1: n = 1, 2: n = 2, 3: n = 3, 4: any n
// with FP32 powers), one translation unit each.
cudaError_t sre_fwd_onepass_n0(OnepassArgs& A, int sm_count, cudaStream_t st);
cudaError_t sre_fwd_onepass_n1(OnepassArgs& A, int sm_count, cudaStream_t st);
cudaError_t sre_fwd_onepass_n2(OnepassArgs& A, int sm_count, cudaStream_t st);
cudaError_t sre_fwd_onepass_n3(OnepassArgs& A, int sm_count, cudaStream_t st);
cudaError_t sre_fwd_onepass_n4(OnepassArgs& A, int sm_count, cudaStream_t st);
cudaError_t sre_fwd_twopass_n0(const TwoPassParams& P, int grid, cudaStream_t st);
cudaError_t sre_fwd_twopass_n1(const TwoPassParams& P, int grid, cudaStream_t st);
cudaError_t sre_fwd_twopass_n2(const TwoPassParams& P, int grid, cudaStream_t st);
cudaError_t sre_fwd_twopass_n3(const TwoPassParams& P, int grid, cudaStream_t st);
cudaError_t sre_fwd_twopass_n4(const TwoPassParams& P, int grid, cudaStream_t st);
cudaError_t sre_fwd_twopass_occ_n0(int N, int* occ);
cudaError_t sre_fwd_twopass_occ_n1(int N, int* occ);
cudaError_t sre_fwd_twopass_occ_n2(int N, int* occ);
cudaError_t sre_fwd_twopass_occ_n3(int N, int* occ);
cudaError_t sre_fwd_twopass_occ_n4(int N, int* occ);

#define HM_SRE_FWD_MODE(M_)                                                                      \
    cudaError_t sre_fwd_onepass_n##M_(OnepassArgs& A, int sm_count, cudaStream_t st) {          \
        return launch_onepass_m<M_>(A, sm_count, st);                                            \
    }                                                                                            \
    cudaError_t sre_fwd_twopass_n##M_(const TwoPassParams& P, int grid, cudaStream_t st) {      \
        return launch_twopass_m<M_>(P, grid, st);                                                \
    }                                                                                            \
    cudaError_t sre_fwd_twopass_occ_n##M_(int N, int* occ) { return twopass_occ_m<M_>(N, occ); }

}  // namespace hm
