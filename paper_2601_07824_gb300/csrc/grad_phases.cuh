// grad_phases.cuh -- the three passes of the M_2 adjoint (see grad.cu for the derivation) as
// device functions, shared by the single-state kernel and the batched persistent kernel.
//
// One state's data for pass 1 (warp-level, K1 = 10 low bits), pass 2 (2^M units x 2^(13-M)
// columns: finish W, accumulate S_2, form R^3 + i I^3 and transform it back in place) and pass 3
// (one X-string x 16 units: transform the low bits again and scatter 32 psi Q into a partial).
#pragma once
#include "common.cuh"
#include "pairs.cuh"
#include "schedule.h"
#include "sre_fwd.h"

namespace hm {

struct G3State {
    const float2* psi;
    int N;
    float2* scratch;  // R slots x A X-strings x 2^(N-1)
    int R, A, U;
    int64_t n_batches;
    int p1, p2, p3;
    unsigned* done1;
    unsigned* done2;
    unsigned* done3;
    int64_t a_base = 0;  // X-string of batch 0, entry 0 (a slice [a_base, a_base + A n_batches))
    int UPW = 2;         // units per pass-1 warp (even)
    int TPT = 1;         // column tiles per pass-2 task
};

struct G3Ctl {
    int* status;
    long long spin_limit;
    unsigned wait_bias;
};

__device__ __forceinline__ float2 cube_parts(float2 w) { return make_float2(w.x * w.x * w.x, w.y * w.y * w.y); }

// gp[z] += 32 psi[zb] Q,  gp[zb] += 32 psi[z] conj(Q)
__device__ __forceinline__ void scatter_pair(float2* __restrict__ gp, const float2* __restrict__ psi, int64_t z,
                                             int64_t zb, float2 q) {
    const float2 pz = ld_amp(psi, z), pb = ld_amp(psi, zb);
    float2 g0 = gp[z], g1 = gp[zb];
    g0.x += 32.f * (pb.x * q.x - pb.y * q.y);
    g0.y += 32.f * (pb.x * q.y + pb.y * q.x);
    g1.x += 32.f * (pz.x * q.x + pz.y * q.y);
    g1.y += 32.f * (pz.y * q.x - pz.x * q.y);
    gp[z] = g0;
    gp[zb] = g1;
}
// a = 0: gp[z] += 32 psi[z] (Re Q + Im Q), gp[z+1] += 32 psi[z+1] (Re Q - Im Q)
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

// ---- pass 1: task r of batch g (each warp: one X-string, two units) ------------------------
template <int M>
__device__ __forceinline__ bool g3_pass1(const G3State& S, const G3Ctl& C, int64_t g, int r, float2* smem) {
    constexpr int K1 = 10, L = K1 + M;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int slot;
    unsigned need;
    if (g3_dependency(g, 1, S.R, S.p1, S.p2, S.p3, slot, need) &&
        !cta_wait_geq(S.done3 + slot, need + C.wait_bias, C.status, C.spin_limit))
        return false;
    const int a_idx = warp % S.A;
    const int64_t unit = ((int64_t)r * S.U + warp / S.A) * S.UPW;
    const int64_t a = S.a_base + g * S.A + a_idx;
    const int64_t dim = int64_t(1) << S.N;
    // with 8 X-strings per batch (U == 1) the CTA's warps read the same state rows (consecutive
    // aligned X-strings): stage them once in shared memory, two units at a time (the caller
    // reserves kStageSlots values after the 8 warps' exchange buffers)
    const int64_t a0 = S.a_base + g * S.A;
    const bool stage = S.U == 1 && a0 < dim;  // CTA-uniform
    // far batch (a0 >= 2^K1): the partner row is staged block-permuted by bits 5..9 of a0, so
    // both pair-product loads are a per-thread base plus a compile-time offset
    const bool far = stage && (a0 >> K1) != 0;
    const uint32_t perm = far ? (uint32_t)((a0 >> 5) & 31) : 0u;
    float2* rows = smem + 8 * tile_slots(10);
    float2* sbase = S.scratch + (size_t)slot * S.A * ((size_t)1 << L);
    float2* sm = smem + warp * tile_slots(10);
    for (int up = 0; up < S.UPW; up += 2) {
        if (stage) {
            if (up > 0) __syncthreads();  // every warp is done with the previous rows
            stage_rows<M>(rows, S.psi, a0, unit + up, perm);
        }
        if (a >= dim) continue;
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
                for (int k = 0; k < 32; ++k) x[k] = pr.value(S.psi, a, lane | (k << 5));
            }
            reg_fwht<5, 0, 5>(x);
            tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
#pragma unroll
            for (int k = 0; k < 32; ++k) __stcg(dst + lane + (k << 5), x[k]);
        }
    }
    __syncthreads();
    if (tid == 224) { red_release_add(S.done1 + slot, 1u); }
    return true;
}

// Lanes of a state's [S_2, S_1] accumulator in the batched launch (pass-2 tasks add into lane
// blockIdx mod kS2Lanes, which keeps the atomics on one address few).
constexpr int kS2Lanes = 16;

// ---- pass 2: tiles r TPT .. r TPT + TPT - 1 of batch g (S.TPT column tiles per task); adds
// 16 sum(R^4+I^4) and 4 sum(R^2+I^2) of each warp's values
// into acc/acc1 of that warp's lane 0 (no CTA barrier for the sums; the caller combines the 8
// warps at the end).  If s2_atomic is given ([kS2Lanes][2] doubles), lane 0 of every warp also
// adds its two sums to lane (8 blockIdx + warp) mod kS2Lanes of it before the task's release.
// FWD: forward only (M_2 without the gradient): no cube, back-transform or store.
template <int M, bool FWD = false>
__device__ __forceinline__ bool g3_pass2(const G3State& S, const G3Ctl& C, int64_t g, int r, float2* smem,
                                         double& acc, double& acc1, double* s2_atomic = nullptr) {
    constexpr int K1 = 10, L = K1 + M, LOGT = 13 - M, T = 1 << LOGT, TILES = 1024 / T;
    constexpr int B0 = LOGT > 8 ? LOGT - 8 : 0;  // round-0 register bits that are columns
    using S2 = TileSched<13, LOGT, 5>;
    constexpr int SL2 = S2::last_shift();
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    int slot;
    unsigned need;
    g3_dependency(g, 2, S.R, S.p1, S.p2, S.p3, slot, need);
    if (!cta_wait_geq(S.done1 + slot, need + C.wait_bias, C.status, C.spin_limit)) return false;
    const int a_idx = r / (TILES / S.TPT);
    const int64_t a = S.a_base + g * S.A + a_idx;
    if (a < (int64_t(1) << S.N)) for (int tile = (r % (TILES / S.TPT)) * S.TPT, te = tile + S.TPT; tile < te; ++tile) {
        float2* src = S.scratch + (size_t)slot * S.A * ((size_t)1 << L) + (size_t)a_idx * ((size_t)1 << L) +
                      (size_t)tile * T;
        float2 x[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint32_t j = deposit<5>(tid, k, 8);
            x[k] = __ldcg(src + ((size_t)(j >> LOGT) << K1) + (j & (T - 1)));
        }
        reg_fwht<5, B0, 5>(x);
        tile_rounds<13, LOGT, 5, 1>(x, smem, tid, SyncCta());
        float q = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float2 sq = mul2(x[k], x[k]);
            s1 += sq.x + sq.y;
            q = fmaf(sq.x, sq.x, fmaf(sq.y, sq.y, q));
            x[k] = cube_parts(x[k]);
        }
        if constexpr (!FWD) {
        // back to the round-0 layout, transform the high bits again, store in place
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 32; ++k) smem[swz(deposit<5>(tid, k, SL2))] = x[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 32; ++k) x[k] = smem[swz(deposit<5>(tid, k, 8))];
        reg_fwht<5, B0, 5>(x);
        tile_rounds<13, LOGT, 5, 1>(x, smem, tid, SyncCta());
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint32_t j = deposit<5>(tid, k, SL2);
            __stcg(src + ((size_t)(j >> LOGT) << K1) + (j & (T - 1)), x[k]);
        }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
        if (lane == 0) {
            const double t0 = 16.0 * (double)q, t1 = 4.0 * (double)s1;
            acc += t0;
            acc1 += t1;
            if (s2_atomic) {
                double* d = s2_atomic + 2 * ((blockIdx.x * 8u + (tid >> 5)) % kS2Lanes);
                atomicAdd(d, t0);
                atomicAdd(d + 1, t1);
            }
        }
    }
    __syncthreads();
    if (tid == 224) { red_release_add(S.done2 + slot, 1u); }
    return true;
}

// ---- pass 3: one X-string x 16 units; scatter into gp (this CTA's partial gradient) ---------
template <int M>
__device__ __forceinline__ bool g3_pass3(const G3State& S, const G3Ctl& C, int64_t g, int r, float2* smem,
                                         float2* __restrict__ gp, const unsigned* extra_ctr = nullptr,
                                         unsigned extra_need = 0) {
    constexpr int K1 = 10, L = K1 + M;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int slot;
    unsigned need;
    g3_dependency(g, 3, S.R, S.p1, S.p2, S.p3, slot, need);
    if (!cta_wait_geq(S.done2 + slot, need + C.wait_bias, C.status, C.spin_limit)) return false;
    if (extra_ctr && !cta_wait_geq(extra_ctr, extra_need + C.wait_bias, C.status, C.spin_limit)) return false;
    constexpr int PER_A = (1 << M) / 16;
    const int a_idx = r / PER_A;
    const int64_t unit0 = (int64_t)(r % PER_A) * 16 + warp * 2;
    const int64_t a = S.a_base + g * S.A + a_idx;
    if (a < (int64_t(1) << S.N)) {
        const float2* sbase = S.scratch + (size_t)slot * S.A * ((size_t)1 << L) + (size_t)a_idx * ((size_t)1 << L);
        float2* sm = smem + warp * tile_slots(10);
        float2 x[32];
        for (int uu = 0; uu < 2; ++uu) {
            const int64_t unit = unit0 + uu;
            const float2* src = sbase + ((size_t)unit << K1);
            // column (k<<5)|lane holds tile index j = k | (lane<<5); with j' = the swap of the
            // two 5-bit halves this is the round-0 layout of the 10-bit schedule
#pragma unroll
            for (int k = 0; k < 32; ++k) x[k] = __ldcg(src + lane + (k << 5));
            reg_fwht<5, 0, 5>(x);
            tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
            // register k now holds Q at j = lane | (k << 5) (the pair-product layout)
            const PairRows<K1, M> pr(a, unit);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const uint32_t j = lane | (k << 5);
                if (a >> K1) {
                    scatter_pair(gp, S.psi, pr.rowA + j, pr.rowB + (int64_t)(j ^ (uint32_t)pr.al), x[k]);
                } else {
                    const int64_t row = (j >> (K1 - 1)) ? pr.rowB : pr.rowA;
                    const int64_t lp = j & ((1u << (K1 - 1)) - 1u);
                    if (a != 0) {
                        const int64_t z = row + insert0(lp, pr.p);
                        scatter_pair(gp, S.psi, z, z ^ a, x[k]);
                    } else {
                        scatter_zero(gp, S.psi, row + (lp << 1), x[k]);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (tid == 224) red_release_add(S.done3 + slot, 1u);
    return true;
}

// One-pass adjoint of a whole state by one group of threads (see grad.cu): X-strings
// a = a_base + i for i = gg, gg + ngroups, ... below count (count < 0: all 2^N X-strings);
// contributions go to gp (this group's partial, 2^N values); the group leader (t == 0)
// receives the group's S_2 and S_1 sums.  FWD: the sums only.
template <int L, bool FWD = false>
__device__ __forceinline__ void grad_onepass_group(const float2* __restrict__ psi, int N, float2* __restrict__ gp,
                                                   int64_t gg, int64_t ngroups, float2* sm, double& acc,
                                                   double& acc1, int64_t a_base = 0, int64_t count = -1) {
    using Sh = OnepassShape<L>;
    constexpr int E = Sh::E, G = Sh::G;
    using S = TileSched<L, 0, E>;
    constexpr int SL = S::last_shift();
    __shared__ float red[16][2];
    const uint32_t tid = threadIdx.x, t = tid % G;
    const int64_t dim = int64_t(1) << N;
    const int64_t cnt = count < 0 ? dim : count;
    const int64_t iters = (cnt + ngroups - 1) / ngroups;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = gg + it * ngroups;
        const int64_t a = a_base + i;
        const bool valid = i < cnt && a < dim;
        const int64_t av = valid ? a : 0;
        const int p = av ? msb64(av) : 0;
        float2 x[1 << E];
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) x[i] = pair_product(psi, deposit<E>(t, i, S::S0), av, p);
        reg_fwht<E, 0, E>(x);
        if constexpr (G <= 32) tile_rounds<L, 0, E, 1>(x, sm, t, SyncWarp());
        else tile_rounds<L, 0, E, 1>(x, sm, t, SyncCta());
        float q = 0.f, s1 = 0.f;
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) {
            const float2 sq = mul2(x[i], x[i]);
            s1 += sq.x + sq.y;
            q = fmaf(sq.x, sq.x, fmaf(sq.y, sq.y, q));
            x[i] = cube_parts(x[i]);
        }
        if constexpr (!FWD) {
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
        }
        if constexpr (G <= 32) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1)
                if (o < G) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
        } else {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) { q += __shfl_xor_sync(0xffffffffu, q, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o); }
            if ((tid & 31) == 0) { red[tid >> 5][0] = q; red[tid >> 5][1] = s1; }
            __syncthreads();
            if (t == 0) {  // this group's warps: [tid/32, tid/32 + G/32)
                float a0 = 0.f, a1 = 0.f;
                for (int w = 0; w < (G >> 5); ++w) { a0 += red[(tid >> 5) + w][0]; a1 += red[(tid >> 5) + w][1]; }
                q = a0; s1 = a1;
            }
            __syncthreads();
        }
        if (t == 0 && valid) { acc += 16.0 * (double)q; acc1 += 4.0 * (double)s1; }
    }
}

}  // namespace hm
