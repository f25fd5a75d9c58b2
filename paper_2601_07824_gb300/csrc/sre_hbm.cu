// sre_hbm.cu -- per-X-string SRE sums for 25 <= N <= 28 (scratch larger than L2), used by the
// uniform-X Monte-Carlo estimator (per-X decomposition of Algorithm 2, Sec. 3.1.2).
//
// Half-length form (common.cuh); the scratch of one X-string is [2^M units][2^13 columns] with
// M = N - 14 = M2 + M3.  Persistent kernel, 256 threads, three passes per batch of one X-string:
//   pass 1: one (a, unit): pair product + transform of the 13 low bits of z' (CTA-level);
//   pass 2: tiles of 2^M2 consecutive units x 2^(13-M2) columns: transform the M2 middle bits,
//           written back in place;
//   pass 3: tiles of 2^M3 units (stride 2^M2) x 2^(13-M3) columns: transform the M3 top bits,
//           reduce, per-(a, tile) partial sums.
// Stage s holds pass 1 of batch s, pass 2 of batch s-1, pass 3 of batch s-2; every bounded wait
// is on an earlier task (R >= 3 slots), so a co-resident grid cannot deadlock.
#include "common.cuh"
#include "pairs.cuh"
#include "sre_fwd.h"

namespace hm {

template <int M2, int M3>
__global__ void __launch_bounds__(256, 2) sre_threepass(HbmParams P) {
    constexpr int K1 = 13, M = M2 + M3, L = K1 + M;
    constexpr int LOG2 = 13 - M2, T2 = 1 << LOG2;
    constexpr int LOG3 = 13 - M3, T3 = 1 << LOG3;
    constexpr int TILES3 = (1 << (K1 + M2)) / T3;  // pass-3 tiles per X-string
    constexpr int TILES2 = (1 << (K1 + M3)) / T2;  // pass-2 tiles per X-string
    extern __shared__ float2 smem[];
    __shared__ float red[8][4];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t dim = int64_t(1) << P.N;
    const int64_t per_stage = (int64_t)P.p1 + P.p2 + P.p3;
    const int64_t total = (P.n_batches + 2) * per_stage;
    const size_t per_a = (size_t)1 << L;

    for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
        const int64_t s = task / per_stage;
        int r = (int)(task % per_stage);
        int kind;
        int64_t g;
        if (r < P.p1) { kind = 1; g = s; }
        else if (r < P.p1 + P.p2) { kind = 2; g = s - 1; r -= P.p1; }
        else { kind = 3; g = s - 2; r -= P.p1 + P.p2; }
        if (g < 0 || g >= P.n_batches) continue;
        const int slot = (int)(g % P.R);
        float2* sbase = P.scratch + (size_t)slot * per_a;
        const int64_t i = g;  // one X-string per batch
        const bool valid = i < P.count;

        if (kind == 1) {
            if (g >= P.R && !cta_wait_geq(P.done3 + slot, (unsigned)((g / P.R) * P.p3) + P.wait_bias, P.status, P.spin_limit))
                return;
            int64_t a = valid ? P.a_list[i] : 0;
            bool ok = valid;
            if (a < 0 || a >= dim) {
                if (valid && tid == 0) atomicOr(P.status, ST_BADARG);
                ok = false;
                a = 0;
            }
            if (ok) {
                const int64_t unit = r;
                const PairRows<K1, M> pr(a, unit);
                float2 x[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) x[k] = pr.value(P.psi, a, deposit<5>(tid, k, 8));
                reg_fwht<5, 0, 5>(x);
                tile_rounds<13, 0, 5, 1>(x, smem, tid, SyncCta());
                constexpr int SL = TileSched<13, 0, 5>::last_shift();
                float2* dst = sbase + ((size_t)unit << K1);
#pragma unroll
                for (int k = 0; k < 32; ++k) __stcg(dst + deposit<5>(tid, k, SL), x[k]);
            }
            __syncthreads();
            if (tid == 0) { __threadfence(); red_release_add(P.done1 + slot, 1u); }
        } else if (kind == 2) {
            if (!cta_wait_geq(P.done1 + slot, (unsigned)((g / P.R + 1) * P.p1) + P.wait_bias, P.status, P.spin_limit))
                return;
            if (valid) {
                // tile: units [uh * 2^M2, (uh+1) * 2^M2) x columns [c0, c0 + T2)
                const int uh = r / ((1 << K1) / T2), ct = r % ((1 << K1) / T2);
                float2* src = sbase + ((size_t)uh << (M2 + K1)) + (size_t)ct * T2;
                float2 x[32];
                using S = TileSched<13, LOG2, 5>;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, 8);
                    x[k] = __ldcg(src + ((size_t)(j >> LOG2) << K1) + (j & (T2 - 1)));
                }
                reg_fwht<5, (LOG2 > 8 ? LOG2 - 8 : 0), 5>(x);
                tile_rounds<13, LOG2, 5, 1>(x, smem, tid, SyncCta());
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, S::last_shift());
                    __stcg(src + ((size_t)(j >> LOG2) << K1) + (j & (T2 - 1)), x[k]);
                }
            }
            __syncthreads();
            if (tid == 0) { __threadfence(); red_release_add(P.done2 + slot, 1u); }
        } else {
            if (!cta_wait_geq(P.done2 + slot, (unsigned)((g / P.R + 1) * P.p2) + P.wait_bias, P.status, P.spin_limit))
                return;
            if (valid) {
                // tile: low-unit index ul, units ul + m * 2^M2 (m < 2^M3) x columns [c0, c0 + T3)
                const int ul = r / ((1 << K1) / T3), ct = r % ((1 << K1) / T3);
                const float2* src = sbase + ((size_t)ul << K1) + (size_t)ct * T3;
                float2 x[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const uint32_t j = deposit<5>(tid, k, 8);
                    x[k] = __ldcg(src + ((size_t)(j >> LOG3) << (K1 + M2)) + (j & (T3 - 1)));
                }
                reg_fwht<5, (LOG3 > 8 ? LOG3 - 8 : 0), 5>(x);
                tile_rounds<13, LOG3, 5, 1>(x, smem, tid, SyncCta());
                Acc<2> ac;
#pragma unroll
                for (int k = 0; k < 32; ++k) ac.add(x[k], 2.0);
                ac.fold();
                float q = ac.q, s1 = ac.s1, u = 0.f;
                double qd = 0.0;
                warp_sum3<2>(q, s1, u, qd, 32);
                if (lane == 0) { red[warp][0] = q; red[warp][1] = s1; }
                __syncthreads();
                if (tid == 0) {
                    double v[3], tot[2] = {0.0, 0.0};
                    for (int w = 0; w < 8; ++w) {
                        finish3<2>(red[w][0], red[w][1], 0.f, 0.0, 2.0, v);
                        tot[0] += v[0]; tot[1] += v[1];
                    }
                    double* o = P.out + ((size_t)i * TILES3 + r) * 3;
                    o[0] = tot[0]; o[1] = tot[1]; o[2] = 0.0;
                }
            }
            __syncthreads();
            if (tid == 0) red_release_add(P.done3 + slot, 1u);
        }
    }
    (void)TILES2;
}

int hbm_tiles_per_a(int N) {
    const int M = N - 14, M2 = (M + 1) / 2, M3 = M - M2;
    return (1 << (13 + M2)) >> (13 - M3);
}

static constexpr size_t kHbmSmem = tile_slots(13) * sizeof(float2);

template <int M2, int M3>
static cudaError_t hbm_launch_t(const HbmParams& P, int sm_count, int* grid, cudaStream_t st) {
    auto k = sre_threepass<M2, M3>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHbmSmem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, kHbmSmem)) != cudaSuccess) return e;
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    k<<<*grid, 256, kHbmSmem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_hbm(const HbmParams& P, int sm_count, int* grid, cudaStream_t st) {
    switch (P.N) {
        case 25: return hbm_launch_t<6, 5>(P, sm_count, grid, st);
        case 26: return hbm_launch_t<6, 6>(P, sm_count, grid, st);
        case 27: return hbm_launch_t<7, 6>(P, sm_count, grid, st);
        case 28: return hbm_launch_t<7, 7>(P, sm_count, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hm
