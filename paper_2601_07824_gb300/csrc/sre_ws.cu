// sre_ws.cu -- warp-specialised persistent exact-SRE kernel for 16 <= N <= 20 (paper Sec. 3.1.2,
// Algorithm 2, in the half-length form of common.cuh).
//
// One 512-thread CTA per SM with two roles that run independently:
//   * warps 0-7, pass 1: each warp takes (X-string, two units) tasks from its own stride of
//     the global pass-1 list, forms the pair products, transforms the 10 low bits of z' in
//     registers + a warp-private shared buffer, stores to the scratch ring and signals with
//     a per-warp release increment.  No CTA-wide barrier is ever needed.
//   * warps 8-15, pass 2 (one 256-thread group, named barrier 1): each task is a tile of all
//     2^M units x 2^(13-M) columns of one X-string.  The group prefetches the next tile with
//     cp.async into the other half of a double buffer while it transforms the current one
//     (in place, dense layout), reduces it, drops its lines from L2 (discard) and signals.
// Dependencies (bounded waits): pass 2 of batch g waits for all pass-1 tasks of batch g; pass 1
// of batch g waits for pass 2 of batch g - R (slot reuse).  A prefetch waits early only when
// that cannot involve the group's own unsignalled task, so the schedule cannot deadlock.
#include "common.cuh"
#include "pairs.cuh"
#include "sre_fwd.h"

namespace hm {

template <int M>
struct WsShape {
    static constexpr int K1 = 10, L = K1 + M, LOGT = 13 - M, T = 1 << LOGT, TILES = 1024 / T;
    static constexpr size_t P1_SLOTS = 8 * tile_slots(10);  // float2 per CTA for pass-1 warps
    static constexpr size_t P2_SLOTS = 2 * 8192;            // double-buffered dense tiles
    static constexpr size_t SMEM = (P1_SLOTS + P2_SLOTS) * sizeof(float2);
};

template <int M, int MODE>
__global__ void __launch_bounds__(512, 1) sre_ws(WsParams P) {
    using Sh = WsShape<M>;
    constexpr int K1 = 10, L = Sh::L, LOGT = Sh::LOGT, T = Sh::T, TILES = Sh::TILES;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float red[8][4];
    __shared__ double redd[8];
    __shared__ int flag;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t dim = int64_t(1) << P.N;
    const size_t per_a = (size_t)1 << L;

    if (warp < 8) {
        // ------------------------------ pass-1 role --------------------------------------
        float2* sm = smem + warp * tile_slots(10);
        const int64_t W1 = (int64_t)gridDim.x * 8;
        const int64_t total1 = P.n_batches * P.p1;
        for (int64_t tau = (int64_t)blockIdx.x * 8 + warp; tau < total1; tau += W1) {
            const int64_t g = tau / P.p1;
            const int r = (int)(tau % P.p1);
            const int slot = (int)(g % P.R);
            if (g >= P.R &&
                !warp_wait_geq(P.done2 + slot, (unsigned)((g / P.R) * P.p2) + P.wait_bias, P.status, P.spin_limit))
                break;
            const int a_idx = r % P.A;
            const int64_t unit = (int64_t)(r / P.A) * 2;
            const int64_t i = g * P.A + a_idx;
            bool valid = i < P.count;
            const int64_t a = valid ? (P.a_list ? P.a_list[i] : i) : 0;
            if (a < 0 || a >= dim) {
                if (valid && lane == 0) atomicOr(P.status, ST_BADARG);
                valid = false;
            }
            if (valid) {
                float2 x[32];
                float2* sbase = P.scratch + ((size_t)slot * P.A + a_idx) * per_a;
                for (int uu = 0; uu < 2; ++uu) {
                    const PairRows<K1, M> pr(a, unit + uu);
                    float2* dst = sbase + ((size_t)(unit + uu) << K1) + lane;
#pragma unroll
                    for (int k = 0; k < 32; ++k) x[k] = pr.value(P.psi, a, lane | (k << 5));
                    reg_fwht<5, 0, 5>(x);
                    tile_rounds<10, 0, 5, 1>(x, sm, lane, SyncWarp());
#pragma unroll
                    for (int k = 0; k < 32; ++k) __stcg(dst + (k << 5), x[k]);
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                red_release_add(P.done1 + slot, 1u);
            }
        }
        return;
    }

    // ------------------------------ pass-2 role ---------------------------------------------
    const uint32_t t2 = tid - 256, w2 = warp - 8;
    SyncNamed<1, 256> bar;
    float2* const bufs = smem + Sh::P1_SLOTS;
    const int64_t total2 = P.n_batches * P.p2;
    double acc[3] = {0.0, 0.0, 0.0};

    auto task_batch = [&](int64_t tau) { return tau / P.p2; };
    auto wait_dep = [&](int64_t tau) -> bool {
        const int64_t g = tau / P.p2;
        const int slot = (int)(g % P.R);
        return group_wait_geq(P.done1 + slot, (unsigned)((g / P.R + 1) * P.p1) + P.wait_bias, P.status,
                              P.spin_limit, 0u, t2 == 0, &flag, bar);
    };
    // source of tile `tau`, or null when the task has no X-string (partial last batch)
    auto tile_src = [&](int64_t tau) -> const float2* {
        const int64_t g = tau / P.p2;
        const int r = (int)(tau % P.p2);
        const int a_idx = r / TILES, tile = r % TILES;
        if (g * P.A + a_idx >= P.count) return nullptr;
        return P.scratch + ((size_t)(g % P.R) * P.A + a_idx) * per_a + (size_t)tile * T;
    };
    auto issue = [&](int64_t tau, float2* buf) {
        const float2* src = tile_src(tau);
        if (src) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {  // 4096 chunks of two values = 2^M rows x T columns
                const uint32_t c = t2 + 256u * q;
                const uint32_t row = c >> (LOGT - 1), col = (c & ((T >> 1) - 1)) << 1;
                cp_async16(buf + (row << LOGT) + col, src + ((size_t)row << K1) + col);
            }
        }
        cp_async_commit();
    };

    int64_t tau = blockIdx.x;
    int cur = 0;
    bool ok = true;
    if (tau < total2) {
        ok = wait_dep(tau);
        if (ok) issue(tau, bufs);
    }
    while (ok && tau < total2) {
        const int64_t tn = tau + gridDim.x;
        bool next_issued = false;
        // wait for the next tile's producers early only if that cannot depend on this task
        if (tn < total2 && task_batch(tn) - task_batch(tau) <= P.R - 1) {
            if (!wait_dep(tn)) { ok = false; break; }
            issue(tn, bufs + (cur ^ 1) * 8192);
            next_issued = true;
        }
        if (next_issued) cp_async_wait<1>(); else cp_async_wait<0>();
        bar();
        const float2* src = tile_src(tau);
        const int64_t g = tau / P.p2;
        if (src) {
            float2* buf = bufs + cur * 8192;
            float2 x[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) x[k] = buf[t2 | (k << 8)];
            reg_fwht<5, 0, 5>(x);
            tile_rounds<13, LOGT, 5, 1>(x, buf, t2, bar, DenseAddr());
            if constexpr (TileSched<13, LOGT, 5>::NR == 1) bar();
            if constexpr (LOGT >= 4) {
                // the tile is in shared memory/registers: drop its scratch lines from L2 unwritten
                constexpr int LPR = (T * 8) / 128;
#pragma unroll
                for (int q = t2; q < (1 << M) * LPR; q += 256)
                    discard_l2_line(src + ((size_t)(q / LPR) << K1) + (q % LPR) * 16);
            }
            Acc<MODE> ac;
#pragma unroll
            for (int k = 0; k < 32; ++k) ac.add(x[k], P.nq);
            ac.fold();
            float q = ac.q, s1 = ac.s1, u = ac.u;
            double qd = ac.qd;
            warp_sum3<MODE>(q, s1, u, qd, 32);
            if (lane == 0) { red[w2][0] = q; red[w2][1] = s1; red[w2][2] = u; redd[w2] = qd; }
            bar();
            if (t2 == 0) {
                double v[3], tot[3] = {0.0, 0.0, 0.0};
                for (int w = 0; w < 8; ++w) {
                    finish3<MODE>(red[w][0], red[w][1], red[w][2], redd[w], P.nq, v);
                    tot[0] += v[0]; tot[1] += v[1]; tot[2] += v[2];
                }
                if (P.per_a) {
                    const int r = (int)(tau % P.p2);
                    double* o = P.out + ((size_t)(g * P.A + r / TILES) * TILES + r % TILES) * 3;
                    o[0] = tot[0]; o[1] = tot[1]; o[2] = tot[2];
                } else {
                    acc[0] += tot[0]; acc[1] += tot[1]; acc[2] += tot[2];
                }
            }
        }
        bar();  // the buffer and red[] are free again
        if (t2 == 0) red_release_add(P.done2 + (int)(g % P.R), 1u);
        if (tn < total2 && !next_issued) {
            if (!wait_dep(tn)) { ok = false; break; }
            issue(tn, bufs + (cur ^ 1) * 8192);
        }
        tau = tn;
        cur ^= 1;
    }
    cp_async_wait<0>();
    if (t2 == 0 && !P.per_a) {
        P.out[blockIdx.x * 3 + 0] = acc[0];
        P.out[blockIdx.x * 3 + 1] = acc[1];
        P.out[blockIdx.x * 3 + 2] = acc[2];
    }
}

template <int M, int MODE>
static cudaError_t ws_prep() {
    return cudaFuncSetAttribute(sre_ws<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WsShape<M>::SMEM);
}

template <int M, int MODE>
static cudaError_t launch_ws_t(const WsParams& P, int grid, cudaStream_t st) {
    cudaError_t e = ws_prep<M, MODE>();
    if (e != cudaSuccess) return e;
    sre_ws<M, MODE><<<grid, 512, WsShape<M>::SMEM, st>>>(P);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_ws_m(const WsParams& P, int grid, cudaStream_t st) {
    switch (P.N) {
        case 16: return launch_ws_t<5, MODE>(P, grid, st);
        case 17: return launch_ws_t<6, MODE>(P, grid, st);
        case 18: return launch_ws_t<7, MODE>(P, grid, st);
        case 19: return launch_ws_t<8, MODE>(P, grid, st);
        case 20: return launch_ws_t<9, MODE>(P, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int ws_tiles_per_a(int N) { return 1024 >> (13 - (N - 11)); }

cudaError_t launch_ws(const WsParams& P, int mode, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: return launch_ws_m<0>(P, grid, st);
        case 1: return launch_ws_m<1>(P, grid, st);
        case 2: return launch_ws_m<2>(P, grid, st);
        case 3: return launch_ws_m<3>(P, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hm
