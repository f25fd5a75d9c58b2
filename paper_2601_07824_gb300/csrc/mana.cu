// mana.cu -- pure-state qutrit mana (paper Sec. 3.3.2, Algorithm 5; Eqs. mana2, mana_FT,
// F3_unnorm_def, z3_FT_tensor_unnorm).
//
// For every a in Z_3^N (base-3 index, digit j = qutrit j):
//   v_x = conj(psi_{x - a}) psi_{-x - a}   (digit-wise mod 3: alpha = amplitudes of X^a psi),
//   chi = F_3^{(x)N} v with (F_3)_{jk} = w^{2jk}, w = e^{2 pi i / 3},
//   m += sum_b |chi_b|,    mana = log2(m / 3^N)   (the 1/3^N of Eq. mana2).
// chi is real (v_{-x} = conj(v_x)), so |chi_b| = |Re chi_b|.
//
// A tile of 3^D values is held as 27 values per thread (three base-3 digits in registers);
// other digits are exchanged through shared memory.  The index x - a (digit-wise) of each
// register is (thread part) + C_0[r0] + C_1[r1] + C_2[r2] with per-thread tables C_j[v] for
// the three register digits, so address arithmetic stays a few integer adds per value.
//   * N <= 8:  one pass, a group of 3^(N-3) threads owns one a.
//   * 9 <= N <= 13: persistent two-pass kernel (same task order and bounded waits as the
//     qubit kernel): pass 1 transforms the 8 low digits of one (a, unit) in a 3^8 tile, pass 2
//     the N-8 high digits of 3^(N-8) units x 3^(16-N) columns and reduces.
//     Since every chi_a is real and F_3^{(x)N} is linear, one complex transform of
//     v_a + i v_a2 gives chi_a (real part) and chi_a2 (imaginary part).  The two-pass kernels
//     transform such pairs: a2 = a + 3^j differs from a in one digit j >= 8, which in pass 1 is
//     a digit of the unit, so the gather indices of a2 are those of a plus one offset per task.
//     Level k (0 <= k < N - 8) pairs the X-strings with digits above j = N - 1 - k equal to 2
//     and digit j equal to 0 with their digit-j-equal-1 partners; the 3^8 X-strings whose top
//     N - 8 digits are all 2 are transformed alone.  About half the transforms remain.
//
// Mixed states (Sec. 3.3.3, Algorithm 6) run the same kernels with MIXED = true: with
// rho = |psi><psi| the value above is rho[-x-a, x-a], and for a general density matrix
//     v_x = rho[-x - a, x - a]   (row-major rho, qutrit j = base-3 digit j of row and column)
// transformed the same way gives every W_u = tr(rho A_u) / 3^N (up to the labelling of u),
// real because rho is Hermitian.  Algorithm 6 sweeps the single-qutrit 9 x 9 map over every leg
// of the 9^N vector Vec_N(rho), N passes over it; here (a, x) -> (-x - a, x - a) is a
// bijection onto the entries of rho, so every entry is read once and the radix-3 transform
// stays on chip.
#include "common.cuh"
#include "extra.h"
#include "mana.h"

namespace hm {
namespace mana {

__host__ __device__ constexpr int pow3(int n) { return n <= 0 ? 1 : 3 * pow3(n - 1); }

// Radix-3 butterfly of F_3: y0 = x0+x1+x2, y1 = x0 + w^2 x1 + w x2, y2 = x0 + w x1 + w^2 x2.
__device__ __forceinline__ void bfly3(float2& x0, float2& x1, float2& x2) {
    const float h = 0.86602540378443864676f;  // sqrt(3)/2
    const float2 s = add2(x1, x2), d = sub2(x1, x2);
    const float2 t = fma2(make_float2(-0.5f, -0.5f), s, x0);
    x0 = add2(x0, s);
    // w^2 x1 + w x2 = -s/2 - i h d,   w x1 + w^2 x2 = -s/2 + i h d
    x1 = make_float2(fmaf(h, d.y, t.x), fmaf(-h, d.x, t.y));
    x2 = make_float2(fmaf(-h, d.y, t.x), fmaf(h, d.x, t.y));
}

// Butterflies over register digits [D0, D1) of an array of 3^E values (digit j has stride 3^j).
// One digit per template level, so that every index into x is a compile-time constant and x
// stays in registers.
template <int E, int D0, int D1>
__device__ __forceinline__ void reg_ft3(float2 (&x)[pow3(E)]) {
    if constexpr (D0 < D1) {
        constexpr int st = pow3(D0);
#pragma unroll
        for (int r = 0; r < pow3(E); ++r)
            if ((r / st) % 3 == 0) bfly3(x[r], x[r + st], x[r + 2 * st]);
        reg_ft3<E, D0 + 1, D1>(x);
    }
}

// Tile element index of register r of thread t when the register digits are [s, s+E):
// thread digits fill the other positions in order.
template <int E>
__device__ __forceinline__ uint32_t deposit3(uint32_t t, uint32_t r, int s) {
    const uint32_t ps = (uint32_t)pow3(s);
    return (t % ps) + r * ps + (t / ps) * ps * (uint32_t)pow3(E);
}

// Round schedule for a tile of 3^D values, transform digits [LO, D), E register digits:
// round 0 holds [D-E, D); round r >= 1 holds [LO + (r-1)E, ...) and transforms digits below D-E.
template <int D, int LO, int E>
struct Sched3 {
    static constexpr int S0 = D - E;
    static constexpr int NR = 1 + ((S0 - LO) > 0 ? ((S0 - LO) + E - 1) / E : 0);
    static constexpr int shift(int r) { return r == 0 ? S0 : LO + (r - 1) * E; }
};

// `act`: threads outside the tile (CTA sizes are not multiples of 3) only join the barriers.
template <int D, int LO, int E, int R, class Sync>
__device__ __forceinline__ void rounds3(float2 (&x)[pow3(E)], float2* sm, uint32_t t, bool act, Sync sync) {
    using S = Sched3<D, LO, E>;
    if constexpr (R < S::NR) {
        constexpr int sp = S::shift(R - 1);
        constexpr int s = S::shift(R);
        constexpr int hi = (s + E < S::S0) ? (s + E) : S::S0;
        sync();
        if (act) {
#pragma unroll
            for (int r = 0; r < pow3(E); ++r) sm[deposit3<E>(t, r, sp)] = x[r];
        }
        sync();
        if (act) {
#pragma unroll
            for (int r = 0; r < pow3(E); ++r) x[r] = sm[deposit3<E>(t, r, s)];
        }
        reg_ft3<E, 0, hi - s>(x);
        rounds3<D, LO, E, R + 1>(x, sm, t, act, sync);
    }
}

// Digit-wise index arithmetic for the pair product.  For a thread whose tile element of
// register r is x = xbase + r * 3^s (register digits at positions s, s+1, s+2 of the whole
// index), idx(x - a) = b1 + C1[0][r0] + C1[1][r1] + C1[2][r2] and idx(-x - a) likewise.
struct PairIdx3 {
    int64_t b1, b2;
    int32_t c1[3][3], c2[3][3];
    // xfix: the full index with the register digits set to 0; pos: position of register digit 0
    template <int E>
    __device__ __forceinline__ void init(int64_t xfix, int64_t a, int N, int pos) {
        b1 = 0; b2 = 0;
        int64_t p = 1, xs = xfix, as = a, ppos = 1;
        for (int j = 0; j < N; ++j) {
            const int xd = (int)(xs % 3), ad = (int)(as % 3);
            xs /= 3; as /= 3;
            if (j < pos) ppos *= 3;
            if (j < pos || j >= pos + E) {
                b1 += ((xd - ad + 3) % 3) * p;
                b2 += ((6 - xd - ad) % 3) * p;
            }
            p *= 3;
        }
        int64_t ar = a / ppos;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int ad = (int)(ar % 3);
            ar /= 3;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                c1[q][v] = q < E ? (int32_t)(((v - ad + 3) % 3) * ppos) : 0;
                c2[q][v] = q < E ? (int32_t)(((6 - v - ad) % 3) * ppos) : 0;
            }
            ppos *= 3;
        }
    }
    // pure: conj(psi[x - a]) psi[-x - a];  mixed: rho[-x - a, x - a] (dim = 3^N, row length)
    template <int R, bool MIXED>
    __device__ __forceinline__ float2 value(const float2* __restrict__ src, int64_t dim) const {
        constexpr int r0 = R % 3, r1 = (R / 3) % 3, r2 = R / 9;
        const int64_t i1 = b1 + c1[0][r0] + c1[1][r1] + c1[2][r2];
        const int64_t i2 = b2 + c2[0][r0] + c2[1][r1] + c2[2][r2];
        if constexpr (MIXED) return ld_amp(src, i2 * dim + i1);
        else return conj_mul(ld_amp(src, i1), ld_amp(src, i2));
    }
};

template <int E, bool MIXED, int R = 0>
__device__ __forceinline__ void load_pairs(float2 (&x)[pow3(E)], const PairIdx3& pi, const float2* __restrict__ src,
                                           int64_t dim) {
    if constexpr (R < pow3(E)) {
        x[R] = pi.value<R, MIXED>(src, dim);
        load_pairs<E, MIXED, R + 1>(x, pi, src, dim);
    }
}

// v_a + i v_a2 where the gather indices of a2 are those of a plus `off` (both of them).
template <int E, bool MIXED, int R = 0>
__device__ __forceinline__ void load_pairs2(float2 (&x)[pow3(E)], const PairIdx3& pi, const float2* __restrict__ src,
                                            int64_t dim, int64_t off) {
    if constexpr (R < pow3(E)) {
        const float2 v = pi.value<R, MIXED>(src, dim);
        PairIdx3 q2 = pi;
        q2.b1 += off;
        q2.b2 += off;
        const float2 w = q2.value<R, MIXED>(src, dim);
        x[R] = make_float2(v.x - w.y, v.y + w.x);
        load_pairs2<E, MIXED, R + 1>(x, pi, src, dim, off);
    }
}

// Work item w of the two-pass kernels (see the file comment): X-string a and its partner
// a2 = a + 3^j (a2 = -1 for a single).
__device__ __forceinline__ void pair_item(int64_t w, int N, int64_t& a, int64_t& a2, int& j) {
    int64_t base = 0, sz = pow3(N - 1);
    for (int k = 0; k < N - 8; ++k, sz /= 3) {
        if (w < sz) {
            a = base + w;
            a2 = a + sz;
            j = N - 1 - k;
            return;
        }
        w -= sz;
        base += 2 * sz;  // digit N - 1 - k is 2 from here on
    }
    a = base + w;
    a2 = -1;
    j = -1;
}

// Accumulate [sum |chi|, sum chi, sum chi^2] over a thread's values; PAIRED: both parts of
// each value are chi values (of two X-strings), else only the real part.
template <int E, bool PAIRED = false>
__device__ __forceinline__ void acc_chi(const float2 (&x)[pow3(E)], float& m, float& s, float& q) {
#pragma unroll
    for (int r = 0; r < pow3(E); ++r) {
        m += fabsf(x[r].x);
        s += x[r].x;
        q = fmaf(x[r].x, x[r].x, q);
        if constexpr (PAIRED) {
            m += fabsf(x[r].y);
            s += x[r].y;
            q = fmaf(x[r].y, x[r].y, q);
        }
    }
}

__device__ __forceinline__ void warp_sum3f(float& m, float& s, float& q) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
}

// CTA reduction of per-thread FP32 triples to FP64 (fixed order); result valid in thread 0.
__device__ __forceinline__ void cta_sum3(float m, float s, float q, double out[3]) {
    __shared__ float red[8][3];
    warp_sum3f(m, s, q);
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = m; red[threadIdx.x >> 5][1] = s; red[threadIdx.x >> 5][2] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = out[1] = out[2] = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { out[0] += red[w][0]; out[1] += red[w][1]; out[2] += red[w][2]; }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------
// One pass (N <= 8): a group of G = 3^(N-3) threads (1 thread for N < 3) owns one a.
template <int N, bool MIXED>
__global__ void __launch_bounds__(256) mana_onepass(const float2* __restrict__ psi, double* __restrict__ out) {
    constexpr int E = N < 3 ? N : 3;
    constexpr int V = pow3(E);
    constexpr int G = pow3(N - E);
    constexpr int GPC = 256 / G;
    constexpr int DIM = pow3(N);
    using S = Sched3<N, 0, E>;
    extern __shared__ float2 smem[];
    const uint32_t tid = threadIdx.x;
    const uint32_t gi = tid / G, t = tid % G;
    const bool active = gi < GPC;
    float2* sm = smem + (active ? gi : 0) * DIM;
    const int64_t ngroups = (int64_t)gridDim.x * GPC;
    const int64_t iters = (DIM + ngroups - 1) / ngroups;
    float m = 0.f, s = 0.f, q = 0.f;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t a = (int64_t)blockIdx.x * GPC + gi + it * ngroups;
        const bool valid = active && a < DIM;
        float2 x[V];
        PairIdx3 pi;
        pi.init<E>(deposit3<E>(t, 0, S::S0), valid ? a : 0, N, S::S0);
        load_pairs<E, MIXED>(x, pi, psi, DIM);
        reg_ft3<E, 0, E>(x);
        rounds3<N, 0, E, 1>(x, sm, t, active, SyncCta());
        float mm = 0.f, ss = 0.f, qq = 0.f;
        if (valid) acc_chi<E>(x, mm, ss, qq);
        m += mm; s += ss; q += qq;
        if ((it & 15) == 15 || it + 1 == iters) {  // flush FP32 partials into FP64 every 16 a's
            double v[3];
            cta_sum3(m, s, q, v);
            if (tid == 0) { acc[0] += v[0]; acc[1] += v[1]; acc[2] += v[2]; }
            m = s = q = 0.f;
        }
    }
    if (tid == 0) { out[blockIdx.x * 3] = acc[0]; out[blockIdx.x * 3 + 1] = acc[1]; out[blockIdx.x * 3 + 2] = acc[2]; }
}

// ---------------------------------------------------------------------------------------
// Two passes (9 <= N <= 13).  Scratch of one a: [3^M units][3^8 columns], M = N - 8.
// Pass-2 tile: 3^M rows x 3^(8-M) columns (3^8 values).  243 active threads of 256.
template <int M, bool MIXED>
__global__ void __launch_bounds__(256, 2) mana_twopass(ManaParams P) {
    constexpr int D = 8, TILE = pow3(D), LOGT3 = D - M, T = pow3(LOGT3), TILES = TILE / T;
    constexpr int N = D + M;
    constexpr int64_t PER_A = (int64_t)pow3(N);
    extern __shared__ float2 smem[];
    const uint32_t tid = threadIdx.x;
    const bool act = tid < 243;
    const uint32_t t = act ? tid : 0;
    const int64_t per_stage = (int64_t)P.p1 + P.p2;
    const int64_t total = P.n_batches * per_stage;
    double acc[3] = {0.0, 0.0, 0.0};

    for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
        int64_t g;
        int kind, r;
        if (task < P.p1) { g = 0; kind = 1; r = (int)task; }
        else {
            const int64_t tt = task - P.p1;
            const int64_t st = 1 + tt / per_stage;
            const int rr = (int)(tt % per_stage);
            if (st < P.n_batches && rr < P.p1) { g = st; kind = 1; r = rr; }
            else { g = st - 1; kind = 2; r = (st < P.n_batches) ? rr - P.p1 : rr; }
        }
        const int slot = (int)(g % P.R);
        float2* sbase = P.scratch + (size_t)slot * P.A * PER_A;
        if (kind == 1) {
            if (g >= P.R && !cta_wait_geq(P.done2 + slot, (unsigned)((g / P.R) * P.p2) + P.wait_bias, P.status, P.spin_limit))
                return;
            // one (work item, unit) per task: tile x = unit * 3^8 + l, registers = digits [5, 8) of l
            const int a_idx = r / pow3(M), unit = r % pow3(M);
            const int64_t w = g * P.A + a_idx;
            if (w < P.count) {
                float2 x[27];
                using S = Sched3<D, 0, 3>;
                int64_t a, a2;
                int jd;
                pair_item(w, N, a, a2, jd);
                PairIdx3 pi;
                pi.init<3>((int64_t)unit * TILE + deposit3<3>(t, 0, S::S0), a, N, S::S0);
                if (a2 >= 0) {
                    // digit jd of a is 0 and of a2 is 1; with x's digit xd (a digit of the unit),
                    // both gather indices move by (xd == 0 ? +2 : -1) 3^jd
                    int64_t pj = 1;
                    for (int q = 8; q < jd; ++q) pj *= 3;
                    const int xd = (int)((unit / pj) % 3);
                    load_pairs2<3, MIXED>(x, pi, P.psi, PER_A, (xd == 0 ? 2 : -1) * pj * TILE);
                } else {
                    load_pairs<3, MIXED>(x, pi, P.psi, PER_A);
                }
                reg_ft3<3, 0, 3>(x);
                rounds3<D, 0, 3, 1>(x, smem, t, act, SyncCta());
                if (act) {
                    float2* dst = sbase + a_idx * PER_A + (int64_t)unit * TILE;
                    constexpr int SL = S::shift(S::NR - 1);
#pragma unroll
                    for (int k = 0; k < 27; ++k) __stcg(dst + deposit3<3>(t, k, SL), x[k]);
                }
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                red_release_add(P.done1 + slot, 1u);
            }
        } else {
            if (!cta_wait_geq(P.done1 + slot, (unsigned)((g / P.R + 1) * P.p1) + P.wait_bias, P.status, P.spin_limit))
                return;
            const int a_idx = r / TILES, tile = r % TILES;
            const int64_t w = g * P.A + a_idx;
            if (w < P.count) {
                const float2* src = sbase + a_idx * PER_A + (int64_t)tile * T;
                float2 x[27];
                using S = Sched3<D, LOGT3, 3>;
#pragma unroll
                for (int k = 0; k < 27; ++k) {
                    const uint32_t j = deposit3<3>(t, k, S::S0);  // row * T + col
                    x[k] = __ldcg(src + (int64_t)(j / T) * TILE + (j % T));
                }
                reg_ft3<3, (LOGT3 > S::S0 ? LOGT3 - S::S0 : 0), 3>(x);
                rounds3<D, LOGT3, 3, 1>(x, smem, t, act, SyncCta());
                float m = 0.f, s = 0.f, q = 0.f;
                if (act) acc_chi<3, true>(x, m, s, q);  // a single's imaginary parts are zero
                double v[3];
                cta_sum3(m, s, q, v);
                if (tid == 0) { acc[0] += v[0]; acc[1] += v[1]; acc[2] += v[2]; }
            }
            __syncthreads();
            if (tid == 0) red_release_add(P.done2 + slot, 1u);
        }
    }
    if (tid == 0) {
        P.out[blockIdx.x * 3] = acc[0];
        P.out[blockIdx.x * 3 + 1] = acc[1];
        P.out[blockIdx.x * 3 + 2] = acc[2];
    }
}

// ---------------------------------------------------------------------------------------
template <int N, bool MIXED>
static cudaError_t launch_onepass_n(const float2* psi, double* out, int sm_count, int* grid, cudaStream_t st) {
    constexpr int E = N < 3 ? N : 3;
    constexpr int G = pow3(N - E);
    constexpr int GPC = 256 / G;
    const size_t smem = (size_t)GPC * pow3(N) * sizeof(float2);
    auto k = mana_onepass<N, MIXED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, smem)) != cudaSuccess) return e;
    int64_t need = (pow3(N) + GPC - 1) / GPC;
    int64_t cap = (int64_t)(occ < 1 ? 1 : occ) * sm_count;
    *grid = (int)(need < cap ? need : cap);
    k<<<*grid, 256, smem, st>>>(psi, out);
    return cudaGetLastError();
}

static constexpr size_t kTwoSmem = (size_t)pow3(8) * sizeof(float2);

template <int M, bool MIXED>
static cudaError_t twopass_prep(int* occ) {
    auto k = mana_twopass<M, MIXED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTwoSmem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, 256, kTwoSmem);
}

}  // namespace mana

int mana_tiles_per_a(int N) { return N <= 8 ? 1 : mana::pow3(8) / mana::pow3(16 - N); }

int64_t mana_pair_items(int N) {
    int64_t n = mana::pow3(8);
    for (int k = 0; k < N - 8; ++k) n += mana::pow3(N - 1 - k);
    return n;
}

cudaError_t launch_mana_onepass(const float2* src, int N, bool mixed, double* out, int sm_count, int* grid,
                                cudaStream_t st) {
#define HM_CASE(NN)                                                                              \
    case NN:                                                                                     \
        return mixed ? mana::launch_onepass_n<NN, true>(src, out, sm_count, grid, st)            \
                     : mana::launch_onepass_n<NN, false>(src, out, sm_count, grid, st);
    switch (N) {
        HM_CASE(1) HM_CASE(2) HM_CASE(3) HM_CASE(4) HM_CASE(5) HM_CASE(6) HM_CASE(7) HM_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef HM_CASE
}

// Mixed states have two-pass variants for N = 9, 10 only (rho is 9^N values: 28 GB at N = 10).
cudaError_t mana_twopass_grid(int N, bool mixed, int sm_count, int* grid) {
    int occ = 0;
    cudaError_t e;
    switch (N * 2 + (mixed ? 1 : 0)) {
        case 18: e = mana::twopass_prep<1, false>(&occ); break;
        case 20: e = mana::twopass_prep<2, false>(&occ); break;
        case 22: e = mana::twopass_prep<3, false>(&occ); break;
        case 24: e = mana::twopass_prep<4, false>(&occ); break;
        case 26: e = mana::twopass_prep<5, false>(&occ); break;
        case 19: e = mana::twopass_prep<1, true>(&occ); break;
        case 21: e = mana::twopass_prep<2, true>(&occ); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_mana_twopass(const ManaParams& P, bool mixed, int grid, cudaStream_t st) {
    switch (P.N * 2 + (mixed ? 1 : 0)) {
#define HM_CASE(NN, MX)                                                               \
    case NN * 2 + MX:                                                                 \
        mana::mana_twopass<NN - 8, MX><<<grid, 256, mana::kTwoSmem, st>>>(P);         \
        return cudaGetLastError();
        HM_CASE(9, 0) HM_CASE(10, 0) HM_CASE(11, 0) HM_CASE(12, 0) HM_CASE(13, 0)
        HM_CASE(9, 1) HM_CASE(10, 1)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hm
