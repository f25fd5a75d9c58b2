// sre_tc.cu -- exact SRE with the Walsh-Hadamard transform on tcgen05 tensor cores.
//
// For every X-string a the half-length vector w (common.cuh) of 2^L complex values, L = N - 1,
// is transformed by H^{(x)L} written as a product of Kronecker blocks, each a dense +-1 matrix
// product on the tensor core (the transform of Algorithm 2 regrouped; see the FWHT structure of
// Sec. 3):
//   pass 1 (tile = 2^13 values sharing z' bits [13, L)):
//     block 1: bits [0, 7)  -- rows (re/im, bits 7..12) x K = 128, times H_128
//     block 2: bits [7, 13) -- rows (bits 0..6) x K = 64, per re/im, times H_64
//   pass 2 (tile = 128 fibres along bits [13, 20), bits [20, L) butterflied in registers first):
//     block 3: bits [13, 20) -- rows (fibres) x K = 128, times H_128, then sum |.|^{2n}.
// Precision form: every operand x is split as x = hi + 2^-11 lo, hi = fp16(x),
// lo = fp16(2^11 (x - hi)) (a normal fp16 number wherever x is, so ~22 significant bits);
// D = hi*H + 2^-11 lo*H accumulates in fp32 in tensor memory (the 2^-11 is the MMA's
// scale-input-d).  The state is first scaled by a power
// of two 2^f (chosen from max|psi|^2) so that every fp16 operand stays in range; the per-CTA
// FP64 sums are unscaled exactly at the end.  FP64 is used only for the cross-tile sums.
//
// Schedule: one CTA of 512 threads per SM, split into two independent groups of 256 threads
// (warps 0-7 and 8-15) with their own named barriers, mbarriers and inter-CTA waits:
//   pass-1 group: staged pair products -> MMA1 -> block-1/block-2 conversion -> MMA2;
//   pass-2 group: scratch -> register butterflies -> MMA3 -> reduction, then the store of the
//                 block-2 result of the matching pass-1 tile to scratch.
// Block 2 has its own tensor-memory columns, handed over by two mbarriers ("full" from the
// MMA2 commit, "free" once the pass-2 group has read it), so the pass-1 group never waits on
// another CTA.  The pair-product inputs of pass 1 (two 8 KiB state rows per eighth of a tile)
// arrive by bulk asynchronous copies into four staging buffers, issued two eighths ahead (and
// across tiles), so the producer reads shared memory only.
#include "common.cuh"
#include "pairs.cuh"
#include "sre_tc.h"
#include "tc.cuh"

namespace hm {

namespace {

// Shared-memory map (bytes from a 1024-byte aligned base).
constexpr uint32_t SM_H = 0;          // H_128, B operand, K-major, no swizzle, 32 KiB
constexpr uint32_t SM_P = 32768;      // pass-1 operands (block 1, then block 2), 64 KiB
constexpr uint32_t SM_Q = 98304;      // pass-2 operand (block 3), 64 KiB
constexpr uint32_t SM_ST = 163840;    // staging: 4 buffers x (own 8 KiB | partner 8 KiB)
constexpr uint32_t SM_BYTES = 229376;
constexpr uint32_t SM_DYN = SM_BYTES + 1024;  // + alignment slack
constexpr uint32_t CHUNK = 1024;              // complex values per staged eighth of a tile

// No-swizzle canonical layouts for 128 rows: core matrices of 8 rows x 16 bytes.
//   K-major, K = 128: core (row/8, kc) at (row/8)*2048 + kc*128;  row%8 at 16 B.
//   MN-major (any K):  core (rc, k/8) at (k/8)*2048 + rc*128;     k%8 at 16 B.
__device__ __forceinline__ uint32_t kmaj(uint32_t row, uint32_t kc) { return (row >> 3) * 2048u + kc * 128u + (row & 7u) * 16u; }
__device__ __forceinline__ uint32_t mnmaj(uint32_t rc, uint32_t k) { return (k >> 3) * 2048u + rc * 128u + (k & 7u) * 16u; }
// MN-major 128-byte swizzle, 128 rows x K = 128: atom (row/64, k/8) of 8 K-rows x 128 B at
// (row/64)*16384 + (k/8)*1024; 16-byte chunk (row%64)/8 of K-row k%8 stored at chunk ^ (k%8).
__device__ __forceinline__ uint32_t mnsw(uint32_t rg, uint32_t k) {  // rg = row / 8
    return (rg >> 3) * 16384u + (k >> 3) * 1024u + (k & 7u) * 128u + (((rg & 7u) ^ (k & 7u)) << 4);
}

// Descriptor strides: LBO = distance of core matrices along K, SBO = along M/N (no swizzle);
// for the swizzled MN-major form LBO = MN-atom distance, SBO = 8-K-row group distance.
constexpr uint32_t KM_LBO = 128, KM_SBO = 2048, KM_STEP = 256;    // K-major, one K=16 step = 2 cores
constexpr uint32_t MN_LBO = 2048, MN_SBO = 128, MN_STEP = 4096;   // MN-major, one K=16 step = 2 K-groups
constexpr uint32_t SW_LBO = 16384, SW_SBO = 1024, SW_STEP = 2048; // MN-major 128B swizzle

constexpr uint32_t ID_B1 = tc::idesc_f16(128, 128, true, false);
constexpr uint32_t ID_B2 = tc::idesc_f16(128, 64, true, false);
constexpr uint32_t ID_B3 = tc::idesc_f16(128, 128, true, false);

// D = (A_hi + 2^-LO_SHIFT A_lo) x H over NK K-steps of 16 (the hi/lo split as a longer K): the lo
// steps accumulate A_lo x H first, then the first hi step scales that partial sum by
// 2^-LO_SHIFT (scale-input-d, exact in fp32) while adding its own product.
template <int NK, uint32_t LBO, uint32_t SBO, uint32_t STEP, uint32_t LAYOUT>
__device__ __forceinline__ void issue_block(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t h, uint32_t idesc) {
#pragma unroll
    for (int j = 0; j < NK; ++j)
        tc::mma_f16(d, tc::sdesc(a_lo + j * STEP, LBO, SBO, LAYOUT), tc::sdesc(h + j * KM_STEP, KM_LBO, KM_SBO), idesc, j > 0);
    tc::mma_f16_scale_d<tc::LO_SHIFT>(d, tc::sdesc(a_hi, LBO, SBO, LAYOUT), tc::sdesc(h, KM_LBO, KM_SBO), idesc);
#pragma unroll
    for (int j = 1; j < NK; ++j)
        tc::mma_f16(d, tc::sdesc(a_hi + j * STEP, LBO, SBO, LAYOUT), tc::sdesc(h + j * KM_STEP, KM_LBO, KM_SBO), idesc, true);
}

// Block-1 operand row group: 8 fibres (m6 = 8 consecutive values, re and im) at K = n, split
// into hi/lo and stored in the swizzled MN-major images (re rows 0..63, im rows 64..127).
__device__ __forceinline__ void put_block1(const float (&re)[8], const float (&im)[8], uint32_t fg, uint32_t n,
                                           uint32_t a_hi, uint32_t a_lo) {
    uint4 hi, lo;
    tc::split8(re, hi, lo);
    tc::sts128(a_hi + mnsw(fg, n), hi);
    tc::sts128(a_lo + mnsw(fg, n), lo);
    tc::split8(im, hi, lo);
    tc::sts128(a_hi + mnsw(8u + fg, n), hi);
    tc::sts128(a_lo + mnsw(8u + fg, n), lo);
}

// Pass-1 producer for a < 2^13 (pairs inside the tile, or the a = 0 row): direct loads.
template <int M>
__device__ __forceinline__ void produce_near(const float2* __restrict__ psi, const PairRows<13, M>& pr, int64_t a,
                                             uint32_t tid, uint32_t a_hi, uint32_t a_lo) {
    const uint32_t n = tid & 127u;
    for (uint32_t fg = tid >> 7; fg < 8u; fg += 2u) {
        float re[8], im[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float2 w = pr.value(psi, a, ((fg * 8u + e) << 7) | n);
            re[e] = w.x;
            im[e] = w.y;
        }
        put_block1(re, im, fg, n, a_hi, a_lo);
    }
}

// All threads wait for phase `ph` of `mbar`; uniform result.  On a timeout the status word is
// set and the threads that gave up wait once more (bounded) so that outstanding asynchronous
// work drains before the caller frees its resources.
// The CTA runs two independent groups of 256 threads (warps 0-7: pass 1, warps 8-15:
// pass 2); each synchronises on its own named barrier (id 1 + group).
__device__ __forceinline__ void gsync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }
__device__ __forceinline__ int gsync_or(int id, int pred) {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.b32 p, %2, 0;\n bar.red.or.pred q, %1, 256, p;\n selp.s32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(id), "r"(pred)
        : "memory");
    return r;
}

// All threads of a group wait for phase `ph` of `mbar`; uniform result.  On a timeout the
// status word is set and the threads that gave up wait once more (bounded) so that
// outstanding asynchronous work drains before the caller frees its resources.
__device__ __forceinline__ bool wait_bar(uint64_t* mbar, uint32_t& ph, int* status, long long limit, int id) {
    const bool good = tc::mbar_wait(mbar, ph, limit);
    const int bad = gsync_or(id, !good);
    if (bad) {
        if ((threadIdx.x & 255u) == 0) atomicOr(status, ST_TIMEOUT);
        if (!good) tc::mbar_wait(mbar, ph, limit);
    }
    ph ^= 1u;
    tc::fence_after();
    return !bad;
}

// Operand writes (generic proxy) -> visible to the MMA, all threads of the group past here.
__device__ __forceinline__ void publish_operands(int id) {
    tc::fence_async_smem();
    tc::fence_before();
    gsync(id);
    tc::fence_after();
}

// Bounded wait of a group on an inter-CTA counter (leader polls); uniform result.
__device__ __forceinline__ bool gwait_geq(const unsigned* ctr, unsigned target, int* status, long long limit, int id,
                                          int* flag) {
    if ((threadIdx.x & 255u) == 0) {
        long long it = 0;
        int good = 1;
        while (ld_acquire(ctr) < target) {
            if (ld_status(status) != 0) { good = 0; break; }
            if (++it > limit) { atomicOr(status, ST_TIMEOUT); good = 0; break; }
            __nanosleep(100);
        }
        if (good && ld_status(status) != 0) good = 0;
        *flag = good;
    }
    gsync(id);
    const int r = *flag;
    gsync(id);
    return r != 0;
}

// Scaled FP64 triple [S_q, S_1, T_1] -> true values.  psi was multiplied by 2^f and the
// reduced values by 2^-RS, so c by sigma = 2^(2f - RS); ls = log2(sigma^2) is an integer.
template <int MODE, int RS>
__device__ __forceinline__ void unscale(const double (&t)[3], int f, double nq, double* out) {
    const int ls = 4 * f - 2 * RS;
    const double S1 = ldexp(t[1], -ls);
    if constexpr (MODE == 1) {
        out[0] = S1;
        out[2] = ldexp(t[2], -ls) - (double)ls * S1;
    } else {
        out[0] = (MODE == 0) ? t[0] * exp2(-nq * ls) : ldexp(t[0], -MODE * ls);
        out[2] = 0.0;
    }
    out[1] = S1;
}

// Pass-1 work of one item: X-string a (far: a >= 2^13), tile h; rows of the state it reads.
struct P1Item {
    int64_t a = -1, h = 0;
    bool far = false;
};

}  // namespace

// ------------------------------------------------------------------------------------------
// Persistent kernel, 512 threads, one CTA per SM, static round-robin over work items.  Work
// item c: stage s = c / T, tile r = c % T (T = 2^M tiles per X-string, one X-string per batch);
// the pass-1 group does pass-1 tile r of batch s (s < n_batches), the pass-2 group pass-2
// tile r of batch s - 2 (s >= 2) and the scratch store of pass-1 tile r of batch s.  R
// scratch slots; batch g uses slot g % R (R >= 3).
// Scratch of one X-string: floats [re/im][h = z' >> 13][q][n][m' & 3] with z' & 8191 =
// (m' << 7) | n and q = m' >> 2 (pass 1 writes 16-byte rows, pass 2 reads 32-byte runs).
template <int MODE, int RB>
__global__ void __launch_bounds__(512, 1) sre_tc(TcParams P) {
    constexpr int M = 7 + RB;         // z' bits above the pass-1 tile
    constexpr int L = 13 + M;
    constexpr int T = 1 << M;         // tiles per X-string (pass 1 and pass 2 alike)
    constexpr int S = 64 >> RB;       // l-slots per pass-2 tile
    constexpr int OCT = S / 8;
    constexpr int ITER2 = (16 * 2 * OCT) / 32;
    // n = 3 sums |c|^6 in fp32: values are brought down by 2^-RS first so that a fully
    // coherent transform (|c| up to 2^L in scaled units) cannot overflow
    constexpr int RS = MODE == 3 ? 8 : 0;
    constexpr float RSF = MODE == 3 ? 1.f / 256.f : 1.f;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mb_p1, mb_p2, mb_d2full, mb_d2free, mb_st[4];
    __shared__ uint32_t tmem_slot;
    __shared__ int gflag[2];
    __shared__ double red64[8][3];
    const uint32_t tid = threadIdx.x, group = tid >> 8, gtid = tid & 255u;
    const uint32_t lane = tid & 31u, gwarp = gtid >> 5;
    const uint32_t quarter = gwarp & 3u, half = gwarp >> 2;
    const int bid = 1 + (int)group;  // this group's named barrier
    const uint32_t sbase = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t sH = sbase + SM_H, sP = sbase + SM_P, sQ = sbase + SM_Q, sST = sbase + SM_ST;

    // H_128 image: row n, K-chunk kc holds H[8kc .. 8kc+7][n] = (-1)^popc(k & n) in fp16.
    for (uint32_t i = tid; i < 128u * 16u; i += 512u) {
        const uint32_t n = i >> 4, kc = i & 15u;
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t k0 = kc * 8u + 2u * e;
            const uint32_t lo = (__popc(k0 & n) & 1) ? 0xBC00u : 0x3C00u;
            const uint32_t hi = (__popc((k0 + 1u) & n) & 1) ? 0xBC00u : 0x3C00u;
            w[e] = lo | (hi << 16);
        }
        tc::sts128(sH + kmaj(n, kc), make_uint4(w[0], w[1], w[2], w[3]));
    }
    if (tid < 32) tc::tmem_alloc(&tmem_slot, 512);
    if (tid == 0) {
        tc::mbar_init(&mb_p1, 1);
        tc::mbar_init(&mb_p2, 1);
        tc::mbar_init(&mb_d2full, 1);
        tc::mbar_init(&mb_d2free, 1);
        for (int b = 0; b < 4; ++b) tc::mbar_init(&mb_st[b], 1);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tq = tmem + ((quarter * 32u) << 16);  // this warp's lane quarter

    const float2* __restrict__ psi = P.psi;
    const int64_t dim = int64_t(1) << P.N;
    const int64_t total = (P.n_batches + 2) * T;
    double accw[3] = {0.0, 0.0, 0.0};  // pass-2 group, lane 0 of each warp: FP64 tile sums
    bool ok = true;

    // X-string of batch g (-1 if the batch does not exist, -2 if the entry is out of range)
    auto xstring = [&](int64_t g) -> int64_t {
        if (g < 0 || g >= P.n_batches || g >= P.count) return -1;
        const int64_t a = P.a_list ? P.a_list[g] : g;
        return (a >= 0 && a < dim) ? a : -2;
    };

    if (group == 0) {
        // ================= pass 1: pair products -> blocks 1 and 2 (the store of block 2 is
        // done by the pass-2 group, which frees its accumulator through mb_d2free) ============
        uint32_t ph1 = 0, phs[4] = {0, 0, 0, 0}, ph_full = 0, ph_free = 0;
        bool mma2_out = false;  // an MMA2 was issued whose completion this group has not seen
        bool d2_used = false;   // block-2 accumulator holds a tile the pass-2 group must store
        int pending[4] = {0, 0, 0, 0};  // staged copies issued and not yet consumed, per buffer
        auto p1_item = [&](int64_t c) {
            P1Item it;
            if (c >= total) return it;
            it.h = c % T;
            it.a = xstring(c / T);
            it.far = it.a >= 8192;
            return it;
        };
        // leader: bulk copies of eighth k of a far item (own and partner rows) into buffer k & 3
        auto stage = [&](const P1Item& it, int k) {
            const PairRows<13, M> pr(it.a, it.h);
            const uint32_t buf = sST + (uint32_t)(k & 3) * 16384u;
            const int64_t jk = (int64_t)k * CHUNK;
            tc::expect_tx(&mb_st[k & 3], 2u * CHUNK * 8u);
            tc::bulk_g2s(buf, psi + pr.rowA + jk, CHUNK * 8u, &mb_st[k & 3]);
            tc::bulk_g2s(buf + 8192u, psi + pr.rowB + (jk ^ (pr.al & 0x1C00)), CHUNK * 8u, &mb_st[k & 3]);
        };
        auto stage4 = [&](const P1Item& it) {  // eighths 0..3 (every buffer)
            if (gtid == 0) for (int k = 0; k < 4; ++k) stage(it, k);
            pending[0] = pending[1] = pending[2] = pending[3] = 1;
        };
        P1Item cur = p1_item(blockIdx.x);
        bool staged = false;  // eighths 0..3 of `cur` are in flight
        if (cur.far) {
            stage4(cur);
            staged = true;
        }
        for (int64_t c = blockIdx.x; c < total && ok; c += gridDim.x) {
            const int64_t g1 = c / T;
            const P1Item nxt = p1_item(c + gridDim.x);
            bool nxt_staged = false;
            if (g1 >= P.n_batches) { cur = nxt; staged = false; continue; }  // group-uniform
            const int64_t a1 = cur.a;
            if (a1 == -2 && gtid == 0) atomicOr(P.status, ST_BADARG);
            const bool do1 = a1 >= 0;
            if (do1) {
                // the previous MMA2 read its operand from the region block 1 is about to overwrite
                if (mma2_out) {
                    if (!wait_bar(&mb_d2full, ph_full, P.status, P.spin_limit, bid)) { ok = false; break; }
                    mma2_out = false;
                }
                // ---- block 1 operand (MN-major, swizzled) from staged or directly loaded rows ----
                const uint32_t a_hi = sP, a_lo = sP + 32768u;
                if (cur.far) {
                    if (!staged) stage4(cur);
                    const uint32_t al_lo = (uint32_t)(PairRows<13, M>(cur.a, cur.h).al) & (CHUNK - 1u);
                    // eighth k holds m6 in [8k, 8k + 8) (fibre group k); step p: thread (n, hh)
                    // builds fibre group 2p + hh from eighth 2p + hh
                    const uint32_t n = gtid & 127u, hh = gtid >> 7;
                    for (int p = 0; p < 4 && ok; ++p) {
                        const int b0 = (2 * p) & 3, b1 = (2 * p + 1) & 3;
                        ok = wait_bar(&mb_st[b0], phs[b0], P.status, P.spin_limit, bid) &&
                             wait_bar(&mb_st[b1], phs[b1], P.status, P.spin_limit, bid);
                        pending[b0] = pending[b1] = 0;
                        if (!ok) break;
                        const uint32_t own = sST + (uint32_t)((2 * p + hh) & 3) * 16384u, par = own + 8192u;
                        float re[8], im[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t jl = ((uint32_t)e << 7) | n;  // j & 1023
                            const float2 u = tc::lds64(own + jl * 8u);
                            const float2 v = tc::lds64(par + (jl ^ al_lo) * 8u);
                            const float2 w = conj_mul(v, u);
                            re[e] = w.x;
                            im[e] = w.y;
                        }
                        put_block1(re, im, 2u * p + hh, n, a_hi, a_lo);
                        gsync(bid);  // buffers b0, b1 consumed
                        if (p < 2 || nxt.far) {
                            if (gtid == 0) {
                                if (p < 2) { stage(cur, 2 * p + 4); stage(cur, 2 * p + 5); }
                                else { stage(nxt, 2 * p - 4); stage(nxt, 2 * p - 3); }
                            }
                            pending[b0] = pending[b1] = 1;
                        }
                    }
                    nxt_staged = nxt.far;
                } else {
                    produce_near<M>(psi, PairRows<13, M>(cur.a, cur.h), cur.a, gtid, a_hi, a_lo);
                }
                if (!ok) break;
                publish_operands(bid);
                if (gtid == 0) {
                    issue_block<8, SW_LBO, SW_SBO, SW_STEP, 2>(tmem, a_hi, a_lo, sH, ID_B1);
                    tc::commit(&mb_p1);
                }
            }
            if (!nxt_staged && nxt.far) {  // this item staged nothing for the next one
                stage4(nxt);
                nxt_staged = true;
            }
            if (do1) {
                // ---- block 1 result (rows (re/im, m6), cols n) -> block 2 operand -> MMA2 ----
                if (!wait_bar(&mb_p1, ph1, P.status, P.spin_limit, bid)) { ok = false; break; }
                const uint32_t row = quarter * 32u + lane, cc = row >> 6, m6 = row & 63u;
                float v[64];
                tc::tmem_ld32(tq + half * 64u, *reinterpret_cast<float(*)[32]>(v));
                tc::tmem_ld32(tq + half * 64u + 32u, *reinterpret_cast<float(*)[32]>(v + 32));
                tc::tmem_wait_ld();
                const uint32_t b_hi = sP + cc * 32768u, b_lo = b_hi + 16384u;
#pragma unroll
                for (int gq = 0; gq < 8; ++gq) {
                    uint4 hi, lo;
                    tc::split8(v + 8 * gq, hi, lo);
                    const uint32_t o = mnmaj(half * 8u + gq, m6);
                    tc::sts128(b_hi + o, hi);
                    tc::sts128(b_lo + o, lo);
                }
                // the block-2 accumulator must have been read out by the pass-2 group
                if (d2_used && !wait_bar(&mb_d2free, ph_free, P.status, P.spin_limit, bid)) { ok = false; break; }
                publish_operands(bid);
                if (gtid == 0) {
                    issue_block<4, MN_LBO, MN_SBO, MN_STEP, 0>(tmem + 256u, sP, sP + 16384u, sH, ID_B2);
                    issue_block<4, MN_LBO, MN_SBO, MN_STEP, 0>(tmem + 320u, sP + 32768u, sP + 49152u, sH, ID_B2);
                    tc::commit(&mb_d2full);
                }
                mma2_out = true;
                d2_used = true;
            }
            cur = nxt;
            staged = nxt_staged;
        }
        // drain staged copies (error exits) and the last MMA2
        for (int b = 0; b < 4; ++b)
            if (pending[b]) tc::mbar_wait(&mb_st[b], phs[b], P.spin_limit);
        if (mma2_out) tc::mbar_wait(&mb_d2full, ph_full, P.spin_limit);
    } else {
        // ================= pass 2: scratch -> block 3 -> sum of |.|^{2n} ======================
        uint32_t ph2 = 0, ph_full = 0;
        for (int64_t c = blockIdx.x; c < total && ok; c += gridDim.x) {
            const int64_t g2 = c / T - 2;
            const int r = (int)(c % T);
            const bool has2 = g2 >= 0 && g2 < P.n_batches;  // group-uniform
            const int slot2 = has2 ? (int)(g2 % P.R) : 0;
            const bool do2 = has2 && xstring(g2) >= 0;
            if (do2) {
                const unsigned need = (unsigned)((g2 / P.R + 1) * T) + P.wait_bias;
                if (!gwait_geq(P.done1 + slot2, need, P.status, P.spin_limit, bid, &gflag[1])) { ok = false; break; }
                const float* scr2 = P.scratch + (size_t)slot2 * ((size_t)2 << L);
                const uint32_t q_hi = sQ, q_lo = sQ + 32768u;
                const uint32_t h7_lo = gtid & 7u, rest = gtid >> 3;
#pragma unroll
                for (int it = 0; it < ITER2; ++it) {
                    const uint32_t combo = rest + 32u * it;
                    const uint32_t oct = combo % OCT, cc = (combo / OCT) & 1u, h7 = ((combo / (2 * OCT)) << 3) | h7_lo;
                    float x[1 << RB][8];
#pragma unroll
                    for (int rc = 0; rc < (1 << RB); ++rc)
                        tc::ldcg256(scr2 + (size_t)cc * ((size_t)1 << L) + (size_t)(h7 + 128u * rc) * 8192u +
                                        (size_t)r * S + oct * 8u,
                                    x[rc]);
#pragma unroll
                    for (int b = 0; b < RB; ++b)
#pragma unroll
                        for (int rc = 0; rc < (1 << RB); ++rc)
                            if (!(rc & (1 << b))) {
#pragma unroll
                                for (int e = 0; e < 8; e += 2) {
                                    const float2 p = make_float2(x[rc][e], x[rc][e + 1]);
                                    const float2 q = make_float2(x[rc | (1 << b)][e], x[rc | (1 << b)][e + 1]);
                                    const float2 s0 = add2(p, q), s1 = sub2(p, q);
                                    x[rc][e] = s0.x; x[rc][e + 1] = s0.y;
                                    x[rc | (1 << b)][e] = s1.x; x[rc | (1 << b)][e + 1] = s1.y;
                                }
                            }
#pragma unroll
                    for (int rc = 0; rc < (1 << RB); ++rc) {
                        uint4 hi, lo;
                        tc::split8(x[rc], hi, lo);
                        const uint32_t o = mnmaj(((rc * 2u + cc) * S + oct * 8u) >> 3, h7);
                        tc::sts128(q_hi + o, hi);
                        tc::sts128(q_lo + o, lo);
                    }
                }
                publish_operands(bid);
                if (gtid == 0) {
                    issue_block<8, MN_LBO, MN_SBO, MN_STEP, 0>(tmem + 128u, q_hi, q_lo, sH, ID_B3);
                    tc::commit(&mb_p2);
                }
                if constexpr (S * 4 >= 128) {
                    // drop the tile's lines from L2 unwritten
                    constexpr int LPR = (S * 4) / 128;
                    for (int qd = gtid; qd < 2 * (1 << M) * LPR; qd += 256) {
                        const int row = qd / LPR;  // (re/im, h)
                        discard_l2_line(scr2 + (size_t)row * 8192u + (size_t)r * S + (qd % LPR) * 32);
                    }
                }
                // the tile's scratch has been read and dropped: the slot may be refilled (the
                // release must follow the discards, or a refill could land before a discard)
                gsync(bid);
                if (gtid == 0) red_release_add(P.done2 + slot2, 1u);
                if (!wait_bar(&mb_p2, ph2, P.status, P.spin_limit, bid)) { ok = false; break; }
                float v[64];
                tc::tmem_ld32(tq + 128u + half * 64u, *reinterpret_cast<float(*)[32]>(v));
                tc::tmem_ld32(tq + 128u + half * 64u + 32u, *reinterpret_cast<float(*)[32]>(v + 32));
                tc::tmem_wait_ld();
                tc::fence_before();
                Acc<MODE> ac;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    float2 w = make_float2(v[2 * k], v[2 * k + 1]);
                    if constexpr (RS != 0) w = mul2(w, make_float2(RSF, RSF));
                    ac.add(w, P.nq);
                }
                ac.fold();
                float q = ac.q, s1 = ac.s1, uu = ac.u;
                double qd = ac.qd;
                warp_sum3<MODE>(q, s1, uu, qd, 32);
                if (lane == 0) {
                    // FP32 warp partial -> FP64; warps accumulate independently
                    double vv[3];
                    finish3<MODE>(q, s1, uu, qd, P.nq, vv);
                    if (P.per_a) unscale<MODE, RS>(vv, *P.scale_exp, P.nq, P.out + (((size_t)g2 * T + r) * 8 + gwarp) * 3);
                    else { accw[0] += vv[0]; accw[1] += vv[1]; accw[2] += vv[2]; }
                }
            } else if (has2 && gtid == 0) {
                red_release_add(P.done2 + slot2, 1u);  // nothing to read (invalid entry): keep counts
            }
            // ---- pass-1 tile of this item: block-2 result (rows n, cols (re/im, m')) -> scratch ----
            const int64_t g1 = c / T;
            if (g1 < P.n_batches) {
                const int slot1 = (int)(g1 % P.R);
                if (g1 >= P.R) {  // the slot is free once pass 2 of batch g1 - R has read it
                    const unsigned need = (unsigned)((g1 / P.R) * T) + P.wait_bias;
                    if (!gwait_geq(P.done2 + slot1, need, P.status, P.spin_limit, bid, &gflag[1])) { ok = false; break; }
                }
                if (xstring(g1) >= 0) {
                    if (!wait_bar(&mb_d2full, ph_full, P.status, P.spin_limit, bid)) { ok = false; break; }
                    float* scr1 = P.scratch + (size_t)slot1 * ((size_t)2 << L);
                    const uint32_t n = quarter * 32u + lane, cc = half;
                    float v[64];
                    tc::tmem_ld32(tq + 256u + cc * 64u, *reinterpret_cast<float(*)[32]>(v));
                    tc::tmem_ld32(tq + 256u + cc * 64u + 32u, *reinterpret_cast<float(*)[32]>(v + 32));
                    tc::tmem_wait_ld();
                    tc::fence_before();
                    gsync(bid);
                    if (gtid == 0) tc::mbar_arrive(&mb_d2free);  // the accumulator may be rewritten
                    float* dst = scr1 + (size_t)cc * ((size_t)1 << L) + (size_t)(c % T) * 8192u + n * 4u;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        __stcg(reinterpret_cast<float4*>(dst + q * 512),
                               make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                }
                gsync(bid);
                if (gtid == 0) red_release_add(P.done1 + slot1, 1u);
            }
        }
    }
    // both groups done: no MMA is in flight (each commit was waited on)
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc(tmem, 512);
    if (!P.per_a) {
        if (group == 1 && lane == 0) { red64[gwarp][0] = accw[0]; red64[gwarp][1] = accw[1]; red64[gwarp][2] = accw[2]; }
        __syncthreads();
        if (tid == 0) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int w = 0; w < 8; ++w) { acc[0] += red64[w][0]; acc[1] += red64[w][1]; acc[2] += red64[w][2]; }
            unscale<MODE, RS>(acc, *P.scale_exp, P.nq, P.out + blockIdx.x * 3);
        }
    }
}

// ------------------------------------------------------------------------------------------
// max |psi_z|^2 as the bit pattern of a non-negative float (atomicMax on the pattern orders it).
__global__ void tc_absmax(const float2* __restrict__ psi, int64_t n, unsigned* __restrict__ out) {
    float m = 0.f;
    for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < n; z += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = __ldg(psi + z);
        m = fmaxf(m, fmaf(v.x, v.x, v.y * v.y));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// psi' = 2^f psi with f = floor(e/2) - extra, e = floor(-log2 max|psi|^2): every |w| <= 2^(-2 extra).
__global__ void tc_scale(const float2* __restrict__ psi, int64_t n, const unsigned* __restrict__ mx, int extra,
                         float2* __restrict__ out, int* __restrict__ f_out) {
    const float m = __uint_as_float(*mx);
    int f = 0;
    if (m > 0.f) {
        const int e = (int)floor(-log2((double)m));
        f = (e >= 0 ? e / 2 : -((-e + 1) / 2)) - extra;
    }
    const float sc = ldexpf(1.f, f);
    for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < n; z += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = __ldg(psi + z);
        out[z] = make_float2(v.x * sc, v.y * sc);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *f_out = f;
}

// ------------------------------------------------------------------------------------------
template <int MODE, int RB>
static cudaError_t tc_prep(int* occ) {
    auto k = sre_tc<MODE, RB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_DYN);
    if (e != cudaSuccess) return e;
    // one CTA with 225 KiB of shared memory needs the largest shared-memory carveout
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, 512, SM_DYN);
}

template <int MODE>
static cudaError_t tc_dispatch(const TcParams* P, int N, int* occ, int grid, cudaStream_t st) {
    switch (N) {
#define HM_CASE(NN)                                                                 \
    case NN:                                                                        \
        if (occ) return tc_prep<MODE, NN - 21>(occ);                                \
        sre_tc<MODE, NN - 21><<<grid, 512, SM_DYN, st>>>(*P);                        \
        return cudaGetLastError();
        HM_CASE(21) HM_CASE(22) HM_CASE(23) HM_CASE(24)
#undef HM_CASE
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t tc_mode(const TcParams* P, int N, int mode, int* occ, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: return tc_dispatch<0>(P, N, occ, grid, st);
        case 1: return tc_dispatch<1>(P, N, occ, grid, st);
        case 2: return tc_dispatch<2>(P, N, occ, grid, st);
        default: return tc_dispatch<3>(P, N, occ, grid, st);
    }
}

cudaError_t tc_max_grid(int N, int mode, int sm_count, int* grid) {
    int occ = 0;
    cudaError_t e = tc_mode(nullptr, N, mode, &occ, 0, nullptr);
    if (e != cudaSuccess) return e;
    if (occ > 1) occ = 1;  // one CTA per SM: 224 KiB of shared memory, 256 TMEM columns
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_tc(const TcParams& P, int mode, int grid, cudaStream_t st) {
    return tc_mode(&P, P.N, mode, nullptr, grid, st);
}

cudaError_t launch_tc_scale(const float2* psi, int N, unsigned* mx, int* f_out, float2* out, cudaStream_t st) {
    const int64_t n = int64_t(1) << N;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    tc_absmax<<<blocks, 256, 0, st>>>(psi, n, mx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tc_scale<<<blocks, 256, 0, st>>>(psi, n, mx, N >= 24 ? 1 : 0, out, f_out);
    return cudaGetLastError();
}

}  // namespace hm
