// pairs.cuh -- pair-product addressing shared by the SRE forward and gradient kernels.
#pragma once
#include "common.cuh"

namespace hm {

template <int K1, int M>
struct TwoPassShape {
    static constexpr int L = K1 + M;
    static constexpr int LOGT = 13 - M;
    static constexpr int T = 1 << LOGT;
    static constexpr int TILES = (1 << K1) / T;
    static constexpr bool DISCARD = LOGT >= 4;  // tile rows cover whole 128-byte lines
};

// Pair product of Algorithm 2 for tile value j of unit `unit` (the X-string scratch layout is
// [unit][j] with K1 bits of j).  a >= 2^K1: rows h (bit p-K1 clear) and h ^ (a >> K1).
// 0 < a < 2^K1: rows unit and unit + 2^M (top bit of j), pair z, z ^ a inside a row.
// a == 0: pairs (2l', 2l'+1) combined as ((e+o) + i(e-o))/2.
template <int K1, int M>
struct PairRows {
    int64_t rowA, rowB;  // element offsets of the two rows (a >= 2^K1)
    int64_t al;          // low K1 bits of a
    int p;               // msb(a) for 0 < a < 2^K1
    __device__ __forceinline__ PairRows(int64_t a, int64_t unit) {
        if (a >> K1) {
            const int64_t ah = a >> K1;
            const int64_t h = insert0(unit, msb64(ah));
            rowA = h << K1;
            rowB = (h ^ ah) << K1;
            al = a & ((int64_t(1) << K1) - 1);
            p = 0;
        } else {
            rowA = unit << K1;
            rowB = (unit + (int64_t(1) << M)) << K1;
            al = a;
            p = a ? msb64(a) : 0;
        }
    }
    // the same from the two rows staged in shared memory (sA = row A, sB = row B, 2^K1 values each)
    __device__ __forceinline__ float2 value_rows(const float2* sA, const float2* sB, int64_t a, uint32_t j) const {
        if (a >> K1) return conj_mul(sB[j ^ (uint32_t)al], sA[j]);
        const float2* row = (j >> (K1 - 1)) ? sB : sA;
        const uint32_t lp = j & ((1u << (K1 - 1)) - 1u);
        if (a != 0) {
            const uint32_t z = (uint32_t)insert0(lp, p);
            return conj_mul(row[z ^ (uint32_t)a], row[z]);
        }
        const float2 u = row[lp << 1], v = row[(lp << 1) + 1];
        float e = fmaf(u.x, u.x, u.y * u.y), o = fmaf(v.x, v.x, v.y * v.y);
        return make_float2(0.5f * (e + o), 0.5f * (e - o));
    }
    __device__ __forceinline__ float2 value(const float2* __restrict__ psi, int64_t a, uint32_t j) const {
        if (a >> K1) return conj_mul(ld_amp(psi, rowB + (int64_t)(j ^ (uint32_t)al)), ld_amp(psi, rowA + j));
        const int64_t row = (j >> (K1 - 1)) ? rowB : rowA;
        const int64_t lp = j & ((1u << (K1 - 1)) - 1u);
        if (a != 0) {
            const int64_t z = row + insert0(lp, p);
            return conj_mul(ld_amp(psi, z ^ a), ld_amp(psi, z));
        }
        const int64_t z = row + (lp << 1);
        float2 u = ld_amp(psi, z), v = ld_amp(psi, z + 1);
        float e = fmaf(u.x, u.x, u.y * u.y), o = fmaf(v.x, v.x, v.y * v.y);
        return make_float2(0.5f * (e + o), 0.5f * (e - o));
    }
};


// Shared-memory slots of a pass-1 row staging (2 units x own/partner row of 2^10 values).
constexpr uint32_t kStageSlots = 4u << 10;

// Copies the four state rows that the pair products of X-string a on units unit and unit + 1
// read (PairRows' row A and row B of each unit, 2^10 values each) into rows[0 .. 4 x 2^10):
// unit uu's rows at rows + 2048 uu (row A) and + 1024 (row B).  With perm != 0 row B is stored
// with its 32-value blocks permuted: staged position (X << 5) | w holds B[((X ^ perm) << 5) | w],
// so that a far X-string's partner value B[j ^ al] (j = (k << 5) | lane, perm = al >> 5) sits at
// (k << 5) | (lane ^ (al & 31)).  cp.async by the 256 threads of the CTA; every thread returns
// once the copy has landed (one CTA barrier).
template <int M>
__device__ __forceinline__ void stage_rows(float2* rows, const float2* __restrict__ psi, int64_t a, int64_t unit,
                                           uint32_t perm = 0) {
    int64_t rb[4];
#pragma unroll
    for (int uu = 0; uu < 2; ++uu) {
        const PairRows<10, M> pr(a, unit + uu);
        rb[2 * uu] = pr.rowA;
        rb[2 * uu + 1] = pr.rowB;
    }
    // 2048 16-byte chunks, 8 per thread: chunk tid + 256 q is in row q / 2 at value offset
    // 2 (tid + 256 (q % 2))
    const uint32_t tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t off = (tid + 256u * (q & 1)) * 2u;
        const uint32_t dst = (q >> 1) & 1 ? ((((off >> 5) ^ perm) << 5) | (off & 31u)) : off;
        cp_async16(rows + (q >> 1) * 1024u + dst, psi + rb[q >> 1] + off);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
}

// Pair product of the half-length form for z' (no unit split; used by the one-pass kernels).
__device__ __forceinline__ float2 pair_product(const float2* __restrict__ psi, int64_t zp, int64_t a, int p) {
    if (a != 0) {
        int64_t z = insert0(zp, p);
        return conj_mul(ld_amp(psi, z ^ a), ld_amp(psi, z));
    }
    int64_t z = zp << 1;
    float2 u = ld_amp(psi, z), v = ld_amp(psi, z + 1);
    float e = fmaf(u.x, u.x, u.y * u.y), o = fmaf(v.x, v.x, v.y * v.y);
    return make_float2(0.5f * (e + o), 0.5f * (e - o));
}

}  // namespace hm
