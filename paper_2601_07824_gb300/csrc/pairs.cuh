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
