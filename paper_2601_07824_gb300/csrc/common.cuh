// common.cuh -- device helpers shared by the hadamag kernels (sm_103a).
//
// Conventions used by every kernel in this library
//   * A qubit state psi has 2^N amplitudes; bit j of the index z is qubit j.
//   * For an X-string a the paper's Algorithm 2 forms v_a(z) = conj(psi_{z^a}) psi_z and
//     takes its unnormalised Walsh-Hadamard transform c_a = H^{(x)N} v_a (Eq. Z_ovN_simplified).
//   * Half-length form used on the GPU (exact, derived from v_a(z^a) = conj(v_a(z))):
//       a != 0, p = msb(a):  w(z') = v_a(z) with z = z' with a 0 inserted at bit p,
//       a == 0:              w(z') = ((e + o) + i (e - o)) / 2, e = |psi_{2z'}|^2, o = |psi_{2z'+1}|^2,
//     W = H^{(x)(N-1)} w, and for every b the value |c_a(b)|^2 is 4 Re(W_b')^2 or 4 Im(W_b')^2
//     (each W entry gives two Pauli strings).  So sum_b |c_a(b)|^{2n} = 4^n sum_b' (Re^{2n} + Im^{2n}).
//   * A length-2^B complex transform is held as 32 complex values per thread (5 "register
//     bits"); the other bits are exchanged through shared memory (padded, conflict-free).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "status_bits.h"

namespace hm {


// ---- packed FP32x2 arithmetic (sm_100-family FADD2/FMUL2/FFMA2 builtins) ---------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one rounding, the same bits as the subtraction, all on the FMA pipe
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---- amplitude loads (complex64 or complex128 input, computed in FP32) ----------------
__device__ __forceinline__ float2 ld_amp(const float2* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float2 ld_amp(const double2* p, int64_t i) {
    double2 v = __ldg(p + i);
    return make_float2((float)v.x, (float)v.y);
}

// conj(b) * a
__device__ __forceinline__ float2 conj_mul(float2 b, float2 a) {
    return make_float2(fmaf(b.x, a.x, b.y * a.y), fmaf(b.x, a.y, -b.y * a.x));
}

__device__ __forceinline__ int64_t insert0(int64_t x, int p) {
    return ((x >> p) << (p + 1)) | (x & ((int64_t(1) << p) - 1));
}
__device__ __forceinline__ int msb64(int64_t a) { return 63 - __clzll((long long)a); }

// ---- tile indexing --------------------------------------------------------------------
// Element index of register i of thread t when the register bits sit at [s, s+E).
template <int E>
__device__ __forceinline__ uint32_t deposit(uint32_t t, uint32_t i, int s) {
    return (t & ((1u << s) - 1u)) | (i << s) | ((t >> s) << (s + E));
}
// Bank-conflict-free placement of complex (8-byte) element j of a tile: one pad slot per 32
// values, so for every register window the address is (thread base) + (compile-time offset).
__device__ __forceinline__ uint32_t swz(uint32_t j) { return j + (j >> 5); }
// Shared-memory slots needed for a tile of 2^B values.
__host__ __device__ constexpr uint32_t tile_slots(int B) { return (1u << B) + ((1u << B) >> 5); }

// In-register radix-2 butterflies over register-index bits [B0, B1).
template <int E, int B0, int B1>
__device__ __forceinline__ void reg_fwht(float2 (&x)[1 << E]) {
#pragma unroll
    for (int b = B0; b < B1; ++b) {
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) {
            if (!(i & (1 << b))) {
                float2 u = x[i], v = x[i | (1 << b)];
                x[i] = add2(u, v);
                x[i | (1 << b)] = sub2(u, v);
            }
        }
    }
}

struct SyncWarp {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct SyncCta {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Transform schedule for a tile of 2^B complex values whose transform bits are [LO, B):
//   round 0 holds tile bits [B-E, B) in registers (done by the caller right after loading);
//   round r >= 1 holds [LO + (r-1)E, LO + rE) and transforms the bits below B-E.
template <int B, int LO, int E>
struct TileSched {
    static constexpr int S0 = B - E;
    static constexpr int NR = 1 + ((S0 - LO) > 0 ? ((S0 - LO) + E - 1) / E : 0);
    static constexpr int shift(int r) { return r == 0 ? S0 : LO + (r - 1) * E; }
    static constexpr int last_shift() { return shift(NR - 1); }
};

struct PadAddr {  // padded placement (conflict-free for every register window)
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return swz(j); }
};
struct DenseAddr {  // dense placement (conflict-free when lanes run over the low tile bits)
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return j; }
};

// Rounds 1..NR-1: exchange through shared memory, then butterflies on the new bits.
template <int B, int LO, int E, int R, class Sync, class Addr = PadAddr>
__device__ __forceinline__ void tile_rounds(float2 (&x)[1 << E], float2* sm, uint32_t t, Sync sync,
                                            Addr addr = Addr()) {
    using S = TileSched<B, LO, E>;
    if constexpr (R < S::NR) {
        constexpr int sp = S::shift(R - 1);
        constexpr int s = S::shift(R);
        constexpr int hi = (s + E < S::S0) ? (s + E) : S::S0;
        sync();
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) sm[addr(deposit<E>(t, i, sp))] = x[i];
        sync();
#pragma unroll
        for (int i = 0; i < (1 << E); ++i) x[i] = sm[addr(deposit<E>(t, i, s))];
        reg_fwht<E, 0, hi - s>(x);
        tile_rounds<B, LO, E, R + 1>(x, sm, t, sync, addr);
    }
}

// Named barrier over `N` threads (id > 0; id 0 is __syncthreads).
template <int ID, int NTHR>
struct SyncNamed {
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NTHR) : "memory"); }
};

// cp.async (LDGSTS) 16-byte global -> shared copies, L2 only.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory"); }

// ---- reductions -----------------------------------------------------------------------
// Per-element terms of sum_b |c|^{2n}: the kernels accumulate, per complex W value,
//   q  = Re^{2n} + Im^{2n}   (n = 2, 3; scaled by 4^n at the end)
//   s1 = Re^2 + Im^2         (scaled by 4)
//   u  = Re^2 log2 Re^2 + Im^2 log2 Im^2   (n = 1 only)
// MODE 1: n = 1, 2: n = 2, 3: n = 3, 0: any n > 0 (q accumulated in FP64 from exp2(n log2)).
// The integer-n sums run as two interleaved FP32 lanes (packed FADD2/FFMA2); `q` and `s1`
// are valid after fold().
template <int MODE>
struct Acc {
    float q = 0.f, s1 = 0.f, u = 0.f;
    double qd = 0.0;
    float2 qv = make_float2(0.f, 0.f), sv = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 w, double nq) {
        float2 sq = mul2(w, w);
        if constexpr (MODE == 2) {
            sv = add2(sv, sq);
            qv = fma2(sq, sq, qv);
            return;
        } else if constexpr (MODE == 3) {
            sv = add2(sv, sq);
            qv = fma2(mul2(sq, sq), sq, qv);
            return;
        }
        s1 += sq.x + sq.y;
        if constexpr (MODE == 1) {
            u += (sq.x > 0.f ? sq.x * log2f(sq.x) : 0.f) + (sq.y > 0.f ? sq.y * log2f(sq.y) : 0.f);
        } else if constexpr (MODE == 4) {
            // FP32 powers (opt-in fast path for non-integer n): sq^n = exp2(n log2 sq), the 4^n of
            // the half-length form applied in finish3; callers keep n (N + 2) <= 100 so that the
            // values stay in FP32's normal range
            const float nf = (float)nq;
            q += (sq.x > 0.f ? exp2f(nf * log2f(sq.x)) : 0.f) + (sq.y > 0.f ? exp2f(nf * log2f(sq.y)) : 0.f);
        } else {
            double px = 4.0 * (double)sq.x, py = 4.0 * (double)sq.y;
            qd += (px > 0.0 ? exp2(nq * log2(px)) : 0.0) + (py > 0.0 ? exp2(nq * log2(py)) : 0.0);
        }
    }
    __device__ __forceinline__ void fold() {
        if constexpr (MODE == 2 || MODE == 3) {
            q = qv.x + qv.y;
            s1 = sv.x + sv.y;
        }
    }
};

template <int MODE>
__device__ __forceinline__ void warp_sum3(float& q, float& s1, float& u, double& qd, int width = 32) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o < width) {
            q += __shfl_xor_sync(0xffffffffu, q, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            if constexpr (MODE == 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            if constexpr (MODE == 0) qd += __shfl_xor_sync(0xffffffffu, qd, o);
        }
    }
}

// Scaled per-a totals in FP64: [S_q, S_1, T_1] with S_q = sum|c|^{2n}, S_1 = sum |c|^2,
// T_1 = sum |c|^2 log2 |c|^2 (n = 1 only).
template <int MODE>
__device__ __forceinline__ void finish3(float q, float s1, float u, double qd, double nq, double out[3]) {
    double S1 = 4.0 * (double)s1;
    out[1] = S1;
    if constexpr (MODE == 2) out[0] = 16.0 * (double)q;
    else if constexpr (MODE == 3) out[0] = 64.0 * (double)q;
    else if constexpr (MODE == 1) out[0] = S1;
    else if constexpr (MODE == 4) out[0] = exp2(2.0 * nq) * (double)q;
    else out[0] = qd;
    // sum 4x^2 log2(4x^2) = 4 (2 sum x^2 + sum x^2 log2 x^2)
    out[2] = (MODE == 1) ? 4.0 * (2.0 * (double)s1 + (double)u) : 0.0;
    (void)nq;
}

// ---- inter-CTA signalling (bounded) ----------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_status(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void discard_l2_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Thread 0 spins (bounded) until *ctr >= target; every thread returns whether the launch is
// still healthy.  On running out of iterations the status word gets ST_TIMEOUT.
// `seen` is a value of *ctr thread 0 read earlier with a relaxed load (0 if none): when it
// already meets the target, an acquire fence replaces the polling, and the status word is not
// read (a failure elsewhere is seen at the next wait that has to poll).
__device__ __forceinline__ bool cta_wait_geq(const unsigned* ctr, unsigned target, int* status,
                                             long long limit, unsigned seen = 0) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        long long it = 0;
        int good = 1;
        if (seen >= target) fence_acquire();
        else {
            while (ld_acquire(ctr) < target) {
                if (ld_status(status) != 0) { good = 0; break; }
                if (++it > limit) { atomicOr(status, ST_TIMEOUT); good = 0; break; }
                __nanosleep(100);
            }
            if (good && ld_status(status) != 0) good = 0;
        }
        ok = good;
    }
    __syncthreads();
    int r = ok;
    __syncthreads();
    return r != 0;
}

// Like cta_wait_geq for a group of threads that synchronise with barrier `Sync`; `leader`
// is the thread that polls.
template <class Sync>
__device__ __forceinline__ bool group_wait_geq(const unsigned* ctr, unsigned target, int* status, long long limit,
                                               unsigned seen, bool leader, int* flag, Sync sync) {
    if (leader) {
        long long it = 0;
        int good = 1;
        if (seen >= target) fence_acquire();
        else while (ld_acquire(ctr) < target) {
            if (ld_status(status) != 0) { good = 0; break; }
            if (++it > limit) { atomicOr(status, ST_TIMEOUT); good = 0; break; }
            __nanosleep(100);
        }
        if (good && ld_status(status) != 0) good = 0;
        *flag = good;
    }
    sync();
    const int r = *flag;
    sync();
    return r != 0;
}

// Warp version: lane 0 polls, the warp converges with __syncwarp.
__device__ __forceinline__ bool warp_wait_geq(const unsigned* ctr, unsigned target, int* status, long long limit) {
    int good = 1;
    if ((threadIdx.x & 31) == 0) {
        long long it = 0;
        while (ld_acquire(ctr) < target) {
            if (ld_status(status) != 0) { good = 0; break; }
            if (++it > limit) { atomicOr(status, ST_TIMEOUT); good = 0; break; }
            __nanosleep(100);
        }
        if (good && ld_status(status) != 0) good = 0;
    }
    good = __shfl_sync(0xffffffffu, good, 0);
    return good != 0;
}

}  // namespace hm
