// tc.cuh -- tcgen05 (5th-generation tensor core) primitives for sm_103a, inline PTX.
//
// Operands live in shared memory, either in the no-swizzle canonical layout -- "core
// matrices" of 8 rows x 16 bytes (8 fp16 values), each 128 contiguous bytes; a K-major operand
// holds 8 consecutive K values of one row in a 16-byte core-matrix row, an MN-major operand 8
// consecutive rows (M or N index) of one K value; the matrix descriptor carries the byte
// distance between core matrices adjacent along K (LBO) and along M/N (SBO) -- or in the
// 128-byte-swizzle layout described at sdesc().
// The accumulator is fp32 in tensor memory (TMEM): row i of D in lane i, column j in column j.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace hm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, descriptor version 1; layout 0 = no swizzle, 2 = 128-byte
// swizzle (atoms of 8 rows x 128 B, 1024-byte aligned, whose 16-byte chunk c of row r sits at
// chunk c ^ r).  For the MN-major 128-byte-swizzle form LBO is the distance between atoms along
// M/N (64 fp16 values) and SBO the distance between groups of 8 K-rows.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)(layout & 7u) << 61);
}

// Instruction descriptor of kind::f16: fp16 A and B, fp32 D, dense, M x N tile.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool a_mn_major, bool b_mn_major) {
    return (1u << 4) | ((a_mn_major ? 1u : 0u) << 15) | ((b_mn_major ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] x B[smem], one elected thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

// D[tmem] = A[smem] x B[smem] + D * 2^-SCALE (the instruction's scale-input-d operand, kind::f16
// and kind::tf32 only, 0 <= SCALE <= 15), one elected thread.
template <int SCALE>
__device__ __forceinline__ void mma_f16_scale_d(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc) {
    static_assert(SCALE >= 0 && SCALE <= 15, "scale-input-d is 0..15");
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p, %4;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "n"(SCALE));
}

// Arrive on `mbar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with parity `parity` of `mbar` to complete.  Each try_wait
// suspends the thread (no issue slots) until the phase completes or 100 us pass; the loop
// gives up after limit / 1024 (at least 16) such periods.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit) {
    const long long n = (limit >> 10) < 16 ? 16 : (limit >> 10);
    for (long long it = 0; it < n; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(mbar)), "r"(parity), "r"(100000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Plain arrive (count 1) on `mbar`.
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy writes to shared memory become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Whole-warp TMEM allocation; the base address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive fp32 columns of this thread's lane (warp w reads lanes 32(w%4) .. +31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t* r = reinterpret_cast<uint32_t*>(v);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Exponent offset of the lo part of the hi/lo split.
constexpr int LO_SHIFT = 11;

// x = hi + 2^-LO_SHIFT lo with hi = fp16(x) and lo = fp16(2^LO_SHIFT (x - hi)): 8 fp32 values ->
// two 16-byte rows.  x - hi is exact in fp32 and |x - hi| <= 2^-11 |x|, so lo has the magnitude
// of x and stays a normal fp16 number down to |x| ~ 2^-14: the pair keeps ~22 significant bits
// over the whole normal fp16 range of x (a lo part stored unscaled would turn subnormal below
// |x| ~ 2^-3 and keep only an absolute precision of 2^-25).  The MMAs undo the offset through
// scale-input-d (issue_block in sre_tc.cu).
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
    const float2 sc = make_float2((float)(1 << LO_SHIFT), (float)(1 << LO_SHIFT));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __half2 hh = __floats2half2_rn(x[2 * k], x[2 * k + 1]);
        const float2 hf = __half22float2(hh);
        const float2 r = __fmul2_rn(__fadd2_rn(make_float2(x[2 * k], x[2 * k + 1]), make_float2(-hf.x, -hf.y)), sc);
        const __half2 ll = __floats2half2_rn(r.x, r.y);
        h[k] = *reinterpret_cast<const uint32_t*>(&hh);
        l[k] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Bulk copy global -> shared (TMA engine, no tensor map); completion is counted in bytes on
// `mbar`.  One thread arrives once per phase with the phase's total byte count (expect_tx),
// then issues the copies of that phase.
__device__ __forceinline__ void expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// 32-byte global load through L2 only (data written earlier in the same launch by other CTAs).
__device__ __forceinline__ void ldcg256(const float* p, float (&v)[8]) {
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}

__device__ __forceinline__ float2 lds64(uint32_t saddr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(saddr));
    return v;
}

__device__ __forceinline__ void sts128(uint32_t saddr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(saddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

}  // namespace tc
}  // namespace hm
