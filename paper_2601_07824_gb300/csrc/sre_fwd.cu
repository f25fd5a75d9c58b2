// sre_fwd.cu -- host dispatch of the exact-SRE forward kernels (paper Sec. 3.1.2, Algorithm 2)
// and the small reduction / conversion kernels they share.  The kernels themselves are in
// sre_fwd_kernels.cuh, instantiated one accumulation mode per translation unit (sre_fwd_n*.cu).
#include "sre_fwd_kernels.cuh"

namespace hm {

// ------------------------------------------------------------------------------------------
// Deterministic FP64 reduction of `n` triples (fixed per-thread strides, fixed tree).
__global__ void sum_triples(const double* __restrict__ in, int64_t n, double* __restrict__ out) {
    __shared__ double s[3][256];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        a0 += in[i * 3]; a1 += in[i * 3 + 1]; a2 += in[i * 3 + 2];
    }
    s[0][threadIdx.x] = a0; s[1][threadIdx.x] = a1; s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s[0][0]; out[1] = s[1][0]; out[2] = s[2][0]; }
}

// Per-X-string sums of `tiles` partial triples: out[i] = sum_t in[i][t].  One warp per X-string:
// lane l adds t = l, l + 32, ... in order, then a fixed xor-shuffle tree combines the lanes, so
// the result depends only on the triples (not on the launch or on which calls made them).
__global__ void sum_tiles(const double* __restrict__ in, int64_t count, int tiles, double* __restrict__ out) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= count) return;  // warp-uniform (blockDim is a multiple of 32)
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int t = lane; t < tiles; t += 32) {
        const double* p = in + ((size_t)i * tiles + t) * 3;
        a0 += p[0]; a1 += p[1]; a2 += p[2];
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) { out[i * 3] = a0; out[i * 3 + 1] = a1; out[i * 3 + 2] = a2; }
}

__global__ void c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = in[i];
        out[i] = make_float2((float)v.x, (float)v.y);
    }
}

// ------------------------------------------------------------------------------------------
// Host dispatch on the accumulation mode.

cudaError_t launch_onepass(OnepassArgs& A, int mode, int sm_count, cudaStream_t st) {
    switch (mode) {
        case 0: return sre_fwd_onepass_n0(A, sm_count, st);
        case 1: return sre_fwd_onepass_n1(A, sm_count, st);
        case 2: return sre_fwd_onepass_n2(A, sm_count, st);
        case 3: return sre_fwd_onepass_n3(A, sm_count, st);
        case 4: return sre_fwd_onepass_n4(A, sm_count, st);
        default: return cudaErrorInvalidValue;
    }
}

// Pass-1 width for N: 10 bits (warp-level) up to N = 20, 13 bits (CTA-level) above, so that
// pass-2 tiles keep rows of >= 16 values whenever possible.
int twopass_k1(int N) { return N <= 20 ? 10 : 13; }

int twopass_tiles_per_a(int N) {
    HM_TWOPASS_SWITCH(N, return (TwoPassShape<KK, MM>::TILES))
}

cudaError_t launch_twopass(const TwoPassParams& P, int mode, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: return sre_fwd_twopass_n0(P, grid, st);
        case 1: return sre_fwd_twopass_n1(P, grid, st);
        case 2: return sre_fwd_twopass_n2(P, grid, st);
        case 3: return sre_fwd_twopass_n3(P, grid, st);
        case 4: return sre_fwd_twopass_n4(P, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t twopass_max_grid(int N, int mode, int sm_count, int* grid) {
    int occ = 0;
    cudaError_t e;
    switch (mode) {
        case 0: e = sre_fwd_twopass_occ_n0(N, &occ); break;
        case 1: e = sre_fwd_twopass_occ_n1(N, &occ); break;
        case 2: e = sre_fwd_twopass_occ_n2(N, &occ); break;
        case 3: e = sre_fwd_twopass_occ_n3(N, &occ); break;
        case 4: e = sre_fwd_twopass_occ_n4(N, &occ); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    *grid = (occ < 1 ? 1 : occ) * sm_count;
    return cudaSuccess;
}

cudaError_t launch_sum_triples(const double* in, int64_t n, double* out, cudaStream_t st) {
    sum_triples<<<1, 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sum_tiles(const double* in, int64_t count, int tiles, double* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    sum_tiles<<<(unsigned)((count * 32 + 255) / 256), 256, 0, st>>>(in, count, tiles, out);
    return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const void* in, float2* out, int64_t n, cudaStream_t st) {
    c128_to_c64<<<1024, 256, 0, st>>>(reinterpret_cast<const double2*>(in), out, n);
    return cudaGetLastError();
}

}  // namespace hm
