// qudit.cu -- mana of N qudits of odd prime dimension d = 5, 7, 11, 13 (Sec. 2: the qutrit
// construction applies to any odd prime d; Algorithm 5 generalised).
//
// From the definitions, A_ab|x> = w^{2a(b-x)} |2b - x> (w = e^{2 pi i / d}), so for every shift a
// (digit-wise mod d)
//     v_x = conj(psi_{x - a}) psi_{-x - a},   chi = F_d^{(x)N} v,  (F_d)_{jk} = w^{2jk},
// and the chi / d^N are the Wigner function W(u); mana = log2(sum |chi| / d^N).  chi is real
// for pure states.
//
// One CTA per shift (grid-stride): the d^N values of v sit in shared memory (d^N <= 25600, so
// N <= 6, 5, 4, 3 for d = 5, 7, 11, 13), the N digits are transformed in place one after the
// other (each thread a set of disjoint d-value fibres, a direct d-point sum with a w^{2jk} table
// in shared memory), then the CTA reduces sum |chi|, sum chi, sum chi^2 (FP32 per thread,
// FP64 per shift, fixed order).  Qutrits (d = 3) use the register-tiled kernels of mana.cu.
#include "common.cuh"
#include "mana.h"

namespace hm {

constexpr int QUDIT_MAXN = 8;
constexpr int QUDIT_MAXDIM = 25600;

template <int D>
__global__ void __launch_bounds__(256) mana_qudit_kernel(const float2* __restrict__ psi, int N, int dim,
                                                         double* __restrict__ out) {
    extern __shared__ float2 v[];  // dim values
    __shared__ float2 tw[D * D];
    __shared__ float red[8][3];
    const int tid = threadIdx.x;
    if (tid < D * D) {
        const int j = tid / D, k = tid % D;
        float sn, cs;
        sincospif(2.0f * (float)((2 * j * k) % D) / (float)D, &sn, &cs);
        tw[tid] = make_float2(cs, sn);
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int a = blockIdx.x; a < dim; a += gridDim.x) {
        int ad[QUDIT_MAXN];
        for (int j = 0, t = a; j < N; ++j, t /= D) ad[j] = t % D;
        __syncthreads();  // the previous shift's reduction has read v; tw is ready
        for (int x = tid; x < dim; x += blockDim.x) {
            int t = x, p = 1, i1 = 0, i2 = 0;
            for (int j = 0; j < N; ++j, t /= D, p *= D) {
                const int xd = t % D;
                i1 += ((xd - ad[j] + D) % D) * p;
                i2 += ((2 * D - xd - ad[j]) % D) * p;
            }
            v[x] = conj_mul(__ldg(psi + i1), __ldg(psi + i2));
        }
        for (int j = 0, s = 1; j < N; ++j, s *= D) {
            __syncthreads();
            for (int f = tid; f < dim / D; f += blockDim.x) {
                const int base = (f / s) * s * D + (f % s);
                float2 xin[D];
#pragma unroll
                for (int m = 0; m < D; ++m) xin[m] = v[base + m * s];
#pragma unroll (D <= 7 ? D : 1)
                for (int k = 0; k < D; ++k) {
                    float re = 0.f, im = 0.f;
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        const float2 w = tw[k * D + m], z = xin[m];
                        re = fmaf(w.x, z.x, fmaf(-w.y, z.y, re));
                        im = fmaf(w.x, z.y, fmaf(w.y, z.x, im));
                    }
                    v[base + k * s] = make_float2(re, im);
                }
            }
        }
        __syncthreads();
        float m = 0.f, s1 = 0.f, q = 0.f;
        for (int x = tid; x < dim; x += blockDim.x) {
            const float r = v[x].x;
            m += fabsf(r);
            s1 += r;
            q = fmaf(r, r, q);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5][0] = m; red[tid >> 5][1] = s1; red[tid >> 5][2] = q; }
        __syncthreads();
        if (tid == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { acc[0] += red[w][0]; acc[1] += red[w][1]; acc[2] += red[w][2]; }
    }
    if (tid == 0) { out[blockIdx.x * 3] = acc[0]; out[blockIdx.x * 3 + 1] = acc[1]; out[blockIdx.x * 3 + 2] = acc[2]; }
}

int mana_qudit_max_n(int d) {
    if (d != 5 && d != 7 && d != 11 && d != 13) return 0;
    int n = 0;
    for (long long p = d; p <= QUDIT_MAXDIM; p *= d) ++n;
    return n < QUDIT_MAXN ? n : QUDIT_MAXN;
}

template <int D>
static cudaError_t launch_qudit_d(const float2* psi, int N, int dim, double* out, int sm_count, int max_grid,
                                  int* grid, cudaStream_t st) {
    const size_t smem = (size_t)dim * sizeof(float2);
    auto k = mana_qudit_kernel<D>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, smem)) != cudaSuccess) return e;
    int g = (occ < 1 ? 1 : occ) * sm_count;
    if (g > dim) g = dim;
    if (g > max_grid) g = max_grid;
    *grid = g;
    k<<<g, 256, smem, st>>>(psi, N, dim, out);
    return cudaGetLastError();
}

cudaError_t launch_mana_qudit(const float2* psi, int N, int d, double* out, int sm_count, int max_grid, int* grid,
                              cudaStream_t st) {
    if (N < 1 || N > mana_qudit_max_n(d)) return cudaErrorInvalidValue;
    int dim = 1;
    for (int j = 0; j < N; ++j) dim *= d;
    switch (d) {
        case 5: return launch_qudit_d<5>(psi, N, dim, out, sm_count, max_grid, grid, st);
        case 7: return launch_qudit_d<7>(psi, N, dim, out, sm_count, max_grid, grid, st);
        case 11: return launch_qudit_d<11>(psi, N, dim, out, sm_count, max_grid, grid, st);
        case 13: return launch_qudit_d<13>(psi, N, dim, out, sm_count, max_grid, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hm
