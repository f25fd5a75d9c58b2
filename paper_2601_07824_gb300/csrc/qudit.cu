// qudit.cu -- mana of N qudits of odd prime dimension d = 5, 7, 11, 13 (Sec. 2: the qutrit
// construction applies to any odd prime d; Algorithm 5 generalised), and the gradient of the
// mana for d = 3, 5, 7, 11, 13.
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
// FP64 per shift, fixed order).  The mana of qutrits (d = 3) uses the register-tiled kernels of
// mana.cu; the gradient kernel below covers d = 3 too.
#include "common.cuh"
#include "mana.h"

namespace hm {

constexpr int QUDIT_MAXN = 9;  // d = 3: 3^9 = 19683 <= QUDIT_MAXDIM
constexpr int QUDIT_MAXDIM = 25600;

// idx(x - a) and idx(-x - a), digit-wise mod D (ad: the digits of a)
template <int D>
__device__ __forceinline__ void qudit_pair_idx(int x, const int* ad, int N, int& i1, int& i2) {
    int t = x, p = 1;
    i1 = 0;
    i2 = 0;
    for (int j = 0; j < N; ++j, t /= D, p *= D) {
        const int xd = t % D;
        i1 += ((xd - ad[j] + D) % D) * p;
        i2 += ((2 * D - xd - ad[j]) % D) * p;
    }
}

__device__ __forceinline__ void qudit_twiddles(float2* tw, int D) {
    if ((int)threadIdx.x < D * D) {
        const int j = threadIdx.x / D, k = threadIdx.x % D;
        float sn, cs;
        sincospif(2.0f * (float)((2 * j * k) % D) / (float)D, &sn, &cs);
        tw[threadIdx.x] = make_float2(cs, sn);
    }
}

// F_D^{(x)N} in place on the dim = D^N values in shared memory, one digit after the other
// (each thread a set of disjoint D-value fibres); a barrier before every digit and at the end.
template <int D>
__device__ __forceinline__ void qudit_transform(float2* v, const float2* tw, int N, int dim) {
    for (int j = 0, s = 1; j < N; ++j, s *= D) {
        __syncthreads();
        for (int f = threadIdx.x; f < dim / D; f += blockDim.x) {
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
}

// CTA sum of per-thread FP32 triples into FP64 acc (valid in thread 0; 256 threads)
__device__ __forceinline__ void qudit_cta_sum(float m, float s1, float q, float (*red)[3], double* acc) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = m; red[threadIdx.x >> 5][1] = s1; red[threadIdx.x >> 5][2] = q; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { acc[0] += red[w][0]; acc[1] += red[w][1]; acc[2] += red[w][2]; }
}

// MIXED: psi is a density matrix rho (dim x dim, row-major) and v_x = rho[-x - a, x - a], which
// for rho = |psi><psi| is conj(psi_{x-a}) psi_{-x-a}; every entry of rho is read once.
template <int D, bool MIXED>
__global__ void __launch_bounds__(256) mana_qudit_kernel(const float2* __restrict__ psi, int N, int dim,
                                                         double* __restrict__ out) {
    extern __shared__ float2 v[];  // dim values
    __shared__ float2 tw[D * D];
    __shared__ float red[8][3];
    const int tid = threadIdx.x;
    qudit_twiddles(tw, D);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int a = blockIdx.x; a < dim; a += gridDim.x) {
        int ad[QUDIT_MAXN];
        for (int j = 0, t = a; j < N; ++j, t /= D) ad[j] = t % D;
        __syncthreads();  // the previous shift's reduction has read v; tw is ready
        for (int x = tid; x < dim; x += blockDim.x) {
            int i1, i2;
            qudit_pair_idx<D>(x, ad, N, i1, i2);
            if constexpr (MIXED) v[x] = __ldg(psi + (int64_t)i2 * dim + i1);
            else v[x] = conj_mul(__ldg(psi + i1), __ldg(psi + i2));
        }
        qudit_transform<D>(v, tw, N, dim);
        float m = 0.f, s1 = 0.f, q = 0.f;
        for (int x = tid; x < dim; x += blockDim.x) {
            const float r = v[x].x;
            m += fabsf(r);
            s1 += r;
            q = fmaf(r, r, q);
        }
        qudit_cta_sum(m, s1, q, red, acc);
    }
    if (tid == 0) { out[blockIdx.x * 3] = acc[0]; out[blockIdx.x * 3 + 1] = acc[1]; out[blockIdx.x * 3 + 2] = acc[2]; }
}

// Gradient of the mana (the adjoint of the kernel above).  With v_x = conj(psi_{x-a}) psi_{-x-a},
// d chi_b(a) / d psi*_w = d conj(chi_b(a)) / d psi*_w = F_{b, w+a} psi_{-w-2a}; for y = w + a and
// G_a = F^{(x)N} (Re chi_a / |chi_a|):  d m / d psi*_{y-a} += psi_{-y-a} G_a(y)  (m = sum |chi|).
// Per shift: forward transform, reduction, the sign vector, a second transform, and the scatter
// into this CTA's FP64 partial gradient (y -> y - a is a bijection, so the threads of a CTA write
// distinct entries for one shift; barriers order consecutive shifts).
template <int D>
__global__ void __launch_bounds__(256) mana_grad_kernel(const float2* __restrict__ psi, int N, int dim,
                                                        double* __restrict__ out, double2* __restrict__ gpart) {
    extern __shared__ float2 v[];
    __shared__ float2 tw[D * D];
    __shared__ float red[8][3];
    const int tid = threadIdx.x;
    qudit_twiddles(tw, D);
    double2* gp = gpart + (size_t)blockIdx.x * dim;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int a = blockIdx.x; a < dim; a += gridDim.x) {
        int ad[QUDIT_MAXN];
        for (int j = 0, t = a; j < N; ++j, t /= D) ad[j] = t % D;
        __syncthreads();
        for (int x = tid; x < dim; x += blockDim.x) {
            int i1, i2;
            qudit_pair_idx<D>(x, ad, N, i1, i2);
            v[x] = conj_mul(__ldg(psi + i1), __ldg(psi + i2));
        }
        qudit_transform<D>(v, tw, N, dim);
        float m = 0.f, s1 = 0.f, q = 0.f;
        for (int x = tid; x < dim; x += blockDim.x) {
            const float2 c = v[x];
            m += fabsf(c.x);
            s1 += c.x;
            q = fmaf(c.x, c.x, q);
            const float r = hypotf(c.x, c.y);
            v[x] = make_float2(r > 0.f ? c.x / r : 0.f, 0.f);
        }
        qudit_cta_sum(m, s1, q, red, acc);
        qudit_transform<D>(v, tw, N, dim);
        for (int y = tid; y < dim; y += blockDim.x) {
            int i1, i2;
            qudit_pair_idx<D>(y, ad, N, i1, i2);
            const float2 g = v[y], p = __ldg(psi + i2);
            double2 cur = gp[i1];
            cur.x += (double)fmaf(p.x, g.x, -p.y * g.y);
            cur.y += (double)fmaf(p.x, g.y, p.y * g.x);
            gp[i1] = cur;
        }
    }
    if (tid == 0) { out[blockIdx.x * 3] = acc[0]; out[blockIdx.x * 3 + 1] = acc[1]; out[blockIdx.x * 3 + 2] = acc[2]; }
}

// grad[w] = sum over CTAs (fixed order) of the partials, times 1 / (m ln 2), m = msum[0]
template <typename T>
__global__ void mana_grad_finalize(const double2* __restrict__ gpart, int parts, int dim, const double* __restrict__ msum,
                                   T* __restrict__ grad) {
    const double scale = 1.0 / (msum[0] * 0.693147180559945309417);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < dim; w += gridDim.x * blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int c = 0; c < parts; ++c) {
            const double2 t = gpart[(size_t)c * dim + w];
            gx += t.x;
            gy += t.y;
        }
        grad[w].x = gx * scale;
        grad[w].y = gy * scale;
    }
}

int mana_qudit_max_n(int d) {
    if (d != 3 && d != 5 && d != 7 && d != 11 && d != 13) return 0;
    int n = 0;
    for (long long p = d; p <= QUDIT_MAXDIM; p *= d) ++n;
    return n < QUDIT_MAXN ? n : QUDIT_MAXN;
}

template <int D, bool GRAD, bool MIXED>
static cudaError_t launch_qudit_d(const float2* psi, int N, int dim, double* out, double2* gpart, int sm_count,
                                  int max_grid, int* grid, cudaStream_t st) {
    const size_t smem = (size_t)dim * sizeof(float2);
    cudaError_t e;
    int occ = 0;
    if constexpr (GRAD) {
        if ((e = cudaFuncSetAttribute(mana_grad_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mana_grad_kernel<D>, 256, smem);
    } else {
        if ((e = cudaFuncSetAttribute(mana_qudit_kernel<D, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mana_qudit_kernel<D, MIXED>, 256, smem);
    }
    if (e != cudaSuccess) return e;
    int g = (occ < 1 ? 1 : occ) * sm_count;
    if (g > dim) g = dim;
    if (g > max_grid) g = max_grid;
    *grid = g;
    if constexpr (GRAD) mana_grad_kernel<D><<<g, 256, smem, st>>>(psi, N, dim, out, gpart);
    else mana_qudit_kernel<D, MIXED><<<g, 256, smem, st>>>(psi, N, dim, out);
    return cudaGetLastError();
}

template <bool GRAD, bool MIXED>
static cudaError_t launch_qudit(const float2* psi, int N, int d, double* out, double2* gpart, int sm_count,
                                int max_grid, int* grid, cudaStream_t st) {
    if (N < 1 || N > mana_qudit_max_n(d)) return cudaErrorInvalidValue;
    int dim = 1;
    for (int j = 0; j < N; ++j) dim *= d;
    switch (d) {
        case 3: return launch_qudit_d<3, GRAD, MIXED>(psi, N, dim, out, gpart, sm_count, max_grid, grid, st);
        case 5: return launch_qudit_d<5, GRAD, MIXED>(psi, N, dim, out, gpart, sm_count, max_grid, grid, st);
        case 7: return launch_qudit_d<7, GRAD, MIXED>(psi, N, dim, out, gpart, sm_count, max_grid, grid, st);
        case 11: return launch_qudit_d<11, GRAD, MIXED>(psi, N, dim, out, gpart, sm_count, max_grid, grid, st);
        case 13: return launch_qudit_d<13, GRAD, MIXED>(psi, N, dim, out, gpart, sm_count, max_grid, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mana_qudit(const float2* psi, int N, int d, double* out, int sm_count, int max_grid, int* grid,
                              cudaStream_t st) {
    return launch_qudit<false, false>(psi, N, d, out, nullptr, sm_count, max_grid, grid, st);
}

cudaError_t launch_mana_qudit_mixed(const float2* rho, int N, int d, double* out, int sm_count, int max_grid,
                                    int* grid, cudaStream_t st) {
    return launch_qudit<false, true>(rho, N, d, out, nullptr, sm_count, max_grid, grid, st);
}

cudaError_t launch_mana_grad(const float2* psi, int N, int d, double* out, double2* gpart, int sm_count, int max_grid,
                             int* grid, cudaStream_t st) {
    return launch_qudit<true, false>(psi, N, d, out, gpart, sm_count, max_grid, grid, st);
}

cudaError_t launch_mana_grad_finalize(const double2* gpart, int parts, int dim, const double* msum, void* grad,
                                      bool c128, cudaStream_t st) {
    const int blocks = (dim + 255) / 256;
    if (c128) mana_grad_finalize<double2><<<blocks, 256, 0, st>>>(gpart, parts, dim, msum, (double2*)grad);
    else mana_grad_finalize<float2><<<blocks, 256, 0, st>>>(gpart, parts, dim, msum, (float2*)grad);
    return cudaGetLastError();
}

}  // namespace hm
