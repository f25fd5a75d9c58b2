// rdm.cu -- reduced density matrix of a pure state of qudits (qutrits by default), the partial
// trace that produces the mixed states of the paper's mixed-state mana example (Sec. 3.3.3,
// Algorithm 6 input):
//     rho_A[r, c] = sum_x psi[(r, x)] conj(psi[(c, x)]),
// r, c over the kept sites (site keep[m] = base-d digit m of r and c), x over the traced-out
// sites.  With A[r, x] = psi[off_keep[r] + off_rest[x]] (per-digit place values tabulated on the
// host) this is the Gram product A A^dagger: a CTA computes a 16 x 16 tile of rho_A, staging
// 16 x 32 gathered blocks of A for its rows and its columns in shared memory; each thread sums
// its entry over a 32-wide chunk in FP32 and adds the chunk into FP64.
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace hm {

constexpr int RDM_TB = 16, RDM_KC = 32;

__global__ void __launch_bounds__(256) rdm_kernel(const float2* __restrict__ psi, const int64_t* __restrict__ off_keep,
                                                  const int64_t* __restrict__ off_rest, int64_t DA, int64_t DB,
                                                  float2* __restrict__ rho) {
    __shared__ float2 Ar[RDM_TB][RDM_KC + 1];
    __shared__ float2 Ac[RDM_TB][RDM_KC + 1];
    const int tx = threadIdx.x % RDM_TB, ty = threadIdx.x / RDM_TB;
    const int64_t r0 = (int64_t)blockIdx.y * RDM_TB, c0 = (int64_t)blockIdx.x * RDM_TB;
    double ax = 0.0, ay = 0.0;
    for (int64_t x0 = 0; x0 < DB; x0 += RDM_KC) {
        for (int i = threadIdx.x; i < RDM_TB * RDM_KC; i += blockDim.x) {
            const int row = i / RDM_KC, k = i % RDM_KC;
            const int64_t xg = x0 + k;
            float2 vr = make_float2(0.f, 0.f), vc = make_float2(0.f, 0.f);
            if (xg < DB) {
                const int64_t o = off_rest[xg];
                if (r0 + row < DA) vr = ld_amp(psi, off_keep[r0 + row] + o);
                if (c0 + row < DA) vc = ld_amp(psi, off_keep[c0 + row] + o);
            }
            Ar[row][k] = vr;
            Ac[row][k] = vc;
        }
        __syncthreads();
        float sx = 0.f, sy = 0.f;
#pragma unroll 8
        for (int k = 0; k < RDM_KC; ++k) {
            const float2 a = Ar[ty][k], b = Ac[tx][k];  // a conj(b)
            sx = fmaf(a.x, b.x, fmaf(a.y, b.y, sx));
            sy = fmaf(a.y, b.x, fmaf(-a.x, b.y, sy));
        }
        ax += sx;
        ay += sy;
        __syncthreads();
    }
    const int64_t r = r0 + ty, c = c0 + tx;
    if (r < DA && c < DA) rho[r * DA + c] = make_float2((float)ax, (float)ay);
}

}  // namespace hm

using namespace hm;

namespace {

// Sites of dimension d: d^N <= 3^16 amplitudes, rho_A of side d^n_keep <= 3^10.
hadamag_status rdm_run(hadamag_ctx_t c, const void* psi, int N, int d, hadamag_dtype dt, const int* keep,
                       int n_keep, void* rho, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !keep || !rho || (reinterpret_cast<uintptr_t>(rho) & 7))
        return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (d < 2 || d > 13) return fail(c, HADAMAG_ERR_INVALID_ARG, "site dimension must be in [2, 13] (got %d)", d);
    long long dimN = 1, dimA = 1;
    for (int j = 0; j < N && dimN <= 43046721; ++j) dimN *= d;
    for (int j = 0; j < n_keep && dimA <= 59049; ++j) dimA *= d;
    if (N < 1 || dimN > 43046721) return fail(c, HADAMAG_ERR_INVALID_ARG, "need 1 <= N and d^N <= 3^16 (N = %d)", N);
    if (n_keep < 1 || n_keep > N || dimA > 59049)
        return fail(c, HADAMAG_ERR_INVALID_ARG, "need 1 <= n_keep <= N and d^n_keep <= 3^10 (got %d)", n_keep);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    std::vector<int> kept(N, 0);
    for (int m = 0; m < n_keep; ++m) {
        if (keep[m] < 0 || keep[m] >= N || kept[keep[m]])
            return fail(c, HADAMAG_ERR_INVALID_ARG, "keep must list distinct sites in [0, N)");
        kept[keep[m]] = 1;
    }
    std::vector<int64_t> place(N);
    for (int j = 0; j < N; ++j) place[j] = j ? place[j - 1] * d : 1;
    std::vector<int> rest;
    for (int j = 0; j < N; ++j)
        if (!kept[j]) rest.push_back(j);
    // off(list)[i] = sum_m digit_m(i) * d^(list[m])  (digits in base d)
    auto offsets = [&](const int* sites, int n) {
        int64_t D = 1;
        for (int m = 0; m < n; ++m) D *= d;
        std::vector<int64_t> off((size_t)D);
        for (int64_t i = 0; i < D; ++i) {
            int64_t v = 0, q = i;
            for (int m = 0; m < n; ++m, q /= d) v += (q % d) * place[sites[m]];
            off[(size_t)i] = v;
        }
        return off;
    };
    const std::vector<int64_t> ok = offsets(keep, n_keep), orr = offsets(rest.data(), (int)rest.size());
    const int64_t DA = (int64_t)ok.size(), DB = (int64_t)orr.size();
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    c->last_error[0] = 0;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    hadamag_status s;
    const float2* p;
    if ((s = as_c64(c, psi, (int64_t)dimN, dt, st, &p))) return s;
    if ((s = ensure_buf(c, c->rdm_idx, (size_t)(DA + DB) * sizeof(int64_t)))) return s;
    int64_t* dok = (int64_t*)c->rdm_idx.ptr;
    int64_t* dor = dok + DA;
    if ((e = cudaMemcpyAsync(dok, ok.data(), DA * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dor, orr.data(), DB * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "copy index tables");
    const dim3 grid((unsigned)((DA + RDM_TB - 1) / RDM_TB), (unsigned)((DA + RDM_TB - 1) / RDM_TB));
    rdm_kernel<<<grid, 256, 0, st>>>(p, dok, dor, DA, DB, reinterpret_cast<float2*>(rho));
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "rdm_kernel");
    return HADAMAG_OK;
}

}  // namespace

extern "C" hadamag_status hadamag_reduced_density_matrix(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt,
                                                         const int* keep, int n_keep, void* rho,
                                                         hadamag_stream_t stream) {
    return rdm_run(c, psi, N, 3, dt, keep, n_keep, rho, stream);
}

extern "C" hadamag_status hadamag_reduced_density_matrix_qudit(hadamag_ctx_t c, const void* psi, int N, int d,
                                                               hadamag_dtype dt, const int* keep, int n_keep,
                                                               void* rho, hadamag_stream_t stream) {
    return rdm_run(c, psi, N, d, dt, keep, n_keep, rho, stream);
}
