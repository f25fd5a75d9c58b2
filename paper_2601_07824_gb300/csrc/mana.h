// mana.h -- launch interface of the qutrit mana kernels (internal to libhadamag).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hm {

struct ManaParams {
    const float2* psi;       // the state, or the density matrix for mixed states
    int N;
    int64_t count;           // number of work items (mana_pair_items(N)): X-string pairs and singles
    float2* scratch;         // R slots x A work items x 3^N values
    int R, A;
    int64_t n_batches;
    int p1, p2;              // tasks per batch (A * 3^(N-8) each)
    unsigned* done1;
    unsigned* done2;
    int* status;
    long long spin_limit;
    unsigned wait_bias;
    double* out;             // per-CTA [grid][3]: sum |chi|, sum chi, sum chi^2
};

int mana_tiles_per_a(int N);
// Work items of the two-pass kernels (9 <= N <= 13): sum_{k < N-8} 3^(N-1-k) pairs + 3^8 singles.
int64_t mana_pair_items(int N);
// mixed = false: src is the N-qutrit state psi (3^N values, Algorithm 5); mixed = true: src is
// a density matrix rho, 3^N x 3^N row-major (Algorithm 6's W via the same transform; the
// two-pass variant exists for N = 9, 10).
cudaError_t launch_mana_onepass(const float2* src, int N, bool mixed, double* out, int sm_count, int* grid,
                                cudaStream_t st);
cudaError_t mana_twopass_grid(int N, bool mixed, int sm_count, int* grid);
cudaError_t launch_mana_twopass(const ManaParams& P, bool mixed, int grid, cudaStream_t st);

// Odd-prime qudits (qudit.cu): largest N with d^N <= 25600 for d = 3, 5, 7, 11, 13 (0 for other
// d); the mana launch (d != 3) writing grid <= max_grid per-CTA triples [sum |chi|, sum chi,
// sum chi^2]; the gradient launch, which also fills grid per-CTA partial gradients of d^N
// double2 each (zeroed by the caller); and the finalize writing grad = (sum of partials) /
// (msum[0] ln 2) as complex64 or complex128.
int mana_qudit_max_n(int d);
cudaError_t launch_mana_qudit(const float2* psi, int N, int d, double* out, int sm_count, int max_grid, int* grid,
                              cudaStream_t st);
cudaError_t launch_mana_grad(const float2* psi, int N, int d, double* out, double2* gpart, int sm_count, int max_grid,
                             int* grid, cudaStream_t st);
// the mana launch for a d^N x d^N density matrix (row-major), v_x = rho[-x - a, x - a]
cudaError_t launch_mana_qudit_mixed(const float2* rho, int N, int d, double* out, int sm_count, int max_grid,
                                    int* grid, cudaStream_t st);
cudaError_t launch_mana_grad_finalize(const double2* gpart, int parts, int dim, const double* msum, void* grad,
                                      bool c128, cudaStream_t st);

}  // namespace hm
