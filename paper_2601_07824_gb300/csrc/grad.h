// grad.h -- launch interface of the M_2 adjoint kernels (internal to libhadamag).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctx.h"
#include "sre_fwd.h"

namespace hm {

struct GradParams {
    const float2* psi;
    int N;
    float2* scratch;         // R slots x A X-strings x 2^(N-1) values
    int R, A, U;
    int64_t n_batches;
    int p1, p2, p3;          // tasks per batch of the three passes
    unsigned* done1;
    unsigned* done2;
    unsigned* done3;
    int* status;
    long long spin_limit;
    unsigned wait_bias;
    float2* gpart;           // per-CTA partial dS_2/dpsi* [grid][2^N] (zeroed before launch)
    double* sums;            // per-CTA [grid][3]: S_2, S_1, 0
    int64_t a_base = 0;      // X-strings a_base .. a_base + A n_batches - 1
    int UPW = 2, TPT = 1;    // units per pass-1 warp, column tiles per pass-2 task
    int lag = 1;             // stages between the passes of a batch (R >= 2 lag + 1)
};

int grad_onepass_gpc(int N);
// X-strings a_base .. a_base + count - 1 (count < 0: all 2^N)
cudaError_t launch_grad_onepass(const float2* psi, int N, double* sums, float2* gpart, int groups_max,
                                int* ngroups, cudaStream_t st, int64_t a_base = 0, int64_t count = -1);
cudaError_t grad_threepass_grid(int N, int sm_count, int* grid);
cudaError_t launch_grad_threepass(const GradParams& P, int grid, cudaStream_t st);
cudaError_t launch_grad_sum_parts(const float2* gpart, int64_t nparts, int64_t dim, double2* out, cudaStream_t st);
cudaError_t launch_grad_scale(const double2* dS, int64_t dim, double S2, void* out, bool c128, cudaStream_t st);
cudaError_t launch_grad_finalize(const float2* gpart, int64_t nparts, int64_t dim, const double* s2, void* out,
                                 bool c128, cudaStream_t st);

hadamag_status enqueue_grad_parts(hadamag_ctx_t c, const float2* p, int N, int64_t a0, int64_t count, cudaStream_t st,
                                  int64_t* nparts_out);

}  // namespace hm
