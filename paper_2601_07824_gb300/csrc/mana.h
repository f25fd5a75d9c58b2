// mana.h -- launch interface of the qutrit mana kernels (internal to libhadamag).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hm {

struct ManaParams {
    const float2* psi;
    int N;
    int64_t count;           // number of X-strings a (3^N)
    float2* scratch;         // R slots x A X-strings x 3^N values
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
cudaError_t launch_mana_onepass(const float2* psi, int N, double* out, int sm_count, int* grid, cudaStream_t st);
cudaError_t mana_twopass_grid(int N, int sm_count, int* grid);
cudaError_t launch_mana_twopass(const ManaParams& P, int grid, cudaStream_t st);

}  // namespace hm
