// batched.h -- launch interface of the batched persistent adjoint kernel (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "grad_phases.cuh"

namespace hm {

struct BatchState {
    const float2* psi;
    float2* grad;              // dM_2/dpsi* out (complex64) or null
    int N;
    int kind;                  // 0: small (one-pass items), 1: large (three passes + finalize)
    int fwd;                   // 1: M_2 only (large: two passes + one finalize task)
    int out_idx;               // position of this state in the caller's arrays
    int64_t task_begin;        // small states: first ticket of this state's segment
    // small states: n_chunks items of 2^N / n_chunks X-strings each (then, if n_chunks > 1, one
    // finalize item that combines them)
    float2* gsmall;            // n_chunks x GPC x 2^N partials, zeroed before launch
    int n_chunks;
    // large states
    float2* scratch;           // R x A x 2^(N-1)
    int R, A, U;
    int UPW, TPT;              // units per pass-1 warp, column tiles per pass-2 task
    int lag;                   // stages between the passes of a batch (R >= 2 lag + 1)
    int64_t n_batches;
    int p1, p2, p3;
    int64_t n_stage_tasks;     // (n_batches + 2 lag) (p1 + p2 + p3); forward: (n_batches + lag) (p1 + p2)
    int n_fin;                 // finalize tasks
    unsigned* ctr;             // [64 done1][64 done2][64 done3], zeroed before launch
    unsigned* fin;             // finalize tasks done (zeroed)
    float2* gpart;             // this state's per-CTA partial gradients [nparts][2^N] (a buffer slot)
    const unsigned* prev_fin;  // fin counter of the previous large state on the same slot, or null
    unsigned prev_nfin;
    double* s2;                // [kS2Lanes][S_2, S_1] accumulated with atomics (zeroed)
};

struct BatchedParams {
    const BatchState* states;  // large states first, then small ones
    int n_states;
    int n_large;
    int64_t total;             // tickets of the small states
    unsigned long long* ticket;
    int nparts;                // = grid; partial-gradient buffers are zero on entry and exit
    double* m2_out;            // [n_states] (device)
    G3Ctl ctl;
};

size_t batched_smem_bytes();
cudaError_t batched_max_grid(int sm_count, int* grid);
cudaError_t launch_batched(const BatchedParams& B, bool fwd, int grid, cudaStream_t st);

}  // namespace hm
