// sre_tc.h -- launch interface of the tensor-core SRE kernel (internal to libhadamag).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hm {

struct TcParams {
    const float2* psi;       // scaled copy 2^f psi (complex64)
    int N;                   // 21 <= N <= 24
    double nq;               // Renyi index n
    int64_t count;           // number of X-strings
    const int64_t* a_list;   // nullptr: a = 0 .. count-1; else a = a_list[i] (checked in range)
    int per_a;               // 1: per-X-string triples out[count][2^(N-14) tiles][8 warps][3]; 0: per-CTA
    float* scratch;          // R slots x 2^N floats (re plane, im plane of one X-string)
    int R;                   // scratch slots, >= 3 (pass 2 runs two batches behind pass 1)
    int64_t n_batches;       // one X-string per batch, 2^(N-14) tiles per pass
    unsigned* done1;         // per slot, monotonic
    unsigned* done2;
    int* status;
    long long spin_limit;
    unsigned wait_bias;
    const int* scale_exp;    // f
    double* out;             // unscaled triples [S_q, S_1, T_1]
};

cudaError_t tc_max_grid(int N, int mode, int sm_count, int* grid);
cudaError_t launch_tc(const TcParams& P, int mode, int grid, cudaStream_t st);
// per-X-string output: triples per X-string (8 warp partials per tile)
inline int tc_tiles_per_a(int N) { return 1 << (N - 14); }
inline int tc_triples_per_a(int N) { return 8 << (N - 14); }
// max|psi|^2 -> f -> out = 2^f psi (two small kernels); *f_out receives f.
cudaError_t launch_tc_scale(const float2* psi, int N, unsigned* mx, int* f_out, float2* out, cudaStream_t st);

}  // namespace hm
