// sre_fwd.h -- launch interface of the SRE forward kernels (internal to libhadamag).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hm {

// Thread layout of the one-pass kernel for a transform of 2^L complex values.
template <int L>
struct OnepassShape {
    static constexpr int E = L < 5 ? L : 5;        // register bits per thread
    static constexpr int G = 1 << (L - E);          // threads per X-string
    static constexpr int NT = G <= 32 ? 256 : G;    // threads per CTA
    static constexpr int GPC = NT / G;              // X-strings in flight per CTA
};

struct OnepassArgs {
    const float2* psi;
    int N;
    double nq;               // Renyi index n
    int64_t count;           // number of X-strings (2^N, or the list length)
    const int64_t* a_list;   // nullptr: a = a_base .. a_base + count-1
    int64_t a_base;
    double* out;             // per_a: [count][3]; else per-CTA [grid][3]
    int per_a;
    int* status;
    int grid;                // 0: choose from occupancy; the launcher writes back the grid used
};

struct TwoPassParams {
    const float2* psi;
    int N;
    double nq;
    int64_t count;
    const int64_t* a_list;
    float2* scratch;         // R slots x A X-strings x 2^(N-1) complex values
    int R, A, U;             // slots, X-strings per batch, warps per X-string in pass 1 (A*U = 8 or 1)
    int UPW, TPT;            // units per pass-1 warp (K1 = 10; even), column tiles per pass-2 task
    int lag;                 // pass 2 of a batch runs `lag` stages after its pass 1 (1 <= lag < R)
    int64_t n_batches;
    int p1, p2;              // pass-1 / pass-2 tasks per batch
    int64_t a_base;          // without a list: X-string of entry i is a_base + i
    unsigned* done1;         // per slot: finished pass-1 tasks (monotonic)
    unsigned* done2;         // per slot: finished pass-2 tasks (monotonic)
    int* status;
    long long spin_limit;
    unsigned wait_bias;      // added to every wait target (fault-injection tests only)
    double* out;             // per_a: [count][tiles][3]; else per-CTA [grid][3]
    int per_a;
};

// Three-pass per-X-string kernel for 25 <= N <= 28 (scratch in HBM), one X-string per batch.
struct HbmParams {
    const float2* psi;
    int N;
    int64_t count;
    const int64_t* a_list;
    float2* scratch;         // R slots x 2^(N-1) values
    int R;
    int64_t n_batches;
    int p1, p2, p3;          // tasks per batch (2^(N-14) each)
    unsigned* done1;
    unsigned* done2;
    unsigned* done3;
    int* status;
    long long spin_limit;
    unsigned wait_bias;
    double* out;             // [count][tiles][3]
};
int hbm_tiles_per_a(int N);
cudaError_t launch_hbm(const HbmParams& P, int sm_count, int* grid, cudaStream_t st);

// Two-pass geometry for N in [15, 24]: pass 1 transforms K1 = twopass_k1(N) bits (10 or 13),
// pass 2 the other N-1-K1 bits, in tiles of 2^13 values; tiles per X-string:
int twopass_tiles_per_a(int N);
// per-X-string output triples of the two-pass kernel (one per tile and warp)
inline int twopass_triples_per_a(int N) { return 8 * twopass_tiles_per_a(N); }
int twopass_k1(int N);

cudaError_t launch_onepass(OnepassArgs& A, int mode, int sm_count, cudaStream_t st);
// Requires a prior twopass_max_grid(N, mode) on the current device (it sets the kernel's
// shared-memory limit).
cudaError_t launch_twopass(const TwoPassParams& P, int mode, int grid, cudaStream_t st);
cudaError_t twopass_max_grid(int N, int mode, int sm_count, int* grid);
cudaError_t launch_sum_triples(const double* in, int64_t n, double* out, cudaStream_t st);
cudaError_t launch_sum_tiles(const double* in, int64_t count, int tiles, double* out, cudaStream_t st);
cudaError_t launch_c128_to_c64(const void* in, float2* out, int64_t n, cudaStream_t st);

}  // namespace hm
