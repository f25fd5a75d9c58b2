// tc_api.cu -- host side of the tensor-core SRE path (sre_tc.cu): scaling of the state,
// scratch planning and launch.
#include "extra.h"
#include "sre_fwd.h"
#include "sre_tc.h"

namespace hm {

// The tensor path exists for 21 <= N <= 24 (pass 1 of 13 bits, pass 2 of 7 MMA bits plus up to
// three register bits).  HADAMAG_PATH_TENSOR selects it there; every other N, and the AUTO and
// CUDACORE settings, use the CUDA-core kernels.
bool use_tensor_path(hadamag_ctx_t c, int N, double n) {
    (void)n;
    return c->path == HADAMAG_PATH_TENSOR && N >= 21 && N <= 24;
}

hadamag_status run_sre_tensor(hadamag_ctx_t c, const float2* psi, int N, double n, int64_t count,
                              const int64_t* a_list, int per_a, double* terms, cudaStream_t st, int64_t* nparts) {
    if (N < 21 || N > 24) return fail(c, HADAMAG_ERR_UNSUPPORTED, "tensor path covers 21 <= N <= 24 (got %d)", N);
    const int mode = sre_mode(n);
    hadamag_status s;
    cudaError_t e;
    const size_t psi_bytes = ((size_t)1 << N) * sizeof(float2);
    if ((s = ensure_buf(c, c->tc_scratch, psi_bytes + 256))) return s;
    float2* ps = (float2*)c->tc_scratch.ptr;
    unsigned* mx = (unsigned*)((char*)c->tc_scratch.ptr + psi_bytes);
    int* fexp = (int*)(mx + 1);
    e = launch_tc_scale(psi, N, mx, fexp, ps, st);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_scale");

    TcParams P{};
    P.psi = ps; P.N = N; P.nq = n; P.count = count; P.a_list = a_list; P.per_a = per_a;
    // scratch of one X-string: 2^N floats (8 MiB at N = 21); pass 2 runs two batches behind
    // pass 1, so three slots are live at once
    P.R = N <= 22 ? 4 : 3;
    P.n_batches = count;
    const size_t scratch_bytes = (size_t)P.R * ((size_t)1 << N) * sizeof(float);
    if ((s = ensure_buf(c, c->scratch, scratch_bytes))) return s;
    if ((s = ensure_buf(c, c->counters, 2 * 64 * sizeof(unsigned)))) return s;
    P.scratch = (float*)c->scratch.ptr;
    P.done1 = (unsigned*)c->counters.ptr;
    P.done2 = P.done1 + 64;
    P.status = (int*)c->status.ptr;
    P.spin_limit = c->spin_limit;
    P.wait_bias = c->wait_bias;
    P.scale_exp = fexp;
    int grid = 0;
    if ((e = tc_max_grid(N, mode, c->sm_count, &grid)) != cudaSuccess) return cuda_fail(c, e, "tc occupancy");
    const int64_t total = (P.n_batches + 2) * (int64_t)tc_tiles_per_a(N);  // work items
    if (grid > total) grid = (int)total;
    const int tiles = tc_triples_per_a(N);
    if (per_a) {
        if ((s = ensure_buf(c, c->tiles, (size_t)count * tiles * 3 * sizeof(double)))) return s;
        P.out = (double*)c->tiles.ptr;
    } else {
        if ((s = ensure_buf(c, c->part, (size_t)grid * 3 * sizeof(double)))) return s;
        P.out = (double*)c->part.ptr;
    }
    if ((e = cudaMemsetAsync(c->counters.ptr, 0, 2 * 64 * sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(c, e, "memset counters");
    e = launch_tc(P, mode, grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sre_tc");
    if (per_a) {
        e = launch_sum_tiles((double*)c->tiles.ptr, count, tiles, terms, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "sum_tiles");
    }
    if (nparts) *nparts = grid;
    return HADAMAG_OK;
}

}  // namespace hm
