// ctx.h -- the context object behind hadamag_ctx_t and internal host helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <vector>

#include "../../include/hadamag.h"
#include "status_bits.h"

namespace hm {

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct TwoPlan {
    int A, U, R, p1, p2, tiles, triples;  // triples: per-X-string output triples (per_a)
    int UPW, TPT;                         // task shapes: units per pass-1 warp, tiles per pass-2 task
    int lag;                              // stages between a batch's pass 1 and its pass 2
    size_t scratch_bytes;
};

// Lag (stages) between dependent passes of a persistent staged kernel: the smallest D with
// D x per_stage >= 1.5 grid tasks, so that a task rarely waits on one that started less than a
// grid round before it; then lowered until the ring of mult D + 1 slots of slot_bytes fits in
// max_bytes and in the 64 per-slot counters.  At least 1.
inline int pipeline_lag(int64_t per_stage, int grid, int mult, size_t slot_bytes, size_t max_bytes) {
    int64_t D = per_stage > 0 ? (3 * (int64_t)grid + 2 * per_stage - 1) / (2 * per_stage) : 1;
    if (D < 1) D = 1;
    while (D > 1 && ((size_t)(mult * D + 1) * slot_bytes > max_bytes || mult * D + 1 > 63)) --D;
    return (int)D;
}

// Two-pass task shapes picked by the context's autotuner for one (N, accumulation mode).
struct TwoShape {
    int UPW = 0, TPT = 0, R = 0, lag = 1;  // UPW 0: not tuned yet
    int onepass = 0;              // N = 15: 1 when the one-pass kernel won
    int pinned = 0;               // set by hadamag_set_twopass_shape (also used for a few X-strings)
};

}  // namespace hm

struct hadamag_ctx_s {
    int device = 0;
    int sm_count = 0;
    hadamag_path path = HADAMAG_PATH_AUTO;
    cudaStream_t own_stream = nullptr;
    hm::DevBuf status, res, part, scratch, counters, tiles, conv, staging, alist, terms;
    hm::DevBuf grad_acc, batch_meta, batch_sums, tc_scratch, ti_state, rdm_idx;
    double* host_res = nullptr;
    int* host_status = nullptr;
    long long spin_limit = hm::kDefaultSpinLimit;
    unsigned wait_bias = 0;
    int autotune = 1;
    hm::TwoShape twopass_shape[25][5];  // [N][mode], filled by the two-pass autotuner
    int twopass_grid[25][5] = {};       // [N][mode]: resident CTAs of the two-pass kernel (0: not queried)
    int grad_xbatch[25] = {};            // [N]: X-strings per batch of the three-pass adjoint (0: untuned, 8)
    int fp32_powers = 0;  // non-integer n: FP32 powers (mode 4) where n <= 4 and n (N + 2) <= 100
    void* host_table = nullptr;  // pinned copy of the batched state table
    size_t host_table_bytes = 0;
    uint64_t launches = 0;
    char last_error[256] = {0};
    std::vector<hm::DevBuf*> all_bufs() {
        return {&status, &res, &part, &scratch, &counters, &tiles, &conv, &staging, &alist, &terms,
                &grad_acc, &batch_meta, &batch_sums, &tc_scratch, &ti_state, &rdm_idx};
    }
};

namespace hm {

hadamag_status fail(hadamag_ctx_t c, hadamag_status s, const char* fmt, ...);
hadamag_status cuda_fail(hadamag_ctx_t c, cudaError_t e, const char* where);
hadamag_status ensure_buf(hadamag_ctx_t c, DevBuf& b, size_t bytes);
bool aligned16(const void* p);
hadamag_status as_c64(hadamag_ctx_t c, const void* psi, int64_t n, hadamag_dtype dt, cudaStream_t st,
                      const float2** out);
int sre_mode(double n);
TwoPlan plan_twopass(int N, int UPW = 2, int TPT = 2, int R = 0, int lag = 1);
hadamag_status run_sre(hadamag_ctx_t c, const float2* psi, int N, double n, int64_t count,
                       const int64_t* a_list, int per_a, double* terms, cudaStream_t st, int64_t* nparts);
hadamag_status launch_twopass_plan(hadamag_ctx_t c, const float2* psi, int N, double n, int mode, const TwoPlan& pl,
                                   int64_t count, const int64_t* a_list, int64_t a_base, int per_a, double* terms,
                                   cudaStream_t st, int64_t* nparts);
hadamag_status tune_twopass(hadamag_ctx_t c, const float2* psi, int N, double n, int mode, cudaStream_t st);
hadamag_status status_word_now(hadamag_ctx_t c, cudaStream_t st);
hadamag_status begin(hadamag_ctx_t c, cudaStream_t st);
hadamag_status finish(hadamag_ctx_t c, const double* res_dev, int n, cudaStream_t st);
hadamag_status status_word(hadamag_ctx_t c);
hadamag_status sre_sums(hadamag_ctx_t c, const float2* p, int N, double n, cudaStream_t st, double sums[3]);
hadamag_status sre_from_sums(hadamag_ctx_t c, int N, double n, const double sums[3], double* M_out,
                             double* lost_out);

}  // namespace hm
