// mana_api.cu -- C ABI entry points for the qutrit mana: pure states (Algorithm 5, Eq. mana2)
// and density matrices (Algorithm 6's Wigner function, Sec. 3.3.3).
#include <cmath>

#include "ctx.h"
#include "mana.h"
#include "sre_fwd.h"

using namespace hm;

namespace {

int64_t ipow3(int n) {
    int64_t r = 1;
    while (n-- > 0) r *= 3;
    return r;
}

// sums = [sum_{a,b} |chi_b(a)|, sum chi_b(a), sum chi_b(a)^2] (device FP64, then host).  psi is
// the state (3^N values) or, with mixed, the density matrix (3^N x 3^N, row-major).
hadamag_status mana_sums(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt, cudaStream_t st,
                         double sums[3], bool mixed) {
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    const int64_t dim = ipow3(N);
    const float2* p;
    if ((s = as_c64(c, psi, mixed ? dim * dim : dim, dt, st, &p))) return s;
    int64_t nparts = 0;
    if (N <= 8) {
        if ((s = ensure_buf(c, c->part, (size_t)c->sm_count * 64 * 3 * sizeof(double)))) return s;
        int grid = 0;
        e = launch_mana_onepass(p, N, mixed, (double*)c->part.ptr, c->sm_count, &grid, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "mana_onepass");
        nparts = grid;
    } else {
        const int M = N - 8;
        const size_t per_a = (size_t)dim * sizeof(float2);
        int A = 8;
        while (A > 1 && (size_t)A * per_a > ((size_t)16 << 20)) A >>= 1;
        ManaParams P{};
        P.psi = p; P.N = N; P.count = mana_pair_items(N); P.R = 3; P.A = A;
        P.n_batches = (P.count + A - 1) / A;
        P.p1 = P.p2 = A * (int)ipow3(M);
        int grid = 0;
        if ((e = mana_twopass_grid(N, mixed, c->sm_count, &grid)) != cudaSuccess) return cuda_fail(c, e, "occupancy");
        const int64_t total = P.n_batches * ((int64_t)P.p1 + P.p2);
        if (grid > total) grid = (int)total;
        if ((s = ensure_buf(c, c->scratch, (size_t)P.R * A * per_a))) return s;
        if ((s = ensure_buf(c, c->counters, 2 * 64 * sizeof(unsigned)))) return s;
        if ((s = ensure_buf(c, c->part, (size_t)grid * 3 * sizeof(double)))) return s;
        P.scratch = (float2*)c->scratch.ptr;
        P.done1 = (unsigned*)c->counters.ptr; P.done2 = P.done1 + 64;
        P.status = (int*)c->status.ptr; P.spin_limit = c->spin_limit; P.wait_bias = c->wait_bias;
        P.out = (double*)c->part.ptr;
        if ((e = cudaMemsetAsync(c->counters.ptr, 0, 2 * 64 * sizeof(unsigned), st)) != cudaSuccess)
            return cuda_fail(c, e, "memset counters");
        e = launch_mana_twopass(P, mixed, grid, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "mana_twopass");
        nparts = grid;
    }
    e = launch_sum_triples((const double*)c->part.ptr, nparts, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    sums[0] = c->host_res[0]; sums[1] = c->host_res[1]; sums[2] = c->host_res[2];
    return HADAMAG_OK;
}

hadamag_status check_args(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt) {
    if (!aligned16(psi)) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 13) return fail(c, HADAMAG_ERR_INVALID_ARG, "mana needs 1 <= N <= 13 (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    return HADAMAG_OK;
}

}  // namespace

extern "C" hadamag_status hadamag_mana(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt,
                                       double* mana_out, double* sum_w_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    hadamag_status s;
    if ((s = check_args(c, psi, N, dt))) return s;
    double sums[3];
    if ((s = mana_sums(c, psi, N, dt, reinterpret_cast<cudaStream_t>(stream), sums, false))) return s;
    const double sw = sums[0] / (double)ipow3(N);  // Eq. (mana2): sum_u |W(u)| = m / 3^N
    double m = std::log2(sw);
    if (m == 0.0) m = 0.0;
    if (mana_out) *mana_out = m;
    if (sum_w_out) *sum_w_out = sw;
    if (!std::isfinite(m)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite mana");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_mana_sums(hadamag_ctx_t c, const void* psi, int N, hadamag_dtype dt,
                                            double* sums_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!sums_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null output");
    hadamag_status s;
    if ((s = check_args(c, psi, N, dt))) return s;
    return mana_sums(c, psi, N, dt, reinterpret_cast<cudaStream_t>(stream), sums_out, false);
}

extern "C" hadamag_status hadamag_mana_qudit(hadamag_ctx_t c, const void* psi, int N, int d, hadamag_dtype dt,
                                             double* mana_out, double* sums_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi)) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    const int nmax = d == 3 ? 13 : mana_qudit_max_n(d);
    if (nmax == 0) return fail(c, HADAMAG_ERR_UNSUPPORTED, "d must be 3, 5, 7, 11 or 13 (got %d)", d);
    if (N < 1 || N > nmax) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, %d] for d = %d (got %d)", nmax, d, N);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double sums[3];
    hadamag_status s;
    int64_t dim = 1;
    for (int j = 0; j < N; ++j) dim *= d;
    if (d == 3) {
        if ((s = mana_sums(c, psi, N, dt, st, sums, false))) return s;
    } else {
        cudaError_t e;
        if ((s = begin(c, st))) return s;
        const float2* p;
        if ((s = as_c64(c, psi, dim, dt, st, &p))) return s;
        const int max_grid = c->sm_count * 8;
        if ((s = ensure_buf(c, c->part, (size_t)max_grid * 3 * sizeof(double)))) return s;
        int grid = 0;
        e = launch_mana_qudit(p, N, d, (double*)c->part.ptr, c->sm_count, max_grid, &grid, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "mana_qudit");
        e = launch_sum_triples((const double*)c->part.ptr, grid, (double*)c->res.ptr, st);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
        if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
        sums[0] = c->host_res[0]; sums[1] = c->host_res[1]; sums[2] = c->host_res[2];
    }
    double m = std::log2(sums[0] / (double)dim);  // sum_u |W(u)|, W = chi / d^N
    if (m == 0.0) m = 0.0;
    if (mana_out) *mana_out = m;
    if (sums_out) { sums_out[0] = sums[0]; sums_out[1] = sums[1]; sums_out[2] = sums[2]; }
    if (!std::isfinite(m)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite mana");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_mana_mixed_qudit(hadamag_ctx_t c, const void* rho, int N, int d, hadamag_dtype dt,
                                                   double* mana_out, double* sums_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (d == 3) return hadamag_mana_mixed(c, rho, N, dt, mana_out, sums_out, stream);
    if (!aligned16(rho)) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    const int nmax = mana_qudit_max_n(d);
    if (nmax == 0) return fail(c, HADAMAG_ERR_UNSUPPORTED, "d must be 3, 5, 7, 11 or 13 (got %d)", d);
    if (N < 1 || N > nmax) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, %d] for d = %d (got %d)", nmax, d, N);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    int64_t dim = 1;
    for (int j = 0; j < N; ++j) dim *= d;
    const float2* p;
    if ((s = as_c64(c, rho, dim * dim, dt, st, &p))) return s;
    const int max_grid = c->sm_count * 8;
    if ((s = ensure_buf(c, c->part, (size_t)max_grid * 3 * sizeof(double)))) return s;
    int grid = 0;
    e = launch_mana_qudit_mixed(p, N, d, (double*)c->part.ptr, c->sm_count, max_grid, &grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mana_qudit_mixed");
    e = launch_sum_triples((const double*)c->part.ptr, grid, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    double m = std::log2(c->host_res[0] / (double)dim);
    if (m == 0.0) m = 0.0;
    if (mana_out) *mana_out = m;
    if (sums_out) { sums_out[0] = c->host_res[0]; sums_out[1] = c->host_res[1]; sums_out[2] = c->host_res[2]; }
    if (!std::isfinite(m)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite mana");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_mana_grad(hadamag_ctx_t c, const void* psi, int N, int d, hadamag_dtype dt,
                                            double* mana_out, void* grad, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(psi) || !aligned16(grad) || !mana_out) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    const int nmax = mana_qudit_max_n(d);
    if (nmax == 0) return fail(c, HADAMAG_ERR_UNSUPPORTED, "d must be 3, 5, 7, 11 or 13 (got %d)", d);
    if (N < 1 || N > nmax) return fail(c, HADAMAG_ERR_INVALID_ARG, "N must be in [1, %d] for d = %d (got %d)", nmax, d, N);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    hadamag_status s;
    cudaError_t e;
    if ((s = begin(c, st))) return s;
    int dim = 1;
    for (int j = 0; j < N; ++j) dim *= d;
    const float2* p;
    if ((s = as_c64(c, psi, dim, dt, st, &p))) return s;
    const int max_grid = c->sm_count * 2;
    const size_t gbytes = (size_t)max_grid * dim * sizeof(double2);
    if ((s = ensure_buf(c, c->part, (size_t)max_grid * 3 * sizeof(double)))) return s;
    if ((s = ensure_buf(c, c->grad_acc, gbytes))) return s;
    if ((e = cudaMemsetAsync(c->grad_acc.ptr, 0, gbytes, st)) != cudaSuccess) return cuda_fail(c, e, "memset");
    int grid = 0;
    e = launch_mana_grad(p, N, d, (double*)c->part.ptr, (double2*)c->grad_acc.ptr, c->sm_count, max_grid, &grid, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mana_grad");
    e = launch_sum_triples((const double*)c->part.ptr, grid, (double*)c->res.ptr, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sum_triples");
    e = launch_mana_grad_finalize((const double2*)c->grad_acc.ptr, grid, dim, (const double*)c->res.ptr, grad,
                                  dt == HADAMAG_C128, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "mana_grad_finalize");
    if ((s = finish(c, (const double*)c->res.ptr, 3, st))) return s;
    double m = std::log2(c->host_res[0] / (double)dim);
    if (m == 0.0) m = 0.0;
    *mana_out = m;
    if (!std::isfinite(m)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite mana");
    return HADAMAG_OK;
}

extern "C" hadamag_status hadamag_mana_mixed(hadamag_ctx_t c, const void* rho, int N, hadamag_dtype dt,
                                             double* mana_out, double* sums_out, hadamag_stream_t stream) {
    if (!c) return HADAMAG_ERR_INVALID_ARG;
    if (!aligned16(rho)) return fail(c, HADAMAG_ERR_INVALID_ARG, "null or misaligned pointer");
    if (N < 1 || N > 10) return fail(c, HADAMAG_ERR_INVALID_ARG, "mixed-state mana needs 1 <= N <= 10 (got %d)", N);
    if (dt != HADAMAG_C64 && dt != HADAMAG_C128) return fail(c, HADAMAG_ERR_INVALID_ARG, "bad dtype");
    double sums[3];
    hadamag_status s;
    if ((s = mana_sums(c, rho, N, dt, reinterpret_cast<cudaStream_t>(stream), sums, true))) return s;
    double m = std::log2(sums[0] / (double)ipow3(N));  // sum_u |W_u|, W_u = tr(rho A_u) / 3^N
    if (m == 0.0) m = 0.0;
    if (mana_out) *mana_out = m;
    if (sums_out) { sums_out[0] = sums[0]; sums_out[1] = sums[1]; sums_out[2] = sums[2]; }
    if (!std::isfinite(m)) return fail(c, HADAMAG_ERR_NONFINITE, "non-finite mana");
    return HADAMAG_OK;
}
