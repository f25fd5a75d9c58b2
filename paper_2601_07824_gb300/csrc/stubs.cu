// stubs.cu -- entry points whose kernels are not built yet report HADAMAG_ERR_UNSUPPORTED.
#include "extra.h"

namespace hm {
bool use_tensor_path(hadamag_ctx_t c, int N, double n) { (void)c; (void)N; (void)n; return false; }
hadamag_status run_sre_tensor(hadamag_ctx_t c, const float2*, int, double, cudaStream_t, int64_t*) {
    return fail(c, HADAMAG_ERR_UNSUPPORTED, "tensor path not built");
}
hadamag_status run_sre_hbm_terms(hadamag_ctx_t c, const float2*, int N, int64_t, const int64_t*, double*,
                                 cudaStream_t) {
    return fail(c, HADAMAG_ERR_UNSUPPORTED, "N = %d needs the HBM schedule (not built)", N);
}
}  // namespace hm

extern "C" hadamag_status hadamag_sre_batched(hadamag_ctx_t c, int, const void* const*, const int*, int,
                                              void* const*, double*, hadamag_stream_t) {
    return hm::fail(c, HADAMAG_ERR_UNSUPPORTED, "batched launch not built");
}
