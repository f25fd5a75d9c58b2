// stubs.cu -- entry points whose kernels are not built yet report HADAMAG_ERR_UNSUPPORTED.
#include "extra.h"

namespace hm {
bool use_tensor_path(hadamag_ctx_t c, int N, double n) { (void)c; (void)N; (void)n; return false; }
hadamag_status run_sre_tensor(hadamag_ctx_t c, const float2*, int, double, cudaStream_t, int64_t*) {
    return fail(c, HADAMAG_ERR_UNSUPPORTED, "tensor path not built");
}
}  // namespace hm

