// sre_fwd_n4.cu -- the exact-SRE forward kernels of sre_fwd_kernels.cuh instantiated for
// non-integer n with FP32 powers (the opt-in fast path; see hadamag_set_fp32_powers).
#include "sre_fwd_kernels.cuh"

namespace hm {

HM_SRE_FWD_MODE(4)

}  // namespace hm
