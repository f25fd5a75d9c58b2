// sre_fwd_n0.cu -- the exact-SRE forward kernels of sre_fwd_kernels.cuh instantiated for
// any other n (FP64 powers).
#include "sre_fwd_kernels.cuh"

namespace hm {

HM_SRE_FWD_MODE(0)

}  // namespace hm
