// sre_fwd_n2.cu -- the exact-SRE forward kernels of sre_fwd_kernels.cuh instantiated for
// n = 2.
#include "sre_fwd_kernels.cuh"

namespace hm {

HM_SRE_FWD_MODE(2)

}  // namespace hm
