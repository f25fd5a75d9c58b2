// sre_fwd_n3.cu -- the exact-SRE forward kernels of sre_fwd_kernels.cuh instantiated for
// n = 3.
#include "sre_fwd_kernels.cuh"

namespace hm {

HM_SRE_FWD_MODE(3)

}  // namespace hm
