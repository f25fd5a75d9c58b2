// sre_fwd_n1.cu -- the exact-SRE forward kernels of sre_fwd_kernels.cuh instantiated for
// n = 1 (Shannon limit).
#include "sre_fwd_kernels.cuh"

namespace hm {

HM_SRE_FWD_MODE(1)

}  // namespace hm
