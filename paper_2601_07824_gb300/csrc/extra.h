// extra.h -- launchers and host paths beyond the exact CUDA-core SRE (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctx.h"

namespace hm {

// Monte-Carlo helpers (mc.cu)
cudaError_t launch_mc_xstrings(uint64_t seed, int64_t count, int N, int64_t* out, cudaStream_t st);
cudaError_t launch_mc_stats(const double* terms, const int64_t* a_list, int64_t count, double* out4, cudaStream_t st);
cudaError_t launch_even_xstrings(int64_t count, int64_t* out, cudaStream_t st);
hadamag_status run_sre_hbm_terms(hadamag_ctx_t c, const float2* psi, int N, int64_t count,
                                 const int64_t* a_list, double* terms, cudaStream_t st);

// Tensor-core path (tc_api.cu, sre_tc.cu)
bool use_tensor_path(hadamag_ctx_t c, int N, double n);
// Same contract as run_sre (api.cu): all X-strings (a_list null) or a list; per-CTA partial
// triples in c->part (*nparts of them) or per-X-string triples in `terms` (device).
hadamag_status run_sre_tensor(hadamag_ctx_t c, const float2* psi, int N, double n, int64_t count,
                              const int64_t* a_list, int per_a, double* terms, cudaStream_t st, int64_t* nparts);

}  // namespace hm
