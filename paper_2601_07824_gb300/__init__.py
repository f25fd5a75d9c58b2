"""GB300-native magic (non-stabilizerness) of state vectors.

Implements the hot path of "Computing quantum magic of state vectors" (arXiv 2601.07824):
the exact stabilizer Renyi entropy M_n (Algorithm 2: one Walsh-Hadamard transform per
X-string), the qutrit mana (Algorithm 5: one Z_3^N Fourier transform per X-string), a
uniform-X Monte-Carlo M_2, the thermodynamic-integration Metropolis estimate of M_2
(Algorithm 3), the mana of qutrit density matrices (Algorithm 6) with the partial trace that
produces them, the Wirtinger gradient dM_2/dpsi*, and a batched persistent launch over many
states.  All arithmetic runs in hand-written sm_103a CUDA kernels in
libhadamag.so behind a C ABI (include/hadamag.h); this package only marshals PyTorch CUDA
tensors into that ABI.

`paper_2601_07824_gb300.inputs` (seeded synthetic states) imports no CUDA code.
"""
from __future__ import annotations

__all__ = ["sre", "sre_host", "sre_terms", "sre_even_sector", "mc_xstrings", "sre_mc", "sre_ti", "mana",
           "mana_sums", "mana_qudit", "mana_grad", "mana_mixed", "reduced_density_matrix", "sre_grad",
           "sre_chunk", "sre_slice", "sre_combine", "sre_grad_slice", "sre_grad_combine",
           "SREFunction",
           "sre_batched",
           "context", "HadamagError", "PATH_AUTO", "PATH_CUDACORE", "PATH_TENSOR"]


def __getattr__(name):
    # The binding (and torch) load lazily so that `inputs` stays importable without them.
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
