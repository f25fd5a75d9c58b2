"""PyTorch-facing calls with the C ABI's names (argument marshalling only).

Tensors must be CUDA, contiguous, complex64 or complex128 (batched: complex64).  Work is
enqueued on torch's current stream of the tensor's device.
"""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np
import torch

from ._lib import (C64, C128, PATH_AUTO, PATH_CUDACORE, PATH_TENSOR, HadamagError, context)

__all__ = ["sre", "sre_host", "sre_terms", "mc_xstrings", "sre_mc", "mana", "mana_sums", "sre_grad",
           "sre_chunk", "sre_slice", "sre_combine", "sre_grad_slice", "sre_grad_combine",
           "SREFunction", "sre_batched", "context", "HadamagError", "PATH_AUTO",
           "PATH_CUDACORE", "PATH_TENSOR"]


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"state must be complex64 or complex128, got {t.dtype}")


def _check_state(psi: torch.Tensor, d: int = 2) -> int:
    if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
        raise TypeError("state must be a CUDA tensor")
    if psi.dim() != 1 or not psi.is_contiguous():
        raise ValueError("state must be a contiguous 1-D tensor")
    n, size = 0, psi.numel()
    while d ** n < size:
        n += 1
    if d ** n != size or n < 1:
        raise ValueError(f"state length {size} is not {d}^N")
    return n


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ctx(t: torch.Tensor):
    return context(t.device.index if t.device.index is not None else torch.cuda.current_device())


@contextlib.contextmanager
def _path(c, path):
    """Select the transform path of context `c` for one call (None: keep the context's)."""
    if path is None:
        yield
        return
    prev = getattr(c, "path", PATH_AUTO)
    c.set_path(path)
    try:
        yield
    finally:
        c.set_path(prev)


def sre(psi: torch.Tensor, n: float = 2.0, path: int | None = None):
    """(M_n, lost_norm): exact SRE, Eq. (sre), by the per-X-string Walsh-Hadamard method.

    path: None (the context's setting), PATH_CUDACORE, or PATH_TENSOR (tcgen05 +-1 Hadamard
    blocks on fp16 hi/lo operands, used for 21 <= N <= 24) -- for this call only."""
    N = _check_state(psi)
    c = _ctx(psi)
    M, ln = ctypes.c_double(), ctypes.c_double()
    with _path(c, path):
        c.check(c.lib.hadamag_sre(c.h, ctypes.c_void_p(psi.data_ptr()), N, float(n), _dtype_code(psi),
                                  ctypes.byref(M), ctypes.byref(ln), _stream(psi)), "hadamag_sre")
    return M.value, ln.value


def sre_host(psi: np.ndarray, n: float = 2.0, device: int = 0):
    """hadamag_sre on a HOST array (the call copies it to the device itself)."""
    a = np.ascontiguousarray(psi)
    if a.dtype == np.complex64:
        code = C64
    elif a.dtype == np.complex128:
        code = C128
    else:
        raise TypeError("state must be complex64 or complex128")
    N = int(a.size).bit_length() - 1
    if 1 << N != a.size:
        raise ValueError("state length must be 2^N")
    c = context(device)
    M, ln = ctypes.c_double(), ctypes.c_double()
    c.check(c.lib.hadamag_sre_host(c.h, ctypes.c_void_p(a.ctypes.data), N, float(n), code,
                                   ctypes.byref(M), ctypes.byref(ln)), "hadamag_sre_host")
    return M.value, ln.value


def sre_terms(psi: torch.Tensor, n: float, a_list: torch.Tensor, path: int | None = None) -> torch.Tensor:
    """Per-X-string sums [sum_b |chi|^{2n}, sum_b |chi|^2, sum_b |chi|^2 log2 |chi|^2] (count x 3)."""
    N = _check_state(psi)
    if a_list.dtype != torch.int64 or a_list.device != psi.device or not a_list.is_contiguous():
        raise ValueError("a_list must be a contiguous int64 tensor on the state's device")
    out = torch.empty((a_list.numel(), 3), dtype=torch.float64, device=psi.device)
    c = _ctx(psi)
    with _path(c, path):
        c.check(c.lib.hadamag_sre_terms(c.h, ctypes.c_void_p(psi.data_ptr()), N, float(n), _dtype_code(psi),
                                        ctypes.c_void_p(a_list.data_ptr()), a_list.numel(),
                                        ctypes.c_void_p(out.data_ptr()), _stream(psi)), "hadamag_sre_terms")
    return out


def mc_xstrings(seed: int, count: int, N: int, device: int = 0) -> torch.Tensor:
    """SplitMix64 X-strings a_i (top N bits of output i), as drawn by sre_mc."""
    out = torch.empty(count, dtype=torch.int64, device=f"cuda:{device}")
    c = context(device)
    c.check(c.lib.hadamag_mc_xstrings(c.h, ctypes.c_uint64(seed & (2 ** 64 - 1)), count, int(N),
                                      ctypes.c_void_p(out.data_ptr()), _stream(out)), "hadamag_mc_xstrings")
    return out


def sre_mc(psi: torch.Tensor, samples: int, seed: int, path: int | None = None):
    """(M2_hat, stderr) of the uniform-X Monte-Carlo estimator."""
    N = _check_state(psi)
    c = _ctx(psi)
    M, se = ctypes.c_double(), ctypes.c_double()
    with _path(c, path):
        c.check(c.lib.hadamag_sre_mc(c.h, ctypes.c_void_p(psi.data_ptr()), N, int(samples),
                                     ctypes.c_uint64(seed & (2 ** 64 - 1)), _dtype_code(psi),
                                     ctypes.byref(M), ctypes.byref(se), _stream(psi)), "hadamag_sre_mc")
    return M.value, se.value


def sre_even_sector(psi: torch.Tensor, n: float = 2.0, path: int | None = None):
    """(M_n, lost_norm) from the even-weight X-strings only, exact for U(1) or prod_j Z_j
    symmetric states (Sec. 3.2), at half the work of `sre`."""
    N = _check_state(psi)
    c = _ctx(psi)
    M, lost = ctypes.c_double(), ctypes.c_double()
    with _path(c, path):
        c.check(c.lib.hadamag_sre_even_sector(c.h, ctypes.c_void_p(psi.data_ptr()), N, float(n), _dtype_code(psi),
                                              ctypes.byref(M), ctypes.byref(lost), _stream(psi)),
                "hadamag_sre_even_sector")
    return M.value, lost.value


def sre_ti(psi: torch.Tensor, L: int, n_s: int, seed: int, burn_in: int = 0, eps: float = 0.0,
           record: bool = False, even_sector: bool = False):
    """Thermodynamic-integration estimate of M_2 (Sec. 3.2, Algorithm 3): (M2_hat, delta M2, chain
    means), delta M2 from Eq. m2error with batch-means variances; with record=True also the
    chains' X-strings after every step as an int64 tensor [L, burn_in + n_s] on the state's
    device.  even_sector=True keeps the chains on even-weight X-strings (U(1) or prod_j Z_j
    symmetric states)."""
    N = _check_state(psi)
    c = _ctx(psi)
    M, err = ctypes.c_double(), ctypes.c_double()
    means = (ctypes.c_double * int(L))()
    traj = torch.empty((int(L), int(burn_in) + int(n_s)), dtype=torch.int64, device=psi.device) if record else None
    c.check(c.lib.hadamag_sre_ti(c.h, ctypes.c_void_p(psi.data_ptr()), N, int(L), int(n_s), int(burn_in),
                                 ctypes.c_uint64(seed & (2 ** 64 - 1)), float(eps), 1 if even_sector else 0,
                                 _dtype_code(psi), ctypes.byref(M), ctypes.byref(err), means,
                                 ctypes.c_void_p(traj.data_ptr()) if record else None, _stream(psi)),
            "hadamag_sre_ti")
    out = (M.value, err.value, list(means))
    return out + (traj,) if record else out


def mana(psi: torch.Tensor):
    """(mana in bits, sum_u |W(u)|) of an N-qutrit state (Algorithm 5, Eq. mana2)."""
    N = _check_state(psi, 3)
    c = _ctx(psi)
    m, sw = ctypes.c_double(), ctypes.c_double()
    c.check(c.lib.hadamag_mana(c.h, ctypes.c_void_p(psi.data_ptr()), N, _dtype_code(psi),
                               ctypes.byref(m), ctypes.byref(sw), _stream(psi)), "hadamag_mana")
    return m.value, sw.value


def mana_qudit(psi: torch.Tensor, d: int):
    """(mana in bits, [sum |chi|, sum chi, sum chi^2]) of N qudits of odd prime dimension d
    (d^N amplitudes; Sec. 2's construction for general odd prime d, Algorithm 5 generalised)."""
    if int(d) < 2:
        raise ValueError("d must be an odd prime")
    N = _check_state(psi, int(d))
    c = _ctx(psi)
    m = ctypes.c_double()
    sums = (ctypes.c_double * 3)()
    c.check(c.lib.hadamag_mana_qudit(c.h, ctypes.c_void_p(psi.data_ptr()), N, int(d), _dtype_code(psi),
                                     ctypes.byref(m), sums, _stream(psi)), "hadamag_mana_qudit")
    return m.value, list(sums)


def mana_grad(psi: torch.Tensor, d: int = 3):
    """(mana in bits, d mana / d psi*) of N qudits of odd prime dimension d (Wirtinger gradient
    on the vector as given; a tensor like psi)."""
    if int(d) < 2:
        raise ValueError("d must be an odd prime")
    N = _check_state(psi, int(d))
    c = _ctx(psi)
    m = ctypes.c_double()
    grad = torch.empty_like(psi)
    c.check(c.lib.hadamag_mana_grad(c.h, ctypes.c_void_p(psi.data_ptr()), N, int(d), _dtype_code(psi),
                                    ctypes.byref(m), ctypes.c_void_p(grad.data_ptr()), _stream(psi)),
            "hadamag_mana_grad")
    return m.value, grad


def mana_mixed(rho: torch.Tensor, d: int = 3):
    """(mana in bits, [sum |chi|, sum chi, sum chi^2]) of a density matrix of N qudits (d = 3:
    qutrits, Algorithm 6's W via the Algorithm 5 transform, Sec. 3.3.3; other odd primes d as
    Sec. 2 allows) given as a d^N x d^N CUDA tensor."""
    if int(d) < 2:
        raise ValueError("d must be an odd prime")
    if not isinstance(rho, torch.Tensor) or not rho.is_cuda:
        raise TypeError("rho must be a CUDA tensor")
    if rho.dim() != 2 or rho.shape[0] != rho.shape[1] or not rho.is_contiguous():
        raise ValueError("rho must be a contiguous square matrix")
    n, D = 0, rho.shape[0]
    while d ** n < D:
        n += 1
    if d ** n != D or n < 1:
        raise ValueError(f"rho must be {d}^N x {d}^N, got {D} x {D}")
    c = _ctx(rho)
    m = ctypes.c_double()
    sums = (ctypes.c_double * 3)()
    c.check(c.lib.hadamag_mana_mixed_qudit(c.h, ctypes.c_void_p(rho.data_ptr()), n, int(d), _dtype_code(rho),
                                           ctypes.byref(m), sums, _stream(rho)), "hadamag_mana_mixed_qudit")
    return m.value, list(sums)


def reduced_density_matrix(psi: torch.Tensor, keep, d: int = 3) -> torch.Tensor:
    """rho_A = tr_B |psi><psi| of N sites of dimension d (qutrits by default) for the sites in
    `keep` (site keep[m] is digit m of rho_A's row and column index); complex64 [d^k, d^k] on
    the state's device."""
    if int(d) < 2:
        raise ValueError("d must be >= 2")
    N = _check_state(psi, int(d))
    keep = [int(k) for k in keep]
    c = _ctx(psi)
    rho = torch.empty((int(d) ** len(keep), int(d) ** len(keep)), dtype=torch.complex64, device=psi.device)
    arr = (ctypes.c_int * max(1, len(keep)))(*keep)
    c.check(c.lib.hadamag_reduced_density_matrix_qudit(c.h, ctypes.c_void_p(psi.data_ptr()), N, int(d),
                                                       _dtype_code(psi), arr, len(keep),
                                                       ctypes.c_void_p(rho.data_ptr()), _stream(psi)),
            "hadamag_reduced_density_matrix")
    return rho


def mana_sums(psi: torch.Tensor):
    """[sum |chi|, sum chi, sum chi^2] over all (a, b); W = chi / 3^N."""
    N = _check_state(psi, 3)
    c = _ctx(psi)
    out = (ctypes.c_double * 3)()
    c.check(c.lib.hadamag_mana_sums(c.h, ctypes.c_void_p(psi.data_ptr()), N, _dtype_code(psi), out,
                                    _stream(psi)), "hadamag_mana_sums")
    return list(out)


def sre_grad(psi: torch.Tensor):
    """(M_2, dM_2/dpsi*) -- the Wirtinger gradient on the unnormalised state."""
    N = _check_state(psi)
    g = torch.empty_like(psi)
    c = _ctx(psi)
    M = ctypes.c_double()
    c.check(c.lib.hadamag_sre_grad(c.h, ctypes.c_void_p(psi.data_ptr()), N, _dtype_code(psi),
                                   ctypes.byref(M), ctypes.c_void_p(g.data_ptr()), _stream(psi)),
            "hadamag_sre_grad")
    return M.value, g


def sre_chunk(N: int) -> int:
    """Chunk size of the X-string slices (slices start and end on multiples of it)."""
    from ._lib import load
    ch = int(load().hadamag_sre_chunk(int(N)))
    if ch <= 0:
        raise ValueError(f"N = {N} outside the exact-SRE range")
    return ch


def sre_slice(psi: torch.Tensor, n: float, a0: int, a1: int, path: int | None = None) -> torch.Tensor:
    """Per-chunk sums [sum |c|^{2n}, sum |c|^2, sum |c|^2 log2 |c|^2] over the X-strings
    a0 <= a < a1, as a float64 tensor [(a1 - a0) / chunk, 3] on the state's device."""
    N = _check_state(psi)
    ch = sre_chunk(N)
    out = torch.empty((max(0, (int(a1) - int(a0)) // ch), 3), dtype=torch.float64, device=psi.device)
    c = _ctx(psi)
    buf = out if out.numel() else torch.empty(3, dtype=torch.float64, device=psi.device)
    with _path(c, path):
        c.check(c.lib.hadamag_sre_slice(c.h, ctypes.c_void_p(psi.data_ptr()), N, float(n), _dtype_code(psi),
                                        int(a0), int(a1), ctypes.c_void_p(buf.data_ptr()), _stream(psi)),
                "hadamag_sre_slice")
    return out


def sre_combine(N: int, n: float, chunks) -> tuple:
    """(M_n, lost_norm) from the chunk sums of every slice, in chunk order (host only)."""
    from ._lib import load
    a = np.ascontiguousarray(np.asarray(chunks.cpu() if isinstance(chunks, torch.Tensor) else chunks,
                                        dtype=np.float64)).reshape(-1, 3)
    M, ln = ctypes.c_double(), ctypes.c_double()
    rc = load().hadamag_sre_combine(int(N), float(n), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    a.shape[0], ctypes.byref(M), ctypes.byref(ln))
    if rc != 0:
        raise HadamagError(rc, "hadamag_sre_combine")
    return M.value, ln.value


def sre_grad_slice(psi: torch.Tensor, a0: int, a1: int):
    """((S_2, S_1) of the slice, dS_2/dpsi* of the slice as complex128 [2^N] on the device)."""
    N = _check_state(psi)
    dS = torch.empty(psi.numel(), dtype=torch.complex128, device=psi.device)
    sums = (ctypes.c_double * 2)()
    c = _ctx(psi)
    c.check(c.lib.hadamag_sre_grad_slice(c.h, ctypes.c_void_p(psi.data_ptr()), N, _dtype_code(psi), int(a0),
                                         int(a1), sums, ctypes.c_void_p(dS.data_ptr()), _stream(psi)),
            "hadamag_sre_grad_slice")
    return (sums[0], sums[1]), dS


def sre_grad_combine(dS: torch.Tensor, S2: float, dtype=torch.complex64):
    """(M_2, dM_2/dpsi*) from the dS_2/dpsi* and S_2 summed over every slice."""
    if dS.dtype != torch.complex128 or not dS.is_cuda or not dS.is_contiguous():
        raise ValueError("dS must be a contiguous complex128 CUDA tensor")
    N = _check_state(dS)
    g = torch.empty(dS.numel(), dtype=dtype, device=dS.device)
    c = _ctx(dS)
    M = ctypes.c_double()
    c.check(c.lib.hadamag_sre_grad_combine(c.h, ctypes.c_void_p(dS.data_ptr()), N, float(S2), _dtype_code(g),
                                           ctypes.byref(M), ctypes.c_void_p(g.data_ptr()), _stream(dS)),
            "hadamag_sre_grad_combine")
    return M.value, g


class SREFunction(torch.autograd.Function):
    """M_2(psi) as a differentiable scalar.  backward returns grad_out * 2 dM_2/dpsi*, which
    is PyTorch's convention for real functions of complex inputs (grad of |z|^2 is 2z)."""

    @staticmethod
    def forward(ctx, psi):
        M2, g = sre_grad(psi.detach().contiguous())
        ctx.save_for_backward(g)
        return torch.tensor(M2, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return (2.0 * grad_out.to(g.real.dtype)) * g


def sre_batched(states, want_grad: bool = False, out=None, grads=None, sync: bool = True):
    """M_2 (and dM_2/dpsi*) of many complex64 states of uneven N (10..18) in one persistent launch.

    Returns (M2 tensor [count] float64, list of gradients or None).  With sync=False nothing
    waits on the host (the call can be captured in a CUDA graph after one uncaptured call with
    the same shapes); pass preallocated `out` / `grads` then."""
    if not states:
        raise ValueError("empty batch")
    dev = states[0].device
    Ns, ptrs = [], []
    for s in states:
        if s.dtype != torch.complex64 or s.device != dev:
            raise ValueError("batched states must be complex64 on one device")
        Ns.append(_check_state(s))
        ptrs.append(s.data_ptr())
    if want_grad and grads is None:
        grads = [torch.empty_like(s) for s in states]
    if out is None:
        out = torch.empty(len(states), dtype=torch.float64, device=dev)
    k = len(states)
    P = (ctypes.c_void_p * k)(*ptrs)
    G = (ctypes.c_void_p * k)(*([g.data_ptr() for g in grads] if want_grad else [0] * k))
    Narr = (ctypes.c_int * k)(*Ns)
    c = _ctx(states[0])
    c.check(c.lib.hadamag_sre_batched(c.h, k, P, Narr, 1 if want_grad else 0, G,
                                      ctypes.c_void_p(out.data_ptr()), _stream(states[0])),
            "hadamag_sre_batched")
    if sync:
        c.check(c.lib.hadamag_batched_status(c.h, _stream(states[0])), "hadamag_batched_status")
    return out, (grads if want_grad else None)
