"""FP64 CPU oracle for the SRE and mana computations.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
/ reference leg of `bench.py` may import this package.  It shares no code with the CUDA
library and never calls it.

Two independent halves:
  * `hadamag_oracle.c` (built here with gcc, loaded with ctypes): the paper's Algorithm 2
    (SRE via one Walsh-Hadamard transform per X-string) and Algorithm 5 (mana via one
    Z_3^N Fourier transform per X-string) written plainly in FP64, plus the M_2 gradient
    and the uniform-X Monte-Carlo estimator.
  * `oracle.brute` (NumPy): the definitions themselves -- every Pauli string or
    phase-space point operator built as a dense matrix -- for tiny N.  Tests pin the C
    half to the brute force, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hadamag_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/liboracle.so."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        U64 = ctypes.c_uint64
        lib.orc_num_threads.argtypes = [I]
        lib.orc_num_threads.restype = I
        lib.orc_sre_terms.argtypes = [P, I, D, L, L, I, P, P, P]
        lib.orc_sre.argtypes = [P, I, D, I, P, P]
        lib.orc_sre_grad.argtypes = [P, I, I, P, P]
        lib.orc_splitmix64.argtypes = [U64, L, P]
        lib.orc_splitmix64.restype = None
        lib.orc_mc_xstrings.argtypes = [U64, L, I, P]
        lib.orc_mc_xstrings.restype = None
        lib.orc_sre_terms_list.argtypes = [P, I, P, L, I, P]
        lib.orc_sre_mc.argtypes = [P, I, L, U64, I, P, P, P]
        lib.orc_mana_terms.argtypes = [P, I, L, L, I, P, P, P, P]
        lib.orc_mana.argtypes = [P, I, I, P, P]
        for f in ("orc_sre_terms", "orc_sre", "orc_sre_grad", "orc_sre_terms_list",
                  "orc_sre_mc", "orc_mana_terms", "orc_mana"):
            getattr(lib, f).restype = I
        _lib = lib
        return lib


def _c128(psi) -> np.ndarray:
    """Upcast to contiguous complex128 (the oracle reads the same amplitudes the GPU reads)."""
    return np.ascontiguousarray(np.asarray(psi).astype(np.complex128))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads(n: int = 0) -> int:
    return _load().orc_num_threads(int(n))


def n_qubits(psi) -> int:
    n = int(np.asarray(psi).size).bit_length() - 1
    if 1 << n != np.asarray(psi).size:
        raise ValueError("qubit state length must be a power of two")
    return n


def n_qutrits(psi) -> int:
    size, n = int(np.asarray(psi).size), 0
    while 3 ** n < size:
        n += 1
    if 3 ** n != size:
        raise ValueError("qutrit state length must be a power of three")
    return n


def sre(psi, q: float, nthreads: int = 0):
    """(M_q, lost_norm) by the paper's Eq. (sre) evaluated with Algorithm 2 in FP64."""
    lib, p = _load(), _c128(psi)
    M, ln = ctypes.c_double(), ctypes.c_double()
    _check(lib.orc_sre(_ptr(p), n_qubits(p), float(q), int(nthreads), ctypes.byref(M),
                       ctypes.byref(ln)), "sre")
    return M.value, ln.value


def sre_terms(psi, q: float, a0: int = 0, a1: int | None = None, nthreads: int = 0):
    """Per-X-string sums for a in [a0, a1): (S_q(a), S_1(a), T_1(a)) with
    S_q(a) = sum_b |chi_b(a)|^{2q}, S_1(a) = sum_b |chi_b(a)|^2,
    T_1(a) = sum_b |chi_b|^2 log2 |chi_b|^2."""
    lib, p = _load(), _c128(psi)
    N = n_qubits(p)
    a1 = (1 << N) if a1 is None else a1
    n = a1 - a0
    Sq, S1, T1 = np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib.orc_sre_terms(_ptr(p), N, float(q), a0, a1, int(nthreads), _ptr(Sq), _ptr(S1),
                             _ptr(T1)), "sre_terms")
    return Sq, S1, T1


def sre_even_sector(psi, q: float, nthreads: int = 0):
    """(M_q, lost_norm) from the even-weight X-strings only (Sec. 3.2): for states with U(1)
    symmetry or the Z_2 symmetry prod_j Z_j, <psi|X_a Z_b|psi> = 0 whenever |a| is odd, so the
    2^(N-1) even-weight X-strings carry the whole sum of Eq. (sre).  Same formulas as `sre`
    (the n -> 1 Shannon limit included) over the restricted sums."""
    p = _c128(psi)
    N = n_qubits(p)
    Sq, S1, T1 = sre_terms(p, q, nthreads=nthreads)
    a = np.arange(1 << N)
    w = np.zeros_like(a)
    for j in range(N):
        w += (a >> j) & 1
    even = (w & 1) == 0
    sq, s1, t1 = float(Sq[even].sum()), float(S1[even].sum()), float(T1[even].sum())
    if q == 1.0:
        M = -t1 / s1 + np.log2(s1) - N
    else:
        M = np.log2(sq / 2.0 ** N) / (1.0 - q)
    return float(M), 1.0 - s1 / 2.0 ** N


def sre_terms_list(psi, a_list, nthreads: int = 0) -> np.ndarray:
    """S(a) = sum_b |chi_b(a)|^4 for an explicit list of X-strings."""
    lib, p = _load(), _c128(psi)
    a = np.ascontiguousarray(np.asarray(a_list, dtype=np.int64))
    out = np.zeros(a.size)
    _check(lib.orc_sre_terms_list(_ptr(p), n_qubits(p), _ptr(a), a.size, int(nthreads),
                                  _ptr(out)), "sre_terms_list")
    return out


def sre_grad(psi, nthreads: int = 0):
    """(M_2, dM_2/dpsi*) -- Wirtinger gradient on the unnormalised psi."""
    lib, p = _load(), _c128(psi)
    M2 = ctypes.c_double()
    g = np.zeros(p.size, dtype=np.complex128)
    _check(lib.orc_sre_grad(_ptr(p), n_qubits(p), int(nthreads), ctypes.byref(M2), _ptr(g)),
           "sre_grad")
    return M2.value, g


def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    _load().orc_splitmix64(ctypes.c_uint64(seed & (2 ** 64 - 1)), count, _ptr(out))
    return out


def mc_xstrings(seed: int, count: int, N: int) -> np.ndarray:
    """Sampled X-strings a_i = top N bits of SplitMix64 output i (i = 0..count-1)."""
    out = np.zeros(count, dtype=np.int64)
    _load().orc_mc_xstrings(ctypes.c_uint64(seed & (2 ** 64 - 1)), count, int(N), _ptr(out))
    return out


def sre_mc(psi, samples: int, seed: int, nthreads: int = 0):
    """(M2_hat, stderr, S per sample) of the uniform-X Monte-Carlo estimator."""
    lib, p = _load(), _c128(psi)
    M, se = ctypes.c_double(), ctypes.c_double()
    S = np.zeros(samples)
    _check(lib.orc_sre_mc(_ptr(p), n_qubits(p), int(samples), ctypes.c_uint64(seed),
                          int(nthreads), ctypes.byref(M), ctypes.byref(se), _ptr(S)), "sre_mc")
    return M.value, se.value, S


def mana(psi, nthreads: int = 0):
    """(mana in bits = log2 sum|W|, sum|W|) by Algorithm 5 with Eq. (mana2)'s 1/3^N."""
    lib, p = _load(), _c128(psi)
    m, sw = ctypes.c_double(), ctypes.c_double()
    _check(lib.orc_mana(_ptr(p), n_qutrits(p), int(nthreads), ctypes.byref(m), ctypes.byref(sw)),
           "mana")
    return m.value, sw.value


def mana_terms(psi, a0: int = 0, a1: int | None = None, nthreads: int = 0):
    """Per-a sums over b of |chi|, Re chi, |chi|^2 and max |Im chi| (a as base-3 index)."""
    lib, p = _load(), _c128(psi)
    N = n_qutrits(p)
    a1 = 3 ** N if a1 is None else a1
    n = a1 - a0
    m, s, q2, mi = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib.orc_mana_terms(_ptr(p), N, a0, a1, int(nthreads), _ptr(m), _ptr(s), _ptr(q2),
                              _ptr(mi)), "mana_terms")
    return m, s, q2, mi
