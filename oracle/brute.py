"""Brute-force definitions for tiny N (NumPy, FP64).  TEST INFRASTRUCTURE ONLY.

These follow the paper's definitions directly, with every operator built as a dense
matrix, and serve to pin the fast FP64 oracle (`hadamag_oracle.c`):

  * SRE, Eq. (sre) of Sec. 2: M_q = 1/(1-q) log2[ sum_P <psi|P|psi>^{2q} / 2^N ] over all
    4^N Hermitian Pauli strings P = (x)_j {I, X, Y, Z}  (q -> 1: Shannon limit).
  * Qutrit Heisenberg-Weyl operators, Eqs. clock_and_shift / pauli_qudit:
    T_ab = w^{-2^{-1} ab} Z^a X^b with 2^{-1} = 2 in Z_3; T_u = (x)_j T_{u_j u'_j}.
  * Phase-space point operators, Eq. phase-space: A_0 = 3^-N sum_u T_u, A_u = T_u A_0 T_u^dag;
    Wigner function W(u) = tr(A_u rho) / 3^N; mana, Eq. (mana): log2 sum_u |W(u)|.
"""
from __future__ import annotations

import itertools

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_X2 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z2 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULIS = (_I2, _X2, _Y2, _Z2)


def kron_sites(mats):
    """Operator acting with mats[j] on site j (site j = digit j, least significant)."""
    out = np.array([[1.0 + 0j]])
    for m in mats:
        out = np.kron(m, out)  # later sites are more significant
    return out


def pauli_expectations(psi: np.ndarray) -> np.ndarray:
    """<psi|P|psi> (real) for all 4^N Hermitian Pauli strings."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = int(psi.size).bit_length() - 1
    vals = []
    for labels in itertools.product(range(4), repeat=N):
        P = kron_sites([PAULIS[k] for k in labels])
        vals.append(np.vdot(psi, P @ psi).real)
    return np.array(vals)


def sre_brute(psi: np.ndarray, q: float):
    """(M_q, lost_norm) straight from Eq. (sre)."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = int(psi.size).bit_length() - 1
    e = pauli_expectations(psi)
    x = e ** 2
    s1 = x.sum()
    if q == 1.0:
        nz = x[x > 0]
        p = nz / s1
        M = -(p * np.log2(p)).sum() - N
    else:
        M = np.log2((x ** q).sum() / 2 ** N) / (1.0 - q)
    return float(M), float(1.0 - s1 / 2 ** N)


# ---- qutrits -------------------------------------------------------------------------

W3 = np.exp(2j * np.pi / 3)
X3 = np.roll(np.eye(3, dtype=np.complex128), 1, axis=0)  # X|k> = |k+1>
Z3 = np.diag([W3 ** k for k in range(3)])                 # Z|k> = w^k |k>
TWO_INV = 2  # inverse of 2 in Z_3


def hw_operator(a: int, b: int) -> np.ndarray:
    """T_ab = w^{-2^{-1} a b} Z^a X^b."""
    return (W3 ** (-(TWO_INV * a * b) % 3)) * (np.linalg.matrix_power(Z3, a)
                                               @ np.linalg.matrix_power(X3, b))


def phase_point_operators(N: int):
    """All 9^N phase-space point operators A_u (list) and A_0."""
    singles = {(a, b): hw_operator(a, b) for a in range(3) for b in range(3)}
    us = list(itertools.product(range(9), repeat=N))
    Ts = [kron_sites([singles[divmod(k, 3)] for k in u]) for u in us]
    A0 = sum(Ts) / 3 ** N
    As = [T @ A0 @ T.conj().T for T in Ts]
    return As, A0


def wigner_brute(psi: np.ndarray) -> np.ndarray:
    """W(u) = tr(A_u rho)/3^N for rho = |psi><psi| (real up to rounding)."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = 0
    while 3 ** N < psi.size:
        N += 1
    As, _ = phase_point_operators(N)
    return np.array([np.vdot(psi, A @ psi) for A in As]) / 3 ** N


def mana_brute(psi: np.ndarray):
    """(mana in bits, sum |W|) from Eq. (mana)."""
    W = wigner_brute(psi)
    s = float(np.abs(W.real).sum())
    return float(np.log2(s)), s


def wigner_mixed_brute(rho: np.ndarray) -> np.ndarray:
    """W(u) = tr(A_u rho)/3^N for a qutrit density matrix (site j = digit j), in the order of
    `phase_point_operators`."""
    rho = np.asarray(rho, dtype=np.complex128)
    N = 0
    while 3 ** N < rho.shape[0]:
        N += 1
    As, _ = phase_point_operators(N)
    return np.array([np.trace(A @ rho) for A in As]) / 3 ** N


def mana_mixed_brute(rho: np.ndarray):
    """(mana in bits, sum |W|) of a qutrit density matrix from Eq. (mana)."""
    W = wigner_mixed_brute(rho)
    s = float(np.abs(W).sum())
    return float(np.log2(s)), s
