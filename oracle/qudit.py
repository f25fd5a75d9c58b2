"""Mana of qudits of odd prime dimension d, FP64 NumPy.  TEST INFRASTRUCTURE ONLY: only
`tests/` may import this module.

Sec. 2 defines the Heisenberg-Weyl operators, phase-space point operators and mana for
qutrits and notes that the construction applies to any odd prime d:
    X|k> = |k+1>,  Z|k> = w^k |k>  (w = e^{2 pi i / d}),  T_ab = w^{-2^{-1} ab} Z^a X^b,
    A_0 = d^-N sum_u T_u,  A_u = T_u A_0 T_u^dag,  W(u) = tr(A_u rho) / d^N,
    mana = log2 sum_u |W(u)|.
Two independent evaluations:
  * `wigner_brute`: the definition with every T_u and A_u built as a dense matrix (tiny N);
  * `mana_fast`: Algorithm 5's per-shift transform for general d.  With
    A_{ab}|x> = w^{2a(b-x)} |2b - x> (from the definitions above), <psi|A_ab|psi> =
    sum_y w^{-2ay} psi_{b+y} conj(psi_{b-y}); for every shift a (digit-wise mod d)
        v_x = conj(psi_{x-a}) psi_{-x-a},   chi = F_d^{(x)N} v,  (F_d)_{jk} = w^{2jk},
    and the values chi / d^N are the W(u) (a relabelling of u); chi is real for pure states.
Sites: site j = base-d digit j of the index (least significant first).
"""
from __future__ import annotations

import itertools

import numpy as np

PRIMES = (3, 5, 7, 11, 13)


def _check_d(d: int):
    if d not in PRIMES:
        raise ValueError(f"d must be an odd prime in {PRIMES}")


def n_sites(dim: int, d: int) -> int:
    N = 0
    while d ** N < dim:
        N += 1
    if d ** N != dim:
        raise ValueError(f"dimension must be {d}^N")
    return N


def hw_operator(a: int, b: int, d: int) -> np.ndarray:
    """T_ab = w^{-2^{-1} ab} Z^a X^b for one qudit."""
    _check_d(d)
    w = np.exp(2j * np.pi / d)
    X = np.roll(np.eye(d, dtype=np.complex128), 1, axis=0)
    Z = np.diag([w ** k for k in range(d)])
    two_inv = (d + 1) // 2
    return (w ** (-(two_inv * a * b) % d)) * (np.linalg.matrix_power(Z, a) @ np.linalg.matrix_power(X, b))


def _kron_sites(mats):
    out = np.array([[1.0 + 0j]])
    for m in mats:
        out = np.kron(m, out)  # later sites are more significant
    return out


def phase_point_operators(N: int, d: int):
    """All d^(2N) phase-space point operators A_u (list, u = per-site (a, b) in row-major order)."""
    singles = {(a, b): hw_operator(a, b, d) for a in range(d) for b in range(d)}
    us = list(itertools.product(range(d * d), repeat=N))
    Ts = [_kron_sites([singles[divmod(k, d)] for k in u]) for u in us]
    A0 = sum(Ts) / d ** N
    return [T @ A0 @ T.conj().T for T in Ts], A0


def wigner_brute(psi, d: int) -> np.ndarray:
    """W(u) = <psi|A_u|psi> / d^N from dense operators (N small)."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = n_sites(psi.size, d)
    As, _ = phase_point_operators(N, d)
    return np.array([np.vdot(psi, A @ psi) for A in As]) / d ** N


def wigner_mixed_brute(rho, d: int) -> np.ndarray:
    """W(u) = tr(A_u rho) / d^N for a density matrix (dense operators, N small)."""
    rho = np.asarray(rho, dtype=np.complex128)
    N = n_sites(rho.shape[0], d)
    As, _ = phase_point_operators(N, d)
    return np.array([np.trace(A @ rho) for A in As]) / d ** N


def mana_mixed_fast(rho, d: int, chunk: int = 256):
    """(mana, sum |W|, sum W, sum W^2) of a density matrix by the per-shift transform with the
    gather v_x = rho[-x - a, x - a] (digit-wise mod d; for rho = |psi><psi| this is
    conj(psi_{x-a}) psi_{-x-a}), F_d^{(x)N} and W = chi / d^N (a relabelling of u)."""
    _check_d(d)
    rho = np.asarray(rho, dtype=np.complex128)
    D = rho.shape[0]
    N = n_sites(D, d)
    dig, pw = _digits(D, N, d), d ** np.arange(N)
    s_abs = s1 = s2 = 0.0
    for a0 in range(0, D, chunk):
        i1, i2 = _shift_indices(dig, dig[a0:a0 + chunk], d, pw)
        chi = _transform_rows(rho[i2, i1], d, N).real / d ** N
        s_abs += float(np.abs(chi).sum())
        s1 += float(chi.sum())
        s2 += float((chi ** 2).sum())
    return float(np.log2(s_abs)), s_abs, s1, s2


def mana_brute(psi, d: int):
    W = wigner_brute(psi, d)
    s = float(np.abs(W.real).sum())
    return float(np.log2(s)), s


def _digits(D: int, N: int, d: int) -> np.ndarray:
    return np.stack([(np.arange(D) // d ** k) % d for k in range(N)], axis=1)  # [index, site]


def _transform_rows(V: np.ndarray, d: int, N: int) -> np.ndarray:
    """F_d^{(x)N} applied to every row of V, (F_d)_{jk} = w^{2jk}."""
    w = np.exp(2j * np.pi / d)
    F = np.array([[w ** ((2 * j * k) % d) for k in range(d)] for j in range(d)])
    t = V.reshape((V.shape[0],) + (d,) * N)  # axis 1 + k holds site N-1-k
    for ax in range(1, N + 1):
        t = np.moveaxis(np.tensordot(F, t, axes=([1], [ax])), 0, ax)
    return t.reshape(V.shape[0], -1)


def _shift_indices(dig: np.ndarray, da: np.ndarray, d: int, pw: np.ndarray):
    """idx(x - a) and idx(-x - a) (digit-wise mod d) for the shifts in da and every x, summed
    site by site from (d x d) tables of ((x_k -+ a_k) mod d) d^k."""
    r = np.arange(d)
    sub = (r[None, :] - r[:, None]) % d   # [a_k, x_k] -> (x_k - a_k) mod d
    neg = (-r[None, :] - r[:, None]) % d  # [a_k, x_k] -> (-x_k - a_k) mod d
    i1 = np.zeros((da.shape[0], dig.shape[0]), dtype=np.int64)
    i2 = np.zeros_like(i1)
    for k in range(dig.shape[1]):
        ia, ix = da[:, k][:, None], dig[None, :, k]
        i1 += (sub * pw[k])[ia, ix]
        i2 += (neg * pw[k])[ia, ix]
    return i1, i2


def chi_fast(psi, d: int, chunk: int = 256) -> np.ndarray:
    """chi[a, b] for every shift a and frequency b (both base-d indices)."""
    _check_d(d)
    psi = np.asarray(psi, dtype=np.complex128)
    N = n_sites(psi.size, d)
    D = psi.size
    dig, pw = _digits(D, N, d), d ** np.arange(N)
    out = np.empty((D, D), dtype=np.complex128)
    for a0 in range(0, D, chunk):
        i1, i2 = _shift_indices(dig, dig[a0:a0 + chunk], d, pw)
        out[a0:a0 + chunk] = _transform_rows(np.conj(psi[i1]) * psi[i2], d, N)
    return out


def mana_grad(psi, d: int, chunk: int = 256, small: float | None = None):
    """(mana, d mana / d psi*) on the unnormalised psi (Wirtinger gradient; mana =
    log2(sum_{a,b} |chi_b(a)| / d^N)).  From v_x = conj(psi_{x-a}) psi_{-x-a}:
        d chi_b(a) / d psi*_w = d conj(chi_b(a)) / d psi*_w = F_{b, w+a} psi_{-w-2a},
    so with y = w + a and G_a = F_d^{(x)N} (Re chi_a / |chi_a|) (F_d symmetric)
        d m / d psi*_{y-a} += psi_{-y-a} G_a(y),   d mana / d psi* = (d m / d psi*) / (m ln 2).
    Defined where no chi_b(a) vanishes (not on stabilizer states).  With `small` given, also
    returns how many |chi_b(a)| are below it (entries whose sign a perturbation of that size
    can flip, each moving d m / d psi* by at most 2 |psi|)."""
    _check_d(d)
    psi = np.asarray(psi, dtype=np.complex128)
    N = n_sites(psi.size, d)
    D = psi.size
    dig, pw = _digits(D, N, d), d ** np.arange(N)
    g = np.zeros(D, dtype=np.complex128)
    m = 0.0
    below = 0
    for a0 in range(0, D, chunk):
        i1, i2 = _shift_indices(dig, dig[a0:a0 + chunk], d, pw)  # i1 = idx(y - a), i2 = idx(-y - a)
        chi = _transform_rows(np.conj(psi[i1]) * psi[i2], d, N)
        m += float(np.abs(chi).sum())
        if small is not None:
            below += int((np.abs(chi) < small).sum())
        G = _transform_rows(chi.real / np.abs(chi), d, N)
        np.add.at(g, i1.ravel(), (psi[i2] * G).ravel())
    out = (float(np.log2(m / d ** N)), g / (m * np.log(2.0)))
    return out + (below,) if small is not None else out


def mana_fast(psi, d: int):
    """(mana in bits, sum |W|, sum W, sum W^2) by the per-shift transform."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = n_sites(psi.size, d)
    chi = chi_fast(psi, d).real / d ** N
    s = float(np.abs(chi).sum())
    return float(np.log2(s)), s, float(chi.sum()), float((chi ** 2).sum())


# ---- qudit states used by the pins ------------------------------------------------------

def zero_state(N: int, d: int) -> np.ndarray:
    v = np.zeros(d ** N, dtype=np.complex128)
    v[0] = 1.0
    return v


def ghz(N: int, d: int) -> np.ndarray:
    """sum_k |k...k> / sqrt d, a stabilizer state."""
    v = np.zeros(d ** N, dtype=np.complex128)
    ones = sum(d ** j for j in range(N))
    for k in range(d):
        v[k * ones] = 1.0 / np.sqrt(d)
    return v


def graph_state(N: int, d: int, edges) -> np.ndarray:
    """prod CZ_ij |+>^N with CZ|x, y> = w^{xy}|x, y>, a stabilizer state."""
    D = d ** N
    dig = np.stack([(np.arange(D) // d ** k) % d for k in range(N)], axis=1)
    ph = np.zeros(D, dtype=np.int64)
    for i, j in edges:
        ph += dig[:, i] * dig[:, j]
    return np.exp(2j * np.pi * (ph % d) / d) / np.sqrt(D)


def apply_1site(psi, U, q: int, N: int, d: int) -> np.ndarray:
    t = np.asarray(psi, dtype=np.complex128).reshape((d,) * N)
    ax = N - 1 - q
    return np.moveaxis(np.tensordot(U, t, axes=([1], [ax])), 0, ax).reshape(-1)


def sum_gate(psi, c: int, t: int, N: int, d: int) -> np.ndarray:
    """|x_c, x_t> -> |x_c, x_t + x_c>."""
    D = d ** N
    idx = np.arange(D)
    xc, xt = (idx // d ** c) % d, (idx // d ** t) % d
    dst = idx + (((xt + xc) % d) - xt) * d ** t
    out = np.zeros(D, dtype=np.complex128)
    out[dst] = np.asarray(psi, dtype=np.complex128)
    return out


def random_clifford_circuit(psi, N: int, d: int, n_gates: int, seed: int) -> np.ndarray:
    """Random gates from {Fourier F_{xy} = w^{xy}/sqrt d, phase w^{x^2}, X, SUM} (all Clifford
    for odd prime d)."""
    rng = np.random.default_rng(seed)
    w = np.exp(2j * np.pi / d)
    F = np.array([[w ** ((x * y) % d) for y in range(d)] for x in range(d)]) / np.sqrt(d)
    P = np.diag([w ** ((x * x) % d) for x in range(d)])
    X = np.roll(np.eye(d), 1, axis=0)
    out = np.asarray(psi, dtype=np.complex128)
    for _ in range(n_gates):
        g = int(rng.integers(4))
        if g < 3 or N == 1:
            out = apply_1site(out, (F, P, X)[g % 3], int(rng.integers(N)), N, d)
        else:
            c, t = rng.choice(N, 2, replace=False)
            out = sum_gate(out, int(c), int(t), N, d)
    return out
