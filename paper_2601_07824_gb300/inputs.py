"""Seeded synthetic input states for the SRE and mana computations.

This module generates *inputs* only: state vectors of N qubits (d = 2) or N qutrits
(d = 3), built by plain NumPy linear algebra from a seed.  It holds none of the
magic-measure arithmetic (no Walsh-Hadamard / Z_3 transforms, no Pauli or
phase-space sums), so both the CUDA path and the FP64 CPU oracle may take their
inputs from here.

Index convention (used everywhere in this project): amplitude index
z = sum_j x_j d^j, i.e. site j is digit j of z, least significant first.

Workloads follow the paper's benchmark states (Sec. 4, Eq. randC: brick-wall
circuits of Haar-random two-site gates drawn as in Mezzadri's QR recipe) plus the
closed-form states the paper's properties fix (Sec. 2: stabilizer states give
M_q = 0 and mana 0; additivity gives product-state values).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_state", "zero_state", "t_state_product", "ghz_state", "graph_state",
    "haar_unitary", "brickwork_haar", "ry_rz_cz_ladder", "batched_ladder_states",
    "strange_product", "qutrit_ghz", "qutrit_graph_state", "apply_1site", "apply_2site",
    "random_clifford_circuit", "random_qutrit_clifford_circuit", "product_state",
    "to_interleaved", "X_STRING_MAX_QUBITS",
]

X_STRING_MAX_QUBITS = 30


def _dim(N: int, d: int) -> int:
    return d ** N


def gaussian_state(N: int, seed: int, d: int = 2, dtype=np.complex128) -> np.ndarray:
    """i.i.d. complex Gaussian amplitudes, normalised (Haar-random after normalisation).

    Draw order: all real parts, then all imaginary parts, from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    n = _dim(N, d)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    g = re + 1j * im
    g /= np.linalg.norm(g)
    return g.astype(dtype)


def _popcount(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.int64)
    c = np.zeros_like(z)
    while np.any(z):
        c += z & 1
        z >>= 1
    return c


def u1_state(N: int, k: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """U(1)-symmetric qubit state: i.i.d. complex Gaussian amplitudes on the basis states of
    Hamming weight k (fixed total magnetisation), zero elsewhere, normalised.

    Draw order: real parts, then imaginary parts of the supported amplitudes in index order."""
    z = np.arange(2 ** N)
    sup = np.nonzero(_popcount(z) == k)[0]
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(sup.size)
    im = rng.standard_normal(sup.size)
    v = np.zeros(2 ** N, dtype=np.complex128)
    v[sup] = re + 1j * im
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def parity_state(N: int, seed: int, parity: int = 0, dtype=np.complex128) -> np.ndarray:
    """Z_2-symmetric qubit state (eigenstate of prod_j Z_j): i.i.d. complex Gaussian amplitudes
    on the basis states of the given Hamming-weight parity, zero elsewhere, normalised."""
    z = np.arange(2 ** N)
    sup = np.nonzero((_popcount(z) & 1) == parity)[0]
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(sup.size)
    im = rng.standard_normal(sup.size)
    v = np.zeros(2 ** N, dtype=np.complex128)
    v[sup] = re + 1j * im
    v /= np.linalg.norm(v)
    return v.astype(dtype)


def zero_state(N: int, d: int = 2, dtype=np.complex128) -> np.ndarray:
    v = np.zeros(_dim(N, d), dtype=dtype)
    v[0] = 1.0
    return v


def product_state(local: np.ndarray, N: int, dtype=np.complex128) -> np.ndarray:
    """|phi>^{(x)N} for a single-site vector `local` (site j = digit j)."""
    out = np.array([1.0 + 0j])
    for _ in range(N):
        # new site becomes the most significant digit
        out = np.kron(np.asarray(local, dtype=np.complex128), out)
    return out.astype(dtype)


def t_state_product(N: int, dtype=np.complex128) -> np.ndarray:
    """|T>^{(x)N}, |T> = (|0> + e^{i pi/4}|1>)/sqrt(2)."""
    t = np.array([1.0, np.exp(1j * np.pi / 4)]) / np.sqrt(2.0)
    return product_state(t, N, dtype)


def ghz_state(N: int, dtype=np.complex128) -> np.ndarray:
    v = np.zeros(2 ** N, dtype=np.complex128)
    v[0] = v[-1] = 1.0 / np.sqrt(2.0)
    return v.astype(dtype)


def graph_state(N: int, edges, dtype=np.complex128) -> np.ndarray:
    """Qubit graph state prod_{(i,j)} CZ_ij |+>^N."""
    z = np.arange(2 ** N)
    phase = np.zeros(2 ** N, dtype=np.int64)
    for (i, j) in edges:
        phase += ((z >> i) & 1) * ((z >> j) & 1)
    v = ((-1.0) ** (phase & 1)) / np.sqrt(2.0 ** N)
    return v.astype(dtype)


def strange_product(N: int, dtype=np.complex128) -> np.ndarray:
    """Qutrit Strange state ((|1> - |2>)/sqrt 2)^{(x)N}."""
    s = np.array([0.0, 1.0, -1.0]) / np.sqrt(2.0)
    return product_state(s, N, dtype)


def qutrit_ghz(N: int, dtype=np.complex128) -> np.ndarray:
    """(|0..0> + |1..1> + |2..2>)/sqrt 3, a qutrit stabilizer state."""
    v = np.zeros(3 ** N, dtype=np.complex128)
    ones = sum(3 ** j for j in range(N))
    for k in range(3):
        v[k * ones] = 1.0 / np.sqrt(3.0)
    return v.astype(dtype)


def _digits(N: int, d: int) -> np.ndarray:
    z = np.arange(d ** N)
    return np.stack([(z // d ** j) % d for j in range(N)], axis=0)


def qutrit_graph_state(N: int, edges, dtype=np.complex128) -> np.ndarray:
    """Generalised qutrit graph state prod CZ_ij |+>^N with CZ|j,k> = w^{jk}, w = e^{2 pi i/3}."""
    x = _digits(N, 3)
    e = np.zeros(3 ** N, dtype=np.int64)
    for (i, j) in edges:
        e += x[i] * x[j]
    v = np.exp(2j * np.pi * (e % 3) / 3.0) / np.sqrt(3.0 ** N)
    return v.astype(dtype)


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(n) by QR of a complex Ginibre matrix with the R-diagonal phase fix
    (Mezzadri's recipe, cited by the paper for its random gates)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r) / np.abs(np.diagonal(r))
    return q * ph[None, :]


def apply_1site(psi: np.ndarray, U: np.ndarray, q: int, N: int, d: int = 2) -> np.ndarray:
    """Apply a d x d matrix to site q (digit q of the index)."""
    t = psi.reshape(d ** (N - q - 1), d, d ** q)
    return np.einsum("ij,ajb->aib", U, t).reshape(-1)


def apply_2site(psi: np.ndarray, U: np.ndarray, q: int, N: int, d: int = 2) -> np.ndarray:
    """Apply a d^2 x d^2 matrix to the adjacent sites (q, q+1).

    The gate's basis index is x_q + d * x_{q+1}."""
    t = psi.reshape(d ** (N - q - 2), d, d, d ** q)  # (high, x_{q+1}, x_q, low)
    U4 = U.reshape(d, d, d, d)  # [r_{q+1}, r_q, c_{q+1}, c_q]
    return np.einsum("ijkl,aklb->aijb", U4, t).reshape(-1)


def brickwork_haar(N: int, depth: int, seed: int, d: int = 2, dtype=np.complex64) -> np.ndarray:
    """Brick-wall circuit of Haar-random two-site gates on |0>^N, open chain (Eq. randC).

    Layers r = 1..depth; odd r acts on pairs (0,1),(2,3),...; even r on (1,2),(3,4),...
    (0-indexed sites).  Gates are drawn in order (layer, pair) from PCG64(seed).
    Simulated in complex128, returned as `dtype`."""
    rng = np.random.default_rng(seed)
    psi = zero_state(N, d, np.complex128)
    for r in range(1, depth + 1):
        start = 0 if (r % 2 == 1) else 1
        for q in range(start, N - 1, 2):
            U = haar_unitary(d * d, rng)
            psi = apply_2site(psi, U, q, N, d)
    return psi.astype(dtype)


def _ry(theta: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def _rz(phi: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)])


def ry_rz_cz_ladder(N: int, layers: int, rng: np.random.Generator, dtype=np.complex64) -> np.ndarray:
    """|0>^N followed by `layers` x [RY(theta) on every qubit; RZ(phi) on every qubit;
    CZ(j, j+1) for j = 0..N-2]; angles U[0, 2 pi) drawn per layer as all RY angles then
    all RZ angles (qubit order)."""
    psi = zero_state(N, 2, np.complex128)
    z = np.arange(2 ** N)
    czphase = np.zeros(2 ** N, dtype=np.int64)
    for j in range(N - 1):
        czphase += ((z >> j) & 1) * ((z >> (j + 1)) & 1)
    cz = (-1.0) ** (czphase & 1)
    for _ in range(layers):
        th = rng.uniform(0.0, 2 * np.pi, N)
        ph = rng.uniform(0.0, 2 * np.pi, N)
        for q in range(N):
            psi = apply_1site(psi, _ry(th[q]), q, N)
        for q in range(N):
            psi = apply_1site(psi, _rz(ph[q]), q, N)
        psi = psi * cz
    return psi.astype(dtype)


def batched_ladder_states(count: int, n_lo: int, n_hi: int, layers: int, seed: int,
                          dtype=np.complex64):
    """`count` states with N_i ~ U{n_lo..n_hi}, each an RY/RZ + CZ-ladder circuit state.

    Draw order from PCG64(seed): the N_i first, then per state, per layer, the angles."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [int(n) for n in Ns], [ry_rz_cz_ladder(int(n), layers, rng, dtype) for n in Ns]


# ---- Clifford circuits (used by invariance tests) ---------------------------------

_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
_S = np.diag([1.0, 1j])


def _cnot(psi: np.ndarray, c: int, t: int, N: int) -> np.ndarray:
    z = np.arange(2 ** N)
    src = np.where(((z >> c) & 1) == 1, z ^ (1 << t), z)
    return psi[src]


def random_clifford_circuit(psi: np.ndarray, N: int, n_gates: int, seed: int) -> np.ndarray:
    """Apply `n_gates` random gates from {H, S, CNOT} (all Clifford) to a qubit state."""
    rng = np.random.default_rng(seed)
    out = psi.astype(np.complex128)
    for _ in range(n_gates):
        g = rng.integers(0, 3)
        if g == 0:
            out = apply_1site(out, _H, int(rng.integers(0, N)), N)
        elif g == 1:
            out = apply_1site(out, _S, int(rng.integers(0, N)), N)
        elif N > 1:
            c, t = rng.choice(N, size=2, replace=False)
            out = _cnot(out, int(c), int(t), N)
    return out


_W3 = np.exp(2j * np.pi / 3)
_F3 = np.array([[_W3 ** (j * k) for k in range(3)] for j in range(3)]) / np.sqrt(3.0)
_P3 = np.diag([1.0, 1.0, _W3])  # qutrit phase gate diag(w^{k(k-1)/2})


def _sum_gate(psi: np.ndarray, c: int, t: int, N: int) -> np.ndarray:
    """Qutrit SUM: |x_c, x_t> -> |x_c, x_t + x_c mod 3>."""
    x = _digits(N, 3)
    z = np.arange(3 ** N)
    xt_new = (x[t] + x[c]) % 3
    dst = z + (xt_new - x[t]) * 3 ** t
    out = np.empty_like(psi)
    out[dst] = psi
    return out


def random_qutrit_clifford_circuit(psi: np.ndarray, N: int, n_gates: int, seed: int) -> np.ndarray:
    """Apply `n_gates` random qutrit Clifford gates from {F, P, SUM}."""
    rng = np.random.default_rng(seed)
    out = psi.astype(np.complex128)
    for _ in range(n_gates):
        g = rng.integers(0, 3)
        if g == 0:
            out = apply_1site(out, _F3, int(rng.integers(0, N)), N, 3)
        elif g == 1:
            out = apply_1site(out, _P3, int(rng.integers(0, N)), N, 3)
        elif N > 1:
            c, t = rng.choice(N, size=2, replace=False)
            out = _sum_gate(out, int(c), int(t), N)
    return out


def to_interleaved(psi: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Complex vector -> interleaved (re, im) real array of the given precision."""
    a = np.empty(2 * psi.size, dtype=dtype)
    a[0::2] = psi.real
    a[1::2] = psi.imag
    return a
