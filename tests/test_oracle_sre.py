"""Pins for the FP64 SRE oracle (Algorithm 2 written plainly) against things other than
itself: the brute-force definition (Eq. sre over dense Pauli matrices), closed forms,
the normalisation sum rule, per-X-string Parseval, Clifford and permutation invariance,
additivity and the Haar band.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2601_07824_gb300 import inputs as I

QS = (0.5, 1.0, 2.0, 3.0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_fwht_oracle_matches_brute_force(N):
    # Eq. (sre) by enumerating all 4^N Hermitian Pauli matrices (Sec. 3.1.1) vs Algorithm 2.
    for seed in (11, 12):
        psi = I.gaussian_state(N, seed + 31 * N)
        for q in QS:
            Mo, lo = oracle.sre(psi, q)
            Mb, lb = brute.sre_brute(psi, q)
            assert abs(Mo - Mb) < 1e-12, (N, q, Mo, Mb)
            assert abs(lo - lb) < 1e-12


def test_unnormalised_state_matches_brute_force():
    # The formula is evaluated as given (no renormalisation); lost_norm = 1 - |psi|^4.
    psi = 1.3 * I.gaussian_state(4, 5)
    for q in QS:
        Mo, lo = oracle.sre(psi, q)
        Mb, lb = brute.sre_brute(psi, q)
        assert abs(Mo - Mb) < 1e-12
        assert abs(lo - lb) < 1e-12
    assert abs(oracle.sre(psi, 2.0)[1] - (1 - 1.3 ** 4)) < 1e-12


def test_t_state_closed_form(golden):
    g = golden["closed_forms"]["sre_t_state_per_qubit"]
    psi = I.t_state_product(g["N"])
    for q, key in ((1.0, "M1"), (2.0, "M2"), (3.0, "M3")):
        M, ln = oracle.sre(psi, q)
        assert abs(M - g[key]) < 1e-12, (q, M)
        assert abs(ln) < 1e-12
    # general q (additivity + single-qubit value)
    for N in (1, 3, 7):
        for q in (0.5, 1.5, 2.5):
            M, _ = oracle.sre(I.t_state_product(N), q)
            assert abs(M - N / (1 - q) * np.log2((1 + 2 ** (1 - q)) / 2)) < 1e-12


@pytest.mark.parametrize("N", [1, 4, 9, 12])
def test_stabilizer_states_zero(N, golden):
    g = golden["closed_forms"]["sre_stabilizer_zero"]
    states = [I.zero_state(N), I.ghz_state(N),
              I.graph_state(N, [(j, (j + 1) % N) for j in range(N)] if N > 2 else [(0, N - 1)]),
              I.random_clifford_circuit(I.zero_state(N), N, 40, seed=N)]
    rng = np.random.default_rng(N)
    if N > 2:
        edges = [(i, j) for i in range(N) for j in range(i + 1, N) if rng.random() < 0.4]
        states.append(I.graph_state(N, edges))
    for psi in states:
        for q in QS:
            M, ln = oracle.sre(psi, q)
            assert abs(M - g["M"]) < 1e-10, (q, M)
            assert abs(ln - g["lost_norm"]) < 1e-12


def test_nonstabilizer_is_positive():
    # faithfulness: M_q > 0 for a non-stabilizer state
    psi = I.gaussian_state(6, 3)
    for q in QS:
        assert oracle.sre(psi, q)[0] > 0.5


def test_lost_norm_and_parseval_per_x():
    # Eq. distNAT: sum_P <P>^2 / 2^N = |psi|^4.  Per X-string, Eq. Z_FT_qubits with Parseval
    # for the unnormalised H: sum_b |chi_b(a)|^2 = 2^N sum_z |psi_z|^2 |psi_{z^a}|^2.
    N = 7
    psi = 0.9 * I.gaussian_state(N, 21)
    _, S1, _ = oracle.sre_terms(psi, 2.0)
    z = np.arange(2 ** N)
    p = np.abs(psi) ** 2
    direct = np.array([2 ** N * np.sum(p * p[z ^ a]) for a in range(2 ** N)])
    assert np.allclose(S1, direct, rtol=1e-12, atol=0)
    assert abs(S1.sum() / 2 ** N - 0.9 ** 4) < 1e-12


def test_per_x_terms_brute_force():
    # chi_b(a) = <psi| X_a Z_b |psi>: build X_a, Z_b as dense matrices (Sec. 3.1.2).
    N = 4
    psi = I.gaussian_state(N, 8)
    Sq, S1, _ = oracle.sre_terms(psi, 2.0)
    X, Z = brute.PAULIS[1], brute.PAULIS[3]
    for a in range(2 ** N):
        s4 = s2 = 0.0
        for b in range(2 ** N):
            P = brute.kron_sites([np.linalg.matrix_power(X, (a >> j) & 1)
                                  @ np.linalg.matrix_power(Z, (b >> j) & 1) for j in range(N)])
            c = np.vdot(psi, P @ psi)
            s2 += abs(c) ** 2
            s4 += abs(c) ** 4
        assert abs(Sq[a] - s4) < 1e-13 and abs(S1[a] - s2) < 1e-13


def test_clifford_and_permutation_invariance():
    N = 6
    psi = I.gaussian_state(N, 77)
    ref = [oracle.sre(psi, q)[0] for q in QS]
    for seed in (1, 2, 3):
        phi = I.random_clifford_circuit(psi, N, 60, seed)
        for q, r in zip(QS, ref):
            assert abs(oracle.sre(phi, q)[0] - r) < 1e-10
    perm = [3, 0, 5, 1, 4, 2]
    t = psi.reshape([2] * N)  # axis k <-> qubit N-1-k
    axes = [N - 1 - perm[N - 1 - k] for k in range(N)]
    phi = np.transpose(t, axes).reshape(-1)
    for q, r in zip(QS, ref):
        assert abs(oracle.sre(phi, q)[0] - r) < 1e-10


def test_additivity():
    a, b = I.gaussian_state(3, 1), I.gaussian_state(4, 2)
    ab = np.kron(b, a)  # a on qubits 0..2, b on 3..6
    for q in QS:
        assert abs(oracle.sre(ab, q)[0] - oracle.sre(a, q)[0] - oracle.sre(b, q)[0]) < 1e-10


def test_haar_band(golden):
    # Sec. 4.1: M_2^Haar = log2(2^N + 3) - 2; a Gaussian draw sits close at N = 12.
    N = 12
    psi = I.gaussian_state(N, 1201)
    M2, ln = oracle.sre(psi, 2.0)
    assert abs(M2 - (np.log2(2 ** N + 3) - 2)) < 0.02
    assert abs(ln) < 1e-12


def test_plausible_mistakes_are_caught():
    """A planted mistake in a copy of the per-X chain (dropped conj, wrong partner index,
    chi^{2q} without the modulus) must disagree with the brute force."""
    N = 3
    psi = I.gaussian_state(N, 4)
    Mb, _ = brute.sre_brute(psi, 3.0)

    def fwht(v):
        v = v.copy()
        h = 1
        while h < v.size:
            for i in range(0, v.size, 2 * h):
                x, y = v[i:i + h].copy(), v[i + h:i + 2 * h].copy()
                v[i:i + h], v[i + h:i + 2 * h] = x + y, x - y
            h *= 2
        return v

    z = np.arange(2 ** N)

    def M3(form):
        s = 0.0
        for a in range(2 ** N):
            if form == "noconj":
                v = psi[z ^ a] * psi
            elif form == "badidx":
                v = np.conj(psi[(z + a) % 2 ** N]) * psi
            else:
                v = np.conj(psi[z ^ a]) * psi
            c = fwht(v)
            s += np.sum(c ** 6).real if form == "nomod" else np.sum(np.abs(c) ** 6)
        return np.log2(s / 2 ** N) / (1 - 3.0)

    assert abs(M3("ok") - Mb) < 1e-12
    for bad in ("noconj", "badidx", "nomod"):
        assert abs(M3(bad) - Mb) > 1e-6, bad
