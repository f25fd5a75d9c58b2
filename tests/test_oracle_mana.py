"""Pins for the FP64 mana oracle (Algorithm 5 written plainly) against the brute-force
Wigner function (Eqs. clock_and_shift, pauli_qudit, phase-space, mana), the reflection
property of A_0, the Wigner sum rules, stabilizer zeros, the Strange-state closed form,
additivity and Clifford invariance.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2601_07824_gb300 import inputs as I


def test_a0_is_reflection():
    # Eq. A0_reflection: A_0 |x> = |-x> (digit-wise mod 3), here built from Eq. phase-space.
    for N in (1, 2):
        _, A0 = brute.phase_point_operators(N)
        for x in range(3 ** N):
            digits = [(x // 3 ** j) % 3 for j in range(N)]
            mx = sum(((3 - d) % 3) * 3 ** j for j, d in enumerate(digits))
            e = np.zeros(3 ** N)
            e[x] = 1
            out = A0 @ e
            assert abs(out[mx] - 1) < 1e-12 and np.abs(np.delete(out, mx)).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3])
def test_fast_oracle_matches_brute_force(N):
    for seed in (5, 6):
        psi = I.gaussian_state(N, seed, d=3)
        m_o, s_o = oracle.mana(psi)
        m_b, s_b = brute.mana_brute(psi)
        assert abs(m_o - m_b) < 1e-12 and abs(s_o - s_b) < 1e-12


def test_brute_force_wigner_is_real_and_normalised(golden):
    psi = I.gaussian_state(2, 9, d=3)
    W = brute.wigner_brute(psi)
    assert np.abs(W.imag).max() < 1e-13
    assert abs(W.real.sum() - golden["closed_forms"]["wigner_normalisation"]["sum_w"]) < 1e-12
    assert abs((W.real ** 2).sum() - 3.0 ** -2) < 1e-12


@pytest.mark.parametrize("N", [2, 4, 6])
def test_oracle_sum_rules(N):
    # sum_u W = 1, sum_u W^2 = 3^-N, chi real (v_{-x} = v_x^*), on the fast oracle's terms.
    psi = I.gaussian_state(N, 40 + N, d=3)
    m, s, q2, mi = oracle.mana_terms(psi)
    assert abs(s.sum() / 3 ** N - 1) < 1e-12
    assert abs(q2.sum() / 9 ** N - 3.0 ** -N) < 1e-14
    assert mi.max() < 1e-12


@pytest.mark.parametrize("N", [1, 3, 5])
def test_stabilizer_states_zero(N, golden):
    states = [I.zero_state(N, d=3), I.qutrit_ghz(N),
              I.qutrit_graph_state(N, [(j, j + 1) for j in range(N - 1)]),
              I.random_qutrit_clifford_circuit(I.zero_state(N, d=3), N, 30, seed=N)]
    for psi in states:
        m, sw = oracle.mana(psi)
        assert abs(m) < 1e-10, m
        assert abs(sw - 1.0) < 1e-10


def test_zero_state_listing(golden):
    g = golden["closed_forms"]["mana_zero_state"]
    m, _ = oracle.mana(I.zero_state(g["N"], d=3))
    assert abs(m - g["mana"]) < 1e-10


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_strange_state_closed_form(N, golden):
    per = golden["closed_forms"]["mana_strange_per_qutrit"]["sum_abs_w_per_qutrit"]
    m, sw = oracle.mana(I.strange_product(N))
    assert abs(m - N * np.log2(per)) < 1e-11
    assert abs(sw - per ** N) < 1e-9 * per ** N


def test_additivity_and_clifford_invariance():
    a, b = I.gaussian_state(2, 1, d=3), I.gaussian_state(3, 2, d=3)
    ab = np.kron(b, a)
    assert abs(oracle.mana(ab)[0] - oracle.mana(a)[0] - oracle.mana(b)[0]) < 1e-10
    psi = I.gaussian_state(4, 3, d=3)
    ref = oracle.mana(psi)[0]
    for seed in (1, 2):
        phi = I.random_qutrit_clifford_circuit(psi, 4, 40, seed)
        assert abs(oracle.mana(phi)[0] - ref) < 1e-10


def test_planted_mistake_is_caught():
    """Integer negation instead of digit-wise negation (a plausible index mistake) must
    disagree with the brute force."""
    N = 2
    psi = I.gaussian_state(N, 12, d=3)
    m_b, _ = brute.mana_brute(psi)
    dim = 3 ** N

    def digits(x):
        return [(x // 3 ** j) % 3 for j in range(N)]

    def undig(d):
        return sum(v * 3 ** j for j, v in enumerate(d))

    w = np.exp(2j * np.pi / 3)
    F = np.array([[w ** (2 * j * k) for k in range(3)] for j in range(3)])
    Fn = F
    for _ in range(N - 1):
        Fn = np.kron(F, Fn)

    def mana_with(neg):
        tot = 0.0
        for a in range(dim):
            da = digits(a)
            v = np.zeros(dim, dtype=complex)
            for x in range(dim):
                dx = digits(x)
                xm = undig([(p - q) % 3 for p, q in zip(dx, da)])
                nx = neg(x, dx)
                nxm = undig([(p - q) % 3 for p, q in zip(digits(nx), da)])
                v[x] = np.conj(psi[xm]) * psi[nxm]
            tot += np.abs(Fn @ v).sum()
        return np.log2(tot / dim)

    good = mana_with(lambda x, dx: undig([(-p) % 3 for p in dx]))
    bad = mana_with(lambda x, dx: (-x) % dim)
    assert abs(good - m_b) < 1e-12
    assert abs(bad - m_b) > 1e-6
