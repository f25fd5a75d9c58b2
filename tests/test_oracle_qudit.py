"""Pins of the odd-prime-qudit mana oracle (Sec. 2, the remark that the qutrit construction
applies to any odd prime d) on the CPU: the per-shift transform against the dense definition
(every A_u built explicitly), the qutrit C oracle at d = 3, the Wigner sum rules, zeros on
stabilizer states, additivity, Clifford invariance and a planted mistake."""
import numpy as np
import pytest

import oracle
from oracle import qudit as Q
from paper_2601_07824_gb300 import inputs as I


@pytest.mark.parametrize("d,N", [(3, 1), (3, 2), (5, 1), (5, 2), (7, 1), (7, 2), (11, 1), (13, 1)])
def test_fast_transform_equals_dense_definition(d, N):
    psi = I.gaussian_state(N, 10 * d + N, d=d)
    W = Q.wigner_brute(psi, d)
    assert np.abs(W.imag).max() < 1e-14
    chi = Q.chi_fast(psi, d)
    assert np.abs(chi.imag).max() < 1e-12
    np.testing.assert_allclose(np.sort(np.abs(chi.real).ravel()) / d ** N, np.sort(np.abs(W.real)), atol=1e-14)
    m, s, s1, s2 = Q.mana_fast(psi, d)
    mb, sb = Q.mana_brute(psi, d)
    assert m == pytest.approx(mb, abs=1e-12) and s == pytest.approx(sb, rel=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_qutrits_agree_with_the_c_oracle(N):
    psi = I.gaussian_state(N, 500 + N, d=3)
    assert Q.mana_fast(psi, 3)[0] == pytest.approx(oracle.mana(psi)[0], abs=1e-12)


@pytest.mark.parametrize("d,N", [(5, 3), (7, 2), (11, 2), (13, 2)])
def test_sum_rules(d, N):
    psi = I.gaussian_state(N, 600 + d + N, d=d)
    _, s, s1, s2 = Q.mana_fast(psi, d)
    assert s1 == pytest.approx(1.0, abs=1e-12)            # sum_u W(u) = tr rho
    assert s2 == pytest.approx(d ** -N, rel=1e-10)         # sum_u W(u)^2 = tr rho^2 / d^N
    assert s >= 1.0 - 1e-12


@pytest.mark.parametrize("d,N", [(5, 1), (5, 3), (7, 2), (11, 2)])
def test_stabilizer_states_have_zero_mana(d, N):
    states = [Q.zero_state(N, d), Q.ghz(N, d)]
    if N >= 2:
        states.append(Q.graph_state(N, d, [(j, j + 1) for j in range(N - 1)]))
    states.append(Q.random_clifford_circuit(Q.zero_state(N, d), N, d, 25, seed=7 * d + N))
    for psi in states:
        assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-12)
        m, s, _, _ = Q.mana_fast(psi, d)
        assert abs(m) < 1e-12, (d, N)
        W = Q.chi_fast(psi, d).real / d ** N
        assert W.min() > -1e-13  # Hudson: non-negative Wigner function


@pytest.mark.parametrize("d", [5, 7])
def test_additivity_and_clifford_invariance(d):
    a, b = I.gaussian_state(1, 70 + d, d=d), I.gaussian_state(2, 71 + d, d=d)
    ab = np.kron(b, a)  # a on site 0, b on sites 1, 2
    assert Q.mana_fast(ab, d)[0] == pytest.approx(Q.mana_fast(a, d)[0] + Q.mana_fast(b, d)[0], abs=1e-12)
    psi = I.gaussian_state(2, 72 + d, d=d)
    c = Q.random_clifford_circuit(psi, 2, d, 30, seed=d)
    assert Q.mana_fast(c, d)[0] == pytest.approx(Q.mana_fast(psi, d)[0], abs=1e-11)


def test_planted_mistake_fails():
    # a dropped conjugate in v_x breaks the match with the dense definition
    d, N = 5, 2
    psi = I.gaussian_state(N, 80, d=d)
    W = Q.wigner_brute(psi, d).real
    D = psi.size
    dig = np.stack([(np.arange(D) // d ** k) % d for k in range(N)], axis=1)
    pw = d ** np.arange(N)
    w = np.exp(2j * np.pi / d)
    F = np.array([[w ** ((2 * j * k) % d) for k in range(d)] for j in range(d)])
    vals = []
    for a in range(D):
        i1 = (((dig - dig[a]) % d) * pw).sum(-1)
        i2 = (((-dig - dig[a]) % d) * pw).sum(-1)
        t = (psi[i1] * psi[i2]).reshape((d,) * N)
        for ax in range(N):
            t = np.moveaxis(np.tensordot(F, t, axes=([1], [ax])), 0, ax)
        vals.append(np.abs(t.ravel()))
    bad = np.sort(np.concatenate(vals)) / d ** N
    assert not np.allclose(bad, np.sort(np.abs(W)), atol=1e-6)


# ---- gradient of the mana ---------------------------------------------------------------

@pytest.mark.parametrize("d,N", [(3, 1), (3, 2), (3, 4), (5, 2), (7, 2)])
def test_mana_gradient_matches_finite_differences(d, N):
    rng = np.random.default_rng(90 + d + N)
    psi = I.gaussian_state(N, 91 + d + N, d=d) * 1.3  # unnormalised on purpose
    m, g = Q.mana_grad(psi, d)
    # mana of the vector as given (sum |chi| scales as |psi|^4)
    assert m == pytest.approx(Q.mana_fast(psi, d)[0], abs=1e-12)
    mf = lambda v: float(np.log2(np.abs(Q.chi_fast(v, d)).sum() / d ** N))  # noqa: E731
    h = 1e-6
    for _ in range(4):
        delta = rng.normal(size=psi.size) + 1j * rng.normal(size=psi.size)
        fd = (mf(psi + h * delta) - mf(psi - h * delta)) / (2 * h)
        assert fd == pytest.approx(2 * np.real(np.vdot(g, delta)), rel=1e-5, abs=1e-8)
    if d == 3:  # the independent C oracle (Algorithm 5) gives the same finite differences
        delta = rng.normal(size=psi.size) + 1j * rng.normal(size=psi.size)
        fd = (oracle.mana(psi + h * delta)[0] - oracle.mana(psi - h * delta)[0]) / (2 * h)
        assert fd == pytest.approx(2 * np.real(np.vdot(g, delta)), rel=1e-5, abs=1e-8)


@pytest.mark.parametrize("d,N", [(3, 3), (5, 2)])
def test_mana_gradient_phase_and_scale_identities(d, N):
    psi = I.gaussian_state(N, 95 + d, d=d) * 0.7
    _, g = Q.mana_grad(psi, d)
    # a global phase does not change mana: Im sum conj(g) psi = 0
    assert abs(np.imag(np.vdot(g, psi))) < 1e-12
    # mana(c psi) = mana(psi) + 2 log2 c: 2 Re sum conj(g) psi = 2 / ln 2
    assert 2 * np.real(np.vdot(g, psi)) == pytest.approx(2 / np.log(2.0), rel=1e-12)


def test_mana_gradient_counts_small_entries():
    psi = I.gaussian_state(2, 97, d=5)
    m, g = Q.mana_grad(psi, 5)
    m0, g0, k0 = Q.mana_grad(psi, 5, small=0.0)
    _, _, kall = Q.mana_grad(psi, 5, small=1e9)
    assert k0 == 0 and kall == 5 ** 4
    assert m0 == m and np.array_equal(g0, g)


# ---- mixed states ---------------------------------------------------------------------

def _random_rho(D, rank, seed):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(D, rank)) + 1j * rng.normal(size=(D, rank))
    r = G @ G.conj().T
    return r / np.trace(r).real


@pytest.mark.parametrize("d,N", [(3, 2), (5, 1), (5, 2), (7, 1), (11, 1)])
def test_mixed_transform_equals_dense_definition(d, N):
    D = d ** N
    for rank in sorted({1, 2, D}):
        rho = _random_rho(D, rank, 40 * d + rank)
        W = Q.wigner_mixed_brute(rho, d)
        assert np.abs(W.imag).max() < 1e-14
        m, s, s1, s2 = Q.mana_mixed_fast(rho, d)
        assert s == pytest.approx(float(np.abs(W.real).sum()), rel=1e-12)
        assert m == pytest.approx(float(np.log2(np.abs(W.real).sum())), abs=1e-12)
        assert s1 == pytest.approx(1.0, abs=1e-12)                                   # sum W = tr rho
        assert s2 * d ** N == pytest.approx(float(np.trace(rho @ rho).real), rel=1e-10)  # d^N sum W^2 = tr rho^2


@pytest.mark.parametrize("d,N", [(5, 2), (7, 2), (13, 1)])
def test_mixed_reduces_to_pure_and_maximally_mixed_is_zero(d, N):
    psi = I.gaussian_state(N, 60 + d, d=d)
    assert Q.mana_mixed_fast(np.outer(psi, psi.conj()), d)[0] == pytest.approx(Q.mana_fast(psi, d)[0], abs=1e-12)
    D = d ** N
    m, s, _, _ = Q.mana_mixed_fast(np.eye(D) / D, d)
    assert abs(m) < 1e-12 and s == pytest.approx(1.0, abs=1e-12)
