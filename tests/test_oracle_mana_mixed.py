"""Pins of the mixed-state mana oracle (Algorithm 6, Sec. 3.3.3) on the CPU.

Every check is against something other than the fast transform itself: the dense definition
W_u = tr(rho A_u) / 3^N over explicit phase-space point operators, the pure-state oracle
(Algorithm 5) on rho = |psi><psi|, closed forms (maximally mixed state, Strange product),
invariants (sum_u W_u = tr rho, W real, additivity, Clifford invariance), partial traces with
known results, and a planted convention mistake that must fail."""
import numpy as np
import pytest

import oracle
from oracle import brute, mixed
from paper_2601_07824_gb300 import inputs as I


def random_rho(N, seed, rank=None):
    rng = np.random.default_rng(seed)
    D = 3 ** N
    k = rank or D
    G = rng.normal(size=(D, k)) + 1j * rng.normal(size=(D, k))
    rho = G @ G.conj().T
    return rho / np.trace(rho).real


@pytest.mark.parametrize("N", [1, 2, 3])
def test_fast_transform_equals_dense_definition_elementwise(N):
    for seed in range(3):
        rho = random_rho(N, 100 * N + seed, rank=1 + seed)
        Wf = mixed.wigner_mixed(rho)
        Wb = brute.wigner_mixed_brute(rho)  # same ordering: site 0 = most significant label
        np.testing.assert_allclose(Wf, Wb, atol=1e-14)
        assert mixed.mana_mixed(rho)[0] == pytest.approx(brute.mana_mixed_brute(rho)[0], abs=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_pure_states_reduce_to_algorithm_5(N):
    psi = I.gaussian_state(N, 70 + N, d=3)
    m, s = mixed.mana_mixed(np.outer(psi, psi.conj()))
    mo, so = oracle.mana(psi)
    assert m == pytest.approx(mo, abs=1e-12)
    assert s == pytest.approx(so, rel=1e-12)


def test_closed_forms():
    # maximally mixed: W_u = 1 / 9^N for every u, mana 0
    for N in (1, 2, 3):
        W = mixed.wigner_mixed(np.eye(3 ** N) / 3 ** N)
        np.testing.assert_allclose(W, np.full(9 ** N, 1.0 / 9 ** N), atol=1e-15)
        assert mixed.mana_mixed(np.eye(3 ** N) / 3 ** N)[0] == pytest.approx(0.0, abs=1e-14)
    # Strange product ((|1> - |2>)/sqrt 2)^N: sum |W| = (5/3)^N, mana = N log2(5/3)
    for N in (1, 2, 3):
        s = I.strange_product(N)
        m, sw = mixed.mana_mixed(np.outer(s, s.conj()))
        assert sw == pytest.approx((5.0 / 3.0) ** N, rel=1e-12)
        assert m == pytest.approx(N * np.log2(5.0 / 3.0), abs=1e-12)
    # |0><0|^N: a stabilizer state, mana 0
    z = np.zeros(27); z[0] = 1.0
    assert mixed.mana_mixed(np.outer(z, z))[0] == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_normalisation_and_reality(N):
    rho = random_rho(N, 7 + N)
    W = mixed.wigner_mixed(rho)
    assert W.sum() == pytest.approx(np.trace(rho), abs=1e-13)  # sum_u A_u = 3^N identity
    assert np.abs(W.imag).max() <= 1e-14  # A_u Hermitian, rho Hermitian
    # sum_u W_u^2 = tr(rho^2) / 3^N (Eq. phase-space orthogonality tr(A_u A_v) = 3^N delta)
    assert np.sum(W.real ** 2) == pytest.approx(np.trace(rho @ rho).real / 3 ** N, rel=1e-12)


def test_additivity_on_products():
    ra, rb = random_rho(1, 31), random_rho(2, 32)
    rab = np.kron(rb, ra)  # sites of ra are the least significant digits
    assert mixed.mana_mixed(rab)[0] == pytest.approx(mixed.mana_mixed(ra)[0] + mixed.mana_mixed(rb)[0],
                                                     abs=1e-12)


def test_clifford_invariance():
    N = 2
    # unitary of a random qutrit Clifford circuit, column by column from basis states
    U = np.stack([I.random_qutrit_clifford_circuit(np.eye(9)[:, k], N, 12, seed=5) for k in range(9)], axis=1)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(9), atol=1e-12)
    rho = random_rho(N, 41)
    assert mixed.mana_mixed(U @ rho @ U.conj().T)[0] == pytest.approx(mixed.mana_mixed(rho)[0], abs=1e-12)


def test_reduced_density_matrix():
    # generic state: a density matrix
    psi = I.gaussian_state(4, 9, d=3)
    rho = mixed.reduced_density_matrix(psi, [0, 2])
    assert rho.shape == (9, 9)
    assert np.trace(rho).real == pytest.approx(1.0, abs=1e-13)
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() >= -1e-14
    # brute-force partial trace over sites 1 and 3 (site k = digit k)
    D = 81
    want = np.zeros((9, 9), dtype=np.complex128)
    for z1 in range(D):
        for z2 in range(D):
            d1 = [(z1 // 3 ** k) % 3 for k in range(4)]
            d2 = [(z2 // 3 ** k) % 3 for k in range(4)]
            if d1[1] == d2[1] and d1[3] == d2[3]:
                want[d1[0] + 3 * d1[2], d2[0] + 3 * d2[2]] += psi[z1] * np.conj(psi[z2])
    np.testing.assert_allclose(rho, want, atol=1e-14)
    # product state: the reduced state is the pure factor; its mana is Algorithm 5's
    a, b = I.gaussian_state(2, 11, d=3), I.gaussian_state(1, 12, d=3)
    prod = np.kron(b, a)  # a on sites 0, 1; b on site 2
    ra = mixed.reduced_density_matrix(prod, [0, 1])
    np.testing.assert_allclose(ra, np.outer(a, a.conj()), atol=1e-14)
    assert mixed.mana_mixed(ra)[0] == pytest.approx(oracle.mana(a)[0], abs=1e-12)
    # qutrit GHZ traced over one site: a uniform mixture of |00>, |11>, |22> (stabilizer
    # mixture, nonnegative Wigner function), mana 0
    rg = mixed.reduced_density_matrix(I.qutrit_ghz(3), [0, 1])
    np.testing.assert_allclose(rg, np.diag([1 / 3 if k in (0, 4, 8) else 0 for k in range(9)]), atol=1e-14)
    assert mixed.mana_mixed(rg)[0] == pytest.approx(0.0, abs=1e-14)


def test_planted_convention_mistake_fails():
    # building M for the printed column-stacked vec (alpha = i + 3j) while Vec_N uses
    # mu = 3i + j transposes rho site by site; the dense definition catches it
    As, _ = brute.phase_point_operators(1)
    Mbad = np.zeros((9, 9), dtype=np.complex128)
    for u in range(9):
        for i in range(3):
            for j in range(3):
                Mbad[u, i + 3 * j] = As[u][j, i]
    rho = random_rho(2, 55)
    v = mixed.vec_n(rho)
    for leg in range(2):
        v = np.einsum("ua,bam->bum", Mbad, v.reshape(-1, 9, 9 ** (1 - leg))).reshape(-1)
    assert not np.allclose(v / 9, brute.wigner_mixed_brute(rho), atol=1e-6)


def _shift_gather_chi(rho):
    """chi_b(a) from v_x = rho[-x - a, x - a] (digit-wise mod 3) and F_3^{(x)N}: the route the
    mixed-state kernels take instead of Algorithm 6's leg sweep (restated here in NumPy)."""
    D = rho.shape[0]
    N = mixed._n_sites(D)
    d = np.stack([(np.arange(D) // 3 ** k) % 3 for k in range(N)], axis=1)
    pw = 3 ** np.arange(N)
    r = (((-d[None, :, :] - d[:, None, :]) % 3) * pw).sum(-1)  # [a, x]
    c = (((d[None, :, :] - d[:, None, :]) % 3) * pw).sum(-1)
    w = np.exp(2j * np.pi / 3)
    F = np.array([[w ** (2 * j * k) for k in range(3)] for j in range(3)])
    t = rho[r, c].reshape((D,) + (3,) * N)  # axis 1 + k: digit N-1-k of x
    for ax in range(1, N + 1):
        t = np.moveaxis(np.tensordot(F, t, axes=([1], [ax])), 0, ax)
    return t.reshape(D, D), r, c


@pytest.mark.parametrize("N", [1, 2, 3])
def test_shift_gather_reproduces_algorithm_6(N):
    # (a, x) -> (-x - a, x - a) reads every entry of rho once; the transformed values are
    # 3^N W_u up to the labelling of u, real for Hermitian rho
    for rank in (1, 2, 3 ** N):
        rho = random_rho(N, 300 + 10 * N + rank, rank)
        chi, r, c = _shift_gather_chi(rho)
        flat = np.sort((r * 3 ** N + c).ravel())
        np.testing.assert_array_equal(flat, np.arange(9 ** N))
        assert np.abs(chi.imag).max() < 1e-13
        W = mixed.wigner_mixed(rho).real
        np.testing.assert_allclose(np.sort(np.abs(chi.real).ravel()) / 3 ** N, np.sort(np.abs(W)), atol=1e-14)
        assert np.log2(np.abs(chi.real).sum() / 3 ** N) == pytest.approx(mixed.mana_mixed(rho)[0], abs=1e-12)
    # on rho = |psi><psi| the route gives the C oracle's Algorithm 5 mana
    psi = I.gaussian_state(N, 330 + N, d=3)
    chi, _, _ = _shift_gather_chi(np.outer(psi, psi.conj()))
    assert np.log2(np.abs(chi.real).sum() / 3 ** N) == pytest.approx(oracle.mana(psi)[0], abs=1e-12)


def test_reduced_density_matrix_of_qudits():
    # d = 5: brute-force partial trace, and a product state's pure factor
    d, N = 5, 3
    psi = I.gaussian_state(N, 77, d=d)
    rho = mixed.reduced_density_matrix(psi, [2, 0], d=d)
    want = np.zeros((25, 25), dtype=np.complex128)
    for z1 in range(d ** N):
        for z2 in range(d ** N):
            a = [(z1 // d ** k) % d for k in range(N)]
            b = [(z2 // d ** k) % d for k in range(N)]
            if a[1] == b[1]:
                want[a[2] + d * a[0], b[2] + d * b[0]] += psi[z1] * np.conj(psi[z2])
    np.testing.assert_allclose(rho, want, atol=1e-14)
    f1, f2 = I.gaussian_state(1, 78, d=d), I.gaussian_state(2, 79, d=d)
    np.testing.assert_allclose(mixed.reduced_density_matrix(np.kron(f2, f1), [1, 2], d=d),
                               np.outer(f2, f2.conj()), atol=1e-14)
