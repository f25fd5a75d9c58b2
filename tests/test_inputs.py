"""The seeded input generators (CPU): shapes, normalisation, unitarity, reproducibility, site
order, and the gate conventions the workloads rely on."""
import numpy as np
import pytest

from paper_2601_07824_gb300 import inputs as I


def test_gaussian_state_seeded_and_normalised():
    for N, d in ((1, 2), (10, 2), (5, 3)):
        a = I.gaussian_state(N, 7, d=d)
        assert a.shape == (d ** N,) and a.dtype == np.complex128
        assert np.linalg.norm(a) == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_array_equal(a, I.gaussian_state(N, 7, d=d))  # same seed, same state
        assert not np.allclose(a, I.gaussian_state(N, 8, d=d))
    assert I.gaussian_state(6, 1, dtype=np.complex64).dtype == np.complex64


def test_haar_unitary_is_unitary():
    rng = np.random.default_rng(0)
    for n in (2, 3, 4, 9):
        U = I.haar_unitary(n, rng)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(n), atol=1e-12)


def test_site_order_and_product_states():
    # site j = digit j: a one-site gate on site q acts on digit q of the index
    N = 3
    psi = I.zero_state(N)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    out = I.apply_1site(psi, X, 1, N)
    assert np.argmax(np.abs(out)) == 2  # |010> = index 2
    local = np.array([0.6, 0.8j])
    p = I.product_state(local, 3)
    np.testing.assert_allclose(p, np.kron(local, np.kron(local, local)), atol=1e-15)
    np.testing.assert_allclose(I.t_state_product(2), np.kron(*(2 * [np.array([1, np.exp(1j * np.pi / 4)]) / np.sqrt(2)])),
                               atol=1e-15)


def test_circuit_states_are_normalised_and_seeded():
    b = I.brickwork_haar(8, 6, seed=3)
    assert b.dtype == np.complex64 and np.linalg.norm(b.astype(np.complex128)) == pytest.approx(1.0, abs=1e-6)
    np.testing.assert_array_equal(b, I.brickwork_haar(8, 6, seed=3))
    q = I.brickwork_haar(4, 4, seed=2, d=3)
    assert q.shape == (81,) and np.linalg.norm(q.astype(np.complex128)) == pytest.approx(1.0, abs=1e-6)
    Ns, states = I.batched_ladder_states(16, 10, 12, 3, seed=4001)
    assert len(Ns) == len(states) == 16 and all(10 <= n <= 12 for n in Ns)
    for n, s in zip(Ns, states):
        assert s.shape == (2 ** n,) and np.linalg.norm(s.astype(np.complex128)) == pytest.approx(1.0, abs=1e-5)
    assert I.batched_ladder_states(16, 10, 12, 3, seed=4001)[0] == Ns


def test_stabilizer_generators():
    for N in (2, 4):
        g = I.ghz_state(N)
        assert abs(g[0]) == pytest.approx(2 ** -0.5) and abs(g[-1]) == pytest.approx(2 ** -0.5)
        gs = I.graph_state(N, [(j, j + 1) for j in range(N - 1)])
        np.testing.assert_allclose(np.abs(gs), np.full(2 ** N, 2 ** (-N / 2)), atol=1e-14)
        qg = I.qutrit_ghz(N)
        assert np.count_nonzero(np.abs(qg) > 1e-12) == 3
    c = I.random_clifford_circuit(I.zero_state(5), 5, 40, seed=1)
    assert np.linalg.norm(c) == pytest.approx(1.0, abs=1e-12)
    # a Clifford circuit keeps the squared amplitudes of a stabilizer state uniform on its support
    nz = np.abs(c[np.abs(c) > 1e-9]) ** 2
    assert np.allclose(nz, nz[0])
    q = I.random_qutrit_clifford_circuit(I.zero_state(3, d=3), 3, 30, seed=2)
    assert np.linalg.norm(q) == pytest.approx(1.0, abs=1e-12)


def test_interleaved_layout():
    psi = np.array([1 + 2j, 3 - 4j], dtype=np.complex128)
    np.testing.assert_array_equal(I.to_interleaved(psi), np.array([1, 2, 3, -4], dtype=np.float32))


def test_symmetric_state_generators():
    # U(1): support on Hamming weight k only; Z_2: support on one weight parity only
    for N, k in ((6, 3), (7, 2), (1, 1)):
        u = I.u1_state(N, k, 9)
        w = np.array([bin(z).count("1") for z in range(2 ** N)])
        assert np.linalg.norm(u) == pytest.approx(1.0, abs=1e-12)
        assert np.all(u[w != k] == 0) and np.count_nonzero(u[w == k]) == int((w == k).sum())
        np.testing.assert_array_equal(u, I.u1_state(N, k, 9))
        assert not np.allclose(u, I.u1_state(N, k, 10))
    for N, par in ((5, 0), (5, 1), (1, 0)):
        p = I.parity_state(N, 11, parity=par)
        w = np.array([bin(z).count("1") for z in range(2 ** N)])
        assert np.linalg.norm(p) == pytest.approx(1.0, abs=1e-12)
        assert np.all(p[(w & 1) != par] == 0)
    assert I.u1_state(8, 4, 1, dtype=np.complex64).dtype == np.complex64
