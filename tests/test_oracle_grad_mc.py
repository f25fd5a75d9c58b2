"""Pins for the oracle's M_2 gradient (central finite differences of the oracle's own,
brute-force-pinned forward; exact phase and scale identities) and for the uniform-X
Monte-Carlo estimator (published SplitMix64 outputs, the identity-list reduction to the
exact M_2, a statistical band).  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2601_07824_gb300 import inputs as I


def f(psi):
    return oracle.sre(psi, 2.0)[0]


@pytest.mark.parametrize("N", [2, 3, 4])
def test_gradient_matches_finite_differences_per_coordinate(N):
    psi = I.gaussian_state(N, 100 + N)
    M2, g = oracle.sre_grad(psi)
    assert abs(M2 - f(psi)) < 1e-12
    h = 1e-5
    for w in range(2 ** N):
        for unit in (1.0, 1j):
            d = np.zeros(2 ** N, dtype=complex)
            d[w] = unit * h
            fd = (f(psi + d) - f(psi - d)) / (2 * h)
            # df = 2 Re sum conj(g) dpsi for the Wirtinger derivative g = df/dpsi*
            assert abs(fd - 2 * np.real(np.conj(g[w]) * unit)) < 1e-7, (w, unit)


def test_gradient_random_direction_unnormalised():
    N = 8
    psi = 1.1 * I.gaussian_state(N, 5)
    rng = np.random.default_rng(0)
    _, g = oracle.sre_grad(psi)
    for _ in range(3):
        d = rng.standard_normal(2 ** N) + 1j * rng.standard_normal(2 ** N)
        d /= np.linalg.norm(d)
        h = 1e-4
        fd = (f(psi + h * d) - f(psi - h * d)) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(g, d))) < 1e-7


def test_gradient_phase_and_scale_identities():
    # M2(e^{i t} psi) = M2(psi)  ->  Im <g, psi> = 0;  M2(l psi) = M2(psi) - 8 log2 l
    # -> 2 Re <g, psi> = -8 / ln 2.  Both hold at any N.
    for N in (5, 9):
        psi = I.gaussian_state(N, 3 + N)
        _, g = oracle.sre_grad(psi)
        ip = np.vdot(g, psi)
        assert abs(ip.imag) < 1e-10
        assert abs(2 * ip.real + 8 / np.log(2)) < 1e-9


def test_splitmix64_published_outputs(golden):
    g = golden["splitmix64"]
    out = oracle.splitmix64(g["seed"], len(g["outputs_hex"]))
    assert [f"{int(x):016x}" for x in out] == g["outputs_hex"]


def test_mc_xstrings_are_top_bits():
    seed, N = 2802, 28
    raw = oracle.splitmix64(seed, 64)
    a = oracle.mc_xstrings(seed, 64, N)
    assert np.array_equal(a, (raw >> np.uint64(64 - N)).astype(np.int64))
    assert a.min() >= 0 and a.max() < 2 ** N


def test_mc_identity_list_reduces_to_exact():
    N = 8
    psi = I.gaussian_state(N, 9)
    S = oracle.sre_terms_list(psi, np.arange(2 ** N))
    Sq, _, _ = oracle.sre_terms(psi, 2.0)
    assert np.allclose(S, Sq, rtol=1e-14, atol=0)
    assert abs(-np.log2(S.mean()) - f(psi)) < 1e-12


def test_mc_estimate_within_band():
    N = 12
    psi = I.gaussian_state(N, 7)
    exact = f(psi)
    M, se, S = oracle.sre_mc(psi, 512, seed=99)
    assert se > 0
    assert abs(M - exact) < 4 * se + 1e-12, (M, exact, se)
    a = oracle.mc_xstrings(99, 512, N)
    assert np.allclose(S, oracle.sre_terms_list(psi, a), rtol=1e-15)


def test_mc_estimator_treats_identity_row_exactly():
    # Sec. 4.2 footnote: the identity is handled exactly, not sampled.  With the X-string a = 0
    # evaluated exactly, S_hat = [S(0) + (2^N - 1) mean_{a_i != 0} S(a_i)] / 2^N.
    N = 6
    psi = I.gaussian_state(N, 3)
    M, se, S = oracle.sre_mc(psi, 300, seed=5)
    a = oracle.mc_xstrings(5, 300, N)
    Sq, _, _ = oracle.sre_terms(psi, 2.0)
    nz = a != 0
    Shat = Sq[0] / 2 ** N + (2 ** N - 1) / 2 ** N * S[nz].mean()
    assert abs(M + np.log2(Shat)) < 1e-12
    # every a != 0 drawn once each -> exact
    exact = f(psi)
    Shat_all = Sq[0] / 2 ** N + (2 ** N - 1) / 2 ** N * Sq[1:].mean()
    assert abs(-np.log2(Shat_all) - exact) < 1e-12


def test_gradient_at_N17_matches_stored_finite_differences():
    # tests/golden/grad_large.json (tests/golden/make_grad_fd_values.py, oracle only): at N = 17
    # the oracle's gradient projected on seeded directions equals central finite differences of
    # its forward M_2 (step 1e-4) -- the same pin as above at a size too slow to rerun here
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "grad_large.json")) as f:
        gold = json.load(f)
    checked = 0
    for name, e in gold.items():
        if name.startswith("_"):
            continue
        for k, fd in enumerate(e["fd"]):
            assert abs(fd - e["proj"][k]) <= 1e-6 * abs(e["proj"][k]) + 1e-10, (name, k, fd, e["proj"][k])
            checked += 1
    assert checked >= 2
