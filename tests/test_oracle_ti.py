"""Pins of the thermodynamic-integration M_2 oracle (Sec. 3.2, Algorithm 3) on the CPU.

Against things other than the estimator itself: the exact M_2 of the FP64 oracle (the
identity with the exact integrand converges at Simpson's fourth order), polynomial exactness
of the quadrature weights, the defining relation <f>_beta = -d ln Z / d beta by finite
differences, closed forms with eps > 0 on a stabilizer state, the stationary distribution of
the Metropolis chains (visit frequencies against Pi_beta), and planted mistakes (the printed
sign, log2 in the energy, an inverted acceptance rule) that must fail."""
import math

import numpy as np
import pytest

import oracle
from oracle import ti
from paper_2601_07824_gb300 import inputs as I


@pytest.mark.parametrize("L", [3, 5, 9, 4, 6, 10])
def test_simpson_weights_integrate_cubics_exactly(L):
    w = ti.simpson_weights(L)
    x = np.linspace(0.0, 1.0, L)
    for k in range(4):
        assert np.dot(w, x ** k) == pytest.approx(1.0 / (k + 1), abs=1e-14)


def test_boltzmann_mean_is_minus_dlnZ_dbeta():
    f = ti.energies(I.gaussian_state(5, 3))
    lnZ = lambda b: float(np.log(np.sum(np.exp(-b * f))))  # noqa: E731
    for beta in (0.0, 0.3, 0.8, 1.0):
        h = 1e-5
        assert ti.boltzmann_mean(f, beta) == pytest.approx(-(lnZ(beta + h) - lnZ(beta - h)) / (2 * h), rel=1e-7)
    # beta = 0: the plain mean; beta = 1: Z_1 = S_2 (natural log in f)
    assert ti.boltzmann_mean(f, 0.0) == pytest.approx(f.mean(), rel=1e-13)
    S2 = oracle.sre_terms(I.gaussian_state(5, 3), 2.0)[0].sum()
    assert np.sum(np.exp(-f)) == pytest.approx(S2, rel=1e-12)


@pytest.mark.parametrize("state", ["gauss", "brick", "tprod"])
def test_exact_integrand_converges_to_exact_m2(state):
    psi = {"gauss": I.gaussian_state(7, 21), "brick": I.brickwork_haar(8, 6, seed=3, dtype=np.complex128),
           "tprod": I.t_state_product(6)}[state]
    M2 = oracle.sre(psi, 2.0)[0]
    e17 = abs(ti.m2_ti_exact(psi, 17) - M2)
    e33 = abs(ti.m2_ti_exact(psi, 33) - M2)
    assert e33 < 2e-6 * max(1.0, M2)
    assert e33 < e17 / 6  # fourth order: halving the step divides the error by ~16
    assert ti.m2_ti_exact(psi, 32) == pytest.approx(M2, abs=5e-6 * max(1.0, M2))  # even L: 3/8 end panel


def test_eps_regularisation_on_a_stabilizer_state():
    # |0...0>: S(a) = 0 for a != 0, so eps > 0 is required; M_2 = -log2(exp(-I) - eps) = 0
    z = I.zero_state(6)
    with pytest.raises(ValueError):
        ti.energies(z)
    for eps in (1e-3, 1e-1):
        assert abs(ti.m2_ti_exact(z, 65, eps=eps)) < 1e-6
    # the identity Z_1 = S_2 + 2^N eps
    f = ti.energies(z, eps=1e-3)
    assert np.sum(np.exp(-f)) == pytest.approx(2 ** 6 + 2 ** 6 * 1e-3, rel=1e-12)


def test_metropolis_chains_sample_the_boltzmann_distribution():
    f = ti.energies(I.gaussian_state(5, 4))
    means, visits = ti.metropolis_means(f, 5, 3, 200000, seed=77, burn_in=1000)
    for l, beta in enumerate((0.0, 0.5, 1.0)):
        p = np.exp(-beta * f)
        p /= p.sum()
        emp = visits[l] / visits[l].sum()
        assert 0.5 * np.abs(emp - p).sum() < 0.03, beta
        assert means[l] == pytest.approx(ti.boltzmann_mean(f, beta), rel=0.03)


def test_metropolis_estimate_and_reproducibility():
    psi = I.gaussian_state(6, 9)
    M2 = oracle.sre(psi, 2.0)[0]
    for seed in (0, 100, 200):
        assert ti.m2_metropolis(psi, 9, 20000, seed, burn_in=500) == pytest.approx(M2, rel=0.02)
    assert ti.m2_metropolis(psi, 5, 500, 7) == ti.m2_metropolis(psi, 5, 500, 7)  # seeded, deterministic


def test_planted_mistakes_fail():
    psi = I.gaussian_state(7, 21)
    M2 = oracle.sre(psi, 2.0)[0]
    f = ti.energies(psi)
    betas = np.linspace(0.0, 1.0, 33)
    I_ = float(np.dot(ti.simpson_weights(33), [ti.boltzmann_mean(f, b) for b in betas]))
    # the printed return value of Algorithm 3 (-1/ln 2 times the quadrature) is -M_2
    assert -I_ / math.log(2.0) == pytest.approx(-M2, rel=1e-5)
    assert abs(-I_ / math.log(2.0) - M2) > 1.0
    # log2 instead of ln in the energy breaks Z_1 = S_2
    f2 = f / math.log(2.0)
    I2 = float(np.dot(ti.simpson_weights(33), [ti.boltzmann_mean(f2, b) for b in betas]))
    assert abs(ti.m2_from_integral(I2) - M2) > 0.1
    # an inverted acceptance rule (min(1, exp(+beta df))) samples the wrong distribution
    g = ti.energies(I.gaussian_state(5, 4))
    _, visits = ti.metropolis_means(-g, 5, 3, 50000, seed=77, burn_in=500)
    p = np.exp(-1.0 * g)
    p /= p.sum()
    assert 0.5 * np.abs(visits[2] / visits[2].sum() - p).sum() > 0.1


def test_energies_on_demand_give_the_same_chains():
    # the cached per-X-string evaluation is the table's arithmetic, one X-string at a time
    psi = I.gaussian_state(8, 13)
    table = ti.energies(psi)
    lazy = ti.energy_fn(psi)
    for a in (0, 1, 77, 255):
        assert lazy(a) == pytest.approx(table[a], rel=1e-14)
    ra, rb = {}, {}
    ma, _ = ti.metropolis_means(table, 8, 4, 300, seed=5, burn_in=20, record=ra)
    mb, vb = ti.metropolis_means(lazy, 8, 4, 300, seed=5, burn_in=20, record=rb)
    assert vb is None
    np.testing.assert_array_equal(ra["traj"], rb["traj"])
    np.testing.assert_allclose(ma, mb, rtol=1e-13)
    with pytest.raises(ValueError):
        ti.energy_fn(I.zero_state(4))(3)  # S(3) = 0 on |0000>


def test_recorded_trajectory_is_a_valid_chain():
    N, L, n_s, burn = 7, 5, 400, 30
    psi = I.gaussian_state(N, 17)
    f = ti.energies(psi)
    rec = {}
    means, visits = ti.metropolis_means(f, N, L, n_s, seed=11, burn_in=burn, record=rec)
    traj, margin = rec["traj"], rec["margin"]
    assert traj.shape == margin.shape == (L, burn + n_s)
    assert np.all((margin >= 0.0) & (margin <= 1.0))
    for l in range(L):
        r = oracle.splitmix64(11 + l, 1 + 2 * (burn + n_s))
        a = int(r[0] >> np.uint64(64 - N))
        for t in range(burn + n_s):
            flip = a ^ (1 << int(r[1 + 2 * t] % np.uint64(N)))
            assert traj[l, t] in (a, flip)  # stay or take the proposed one-bit flip
            a = int(traj[l, t])
        assert means[l] == pytest.approx(f[traj[l, burn:]].mean(), rel=1e-12)
        np.testing.assert_array_equal(np.bincount(traj[l, burn:], minlength=1 << N), visits[l])
    # beta = 0 accepts every proposal
    assert np.all(traj[0] != np.concatenate(([int(oracle.splitmix64(11, 1)[0] >> np.uint64(64 - N))], traj[0, :-1])))


# ---- even sector (Sec. 3.2: U(1) / Z_2^Z symmetric states, odd-weight X-sectors vanish) ----

def symmetric_states():
    # U(1) states at half filling (k = N/2 or (N-1)/2): X_a can map weight-k states onto
    # weight-k states only if |a|/2 <= min(k, N-k), so away from half filling some even-weight
    # sectors vanish as well (see the next test)
    return [("u1", I.u1_state(8, 4, 21)), ("u1_odd_N", I.u1_state(7, 3, 22)), ("z2_even", I.parity_state(8, 23)),
            ("z2_odd", I.parity_state(7, 24, parity=1))]


def test_u1_away_from_half_filling_keeps_vanishing_even_sectors():
    N, k = 8, 3
    Sq, _, _ = oracle.sre_terms(I.u1_state(N, k, 21), 2.0)
    a = np.arange(1 << N)
    wt = np.array([bin(x).count("1") for x in a])
    assert np.abs(Sq[wt > 2 * min(k, N - k)]).max() < 1e-14  # |a| = 8 > 6: S(a) = 0
    assert Sq[(wt % 2 == 0) & (wt <= 2 * min(k, N - k))].min() > 0.0
    with pytest.raises(ValueError):  # the even-sector chain then needs eps > 0 too
        ti.energies_sector(I.u1_state(N, k, 21), 0.0, "even")
    assert ti.m2_ti_exact(I.u1_state(N, k, 21), 65, eps=1e-9, sector="even") == pytest.approx(
        oracle.sre(I.u1_state(N, k, 21), 2.0)[0], abs=1e-4)


@pytest.mark.parametrize("label,psi", symmetric_states())
def test_odd_sectors_vanish_and_even_sector_sre_is_exact(label, psi):
    N = int(round(math.log2(psi.size)))
    Sq, S1, _ = oracle.sre_terms(psi, 2.0)
    odd = ~ti.even_mask(N)
    assert np.abs(Sq[odd]).max() < 1e-14 and np.abs(S1[odd]).max() < 1e-14
    for q in (0.5, 1.0, 2.0, 2.5, 3.0):
        M, lost = oracle.sre(psi, q)
        Me, loste = oracle.sre_even_sector(psi, q)
        assert Me == pytest.approx(M, abs=1e-11), q
        assert loste == pytest.approx(lost, abs=1e-12)


def test_even_sector_sre_differs_on_a_generic_state():
    psi = I.gaussian_state(7, 25)
    assert abs(oracle.sre_even_sector(psi, 2.0)[0] - oracle.sre(psi, 2.0)[0]) > 0.1


@pytest.mark.parametrize("label,psi", symmetric_states())
def test_even_sector_integral_converges_to_exact_m2(label, psi):
    M2 = oracle.sre(psi, 2.0)[0]
    e17 = abs(ti.m2_ti_exact(psi, 17, sector="even") - M2)
    e33 = abs(ti.m2_ti_exact(psi, 33, sector="even") - M2)
    assert e33 < 2e-6 * max(1.0, M2) and e33 < e17 / 6
    # without the sector the odd X-strings have S = 0: only eps > 0 makes the full chain valid,
    # and then both agree with M_2 up to the eps bias
    with pytest.raises(ValueError):
        ti.energies(psi)


def test_even_sector_chains_stay_in_the_sector_and_sample_it():
    psi = I.u1_state(7, 3, 26)
    N = 7
    f = ti.energy_table(psi, 0.0, "even")
    rec = {}
    means, visits = ti.metropolis_means(f, N, 3, 100000, seed=31, burn_in=1000, record=rec, sector="even")
    w = np.array([[bin(int(a)).count("1") % 2 for a in row] for row in rec["traj"]])
    assert not w.any()
    even = ti.even_mask(N)
    for l, beta in enumerate((0.0, 0.5, 1.0)):
        p = np.where(even, np.exp(-beta * np.where(even, f, 0.0)), 0.0)
        p /= p.sum()
        emp = visits[l] / visits[l].sum()
        assert 0.5 * np.abs(emp - p).sum() < 0.04, beta
    M2 = oracle.sre(psi, 2.0)[0]
    assert ti.m2_metropolis(psi, 9, 20000, 5, burn_in=500, sector="even") == pytest.approx(M2, rel=0.02)


def test_even_sector_planted_mistakes_fail():
    psi = I.parity_state(7, 27)
    M2 = oracle.sre(psi, 2.0)[0]
    f = ti.energies_sector(psi, 0.0, "even")
    betas = np.linspace(0.0, 1.0, 33)
    I_ = float(np.dot(ti.simpson_weights(33), [ti.boltzmann_mean(f, b) for b in betas]))
    # dropping the log2(2^N / Z_0) = 1 shift is off by one bit
    assert abs(ti.m2_from_integral(I_) - M2) == pytest.approx(1.0, abs=1e-5)
    assert ti.m2_from_integral(I_, sector="even") == pytest.approx(M2, abs=1e-5)
    # one-bit proposals leave the sector at the first step
    rec = {}
    ti.metropolis_means(ti.energies(psi, 1e-3), 7, 3, 50, seed=3, record=rec)
    assert any(bin(int(a)).count("1") % 2 for a in rec["traj"].ravel())


# ---- statistical error (Eqs. Var_I_eps, m2error; batch-means reading) ----------------------

def test_batch_sums_partition_the_recorded_energies():
    psi = I.gaussian_state(6, 41)
    f = ti.energies(psi)
    for n_s in (1, 7, 32, 100, 1000):
        rec = {}
        means, _ = ti.metropolis_means(f, 6, 3, n_s, seed=5, burn_in=3, record=rec)
        B = ti.n_batches(n_s)
        K = n_s // B
        assert rec["batch_sums"].shape == (3, B)
        for l in range(3):
            fr = f[rec["traj"][l, 3:]]
            np.testing.assert_allclose(rec["batch_sums"][l], fr[:B * K].reshape(B, K).sum(1), rtol=1e-13)
            assert means[l] == pytest.approx(fr.mean(), rel=1e-13)
    assert ti.m2_stderr(np.ones((3, 1)), 1, 1.0) == 0.0


def test_reported_error_matches_the_spread_over_seeds():
    # the batch-means error must describe the actual scatter of independent estimates
    psi = I.gaussian_state(6, 42)
    L, n_s, burn = 5, 3000, 200
    f = ti.energies(psi)
    est, errs = [], []
    for seed in range(40):
        rec = {}
        means, _ = ti.metropolis_means(f, 6, L, n_s, seed=1000 * seed, burn_in=burn, record=rec)
        I_ = float(np.dot(ti.simpson_weights(L), means))
        est.append(ti.m2_from_integral(I_))
        errs.append(ti.m2_stderr(rec["batch_sums"], n_s, I_))
    spread, typical = float(np.std(est, ddof=1)), float(np.median(errs))
    assert 0.6 < spread / typical < 1.6, (spread, typical)
    # and the estimates scatter around the exact M_2 accordingly
    M2 = oracle.sre(psi, 2.0)[0]
    assert abs(np.mean(est) - M2) < 4 * spread / np.sqrt(len(est)) + 2e-3


def test_error_slope_with_eps():
    # M_2 = -log2(exp(-I) - eps): d M_2 / d I = exp(-I) / ((exp(-I) - eps) ln 2)
    bs = np.array([[1.0, 2.0, 3.0, 5.0], [2.0, 2.0, 4.0, 1.0], [0.0, 1.0, 0.0, 2.0]])
    e0 = ti.m2_stderr(bs, 8, 0.7)
    e1 = ti.m2_stderr(bs, 8, 0.7, eps=0.1)
    assert e1 / e0 == pytest.approx(np.exp(-0.7) / (np.exp(-0.7) - 0.1), rel=1e-12)
    h = 1e-6
    slope = (ti.m2_from_integral(0.7 + h, 0.1) - ti.m2_from_integral(0.7 - h, 0.1)) / (2 * h)
    assert e1 / e0 == pytest.approx(slope * np.log(2.0), rel=1e-6)
