"""Statistical pins of the Monte-Carlo standard error reported by the oracle's uniform-X
estimator (`orc_sre_mc`), CPU only.

The estimator evaluates the X-string a = 0 exactly and samples the others uniformly:
    S_hat = S(0)/2^N + w mean_{a_i != 0} S(a_i),  w = 1 - 2^-N,  M2_hat = -log2 S_hat,
and propagates the sample variance to the estimate as the paper propagates a sampling error
to M2 (Sec. 3.2, Eq. M2mNcerror):
    dM2 = w sd(S(a_i)) / sqrt(n) / (S_hat ln 2),  n = number of draws with a_i != 0.

The pins compare it with quantities the estimator does not compute:
  * the exact variance of S_hat over the draw, w^2 var_pop E[1/n], from the population
    variance of S(a) over all 2^N - 1 non-zero X-strings (the exhaustive per-X sums, pinned to
    brute force elsewhere), against the mean over seeds of (dM2 S_hat ln 2)^2;
  * the scatter of M2_hat over seeds, against the RMS of the reported dM2.
Each holds within five standard errors of its own estimate (computed from the seeds).  Small
N makes the factor w visible (3/4 at N = 2, 7/8 at N = 3).  Copies of the reported error with
a plausible mistake (the 1/sqrt(n) dropped, w dropped, natural log for log2) fail the pins."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_07824_gb300 import inputs as I

CASES = [(2, 24, 4000), (3, 32, 4000), (10, 64, 600)]  # (N, samples per estimate, seeds)


def _draws(N, samples, K):
    psi = I.gaussian_state(N, 40 + N)
    S_all = np.asarray(oracle.sre_terms(psi, 2.0)[0])
    M = np.empty(K)
    se = np.empty(K)
    inv_n = np.empty(K)
    for k in range(K):
        seed = 10_000 + k
        M[k], se[k], _ = oracle.sre_mc(psi, samples, seed=seed)
        n = np.count_nonzero(oracle.mc_xstrings(seed, samples, N))
        inv_n[k] = 1.0 / n if n else np.nan
    keep = np.isfinite(inv_n)
    return S_all, M[keep], se[keep], inv_n[keep]


def _variance_pin(N, S_all, M, se, inv_n):
    """(ratio, standard error of the ratio): mean (dM2 S_hat ln 2)^2 over exact Var[S_hat]."""
    w = 1.0 - 2.0 ** -N
    exact = w * w * float(np.var(S_all[1:])) * float(np.mean(inv_n))
    d2 = (se * 2.0 ** -M * math.log(2.0)) ** 2
    return float(np.mean(d2)) / exact, float(np.std(d2, ddof=1) / math.sqrt(len(d2))) / exact


def _scatter_pin(M, se):
    """(ratio, standard error): std over seeds of M2_hat over the RMS of the reported dM2."""
    K = len(M)
    r = float(np.std(M, ddof=1)) / math.sqrt(float(np.mean(se ** 2)))
    # std of a sample standard deviation ~ s / sqrt(2 (K - 1)), plus the spread of the se^2 mean
    e = r * (1.0 / math.sqrt(2 * (K - 1)) + 0.5 * float(np.std(se ** 2, ddof=1) / np.mean(se ** 2)) / math.sqrt(K))
    return r, e


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"N{c[0]}")
def draws(request):
    N, samples, K = request.param
    return (N,) + _draws(N, samples, K)


def test_reported_variance_matches_exact_variance_of_the_draw(draws):
    N, S_all, M, se, inv_n = draws
    r, e = _variance_pin(N, S_all, M, se, inv_n)
    assert abs(r - 1.0) <= 5 * e, (N, r, e)
    # the exact variance itself matches the scatter of S_hat over the seeds
    w = 1.0 - 2.0 ** -N
    exact = w * w * float(np.var(S_all[1:])) * float(np.mean(inv_n))
    v = float(np.var(2.0 ** -M, ddof=1))
    assert abs(v / exact - 1.0) <= 5 * math.sqrt(2.0 / (len(M) - 1)) * 2, (N, v / exact)


def test_scatter_of_estimates_matches_reported_error(draws):
    N, S_all, M, se, inv_n = draws
    r, e = _scatter_pin(M, se)
    assert abs(r - 1.0) <= 5 * e, (N, r, e)


def test_planted_mistakes_fail_the_pins(draws):
    N, S_all, M, se, inv_n = draws
    w = 1.0 - 2.0 ** -N
    n = 1.0 / inv_n
    mistakes = {
        "1/sqrt(n) dropped": se * np.sqrt(n),
        "natural log instead of log2": se * math.log(2.0),
    }
    if N <= 3:
        mistakes["factor w dropped"] = se / w
    for name, bad in mistakes.items():
        r1, e1 = _variance_pin(N, S_all, M, bad, inv_n)
        r2, e2 = _scatter_pin(M, bad)
        assert abs(r1 - 1.0) > 5 * e1 and abs(r2 - 1.0) > 5 * e2, (N, name, r1, e1, r2, e2)
