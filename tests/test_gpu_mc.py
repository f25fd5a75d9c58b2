"""Uniform-X Monte-Carlo M_2 (N = 28, 4096 sampled X-strings, and smaller cases) on the GPU: bit-exact X-strings, per-sample
sums against the FP64 oracle (including the three-pass HBM schedule at N = 25 and 28), and the
estimator against the exact value / Haar band.  Per-sample tolerance 2e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402

DEV = torch.device("cuda:0")


def on_dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV)


def test_mc_equals_exact_in_expectation_small():
    # the estimator is unbiased for S_2 / 2^N (4 sigma band on a Haar-like state)
    psi = I.gaussian_state(14, 77)
    t = on_dev(psi)
    exact, _ = hm.sre(t, 2.0)
    M, se = hm.sre_mc(t, 4096, 123)
    assert abs(M - exact) < 4 * se + 1e-9, (M, exact, se)
    Mo, seo, _ = oracle.sre_mc(psi, 4096, 123)
    assert abs(M - Mo) <= 1e-6 * abs(Mo)


@pytest.mark.parametrize("N", [25])
def test_hbm_schedule_terms_vs_oracle(N):
    psi = I.gaussian_state(N, 2500 + N, dtype=np.complex64)
    dim = 2 ** N
    rng = np.random.default_rng(N)
    a = np.array([0, 1, 8191, 8192, dim - 1] + list(rng.integers(0, dim, 3)), dtype=np.int64)
    got = hm.sre_terms(on_dev(psi), 2.0, torch.from_numpy(a).to(DEV)).cpu().numpy()
    want = oracle.sre_terms_list(psi, a)
    np.testing.assert_allclose(got[:, 0], want, rtol=2e-5)


def test_mc_N28_4096_samples():
    N, samples = 28, 4096
    psi = I.gaussian_state(N, 2801, dtype=np.complex64)
    t = on_dev(psi)
    M, se = hm.sre_mc(t, samples, 2802)
    # i.i.d. Gaussian (Haar after normalisation): M_2 ~ log2(2^N + 3) - 2 (Sec. 4.1)
    assert abs(M - (np.log2(2.0 ** N + 3) - 2)) < 4 * se + 1e-6, (M, se)
    # per-sample sums of the first few sampled X-strings against the oracle
    a = oracle.mc_xstrings(2802, 3, N)
    got = hm.sre_terms(t, 2.0, torch.from_numpy(a).to(DEV)).cpu().numpy()
    want = oracle.sre_terms_list(psi, a)
    np.testing.assert_allclose(got[:, 0], want, rtol=2e-5)
