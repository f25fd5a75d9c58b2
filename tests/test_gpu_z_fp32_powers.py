"""The opt-in FP32-powers path for non-integer n (hadamag_set_fp32_powers) against the FP64
oracle.  Tolerance: the documented bound (2 + 2 ln2 n N) 2^-23 on each term's relative error,
so (2 + 2 ln2 n N) 2^-23 / (ln2 |1 - n|) on M_n, plus the FP32 transform's 1e-6 max(1, |M|)
(per-X-string sums: the FP32 path's 2e-5).  The context is shared by the test session, so the
path is switched off again after every test."""
import math

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


@pytest.fixture
def fp32_powers():
    c = hm.context(0)
    c.set_fp32_powers(True)
    try:
        yield c
    finally:
        c.set_fp32_powers(False)


def term_bound(n, N):
    return (2 + 2 * math.log(2) * n * N) * 2.0 ** -23


@pytest.mark.parametrize("N,n", [(3, 0.5), (8, 0.5), (10, 1.5), (12, 2.5), (14, 3.5)])
def test_full_sre_vs_oracle(fp32_powers, N, n):
    psi = I.gaussian_state(N, 5000 + N, dtype=np.complex64)
    M, lost = hm.sre(torch.from_numpy(psi).to(DEV), n)
    Mo, losto = oracle.sre(psi, n)
    tol = term_bound(n, N) / (math.log(2) * abs(1 - n)) + 1e-6 * max(1.0, abs(Mo))
    assert abs(M - Mo) <= tol, (N, n, M, Mo, tol)
    assert abs(lost - losto) <= 2e-6


@pytest.mark.parametrize("N,n", [(16, 2.5), (18, 0.75)])
def test_two_pass_per_x_sums_vs_oracle(fp32_powers, N, n):
    psi = I.brickwork_haar(N, 8, seed=5100 + N)
    a0, a1 = 1000, 1064
    a = torch.arange(a0, a1, dtype=torch.int64, device=DEV)
    t = hm.sre_terms(torch.from_numpy(psi).to(DEV), n, a).cpu().numpy()
    Sq, S1, _ = oracle.sre_terms(psi, n, a0, a1)
    np.testing.assert_allclose(t[:, 0], Sq, rtol=term_bound(n, N) + 2e-5)
    np.testing.assert_allclose(t[:, 1], S1, rtol=2e-5)


def test_off_by_default_and_outside_its_range(fp32_powers):
    # n (N + 2) > 100 keeps FP64 powers: the result equals the default path's exactly
    c = fp32_powers
    psi = torch.from_numpy(I.gaussian_state(10, 5200, dtype=np.complex64)).to(DEV)
    fast = hm.sre(psi, 9.5)
    c.set_fp32_powers(False)
    assert hm.sre(psi, 9.5) == fast
    assert c.lib.hadamag_set_fp32_powers(c.h, 2) == 1  # INVALID_ARG
