"""GPU parity of the exact SRE (C ABI via the torch binding) against the FP64 oracle.

Tolerance (stated for the FP32 path): |dM| <= 1e-6 * max(1, |M|), i.e. 1e-6 relative for
|M| >= 1 and 1e-6 absolute near stabilizer states where M = 0; per-X-string sums agree to
2e-5 relative (FP32 transform of 2^(N-1) values, FP32 partial sums).  Index work (the
SplitMix64 X-strings) is compared bit for bit."""
import ctypes

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
TOL_M = 1e-6


def close_M(a, b, tol=TOL_M):
    return abs(a - b) <= tol * max(1.0, abs(b))


def on_dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV)


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_onepass_sweep_vs_oracle(N):
    psi = I.gaussian_state(N, 500 + N, dtype=np.complex64)
    t = on_dev(psi)
    for n in (1.0, 2.0, 3.0, 2.5):
        M, ln = hm.sre(t, n)
        Mo, lno = oracle.sre(psi, n)
        assert close_M(M, Mo), (N, n, M, Mo)
        assert abs(ln - lno) < 1e-6


def test_N12_complex128_closed_forms(golden):
    g = golden["closed_forms"]["sre_t_state_per_qubit"]
    t = on_dev(I.t_state_product(12))
    for n, key in ((1.0, "M1"), (2.0, "M2"), (3.0, "M3")):
        M, ln = hm.sre(t, n)
        assert close_M(M, g[key]), (n, M)
        assert abs(ln) < 1e-6
    ghz = on_dev(I.ghz_state(12))
    for n in (1.0, 2.0, 3.0):
        M, _ = hm.sre(ghz, n)
        assert abs(M) < 1e-6


def test_N12_gaussian_complex128_vs_oracle():
    psi = I.gaussian_state(12, 1201)  # complex128 input
    t = on_dev(psi)
    for n in (1.0, 2.0, 3.0):
        M, ln = hm.sre(t, n)
        Mo, lno = oracle.sre(psi, n)
        assert close_M(M, Mo), (n, M, Mo)
        assert abs(ln - lno) < 1e-6


@pytest.mark.parametrize("N", [4, 12, 16, 17])
def test_per_x_terms_vs_oracle(N):
    psi = I.gaussian_state(N, 900 + N, dtype=np.complex64)
    dim = 2 ** N
    rng = np.random.default_rng(N)
    a = np.unique(np.concatenate([[0, 1, 2, dim - 1, dim // 2, min(1023, dim - 1), min(1024, dim - 1)],
                                  rng.integers(0, dim, 40)]))
    at = torch.from_numpy(a.astype(np.int64)).to(DEV)
    for n in (1.0, 2.0, 3.0):
        got = hm.sre_terms(on_dev(psi), n, at).cpu().numpy()
        want = np.array([[v[0] for v in oracle.sre_terms(psi, n, int(ai), int(ai) + 1)] for ai in a])
        np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=2e-5)
        np.testing.assert_allclose(got[:, 1], want[:, 1], rtol=2e-5)
        if n == 1.0:
            np.testing.assert_allclose(got[:, 2], want[:, 2], rtol=2e-5, atol=1e-7 * np.abs(want[:, 2]).max())


def test_twopass_full_vs_oracle_N16():
    psi = I.brickwork_haar(16, 6, seed=1601)
    for n in (2.0, 3.0, 1.0):
        M, ln = hm.sre(on_dev(psi), n)
        Mo, lno = oracle.sre(psi, n)
        assert close_M(M, Mo), (n, M, Mo)
        assert abs(ln - lno) < 1e-6


@pytest.mark.parametrize("N", [18, 20, 22, 24])
def test_twopass_sampled_terms_and_exact_identities(N):
    psi = I.gaussian_state(N, 2200 + N, dtype=np.complex64)
    t = on_dev(psi)
    dim = 2 ** N
    rng = np.random.default_rng(N)
    a = np.unique(np.concatenate([[0, 1, 1023, 1024, dim - 1], rng.integers(0, dim, 3)]))
    got = hm.sre_terms(t, 2.0, torch.from_numpy(a.astype(np.int64)).to(DEV)).cpu().numpy()
    want = oracle.sre_terms_list(psi, a)
    np.testing.assert_allclose(got[:, 0], want, rtol=2e-5)
    # sum_b |chi_b(a)|^2 = 2^N sum_z |psi_z|^2 |psi_{z^a}|^2 (Parseval, Eq. Z_FT_qubits)
    p = np.abs(psi.astype(np.complex128)) ** 2
    z = np.arange(dim)
    s1 = np.array([dim * np.sum(p * p[z ^ ai]) for ai in a])
    np.testing.assert_allclose(got[:, 1], s1, rtol=2e-5)
    if N <= 20:
        M, ln = hm.sre(t, 2.0)
        # lost_norm = 1 - |psi|^4 exactly (Eq. distNAT), at any N
        assert abs(ln - (1.0 - np.sum(p) ** 2)) < 1e-6
        assert 0.0 < M < N


def test_brickwork_N20_total_equals_sum_of_terms():
    psi = I.brickwork_haar(20, 10, seed=2001)  # complex64
    t = on_dev(psi)
    M, ln = hm.sre(t, 2.0)
    allx = torch.arange(2 ** 20, dtype=torch.int64, device=DEV)
    terms = hm.sre_terms(t, 2.0, allx).cpu().numpy()
    S2 = terms[:, 0].sum()
    assert abs(M - (-np.log2(S2 / 2 ** 20))) < 1e-9 * abs(M)
    rng = np.random.default_rng(2001)
    a = rng.integers(0, 2 ** 20, 6)
    np.testing.assert_allclose(terms[a, 0], oracle.sre_terms_list(psi, a), rtol=2e-5)


def test_deterministic_repeat():
    psi = on_dev(I.gaussian_state(20, 77, dtype=np.complex64))
    r1 = hm.sre(psi, 2.0)
    r2 = hm.sre(psi, 2.0)
    assert r1 == r2
    psi = on_dev(I.gaussian_state(13, 77, dtype=np.complex64))
    assert hm.sre(psi, 3.0) == hm.sre(psi, 3.0)


def test_zero_state_large():
    for N in (15, 16, 20):
        M, ln = hm.sre(on_dev(I.zero_state(N, dtype=np.complex64)), 2.0)
        assert abs(M) < 1e-6 and abs(ln) < 1e-6


def test_mc_xstrings_bit_exact():
    for N in (5, 20, 28):
        got = hm.mc_xstrings(2802, 1000, N).cpu().numpy()
        assert np.array_equal(got, oracle.mc_xstrings(2802, 1000, N))


def test_mc_matches_oracle_estimator():
    psi = I.brickwork_haar(12, 4, seed=7)
    M, se = hm.sre_mc(on_dev(psi), 700, 99)
    Mo, seo, _ = oracle.sre_mc(psi, 700, 99)
    assert close_M(M, Mo), (M, Mo)
    assert abs(se - seo) < 1e-4 * seo


def test_invalid_arguments():
    t = on_dev(I.gaussian_state(6, 1, dtype=np.complex64))
    with pytest.raises(hm.HadamagError) as e:
        hm.sre(t, -1.0)
    assert e.value.code == 1
    bad = torch.tensor([0, 64], dtype=torch.int64, device=DEV)
    with pytest.raises(hm.HadamagError) as e:
        hm.sre_terms(t, 2.0, bad)
    assert e.value.code == 1
    # the context stays usable
    assert close_M(hm.sre(t, 2.0)[0], oracle.sre(I.gaussian_state(6, 1, dtype=np.complex64), 2.0)[0])


def test_wait_timeout_is_reported_and_recoverable():
    from paper_2601_07824_gb300._lib import Context
    c = Context(0)
    try:
        c.set_wait_limit(2000, bias=1)  # every wait target unreachable -> bounded wait runs out
        t = on_dev(I.gaussian_state(16, 3, dtype=np.complex64))
        import ctypes
        M = ctypes.c_double()
        rc = c.lib.hadamag_sre(c.h, ctypes.c_void_p(t.data_ptr()), 16, 2.0, 0, ctypes.byref(M), None,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 5
        c.set_wait_limit(1 << 25, bias=0)
        rc = c.lib.hadamag_sre(c.h, ctypes.c_void_p(t.data_ptr()), 16, 2.0, 0, ctypes.byref(M), None,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        assert close_M(M.value, hm.sre(t, 2.0)[0], 1e-12)
    finally:
        c.close()


@pytest.mark.parametrize("N", [16, 18, 20])
def test_autotuned_shape_matches_default_shape(N):
    # the two-pass autotuner picks task shapes per (N, n); every shape computes the same sums
    # (up to the order of the FP64 partials), and a tuned context reports its choice
    from paper_2601_07824_gb300._lib import Context
    psi = torch.from_numpy(I.brickwork_haar(N, 6, seed=880 + N, dtype=np.complex64)).to(DEV)
    tuned, plain = Context(0), Context(0)
    try:
        plain.set_autotune(False)
        out = {}
        for c in (tuned, plain):
            M, ln = ctypes.c_double(), ctypes.c_double()
            c.check(c.lib.hadamag_sre(c.h, ctypes.c_void_p(psi.data_ptr()), N, 2.0, 0, ctypes.byref(M),
                                      ctypes.byref(ln), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                    "hadamag_sre")
            out[id(c)] = M.value
        shape = tuned.twopass_shape(N, 2.0)
        assert shape[0] in (2, 4) and shape[1] in (2, 4) and shape[3] == 8, shape
        # a lag of 1 or 2 stages in 2 to 4 ring slots, or a deeper lag with lag + 1 slots
        assert (shape[2] in (2, 3, 4) and shape[4] in (1, 2)) or (shape[4] > 2 and shape[2] == shape[4] + 1), shape
        assert 1 <= shape[4] < shape[2] <= 63, shape
        assert plain.twopass_shape(N, 2.0) == [0, 0, 0, 0, 0]
        assert abs(out[id(tuned)] - out[id(plain)]) <= 1e-12 * abs(out[id(plain)])
    finally:
        tuned.close()
        plain.close()


def _sre_with(c, psi, N, n):
    M, ln = ctypes.c_double(), ctypes.c_double()
    c.check(c.lib.hadamag_sre(c.h, ctypes.c_void_p(psi.data_ptr()), N, float(n), 0, ctypes.byref(M),
                              ctypes.byref(ln), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
            "hadamag_sre")
    return M.value, ln.value


@pytest.mark.parametrize("n", [2.0, 1.0, 3.0])
def test_N15_one_pass_and_two_pass_splits_vs_oracle(n):
    # N = 15 runs either the one-pass kernel (whole transform in one CTA's shared memory) or two
    # passes through L2 (10 + 4 bits), whichever the tuner picks; both against the oracle
    from paper_2601_07824_gb300._lib import Context
    N = 15
    psi_np = I.gaussian_state(N, 1515, dtype=np.complex64)
    psi = torch.from_numpy(psi_np).to(DEV)
    Mo, lno = oracle.sre(psi_np, n)
    c = Context(0)
    try:
        for upw, tpt, R, lag in ((-1, 0, 0, 1), (2, 1, 0, 1), (2, 2, 0, 2), (4, 1, 0, 2), (4, 2, 0, 1), (4, 2, 0, 3),
                                 (2, 1, 21, 20), (4, 2, 63, 62)):
            c.set_twopass_shape(N, n, upw, tpt, R, lag)
            M, ln = _sre_with(c, psi, N, n)
            assert abs(M - Mo) <= TOL_M * max(1.0, abs(Mo)), (upw, tpt, R, lag, M, Mo)
            assert abs(ln - lno) <= 1e-6
            assert c.twopass_shape(N, n) == ([-1] * 5 if upw == -1 else [upw, tpt, R or 4, 8, lag])
        with pytest.raises(Exception):
            c.set_twopass_shape(N, n, 3, 1)
    finally:
        c.close()
