"""GPU parity of the tensor-core SRE path: the Walsh-Hadamard transform as +-1 Kronecker blocks
on tcgen05 tensor cores (fp16 hi/lo operands, fp32 accumulation in tensor memory), 21 <= N <= 24.

Tolerances.  Per-X-string sums: 2e-5 relative of the FP64 oracle, the bound used for the FP32
CUDA-core path (each operand keeps ~22 significant bits after the hi/lo split, whose lo part
carries its own 2^11 scale, and the accumulation is fp32).  M_n: |dM| <= 1e-6 * max(1, |M|) against closed forms and against the CUDA-core path,
which is itself pinned to the oracle."""
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
from paper_2601_07824_gb300 import PATH_CUDACORE, PATH_TENSOR  # noqa: E402

DEV = torch.device("cuda:0")
TOL_M = 1e-6


def close_M(a, b, tol=TOL_M):
    return abs(a - b) <= tol * max(1.0, abs(b))


def on_dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV)


def sample_a(N, seed, extra=6):
    """X-strings covering every producer branch: a = 0, 0 < a < 2^13 (pairs inside a pass-1
    tile), and a >= 2^13 with each of the eight values of a & 7, plus random ones."""
    dim = 2 ** N
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 5, 4095, 8191, dim - 1, dim // 2 + 3]
    fixed += [(8192 * (3 + k)) | k for k in range(8)]  # a >= 2^13, a & 7 = k
    return np.unique(np.concatenate([fixed, rng.integers(0, dim, extra)])).astype(np.int64)


@pytest.mark.parametrize("N", [21, 22, 23, 24])
def test_tc_sampled_terms_vs_oracle(N):
    psi = I.gaussian_state(N, 3100 + N, dtype=np.complex64)
    t = on_dev(psi)
    a = sample_a(N, N)
    at = torch.from_numpy(a).to(DEV)
    got = hm.sre_terms(t, 2.0, at, path=PATH_TENSOR).cpu().numpy()
    want = oracle.sre_terms_list(psi, a)
    np.testing.assert_allclose(got[:, 0], want, rtol=2e-5)
    # sum_b |chi_b(a)|^2 = 2^N sum_z |psi_z|^2 |psi_{z^a}|^2 (Parseval)
    p = np.abs(psi.astype(np.complex128)) ** 2
    z = np.arange(2 ** N)
    s1 = np.array([2 ** N * np.sum(p * p[z ^ ai]) for ai in a])
    np.testing.assert_allclose(got[:, 1], s1, rtol=2e-5)


@pytest.mark.parametrize("n", [1.0, 3.0, 2.5])
def test_tc_sampled_terms_other_indices(n):
    N = 21
    psi = I.brickwork_haar(N, 8, seed=2101)
    a = sample_a(N, 7, extra=2)
    got = hm.sre_terms(on_dev(psi), n, torch.from_numpy(a).to(DEV), path=PATH_TENSOR).cpu().numpy()
    for k, ai in enumerate(a):
        Sq, S1, T1 = oracle.sre_terms(psi, n, int(ai), int(ai) + 1)
        np.testing.assert_allclose(got[k, 0], Sq[0], rtol=2e-5)
        np.testing.assert_allclose(got[k, 1], S1[0], rtol=2e-5)
        if n == 1.0:
            np.testing.assert_allclose(got[k, 2], T1[0], rtol=2e-5, atol=1e-7 * abs(T1[0]) + 1e-12)


def test_tc_closed_forms_N21(golden):
    N = 21
    g = golden["closed_forms"]["sre_t_state_per_qubit"]
    t = on_dev(I.t_state_product(N, dtype=np.complex64))
    # full-size runs at n = 2; n = 1, 3 and 2.5 are covered per X-string against the oracle
    for n, key in ((2.0, "M2"),):
        M, ln = hm.sre(t, n, path=PATH_TENSOR)
        assert close_M(M, N * g[key] / g["N"]), (n, M)  # additive: per-qubit value x N
        assert abs(ln) < 1e-6
    for psi in (I.ghz_state(N, dtype=np.complex64), I.zero_state(N, dtype=np.complex64)):
        M, ln = hm.sre(on_dev(psi), 2.0, path=PATH_TENSOR)
        assert abs(M) < 1e-6 and abs(ln) < 1e-6


def random_product_state(N, seed):
    """A random product state and the oracle's single-qubit M_2 of each factor."""
    rng = np.random.default_rng(seed)
    sites = []
    for _ in range(N):
        v = rng.normal(size=2) + 1j * rng.normal(size=2)
        sites.append(v / np.linalg.norm(v))
    psi = sites[0]
    for v in sites[1:]:
        psi = np.kron(v, psi)  # qubit j = bit j
    return psi.astype(np.complex64), sum(oracle.sre(v, 2.0)[0] for v in sites)


def test_tc_product_state_additivity_N21():
    # M_n is additive over tensor factors: a random product state's M_2 is the sum of its
    # single-qubit values, each given by the oracle at N = 1.  The amplitudes of a random product
    # state spread over many decades, which tests the hi/lo split far below the largest value.
    N = 21
    psi, want = random_product_state(N, 2202)
    t = on_dev(psi)
    M, ln = hm.sre(t, 2.0, path=PATH_TENSOR)
    assert close_M(M, want), (M, want)
    assert abs(ln) < 1e-6
    Mc, _ = hm.sre(t, 2.0, path=PATH_CUDACORE)
    assert close_M(Mc, want), (Mc, want)


@pytest.mark.parametrize("path", [PATH_TENSOR, PATH_CUDACORE], ids=["tensor", "cudacore"])
@pytest.mark.parametrize("state", ["t_product", "ghz", "random_product"])
def test_full_size_closed_forms_N22(golden, path, state):
    # exact M_2 of whole N = 22 states on both paths against values fixed independently of the
    # GPU: |T>^22 gives 22 log2(4/3) (additivity of the per-qubit closed form), GHZ gives 0
    # (a stabilizer state), a random product state the sum of the oracle's N = 1 values
    N = 22
    if state == "t_product":
        psi = I.t_state_product(N, dtype=np.complex64)
        g = golden["closed_forms"]["sre_t_state_per_qubit"]
        want = N * g["M2"] / g["N"]
        assert abs(want - N * math.log2(4.0 / 3.0)) < 1e-12
    elif state == "ghz":
        psi, want = I.ghz_state(N, dtype=np.complex64), 0.0
    else:
        psi, want = random_product_state(N, 2203)
    M, ln = hm.sre(on_dev(psi), 2.0, path=path)
    assert close_M(M, want), (state, M, want)
    assert abs(ln) < 2e-6


def test_tc_matches_cudacore_N21():
    N = 21
    for psi in (I.brickwork_haar(N, 10, seed=2122),):
        t = on_dev(psi)
        Mt, lt = hm.sre(t, 2.0, path=PATH_TENSOR)
        Mc, lc = hm.sre(t, 2.0, path=PATH_CUDACORE)
        assert close_M(Mt, Mc), (Mt, Mc)
        # lost_norm = 1 - S_1 / 2^N: S_1 carries the hi/lo split error (~1e-6 relative)
        assert abs(lt - lc) < 2e-6


def test_tc_deterministic_and_path_restored():
    t = on_dev(I.gaussian_state(21, 5, dtype=np.complex64))
    a = torch.from_numpy(sample_a(21, 5)).to(DEV)
    r1 = hm.sre_terms(t, 2.0, a, path=PATH_TENSOR)
    r2 = hm.sre_terms(t, 2.0, a, path=PATH_TENSOR)
    assert torch.equal(r1, r2)  # static task order, fixed reduction order
    # outside the supported sizes the tensor setting uses the CUDA-core kernels
    s = on_dev(I.gaussian_state(12, 6, dtype=np.complex64))
    assert close_M(hm.sre(s, 2.0, path=PATH_TENSOR)[0], oracle.sre(I.gaussian_state(12, 6, dtype=np.complex64), 2.0)[0])


def test_tc_mc_estimator_N22():
    psi = I.gaussian_state(22, 2222, dtype=np.complex64)
    t = on_dev(psi)
    Mt, st = hm.sre_mc(t, 64, 11, path=PATH_TENSOR)
    Mc, sc = hm.sre_mc(t, 64, 11, path=PATH_CUDACORE)
    assert close_M(Mt, Mc), (Mt, Mc)
    assert abs(st - sc) <= 1e-4 * sc


def test_tc_timeout_is_reported_and_recoverable():
    import ctypes
    from paper_2601_07824_gb300._lib import Context
    c = Context(0)
    try:
        c.set_path(PATH_TENSOR)
        t = on_dev(I.gaussian_state(21, 3, dtype=np.complex64))
        a = torch.arange(4, dtype=torch.int64, device=DEV)
        out = torch.empty((4, 3), dtype=torch.float64, device=DEV)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        c.set_wait_limit(2000, bias=1)  # every inter-CTA wait target unreachable
        rc = c.lib.hadamag_sre_terms(c.h, ctypes.c_void_p(t.data_ptr()), 21, 2.0, 0, ctypes.c_void_p(a.data_ptr()),
                                     4, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 5
        c.set_wait_limit(1 << 25, bias=0)
        rc = c.lib.hadamag_sre_terms(c.h, ctypes.c_void_p(t.data_ptr()), 21, 2.0, 0, ctypes.c_void_p(a.data_ptr()),
                                     4, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        np.testing.assert_allclose(out[:, 0].cpu().numpy(),
                                   oracle.sre_terms_list(I.gaussian_state(21, 3, dtype=np.complex64), np.arange(4)),
                                   rtol=2e-5)
    finally:
        c.close()
