"""GPU adjoint dM_2/dpsi* against the FP64 oracle gradient, FP64 finite differences of the
oracle's (brute-force-pinned) forward, and the exact phase/scale identities.

Tolerance: ||g_gpu - g_oracle||_2 <= 1e-5 ||g_oracle||_2 (FP32 transforms, FP32 partial
gradients over at most 2^N / (number of partials) X-strings each, FP64 reduction)."""
import ctypes
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


def on_dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 6, 9, 12, 14, 15, 16])
def test_grad_vs_oracle(N):
    psi = I.gaussian_state(N, 600 + N, dtype=np.complex64)
    M2, g = hm.sre_grad(on_dev(psi))
    M2o, go = oracle.sre_grad(psi)
    assert abs(M2 - M2o) <= 1e-6 * max(1.0, abs(M2o))
    assert rel(g.cpu().numpy().astype(np.complex128), go) <= 1e-5


@pytest.mark.parametrize("N", [16, 17])
def test_grad_xbatches_agree(N):
    # the three-pass adjoint with 8, 4 and 2 X-strings per batch (the tuner's candidates): the
    # same M_2 and gradient up to the order of the partial sums; N = 16 also against the oracle
    from paper_2601_07824_gb300._lib import Context
    psi = I.gaussian_state(N, 640 + N, dtype=np.complex64)
    t = on_dev(psi)
    c = Context(0)
    try:
        out = {}
        for A in (8, 4, 2):
            c.set_grad_xbatch(N, A)
            g = torch.empty_like(t)
            M = ctypes.c_double()
            c.check(c.lib.hadamag_sre_grad(c.h, ctypes.c_void_p(t.data_ptr()), N, 0,
                                           ctypes.byref(M), ctypes.c_void_p(g.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                    "hadamag_sre_grad")
            out[A] = (M.value, g.cpu().numpy().astype(np.complex128))
        for A in (4, 2):
            assert abs(out[A][0] - out[8][0]) <= 1e-9 * abs(out[8][0])
            assert rel(out[A][1], out[8][1]) <= 1e-6
        if N == 16:
            M2o, go = oracle.sre_grad(psi)
            assert abs(out[2][0] - M2o) <= 1e-6 * max(1.0, abs(M2o))
            assert rel(out[2][1], go) <= 1e-5
        with pytest.raises(Exception):
            c.set_grad_xbatch(N, 3)
    finally:
        c.close()


def test_grad_unnormalised_complex128_vs_oracle():
    psi = 1.2 * I.gaussian_state(11, 5)
    M2, g = hm.sre_grad(on_dev(psi))
    assert g.dtype == torch.complex128
    M2o, go = oracle.sre_grad(psi)
    assert abs(M2 - M2o) <= 1e-6 * abs(M2o)
    assert rel(g.cpu().numpy(), go) <= 1e-5


@pytest.mark.parametrize("N", [10, 12])
def test_batched_ladder_states_finite_differences(N):
    # RY/RZ + CZ-ladder state (depth 8, random angles); central FD in FP64 with step 1e-4
    rng = np.random.default_rng(4001 + N)
    psi = I.ry_rz_cz_ladder(N, 8, rng, dtype=np.complex128)
    _, g = hm.sre_grad(on_dev(psi))
    g = g.cpu().numpy()
    h = 1e-4
    for _ in range(3):
        d = rng.standard_normal(2 ** N) + 1j * rng.standard_normal(2 ** N)
        d /= np.linalg.norm(d)
        fd = (oracle.sre(psi + h * d, 2.0)[0] - oracle.sre(psi - h * d, 2.0)[0]) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(g, d))) <= 1e-5 * max(1.0, abs(fd))


@pytest.mark.parametrize("N", [17, 18, 20])
def test_grad_identities_large(N):
    # phase invariance: Im <g, psi> = 0; scale: M2(l psi) = M2(psi) - 8 log2 l -> 2 Re <g, psi> = -8/ln 2
    psi = I.gaussian_state(N, 700 + N, dtype=np.complex64)
    t = on_dev(psi)
    M2, g = hm.sre_grad(t)
    M2f, _ = hm.sre(t, 2.0)
    assert abs(M2 - M2f) <= 1e-9 * abs(M2f)
    ip = np.vdot(g.cpu().numpy().astype(np.complex128), psi.astype(np.complex128))
    assert abs(2 * ip.real + 8 / math.log(2)) <= 1e-5 * 8 / math.log(2)
    assert abs(ip.imag) <= 1e-5 * 8 / math.log(2)


def test_autograd_function_matches_adjoint():
    psi = on_dev(I.gaussian_state(8, 3, dtype=np.complex64)).requires_grad_(True)
    out = hm.SREFunction.apply(psi)
    (gt,) = torch.autograd.grad(out, psi)
    _, g = hm.sre_grad(psi.detach())
    assert torch.allclose(gt, 2 * g, rtol=1e-6, atol=0)
    # torch convention: d/dt M2(psi + t d) = Re <grad, d>
    d = torch.randn_like(psi.detach())
    with torch.no_grad():
        fd = (hm.sre(psi.detach() + 1e-3 * d, 2.0)[0] - hm.sre(psi.detach() - 1e-3 * d, 2.0)[0]) / 2e-3
    assert abs(fd - torch.real(torch.vdot(gt, d)).item()) <= 1e-3 * max(1.0, abs(fd))
