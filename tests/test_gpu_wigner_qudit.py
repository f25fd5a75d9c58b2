"""Mana of odd-prime qudits (Sec. 2's construction for any odd prime d; Algorithm 5
generalised) on the GPU against the FP64 oracle (`oracle/qudit.py`, pinned to the dense
definition), the Wigner sum rules and zeros on stabilizer states.

Tolerances as for qutrit mana: generic states 1e-6 max(1, |mana|); stabilizer states carry
FP32 residue in their exact zeros, bounded by 4 * d^(N/2) * 2^-24 / ln 2 + 1e-7."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from oracle import qudit as Q
from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402
from paper_2601_07824_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda:0")
# oracle comparisons up to one size below each d's largest (the NumPy oracle needs over a
# minute at 5^6, 7^5, 11^4); the largest sizes are checked by the sum rules below
CASES = [(5, n) for n in range(1, 6)] + [(7, n) for n in range(1, 5)] + [(11, n) for n in range(1, 4)] + \
        [(13, n) for n in range(1, 4)]
LARGEST = [(5, 6), (7, 5), (11, 4), (13, 3)]


def on_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def stab_tol(d, N):
    return 4 * d ** (N / 2) * 2.0 ** -24 / math.log(2) + 1e-7


@pytest.mark.parametrize("d,N", CASES)
def test_gaussian_states_vs_oracle(d, N):
    psi = I.gaussian_state(N, 1000 * d + N, d=d, dtype=np.complex64)
    m, sums = hm.mana_qudit(on_dev(psi), d)
    mo, so, s1, s2 = Q.mana_fast(psi, d)
    assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo)), (d, N, m, mo)
    assert abs(sums[0] / d ** N - so) <= 1e-6 * so
    assert abs(sums[1] / d ** N - 1.0) < 1e-5  # sum_u W(u) = 1
    assert abs(sums[2] / d ** N - 1.0) < 1e-5  # sum_u W(u)^2 = d^-N


@pytest.mark.parametrize("d,N", LARGEST)
def test_largest_sizes_sum_rules(d, N):
    # sum_u W = 1 and d^N sum_u W^2 = 1 for a normalised pure state: both are sensitive to every
    # value of the transform; by Cauchy-Schwarz sum |W| <= (d^{2N} sum W^2)^(1/2) = d^(N/2)
    psi = I.gaussian_state(N, 1000 * d + N, d=d, dtype=np.complex64)
    m, sums = hm.mana_qudit(on_dev(psi), d)
    norm2 = float(np.sum(np.abs(psi.astype(np.complex128)) ** 2))
    assert abs(sums[1] / d ** N - norm2) < 1e-5
    assert abs(sums[2] / d ** N - norm2 ** 2) < 1e-5
    assert 0.0 < m <= 0.5 * N * np.log2(d) + 1e-6
    # the mixed-state route on |psi><psi| agrees with the pure-state kernel
    p = on_dev(psi)
    mm, _ = hm.mana_mixed(torch.outer(p, p.conj()).contiguous(), d)
    assert abs(mm - m) <= 1e-6 * max(1.0, abs(m))


def test_qutrits_take_the_qutrit_kernels():
    psi = I.gaussian_state(7, 1700, d=3, dtype=np.complex64)
    m, _ = hm.mana_qudit(on_dev(psi), 3)
    assert m == hm.mana(on_dev(psi))[0]
    assert abs(m - oracle.mana(psi)[0]) <= 1e-6 * max(1.0, abs(m))


@pytest.mark.parametrize("d,N", [(5, 4), (7, 3), (11, 2), (13, 2)])
def test_stabilizer_states_have_zero_mana(d, N):
    states = [Q.zero_state(N, d), Q.ghz(N, d), Q.graph_state(N, d, [(j, j + 1) for j in range(N - 1)]),
              Q.random_clifford_circuit(Q.zero_state(N, d), N, d, 30, seed=d * 10 + N)]
    for psi in states:
        m, _ = hm.mana_qudit(on_dev(psi.astype(np.complex64)), d)
        assert abs(m) <= stab_tol(d, N), (d, N, m)


def test_complex128_input():
    psi = I.gaussian_state(4, 1800, d=5)
    m128, _ = hm.mana_qudit(on_dev(psi), 5)
    m64, _ = hm.mana_qudit(on_dev(psi.astype(np.complex64)), 5)
    assert m128 == m64  # complex128 is rounded to complex64 on the device first
    assert abs(m128 - Q.mana_fast(psi, 5)[0]) <= 1e-6 * max(1.0, abs(m128))


def test_invalid_arguments():
    lib = _lib.load()
    c = hm.context(0)
    m = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    buf = torch.zeros(5 ** 7, dtype=torch.complex64, device=DEV)
    buf[0] = 1.0
    ptr = ctypes.c_void_p(buf.data_ptr())
    assert lib.hadamag_mana_qudit(c.h, ptr, 2, 9, 0, ctypes.byref(m), None, stream) == 2   # d not an odd prime
    assert lib.hadamag_mana_qudit(c.h, ptr, 2, 4, 0, ctypes.byref(m), None, stream) == 2
    assert lib.hadamag_mana_qudit(c.h, ptr, 7, 5, 0, ctypes.byref(m), None, stream) == 1   # 5^7 > 25600
    assert lib.hadamag_mana_qudit(c.h, ptr, 0, 5, 0, ctypes.byref(m), None, stream) == 1
    with pytest.raises(ValueError):
        hm.mana_qudit(buf[:24].contiguous(), 5)
    # the context stays usable: |0...0> of 6 qudits has mana 0
    assert abs(hm.mana_qudit(buf[:5 ** 6].contiguous(), 5)[0]) <= stab_tol(5, 6)


# ---- gradient of the mana ---------------------------------------------------------------
# Mana is not differentiable where some chi_b(a) = 0: an entry within the FP32 error of zero
# can take the other sign on the GPU, moving d m / d psi* by up to 2 |psi| (so d mana / d psi*
# by 2 |psi| / (m ln 2)).  The tolerance is 1e-5 |g| plus that bound times the number K of
# oracle entries below delta = 4 N d 2^-24 |psi|^2 (the FP32 error bound of a transformed
# value).  The phase and scale identities hold for any sign pattern and stay strict.

GRAD_CASES = [(3, 1), (3, 2), (3, 4), (3, 6), (3, 7), (5, 3), (7, 2), (7, 3), (11, 2), (13, 2)]


@pytest.mark.parametrize("d,N", GRAD_CASES)
def test_mana_gradient_vs_oracle(d, N):
    psi = (I.gaussian_state(N, 3000 * d + N, d=d) * 1.2).astype(np.complex64)
    m, g = hm.mana_grad(on_dev(psi), d)
    g = g.cpu().numpy().astype(np.complex128)
    p = psi.astype(np.complex128)
    delta = 4 * N * d * 2.0 ** -24 * float(np.vdot(p, p).real)
    mo, go, K = Q.mana_grad(p, d, small=delta)
    assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo))
    msum = d ** N * 2.0 ** mo
    tol = 1e-5 * np.linalg.norm(go) + 2 * np.linalg.norm(p) * K / (msum * math.log(2.0))
    assert np.linalg.norm(g - go) <= tol, (d, N, K, np.linalg.norm(g - go) / np.linalg.norm(go))


@pytest.mark.parametrize("d,N,dtype", [(3, 9, np.complex64), (5, 4, np.complex128), (13, 3, np.complex64)])
def test_mana_gradient_identities(d, N, dtype):
    psi = (I.gaussian_state(N, 3100 * d + N, d=d) * 0.8).astype(dtype)
    m, g = hm.mana_grad(on_dev(psi), d)
    assert g.dtype == on_dev(psi).dtype
    g = g.cpu().numpy().astype(np.complex128)
    p = psi.astype(np.complex128)
    # phase invariance and mana(c psi) = mana(psi) + 2 log2 c
    assert abs(np.imag(np.vdot(g, p))) <= 1e-5 * np.linalg.norm(g) * np.linalg.norm(p)
    assert 2 * np.real(np.vdot(g, p)) == pytest.approx(2 / math.log(2.0), rel=1e-5)
    assert abs(m - hm.mana_qudit(on_dev(psi), d)[0]) <= 1e-6 * max(1.0, abs(m))


def test_mana_gradient_invalid_arguments():
    buf = torch.zeros(3 ** 10, dtype=torch.complex64, device=DEV)
    with pytest.raises(hm.HadamagError) as e:
        hm.mana_grad(buf, 3)  # 3^10 > 25600
    assert e.value.code == 1
    with pytest.raises(ValueError):
        hm.mana_grad(buf[:10].contiguous(), 3)


# ---- mixed states of qudits -----------------------------------------------------------

@pytest.mark.parametrize("d,N", [(5, 1), (5, 2), (5, 3), (7, 2), (11, 2), (13, 2)])
def test_mixed_qudit_states_vs_oracle(d, N):
    D = d ** N
    rng = np.random.default_rng(4000 + d + N)
    for rank in sorted({1, 3, D}):
        G = rng.normal(size=(D, rank)) + 1j * rng.normal(size=(D, rank))
        rho = G @ G.conj().T
        rho = (rho / np.trace(rho).real).astype(np.complex64)
        m, sums = hm.mana_mixed(on_dev(rho), d)
        mo, so, s1, s2 = Q.mana_mixed_fast(rho.astype(np.complex128), d)
        assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo)), (d, N, rank, m, mo)
        assert abs(sums[1] / D - s1) < 1e-5 and abs(sums[2] / D - s2 * D) < 1e-5  # tr rho, tr rho^2


@pytest.mark.parametrize("d,N", [(5, 4), (7, 3)])
def test_mixed_qudit_pure_and_maximally_mixed(d, N):
    psi = I.gaussian_state(N, 4100 + d, d=d, dtype=np.complex64)
    p = on_dev(psi)
    m, _ = hm.mana_mixed(torch.outer(p, p.conj()).contiguous(), d)
    assert abs(m - hm.mana_qudit(p, d)[0]) <= 1e-6 * max(1.0, abs(m))
    D = d ** N
    mm, _ = hm.mana_mixed(on_dev(np.eye(D, dtype=np.complex64) / D), d)
    assert abs(mm) <= stab_tol(d, N)


@pytest.mark.parametrize("d,N,keep", [(5, 3, [2, 0]), (7, 3, [1]), (5, 5, [4, 0, 2]), (2, 10, [9, 0, 3, 5])])
def test_qudit_partial_trace_vs_oracle(d, N, keep):
    from oracle import mixed
    psi = I.gaussian_state(N, 4200 + d + N, d=d, dtype=np.complex64)
    rho = hm.reduced_density_matrix(on_dev(psi), keep, d).cpu().numpy()
    ro = mixed.reduced_density_matrix(psi, keep, d=d)
    np.testing.assert_allclose(rho, ro, rtol=0, atol=2e-6 * np.abs(ro).max())


def test_qudit_partial_trace_then_mana():
    from oracle import mixed
    d, N, keep = 5, 4, [3, 1]
    psi = I.gaussian_state(N, 4300, d=d)
    m, _ = hm.mana_mixed(hm.reduced_density_matrix(on_dev(psi), keep, d), d)
    mo = Q.mana_mixed_fast(mixed.reduced_density_matrix(psi, keep, d=d), d)[0]
    assert abs(m - mo) <= 1e-5 * max(1.0, abs(mo))  # rho rounded to complex64 on output
