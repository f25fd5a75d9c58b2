"""Mixed-state mana (Sec. 3.3.3, Algorithm 6) and the reduced density matrix on the GPU,
against the FP64 oracle (`oracle/mixed.py`, itself pinned to the dense definition
tr(rho A_u) / 3^N), the pure-state oracle (Algorithm 5), closed forms and sum rules.

Tolerances as for pure-state mana (same FP32 radix-3 transform, FP64 sums): generic states
|d mana| <= 1e-6 max(1, |mana|); states whose Wigner function has many exact zeros carry
FP32 residue in them, bounded by 4 * 3^(N/2) * 2^-24 / ln 2 + 1e-7.  The reduced density
matrix (FP32 products summed in FP64 per 32-term chunk) is compared entry by entry within
2e-6 of the largest entry."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402
from paper_2601_07824_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda:0")


def stab_tol(N):
    return 4 * 3 ** (N / 2) * 2.0 ** -24 / math.log(2) + 1e-7


def random_rho(N, seed, rank):
    rng = np.random.default_rng(seed)
    D = 3 ** N
    G = rng.normal(size=(D, rank)) + 1j * rng.normal(size=(D, rank))
    rho = G @ G.conj().T
    return (rho / np.trace(rho).real).astype(np.complex64)


def on_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_random_density_matrices_vs_algorithm_6(N):
    for rank in sorted({1, 2, 3 ** N}):
        rho = random_rho(N, 700 + 10 * N + rank, rank)
        m, sums = hm.mana_mixed(on_dev(rho))
        mo, swo = mixed.mana_mixed(rho)
        assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo)), (N, rank, m, mo)
        assert abs(sums[0] / 3 ** N - swo) <= 1e-6 * swo
        r = rho.astype(np.complex128)
        assert abs(sums[1] / 3 ** N - np.trace(r).real) < 1e-5  # sum_u W_u = tr rho
        assert abs(sums[2] / 3 ** N - np.sum(np.abs(r) ** 2)) < 1e-5  # 3^N sum W^2 = tr rho^2


@pytest.mark.parametrize("N", [6, 7, 8, 9])
def test_pure_density_matrices_equal_algorithm_5(N):
    # rho = |psi><psi| built on the device: the mixed-state kernels (one-pass up to 8 qutrits,
    # two-pass at 9) must give the pure-state oracle's mana
    psi_np = I.gaussian_state(N, 800 + N, d=3, dtype=np.complex64)
    psi = on_dev(psi_np)
    rho = torch.outer(psi, psi.conj()).contiguous()
    m, sums = hm.mana_mixed(rho)
    del rho
    mo, swo = oracle.mana(psi_np)
    assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo)), (N, m, mo)
    assert abs(sums[0] / 3 ** N - swo) <= 1e-6 * swo


def test_ten_qutrits_closed_forms():
    # the two-pass variant at its largest size (rho: 3^20 values, 28 GB): the Strange product
    # (sum |W| = (5/3)^N) and the maximally mixed state (W = 9^-N everywhere, mana 0)
    N = 10
    s = on_dev(I.strange_product(N, dtype=np.complex64))
    rho = torch.outer(s, s.conj()).contiguous()
    m, sums = hm.mana_mixed(rho)
    assert abs(m - N * math.log2(5 / 3)) <= 1e-6 * N * math.log2(5 / 3)
    rho.zero_()
    rho.diagonal().fill_(1.0 / 3 ** N)
    m, sums = hm.mana_mixed(rho)
    del rho
    assert abs(m) <= stab_tol(N)
    assert abs(sums[1] / 3 ** N - 1.0) < 1e-5 and abs(sums[2] - 1.0) < 1e-5  # tr rho^2 = 3^-N


@pytest.mark.parametrize("N", [1, 3, 6, 8])
def test_maximally_mixed_and_stabilizer_mixtures(N):
    D = 3 ** N
    m, sums = hm.mana_mixed(on_dev(np.eye(D, dtype=np.complex64) / D))
    assert abs(m) <= stab_tol(N)
    # the qutrit GHZ marginal: a uniform mixture of |0..0>, |1..1>, |2..2>, mana 0
    if N >= 2:
        rg = mixed.reduced_density_matrix(I.qutrit_ghz(N + 1), list(range(N))).astype(np.complex64)
        m, _ = hm.mana_mixed(on_dev(rg))
        assert abs(m) <= stab_tol(N)


@pytest.mark.parametrize("N,keep", [(4, [0, 2]), (5, [4, 1, 3]), (3, [2]), (4, [3, 2, 1, 0]), (9, [8, 0, 4, 2]),
                                    (11, [1, 3, 5, 7, 9]), (12, [11, 10, 0, 1, 2, 5])])
def test_reduced_density_matrix_vs_oracle(N, keep):
    psi = I.gaussian_state(N, 900 + N, d=3, dtype=np.complex64)
    rho = hm.reduced_density_matrix(on_dev(psi), keep).cpu().numpy()
    ro = mixed.reduced_density_matrix(psi, keep)
    assert rho.shape == ro.shape
    np.testing.assert_allclose(rho, ro, rtol=0, atol=2e-6 * np.abs(ro).max())


def test_partial_trace_then_mana_and_complex128():
    psi = I.gaussian_state(8, 950, d=3)
    keep = [6, 1, 3, 4]
    rho = hm.reduced_density_matrix(on_dev(psi), keep)  # complex128 state in, complex64 rho out
    m, _ = hm.mana_mixed(rho)
    mo, _ = mixed.mana_mixed(mixed.reduced_density_matrix(psi, keep))
    assert abs(m - mo) <= 1e-5 * max(1.0, abs(mo))  # rho rounded to complex64 on output
    # a complex128 density matrix is rounded to complex64 on the device: same result
    r64 = rho.cpu().numpy()
    m64, _ = hm.mana_mixed(on_dev(r64))
    m128, _ = hm.mana_mixed(on_dev(r64.astype(np.complex128)))
    assert m64 == m128 == m


def test_invalid_arguments():
    lib = _lib.load()
    c = hm.context(0)
    rho = on_dev(np.eye(9, dtype=np.complex64) / 9)
    m = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    for N in (0, 11):
        assert lib.hadamag_mana_mixed(c.h, ctypes.c_void_p(rho.data_ptr()), N, 0, ctypes.byref(m), None, stream) == 1
    assert lib.hadamag_mana_mixed(c.h, ctypes.c_void_p(rho.data_ptr() + 8), 2, 0, ctypes.byref(m), None, stream) == 1
    with pytest.raises(ValueError):
        hm.mana_mixed(on_dev(np.eye(8, dtype=np.complex64)))
    psi = on_dev(I.gaussian_state(4, 1, d=3, dtype=np.complex64))
    for keep in ([0, 0], [4], [], [0, 1, 2, 3, 0]):
        with pytest.raises(hm.HadamagError) as e:
            hm.reduced_density_matrix(psi, keep)
        assert e.value.code == 1
    # the context stays usable
    assert abs(hm.mana_mixed(rho)[0]) <= stab_tol(2)
