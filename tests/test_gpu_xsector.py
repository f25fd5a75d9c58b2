"""Exact M_n over the even-weight X-sectors (Sec. 3.2 symmetry remark) on the GPU.

For U(1) or prod_j Z_j symmetric states every odd-weight X-sector has S(a) = 0, so the
2^(N-1) even-weight X-strings carry all of Eq. (sre).  Checked against the FP64 oracle's
full M_n (the oracle pins that the two coincide on such states) and, on a generic state,
against the oracle's even-sector sum itself.  Tolerance: the exact-SRE bound
1e-6 max(1, |M|); tensor path as in the tensor-path tests."""
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


def on_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("label,psi", [
    ("u1_N8", I.u1_state(8, 4, 3701, dtype=np.complex64)),
    ("z2_N11", I.parity_state(11, 3702, parity=1, dtype=np.complex64)),
    ("u1_N13", I.u1_state(13, 6, 3703, dtype=np.complex64)),
    ("u1_N13_k3", I.u1_state(13, 3, 3705, dtype=np.complex64)),  # off half filling: odd sectors still vanish
    ("z2_N16", I.parity_state(16, 3704, dtype=np.complex64)),
])
def test_even_sector_equals_full_sre_on_symmetric_states(label, psi):
    # n = 0.5 ... 3 up to 13 qubits (FP64 powers for the non-integer ones); n = 2 at 16, where
    # each FP64 oracle call costs seconds
    for n in ((0.5, 1.0, 2.0, 2.5, 3.0) if psi.size <= 2 ** 13 else (2.0,)):
        M, lost = hm.sre_even_sector(on_dev(psi), n)
        Mo, losto = oracle.sre(psi, n)
        assert abs(M - Mo) <= 1e-6 * max(1.0, abs(Mo)), (label, n, M, Mo)
        assert abs(lost - losto) <= 2e-6


def test_generic_state_gives_the_even_sector_part():
    psi = I.gaussian_state(10, 3706, dtype=np.complex64)
    M, _ = hm.sre_even_sector(on_dev(psi), 2.0)
    Me, _ = oracle.sre_even_sector(psi, 2.0)
    assert abs(M - Me) <= 1e-6 * max(1.0, abs(Me))
    assert abs(M - oracle.sre(psi, 2.0)[0]) > 0.1


def test_large_symmetric_states_match_the_full_transform():
    # at N = 20 the full oracle is out of reach: the half-work sum must equal the library's full
    # sum (itself parity-tested), the odd sectors contributing nothing
    psi = on_dev(I.parity_state(20, 3707, dtype=np.complex64))
    M, lost = hm.sre_even_sector(psi, 2.0)
    Mf, lostf = hm.sre(psi, 2.0)
    assert abs(M - Mf) <= 1e-6 * max(1.0, abs(Mf))
    assert abs(lost - lostf) <= 2e-6
    # tensor-core path at N = 21 (U(1), half filling up to one)
    psi21 = on_dev(I.u1_state(21, 10, 3708, dtype=np.complex64))
    Mt, _ = hm.sre_even_sector(psi21, 2.0, path=hm.PATH_TENSOR)
    Mc, _ = hm.sre(psi21, 2.0)
    assert abs(Mt - Mc) <= 1e-6 * max(1.0, abs(Mc))


def test_invalid_arguments():
    psi = on_dev(I.parity_state(4, 1, dtype=np.complex64))
    with pytest.raises(hm.HadamagError) as e:
        hm.sre_even_sector(psi, -1.0)
    assert e.value.code == 1


@pytest.mark.parametrize("N", [1, 2, 3])
def test_smallest_sizes(N):
    # N = 1: the even sector is {a = 0} alone; N = 2: {0, 3}
    for psi in (I.parity_state(N, 3710 + N, dtype=np.complex64),
                I.parity_state(N, 3720 + N, parity=1, dtype=np.complex64)):
        for n in (1.0, 2.0):
            M, lost = hm.sre_even_sector(on_dev(psi), n)
            Mo, losto = oracle.sre(psi, n)
            assert abs(M - Mo) <= 1e-6 * max(1.0, abs(Mo)), (N, n, M, Mo)
            assert abs(lost - losto) <= 2e-6
