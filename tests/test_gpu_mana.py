"""GPU parity of the qutrit mana (Algorithm 5) against the FP64 oracle, closed forms and the
Wigner sum rules.

Tolerances.  Generic states: |d mana| <= 1e-6 * max(1, |mana|).  Stabilizer states have
mana = 0 exactly, and sum_u |W| then counts FP32 cancellation residue in the 9^N - 3^N
entries that are exactly zero: each is ~ 3^(-N/2) eps, so the bias of sum |W| grows like
3^(N/2) eps (eps = 2^-24); the test bound for them is 4 * 3^(N/2) * 2^-24 / ln 2 + 1e-7."""
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


def stab_tol(N):
    return 4 * 3 ** (N / 2) * 2.0 ** -24 / math.log(2) + 1e-7


@pytest.mark.parametrize("N", list(range(1, 10)))
def test_gaussian_vs_oracle(N):
    psi = I.gaussian_state(N, 300 + N, d=3, dtype=np.complex64)
    m, sw = hm.mana(on_dev(psi))
    mo, swo = oracle.mana(psi)
    assert abs(m - mo) <= 1e-6 * max(1.0, abs(mo)), (N, m, mo)
    assert abs(sw - swo) <= 1e-6 * swo


def test_N11_gaussian_and_strange_closed_form(golden):
    psi = I.gaussian_state(11, 1101, d=3, dtype=np.complex64)
    m, sw = hm.mana(on_dev(psi))
    # additivity-free check at full size: sum|W| >= sum W = 1 and the Haar-typical magnitude
    assert 1.0 < sw and 0.0 < m < 11 * math.log2(3)
    per = golden["closed_forms"]["mana_strange_per_qutrit"]["sum_abs_w_per_qutrit"]
    m, sw = hm.mana(on_dev(I.strange_product(11, dtype=np.complex64)))
    assert abs(m - 11 * math.log2(per)) <= 1e-6 * 11 * math.log2(per)
    # natural-log convention: ln sum|W| = N ln(5/3)
    assert abs(math.log(sw) - 11 * math.log(5 / 3)) <= 1e-6 * 11 * math.log(5 / 3)


@pytest.mark.parametrize("N", [2, 5, 9, 12])
def test_wigner_sum_rules(N):
    psi = I.gaussian_state(N, 40 + N, d=3, dtype=np.complex64)
    s_abs, s_sum, s_sq = hm.mana_sums(on_dev(psi))
    norm2 = float(np.sum(np.abs(psi.astype(np.complex128)) ** 2))
    # sum_u W(u) = tr(rho) and sum_u W(u)^2 = tr(rho^2) / 3^N (Sec. 2)
    assert abs(s_sum / 3 ** N - norm2) < 1e-5
    assert abs(s_sq / 9 ** N - norm2 ** 2 / 3 ** N) < 1e-5 / 3 ** N
    assert s_abs / 3 ** N >= s_sum / 3 ** N - 1e-6


@pytest.mark.parametrize("N", [1, 4, 8, 10, 11, 13])
def test_stabilizer_states_zero(N):
    states = [I.qutrit_graph_state(N, [(j, j + 1) for j in range(N - 1)], dtype=np.complex64)]
    if N <= 11:  # at the largest size (about a minute per state) the graph state alone
        states += [I.zero_state(N, d=3, dtype=np.complex64), I.qutrit_ghz(N, dtype=np.complex64)]
    for psi in states:
        m, sw = hm.mana(on_dev(psi))
        assert abs(m) <= stab_tol(N), (N, m)


def test_complex128_input_and_repeatability():
    psi = I.gaussian_state(9, 5, d=3)
    t = on_dev(psi)
    r1 = hm.mana(t)
    assert r1 == hm.mana(t)
    mo, _ = oracle.mana(psi)
    assert abs(r1[0] - mo) <= 1e-6 * max(1.0, abs(mo))


def test_mana_invalid_arguments():
    t = on_dev(I.gaussian_state(3, 1, d=3, dtype=np.complex64))
    with pytest.raises(ValueError):
        hm.mana(t[:26].contiguous())
    big = torch.zeros(3 ** 14, dtype=torch.complex64, device=DEV)
    with pytest.raises(hm.HadamagError) as e:
        hm.mana(big)
    assert e.value.code == 1
