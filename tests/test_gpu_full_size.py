"""Full-size GPU results against FP64 oracle values stored in tests/golden/ (computed by the
committed scripts there, which call only the oracle; a full run at these sizes takes the
oracle minutes to hours, too long for a test):

  * exact mana of the N = 11 qutrit Gaussian state (Eq. mana2, Algorithm 5) and exact M_2 of
    the N = 20 brick-wall Haar state (Eq. sre, Algorithm 2) -- the bench workloads -- within
    the exact-path tolerance 1e-6 max(1, |M|);
  * the adjoint dM_2/dpsi* at N = 17 and 18 (single-state call and the batched launch): the
    projections 2 Re <g, d_k> on 16 seeded random directions against the oracle gradient's, and
    against finite differences of the oracle's forward.  For an error vector e the projection
    errors are ~ |e| sqrt(2 / 2^N) each, so their RMS estimates |e|; the test holds that
    estimate to 2e-5 |g| (the element-wise bound of the smaller-N gradient tests is 1e-5)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402

DEV = torch.device("cuda:0")
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def direction(k, dim):
    # the directions of tests/golden/make_grad_fd_values.py
    rng = np.random.default_rng(91000 + k)
    d = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    return d / np.linalg.norm(d)


def test_mana_N11_gaussian_vs_stored_oracle():
    ref = load("oracle_full_size.json")["mana_gaussian_N11_seed1101"]
    q = torch.from_numpy(I.gaussian_state(11, 1101, d=3, dtype=np.complex64)).to(DEV)
    m, sw = hm.mana(q)
    assert abs(m - ref["mana"]) <= 1e-6 * max(1.0, abs(ref["mana"])), (m, ref["mana"])
    assert abs(sw - ref["sum_abs_w"]) <= 1e-6 * ref["sum_abs_w"]


def test_sre_N20_brickwork_vs_stored_oracle():
    ref = load("oracle_full_size.json")["sre_brickwork_N20_depth10_seed2001"]
    psi = torch.from_numpy(I.brickwork_haar(20, 10, seed=2001, dtype=np.complex64)).to(DEV)
    M, ln = hm.sre(psi, 2.0)
    assert abs(M - ref["M2"]) <= 1e-6 * max(1.0, abs(ref["M2"])), (M, ref["M2"])
    assert abs(ln - ref["lost_norm"]) <= 1e-6


def _check_projections(name, ref, g):
    g = g.astype(np.complex128)
    dim = g.size
    p = np.array([2 * np.real(np.vdot(g, direction(k, dim))) for k in range(len(ref["proj"]))])
    po = np.array(ref["proj"])
    err_norm = math.sqrt(float(np.mean((p - po) ** 2)) * dim / 2.0)  # RMS projection error -> |e|
    assert err_norm <= 2e-5 * ref["grad_norm"], (name, err_norm / ref["grad_norm"])
    for k, fd in enumerate(ref["fd"]):
        # finite differences of the oracle's forward pin the same directional derivatives
        assert abs(fd - p[k]) <= 2e-5 * ref["grad_norm"] * math.sqrt(2.0 / dim) * 5 + 1e-7, (name, k, fd, p[k])


def test_adjoint_N17_vs_stored_oracle_gradient():
    ref = load("grad_large.json")["gauss17"]
    psi = torch.from_numpy(I.gaussian_state(17, 717, dtype=np.complex64)).to(DEV)
    M2, g = hm.sre_grad(psi)
    assert abs(M2 - ref["M2"]) <= 1e-6 * max(1.0, abs(ref["M2"]))
    _check_projections("gauss17", ref, g.cpu().numpy())


def test_batched_adjoint_N17_N18_vs_stored_oracle_gradient():
    gold = load("grad_large.json")
    Ns, states = I.batched_ladder_states(64, 10, 18, 8, seed=4001)
    ts = [torch.from_numpy(s).to(DEV) for s in states]
    m2, grads = hm.sre_batched(ts, want_grad=True)
    m2 = m2.cpu().numpy()
    for name in ("ladder17", "ladder18"):
        ref = gold[name]
        i = ref["batch_index"]
        assert Ns[i] == ref["N"]
        assert abs(m2[i] - ref["M2"]) <= 1e-6 * max(1.0, abs(ref["M2"]))
        _check_projections(name, ref, grads[i].cpu().numpy())
