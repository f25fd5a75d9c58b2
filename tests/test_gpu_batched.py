"""Batched persistent launch: 64 states, N_i ~ U{10..18}, RY/RZ + CZ-ladder
circuits of depth 8, M_2 and dM_2/dpsi* in one launch.  Checked against the single-state
adjoint (itself checked against the oracle), the FP64 oracle on the small states, FP64
finite differences (step 1e-4), and a CUDA-graph capture + replay."""
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


@pytest.fixture(scope="module")
def batch():
    Ns, states = I.batched_ladder_states(64, 10, 18, 8, seed=4001)
    return Ns, states, [torch.from_numpy(s).to(DEV) for s in states]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batched_matches_single_state_adjoint(batch):
    Ns, states, ts = batch
    m2, grads = hm.sre_batched(ts, want_grad=True)
    m2 = m2.cpu().numpy()
    for i, t in enumerate(ts):
        M, g = hm.sre_grad(t)
        assert abs(m2[i] - M) <= 1e-6 * max(1.0, abs(M)), (i, Ns[i], m2[i], M)
        assert rel(grads[i].cpu().numpy().astype(np.complex128), g.cpu().numpy().astype(np.complex128)) <= 1e-5


def test_batched_small_states_vs_oracle_and_fd(batch):
    Ns, states, ts = batch
    m2, grads = hm.sre_batched(ts, want_grad=True)
    small = [i for i, n in enumerate(Ns) if n <= 11][:3]
    assert small
    rng = np.random.default_rng(5)
    for i in small:
        M2o, go = oracle.sre_grad(states[i])
        assert abs(m2[i].item() - M2o) <= 1e-6 * abs(M2o)
        g = grads[i].cpu().numpy().astype(np.complex128)
        assert rel(g, go) <= 1e-5
        psi = states[i].astype(np.complex128)
        d = rng.standard_normal(psi.size) + 1j * rng.standard_normal(psi.size)
        d /= np.linalg.norm(d)
        h = 1e-4
        fd = (oracle.sre(psi + h * d, 2.0)[0] - oracle.sre(psi - h * d, 2.0)[0]) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(g, d))) <= 1e-5 * max(1.0, abs(fd))


def test_batched_forward_only_and_graph_replay(batch):
    Ns, states, ts = batch
    ref, _ = hm.sre_batched(ts, want_grad=False)
    out = torch.empty(len(ts), dtype=torch.float64, device=DEV)
    grads = [torch.empty_like(t) for t in ts]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        hm.sre_batched(ts, want_grad=True, out=out, grads=grads)  # uncaptured call (buffers, tuning)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        hm.sre_batched(ts, want_grad=True, out=out, grads=grads, sync=False)
    out.zero_()
    for gr in grads:
        gr.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-6)
    i = int(np.argmax(Ns))
    _, gi = hm.sre_grad(ts[i])
    assert rel(grads[i].cpu().numpy().astype(np.complex128), gi.cpu().numpy().astype(np.complex128)) <= 1e-5
