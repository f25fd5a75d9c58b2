"""X-string slices of one state's exact SRE and adjoint on the GPU (the a-loop of Algorithm 2
split as Sec. 4.1 splits it over ranks and GPUs), through the C ABI.

  * K chunk-aligned slices evaluated by separate calls reassemble the chunk triples of the
    single full-range call bit for bit (so any number of GPUs combines to the same bits);
  * the combined M_n matches hadamag_sre (a different summation order) to 1e-12 relative and
    the oracle to the exact-SRE tolerance 1e-6 max(1, |M|);
  * adjoint slices summed and scaled match hadamag_sre_grad;
  * misaligned or out-of-range slices are rejected."""
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
from paper_2601_07824_gb300 import PATH_CUDACORE, PATH_TENSOR, shard  # noqa: E402

DEV = torch.device("cuda:0")


def on_dev(psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV)


@pytest.mark.parametrize("N,K,path", [(9, 1, PATH_CUDACORE), (14, 3, PATH_CUDACORE), (17, 5, PATH_CUDACORE),
                                      (21, 4, PATH_TENSOR)])
def test_k_slices_reassemble_bit_for_bit(N, K, path):
    psi = on_dev(I.gaussian_state(N, 600 + N, dtype=np.complex64))
    ch = hm.sre_chunk(N)
    full = hm.sre_slice(psi, 2.0, 0, 2 ** N, path=path).cpu().numpy()
    parts = []
    for r in range(K):
        a0, a1 = shard.xstring_slice(N, r, K, ch)
        parts.append(hm.sre_slice(psi, 2.0, a0, a1, path=path).cpu().numpy())
    assert np.array_equal(np.concatenate(parts), full)
    # a repeated call is bit-identical too
    assert np.array_equal(hm.sre_slice(psi, 2.0, 0, 2 ** N, path=path).cpu().numpy(), full)
    M, ln = hm.sre_combine(N, 2.0, full)
    Mr, lnr = hm.sre(psi, 2.0, path=path)
    assert abs(M - Mr) <= 1e-12 * max(1.0, abs(Mr)) and abs(ln - lnr) <= 1e-12


@pytest.mark.parametrize("N,n", [(12, 1.0), (12, 3.0), (16, 2.0), (13, 2.5)])
def test_combined_slices_match_the_oracle(N, n):
    psi = I.gaussian_state(N, 620 + N, dtype=np.complex64)
    t = on_dev(psi)
    ch = hm.sre_chunk(N)
    parts = [hm.sre_slice(t, n, *shard.xstring_slice(N, r, 2, ch)) for r in range(2)]
    M, ln = hm.sre_combine(N, n, torch.cat(parts).cpu().numpy())
    Mo, lno = oracle.sre(psi, n)
    assert abs(M - Mo) <= 1e-6 * max(1.0, abs(Mo)), (M, Mo)
    assert abs(ln - lno) <= 1e-6


@pytest.mark.parametrize("N,K", [(10, 1), (13, 2), (16, 3), (18, 2)])
def test_gradient_slices_sum_to_the_gradient(N, K):
    psi = on_dev(I.gaussian_state(N, 640 + N, dtype=np.complex64))
    ch = hm.sre_chunk(N)
    dS = torch.zeros(2 ** N, dtype=torch.complex128, device=DEV)
    S2 = 0.0
    for r in range(K):
        (s2, _), d = hm.sre_grad_slice(psi, *shard.xstring_slice(N, r, K, ch))
        dS += d
        S2 += s2
    M2, g = hm.sre_grad_combine(dS, S2, torch.complex64)
    M2r, gr = hm.sre_grad(psi)
    assert abs(M2 - M2r) <= 1e-9 * max(1.0, abs(M2r))
    gg, ggr = g.cpu().numpy().astype(np.complex128), gr.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(gg - ggr) <= 1e-6 * np.linalg.norm(ggr)
    if N <= 13:
        M2o, go = oracle.sre_grad(psi.cpu().numpy())
        assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)


def test_sharded_helpers_on_one_rank():
    psi = on_dev(I.gaussian_state(15, 15, dtype=np.complex64))
    M, _ = shard.sre_sharded(psi, 2.0)
    assert abs(M - hm.sre(psi, 2.0)[0]) <= 1e-12 * max(1.0, abs(M))
    M2, g = shard.sre_grad_sharded(psi)
    M2r, gr = hm.sre_grad(psi)
    assert abs(M2 - M2r) <= 1e-9 * max(1.0, abs(M2r))
    assert torch.linalg.norm(g - gr) <= 1e-6 * torch.linalg.norm(gr)


def test_bad_slices_are_rejected():
    from paper_2601_07824_gb300 import _lib
    c = _lib.context(0)
    psi = on_dev(I.gaussian_state(14, 1, dtype=np.complex64))
    out = torch.empty((8, 3), dtype=torch.float64, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    for a0, a1 in [(1, 4096), (0, 4095), (4096, 0), (-4096, 0), (0, 2 ** 14 + 4096)]:
        rc = c.lib.hadamag_sre_slice(c.h, ctypes.c_void_p(psi.data_ptr()), 14, 2.0, 0, a0, a1,
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 1, (a0, a1)
    # an empty slice is valid and writes nothing
    assert c.lib.hadamag_sre_slice(c.h, ctypes.c_void_p(psi.data_ptr()), 14, 2.0, 0, 4096, 4096,
                                   ctypes.c_void_p(out.data_ptr()), stream) == 0
    with pytest.raises(ValueError):
        hm.sre_chunk(25)
