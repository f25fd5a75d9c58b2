"""hadamag_sre_noalloc -- the allocation-free exact-SRE call, for callers that cannot allocate
device memory where they need M_n (a host framework that owns all device memory through its own
pool or a fixed budget, latency-critical loops that must not pay cudaMalloc's device-wide
synchronisation, plugins that must not grow the device footprint) -- checked through the C ABI
against hadamag_sre on two calls in a row.  This file is collected last on purpose: the call
keeps its scratch in a library-wide device array, and the checks must hold both in a fresh
process and after every other test."""
import ctypes

import numpy as np
import pytest

from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402
from paper_2601_07824_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-6  # the FP32-path tolerance of the other SRE tests: 1e-6 * max(1, |M|)


def noalloc(psi: torch.Tensor, n: float):
    lib = _lib.load()
    N = int(psi.numel()).bit_length() - 1
    out = torch.full((3,), -1.0, dtype=torch.float64, device=psi.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(psi.device).cuda_stream)
    rc = lib.hadamag_sre_noalloc(ctypes.c_void_p(psi.data_ptr()), N, float(n),
                                 ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == 0, rc
    torch.cuda.synchronize(psi.device)
    return out.cpu().numpy()


@pytest.mark.parametrize("N", [16, 18, 20])
def test_noalloc_matches_sre_twice(N):
    psi = torch.from_numpy(I.gaussian_state(N, 5000 + N, dtype=np.complex64)).to(DEV)
    for n in (2.0, 1.0):
        M, ln = hm.sre(psi, n)
        for _ in range(2):  # two calls in a row share the library's scratch array
            r = noalloc(psi, n)
            assert r[2] == 0.0
            assert abs(r[0] - M) <= TOL * max(1.0, abs(M)), (N, n, r[0], M)
            assert abs(r[1] - ln) <= TOL


def test_noalloc_rejects_sizes_beyond_its_array():
    lib = _lib.load()
    t = torch.zeros(2 ** 21, dtype=torch.complex64, device=DEV)
    out = torch.zeros(3, dtype=torch.float64, device=DEV)
    rc = lib.hadamag_sre_noalloc(ctypes.c_void_p(t.data_ptr()), 21, 2.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 2  # HADAMAG_ERR_UNSUPPORTED
