"""The thermodynamic-integration kernels' per-chain arithmetic (ti.cuh: start pattern, moves,
acceptance variate, beta grid, decision, Simpson weights, M_2, batch-means error), compiled for
the host and run in the kernels' order on exact FP64 energies, must give the oracle's chains
(Algorithm 3) step for step and the same means, M_2 and delta M_2.  CPU only: needs nvcc, no
GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import ti
from paper_2601_07824_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_07824_gb300", "csrc")


@pytest.fixture(scope="module")
def replay(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("ti") / "ti_chain_replay")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(HERE, "ti_chain_replay.cu")],
                   check=True, capture_output=True)
    return exe, tmp_path_factory.mktemp("io")


CASES = [  # (label, state, L, n_s, burn_in, seed, eps, sector)
    ("gauss_N8_L5", lambda: I.gaussian_state(8, 1), 5, 500, 20, 3, 0.0, None),
    ("gauss_N8_L6", lambda: I.gaussian_state(8, 2), 6, 400, 0, 99, 0.0, None),
    ("gauss_N10_seed_wraps", lambda: I.gaussian_state(10, 3), 4, 300, 50, 2 ** 64 - 2, 0.0, None),
    ("N1", lambda: I.gaussian_state(1, 4), 3, 200, 5, 7, 0.0, None),
    ("N2_one_step", lambda: I.gaussian_state(2, 5), 7, 1, 0, 12, 0.0, None),
    ("zero_eps", lambda: I.zero_state(6), 5, 300, 10, 1, 1e-3, None),
    ("T_eps", lambda: I.t_state_product(7), 8, 300, 10, 4, 1e-2, None),
    ("even_u1_N8", lambda: I.u1_state(8, 4, 21), 5, 400, 10, 3, 0.0, "even"),
    ("even_z2_N7", lambda: I.parity_state(7, 24, parity=1), 6, 300, 0, 11, 0.0, "even"),
    ("even_N2", lambda: I.parity_state(2, 5), 3, 50, 0, 2 ** 64 - 1, 0.0, "even"),
    ("even_u1_off_half_eps", lambda: I.u1_state(8, 3, 21), 4, 300, 5, 7, 1e-3, "even"),
]


@pytest.mark.parametrize("label,make,L,n_s,burn,seed,eps,sector", CASES, ids=[c[0] for c in CASES])
def test_kernel_chain_arithmetic_reproduces_the_oracle(replay, label, make, L, n_s, burn, seed, eps, sector):
    exe, io = replay
    psi = make()
    N = int(psi.size).bit_length() - 1
    S = oracle.sre_terms(psi, 2.0)[0]
    sfile, ofile = str(io / f"{label}_S.bin"), str(io / f"{label}_out.bin")
    S.astype(np.float64).tofile(sfile)
    subprocess.run([exe, sfile, str(N), str(L), str(n_s), str(burn), str(seed), repr(eps),
                    "1" if sector else "0", ofile], check=True)
    raw = open(ofile, "rb").read()
    nonpos = int(np.frombuffer(raw[:4], dtype=np.int32)[0])
    out = np.frombuffer(raw[4:4 + 8 * (L + 3)], dtype=np.float64)
    traj = np.frombuffer(raw[4 + 8 * (L + 3):], dtype=np.int64).reshape(L, burn + n_s)
    rec = {}
    means, _ = ti.metropolis_means(ti.energy_table(psi, eps, sector), N, L, n_s, seed, burn, record=rec,
                                   sector=sector)
    I_ = float(np.dot(ti.simpson_weights(L), means))
    assert nonpos == 0
    np.testing.assert_array_equal(traj, rec["traj"])
    np.testing.assert_allclose(out[:L], means, rtol=0, atol=1e-12)
    assert out[L] == pytest.approx(I_, abs=1e-12)
    assert out[L + 1] == pytest.approx(ti.m2_from_integral(I_, eps, sector), abs=1e-12)
    assert out[L + 2] == pytest.approx(ti.m2_stderr(rec["batch_sums"], n_s, I_, eps), rel=1e-10, abs=1e-15)


def test_vanishing_sum_is_flagged(replay):
    # |0000> with eps = 0: S(a) = 0 for a != 0, which the kernels report as non-finite
    exe, io = replay
    sfile, ofile = str(io / "zero_S.bin"), str(io / "zero_out.bin")
    oracle.sre_terms(I.zero_state(4), 2.0)[0].tofile(sfile)
    subprocess.run([exe, sfile, "4", "3", "50", "0", "1", "0.0", "0", ofile], check=True)
    assert int(np.frombuffer(open(ofile, "rb").read()[:4], dtype=np.int32)[0]) == 1
