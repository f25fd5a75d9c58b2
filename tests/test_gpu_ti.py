"""Thermodynamic-integration M_2 (Sec. 3.2, Algorithm 3) on the GPU against the FP64 oracle.

Both sides run the same chains: the proposals and acceptance variates come from one
counter-based generator (SplitMix64 seeded with seed + l), so the X-strings proposed are
compared bit for bit.  The accept/reject decisions are taken in FP64 on both sides, but on
energies f = -ln S(a) that the GPU computes with FP32 transforms; a decision whose margin
|u - p_acc| in the oracle's run is below DELTA could legitimately go either way, so the
chains must agree step for step except that they may part at such a decision, after which
the GPU chain must still make only valid moves (stay, or take the proposed one-bit flip).

Tolerances, from the per-X-string bound of the FP32 path (S(a) within 2e-5 relative of the
oracle): f within 2e-5 absolute, so each chain mean within TOL_F = 2e-5, p_acc = exp(-beta df)
within 4e-5 relative (DELTA = 1e-4), and M_2 = sum_l w_l <f>_l / ln 2 (sum_l w_l = 1) within
TOL_M = 2e-5 / ln 2 (the eps > 0 cases here raise the slope dM_2/dI by under 1 %, covered by the
rounding up to 3e-5).  Unlike exact M_n, whose FP32 errors average over all 2^N X-strings, the
estimate averages -ln S(a) over the few hundred X-strings the chains visit, so the exact-SRE
bound 1e-6 max(1, |M|) is not what the arithmetic guarantees here."""
import numpy as np
import pytest

import oracle
from oracle import ti
from paper_2601_07824_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_07824_gb300 as hm  # noqa: E402

DEV = torch.device("cuda:0")
DELTA = 1e-4
TOL_F = 2e-5
TOL_M = 3e-5


def move_mask(r, N, sector):
    """The generator's move for output r (the oracle's rule, restated for the validity check)."""
    b1 = int(r % np.uint64(N))
    if sector != "even":
        return 1 << b1
    b2 = int((r // np.uint64(N)) % np.uint64(N - 1))
    return (1 << b1) | (1 << (b2 + (b2 >= b1)))


def check_against_oracle(psi_np, L, n_s, burn, seed, eps=0.0, sector=None):
    N = int(psi_np.size).bit_length() - 1
    psi = torch.from_numpy(psi_np).to(DEV)
    M2, err, means, traj = hm.sre_ti(psi, L, n_s, seed, burn_in=burn, eps=eps, record=True,
                                     even_sector=sector == "even")
    traj = traj.cpu().numpy()
    rec = {}
    f = ti.energy_table(psi_np, eps, sector) if N <= 12 else ti.energy_fn(psi_np, eps)
    means_o, _ = ti.metropolis_means(f, N, L, n_s, seed, burn, record=rec, sector=sector)
    I_o = float(np.dot(ti.simpson_weights(L), means_o))
    M2_o = ti.m2_from_integral(I_o, eps, sector)
    T = burn + n_s
    assert traj.shape == (L, T)
    parted = []
    for l in range(L):
        diff = np.nonzero(traj[l] != rec["traj"][l])[0]
        if diff.size == 0:
            continue
        t0 = int(diff[0])
        assert rec["margin"][l, t0] < DELTA, (l, t0, rec["margin"][l, t0])
        r = oracle.splitmix64(seed + l, 1 + 2 * T)
        a = int(rec["traj"][l, t0 - 1]) if t0 > 0 else int(r[0] >> np.uint64(64 - N))
        if t0 == 0 and sector == "even" and bin(a).count("1") % 2:
            a ^= 1
        for t in range(t0, T):
            flip = a ^ move_mask(r[1 + 2 * t], N, sector)
            assert traj[l, t] in (a, flip), (l, t)
            a = int(traj[l, t])
        parted.append(l)
    for l in range(L):
        if l not in parted:
            assert means[l] == pytest.approx(means_o[l], abs=TOL_F), l
    if not parted:
        assert M2 == pytest.approx(M2_o, abs=TOL_M)
        # batch means move by at most 2 TOL_F, the error by at most 2 TOL_F / (sqrt(B - 1) ln 2)
        assert err == pytest.approx(ti.m2_stderr(rec["batch_sums"], n_s, I_o, eps), abs=TOL_M)
    return M2, M2_o, parted


@pytest.mark.parametrize("N,L,n_s,burn,seed", [(10, 5, 400, 20, 3), (13, 6, 300, 0, 17), (15, 4, 200, 10, 5)])
def test_onepass_sizes_follow_the_oracle_chains(N, L, n_s, burn, seed):
    psi = I.gaussian_state(N, 3100 + N, dtype=np.complex64)
    check_against_oracle(psi, L, n_s, burn, seed)


@pytest.mark.parametrize("N,L,n_s,burn,seed", [(16, 3, 120, 5, 9), (18, 4, 150, 10, 3)])
def test_twopass_sizes_follow_the_oracle_chains(N, L, n_s, burn, seed):
    psi = I.brickwork_haar(N, 8, seed=3200 + N) if N == 16 else I.gaussian_state(N, 3200 + N, dtype=np.complex64)
    check_against_oracle(psi, L, n_s, burn, seed)


def test_edge_cases():
    # one qubit (the flipped bit is always bit 0), one recorded step, seeds near 2^64
    check_against_oracle(I.gaussian_state(1, 41, dtype=np.complex64), 3, 200, 5, 7)
    check_against_oracle(I.gaussian_state(2, 42, dtype=np.complex64), 7, 1, 0, 2 ** 64 - 3)
    # stabilizer states: S(a) = 0 off the stabilizer group, so eps > 0 (exact zeros on both sides)
    check_against_oracle(I.zero_state(6).astype(np.complex64), 5, 300, 10, 1, eps=1e-3)
    check_against_oracle(I.ghz_state(6).astype(np.complex64), 3, 300, 0, 8, eps=1e-1)
    check_against_oracle(I.t_state_product(7).astype(np.complex64), 8, 300, 10, 4, eps=1e-2)


@pytest.mark.parametrize("label", ["u1_N10", "z2_N13", "u1_N16", "u1_N9_eps", "N2"])
def test_even_sector_chains_follow_the_oracle(label):
    # Sec. 3.2: chains restricted to even-weight X-strings for U(1) / prod Z symmetric states
    psi, L, n_s, burn, seed, eps = {
        "u1_N10": (I.u1_state(10, 5, 3601, dtype=np.complex64), 5, 300, 10, 3, 0.0),
        "z2_N13": (I.parity_state(13, 3602, dtype=np.complex64), 4, 200, 0, 8, 0.0),
        "u1_N16": (I.u1_state(16, 8, 3603, dtype=np.complex64), 3, 100, 5, 21, 0.0),
        "u1_N9_eps": (I.u1_state(9, 3, 3604, dtype=np.complex64), 4, 200, 5, 4, 1e-3),  # off half filling
        "N2": (I.parity_state(2, 3605, dtype=np.complex64), 3, 100, 0, 2 ** 64 - 1, 0.0),
    }[label]
    check_against_oracle(psi, L, n_s, burn, seed, eps, sector="even")


def test_even_sector_invalid_for_one_qubit():
    psi = torch.from_numpy(I.parity_state(1, 1, dtype=np.complex64)).to(DEV)
    with pytest.raises(hm.HadamagError) as e:
        hm.sre_ti(psi, 3, 10, 1, even_sector=True)
    assert e.value.code == 1


def test_complex128_input_and_unrecorded_run():
    psi_np = I.gaussian_state(12, 3300)
    psi = torch.from_numpy(psi_np).to(DEV)
    M2a, erra, means_a, _ = hm.sre_ti(psi, 5, 200, 11, burn_in=10, record=True)
    M2b, errb, means_b = hm.sre_ti(psi, 5, 200, 11, burn_in=10)  # no trajectory buffer
    assert M2a == M2b and erra == errb and means_a == means_b and erra > 0.0
    # the GPU reads complex128 input rounded to complex64: same chains as the complex64 state
    M2c, _, _ = hm.sre_ti(psi.to(torch.complex64), 5, 200, 11, burn_in=10)
    assert M2c == M2a
    M2_o = ti.m2_metropolis(psi_np.astype(np.complex64), 5, 200, 11, burn_in=10)
    assert M2a == pytest.approx(M2_o, abs=TOL_M)


def test_launches_are_the_library_kernels():
    # start, one per-X evaluation, init, then per step one per-X evaluation and one ti_step,
    # then ti_finish (one-pass per-X kernel below 16 qubits: one launch per evaluation)
    psi = torch.from_numpy(I.gaussian_state(10, 3400, dtype=np.complex64)).to(DEV)
    c = hm.context(0)
    before = c.launch_count()
    hm.sre_ti(psi, 4, 50, 5, burn_in=7)
    assert c.launch_count() - before == 4 + 2 * 57


def test_vanishing_energy_and_invalid_arguments():
    z = torch.from_numpy(I.zero_state(4).astype(np.complex64)).to(DEV)
    with pytest.raises(hm.HadamagError) as e:
        hm.sre_ti(z, 3, 50, 1)  # S(a) = 0 for a != 0 and eps = 0
    assert e.value.code == 6
    psi = torch.from_numpy(I.gaussian_state(8, 3500, dtype=np.complex64)).to(DEV)
    for kw in (dict(L=2, n_s=10), dict(L=3, n_s=0), dict(L=3, n_s=10, burn_in=-1), dict(L=3, n_s=10, eps=-1e-3),
               dict(L=4097, n_s=10)):
        args = dict(seed=1, burn_in=0, eps=0.0)
        args.update(kw)
        with pytest.raises(hm.HadamagError) as e:
            hm.sre_ti(psi, args.pop("L"), args.pop("n_s"), **args)
        assert e.value.code == 1
    # the context stays usable
    M2, err, _ = hm.sre_ti(psi, 3, 20, 1)
    assert np.isfinite(M2) and err > 0.0
    assert hm.sre_ti(psi, 3, 1, 1)[1] == 0.0  # one recorded step: no error estimate
