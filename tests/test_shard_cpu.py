"""The X-string partition of one state over ranks (Sec. 4.1 distributes Algorithm 2's a-loop
over processes and GPUs), exercised with two gloo ranks on the CPU.

The per-slice evaluations are stand-ins built from the FP64 oracle (per-X-string sums, and the
adjoint restricted to a slice); what is under test is the partition, the exchange of partial
results and their combination:
  * the slices tile [0, 2^N) on chunk boundaries for any world size;
  * two ranks reassemble exactly the chunk triples a single rank produces (bit for bit), and
    the library's host-only combination gives the oracle's M_n;
  * the all-reduced adjoint of two slices equals the oracle's gradient."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2601_07824_gb300 import inputs as I
from paper_2601_07824_gb300 import shard


@pytest.mark.parametrize("N,chunk", [(1, 2), (5, 32), (12, 4096), (20, 4096)])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_slices_tile_the_xstrings(N, chunk, world):
    edges = [shard.xstring_slice(N, r, world, chunk) for r in range(world)]
    assert edges[0][0] == 0 and edges[-1][1] == 2 ** N
    for (a0, a1), (b0, _) in zip(edges, edges[1:]):
        assert a1 == b0
    for a0, a1 in edges:
        assert a0 % chunk == 0 and a1 % chunk == 0 and a1 >= a0
    sizes = [a1 - a0 for a0, a1 in edges]
    assert max(sizes) - min(sizes) <= chunk


def _oracle_chunks(psi, n, a0, a1, chunk):
    """Stand-in slice evaluation: the oracle's per-X-string triples, summed per chunk in order."""
    Sq, S1, T1 = oracle.sre_terms(psi, n, a0, a1)
    t = np.stack([Sq, S1, T1], axis=1).reshape(-1, chunk, 3)
    out = np.zeros((t.shape[0], 3))
    for k in range(chunk):
        out += t[:, k]
    return torch.from_numpy(out)


def _slice_grad(psi, a0, a1):
    """Stand-in adjoint of a slice: dS_2/dpsi*_w = sum_{a in slice} psi_{w^a}[G_a(w) + conj G_a(w^a)],
    G_a = H(2|c_a|^2 c_a), c_a = H v_a, v_a(z) = conj(psi_{z^a}) psi_z (plain dense N <= 8)."""
    p = psi.numpy().astype(np.complex128)
    N = int(p.size).bit_length() - 1
    z = np.arange(2 ** N)
    H = np.array([[1.0]])
    for _ in range(N):
        H = np.kron(H, np.array([[1.0, 1.0], [1.0, -1.0]]))
    dS = np.zeros(2 ** N, dtype=np.complex128)
    S2 = S1 = 0.0
    for a in range(a0, a1):
        c = H @ (np.conj(p[z ^ a]) * p)
        S2 += float(np.sum(np.abs(c) ** 4))
        S1 += float(np.sum(np.abs(c) ** 2))
        G = H @ (2 * np.abs(c) ** 2 * c)
        dS += p[z ^ a] * (G + np.conj(G[z ^ a]))
    return (S2, S1), torch.from_numpy(dS)


def _combine_grad(dS, S2, dtype):
    N = int(dS.numel()).bit_length() - 1
    return -np.log2(S2 / 2 ** N), (-dS / (np.log(2.0) * S2)).to(torch.complex128)


def _worker(rank, world, port, N, chunk, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        psi = torch.from_numpy(I.gaussian_state(N, 70 + N))
        res = {}
        for n in (2.0, 1.0):
            a0, a1 = shard.xstring_slice(N, rank, world, chunk)
            local = _oracle_chunks(psi.numpy(), n, a0, a1, chunk)
            res[f"chunks{n}"] = shard.gather_chunks(local, N, chunk).numpy()
            res[f"M{n}"] = shard.sre_sharded(psi, n, slice_fn=lambda p, nn, b0, b1: _oracle_chunks(
                p.numpy(), nn, b0, b1, chunk), chunk=chunk)
        gN = 6
        g_psi = torch.from_numpy(I.gaussian_state(gN, 90))
        res["grad"] = shard.sre_grad_sharded(g_psi, grad_slice_fn=_slice_grad, combine_fn=_combine_grad, chunk=8)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reassemble_the_single_rank_result(world):
    from paper_2601_07824_gb300 import api
    N = 14
    chunk = api.sre_chunk(N)  # the library's chunk (host-only call): 4096, so 4 chunks here
    psi = I.gaussian_state(N, 70 + N)
    one = {n: _oracle_chunks(psi, n, 0, 2 ** N, chunk).numpy() for n in (2.0, 1.0)}
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as sk:  # a free local port for the rendezvous
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, chunk, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = dict(q.get(timeout=300) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    for p in procs:
        assert p.exitcode == 0
    for n in (2.0, 1.0):
        want_M = oracle.sre(psi, n)[0]
        for r in range(world):
            # bit-identical reassembly of the single-rank chunk triples
            assert np.array_equal(out[r][f"chunks{n}"], one[n]), (r, n)
            M, _ = out[r][f"M{n}"]
            assert M == api.sre_combine(N, n, one[n])[0]
            assert abs(M - want_M) <= 1e-12 * max(1.0, abs(want_M)), (n, M, want_M)
    gpsi = I.gaussian_state(6, 90)
    M2o, go = oracle.sre_grad(gpsi)
    for r in range(world):
        M2, g = out[r]["grad"]
        assert abs(M2 - M2o) < 1e-12
        assert np.linalg.norm(g.numpy() - go) <= 1e-12 * np.linalg.norm(go)
