"""One state's exact SRE (and its adjoint) split by X-string over the ranks of a process group.

The a-loop of Algorithm 2 is a sum of independent per-X-string terms; Sec. 4.1 distributes it
over threads, processes and GPUs and combines the partial sums with one reduction.  Here each
rank evaluates one contiguous, chunk-aligned slice of [0, 2^N) on its own GPU:

  * forward: the ranks all-gather their per-chunk FP64 triples (3 doubles per chunk of
    `sre_chunk(N)` X-strings; a few KB at N = 20) and every rank adds them in chunk order
    (hadamag_sre_combine).  A chunk's triple depends only on the chunk, so the result is the
    same bits for any number of ranks;
  * adjoint: the ranks all-reduce (sum) their 2^N complex128 dS_2/dpsi* and their S_2 part,
    then scale (hadamag_sre_grad_combine).

Only marshalling and the collectives live here; the slice evaluation, the combination and the
scaling are library calls.  The slice functions can be replaced (`slice_fn`, `grad_slice_fn`),
which is how the partition and exchange logic is exercised on CPU process groups.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import api


def _nqubits(psi: torch.Tensor) -> int:
    n = int(psi.numel()).bit_length() - 1
    if psi.dim() != 1 or (1 << n) != psi.numel() or n < 1:
        raise ValueError("state length must be 2^N")
    return n


def xstring_slice(N: int, rank: int, world: int, chunk: int) -> tuple[int, int]:
    """Rank `rank`'s slice [a0, a1) of the 2^N X-strings: contiguous whole chunks, as even as
    the chunk count allows (ranks beyond the chunk count get empty slices)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    nch = (1 << N) // chunk
    c0, c1 = rank * nch // world, (rank + 1) * nch // world
    return c0 * chunk, c1 * chunk


def _chunks_per_rank(N: int, world: int, chunk: int) -> list[int]:
    return [(xstring_slice(N, r, world, chunk)[1] - xstring_slice(N, r, world, chunk)[0]) // chunk
            for r in range(world)]


def gather_chunks(local: torch.Tensor, N: int, chunk: int, group=None) -> torch.Tensor:
    """All ranks' chunk triples in chunk order ([2^N / chunk, 3] float64, on local's device)."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        return local
    counts = _chunks_per_rank(N, world, chunk)
    m = max(counts)
    pad = torch.zeros((m, 3), dtype=torch.float64, device=local.device)
    pad[:local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[:k] for b, k in zip(bufs, counts)])


def sre_sharded(psi: torch.Tensor, n: float = 2.0, group=None, path: int | None = None, slice_fn=None,
                chunk: int | None = None):
    """(M_n, lost_norm) of psi, each rank of `group` evaluating its slice of the X-strings.
    Every rank passes the same state and receives the same result."""
    N = _nqubits(psi)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    ch = chunk or api.sre_chunk(N)
    a0, a1 = xstring_slice(N, rank, world, ch)
    local = slice_fn(psi, n, a0, a1) if slice_fn else api.sre_slice(psi, n, a0, a1, path=path)
    allc = gather_chunks(local, N, ch, group)
    return api.sre_combine(N, n, allc.cpu().numpy())


def sre_grad_sharded(psi: torch.Tensor, group=None, grad_slice_fn=None, combine_fn=None,
                     chunk: int | None = None):
    """(M_2, dM_2/dpsi*) of psi, each rank of `group` evaluating its slice of the X-strings;
    the 2^N dS_2/dpsi* and S_2 are all-reduced (sum).  Every rank receives the result."""
    N = _nqubits(psi)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    ch = chunk or api.sre_chunk(N)
    a0, a1 = xstring_slice(N, rank, world, ch)
    (S2, _), dS = (grad_slice_fn or api.sre_grad_slice)(psi, a0, a1)
    s = torch.tensor([S2], dtype=torch.float64, device=dS.device)
    if world > 1:
        dist.all_reduce(dS, group=group)
        dist.all_reduce(s, group=group)
    return (combine_fn or api.sre_grad_combine)(dS, float(s.item()), psi.dtype)
