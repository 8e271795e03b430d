"""Right-hand-side sharding of the response solve across processes (one per GPU).

After the ground state (T, Lambda; replicated on every rank), every
(component, frequency) right-hand side of Eq. 29 and Eq. 32 is independent.
alpha_AB(omega) = -(g_AB + conj g_BA)/2 (Eq. 35) pairs components at the same
frequency, so the unit of work is one frequency with all components: each rank
solves the frequencies assigned to it and the only exchange is a gather of the
resulting alpha blocks (n_c x n_c complex numbers per frequency) on the host.
"""
from __future__ import annotations

import numpy as np


def partition(n_w: int, world: int, rank: int) -> list[int]:
    """Frequencies of this rank: contiguous, balanced blocks (sizes differ by
    at most one; ranks beyond n_w get none)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_w, world)
    start = rank * base + min(rank, extra)
    size = base + (1 if rank < extra else 0)
    return list(range(start, start + size))


def gather_alpha(local_idx, local_alpha, n_w: int, n_c: int, group=None) -> np.ndarray:
    """Assemble alpha [n_w, n_c, n_c] from every rank's blocks (all ranks get
    the full array).  Uses torch.distributed.all_gather_object on the host."""
    import torch.distributed as dist
    mine = (list(local_idx), np.asarray(local_alpha, dtype=np.complex128).reshape(len(local_idx), n_c, n_c))
    if dist.is_available() and dist.is_initialized():
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, mine, group=group)
    else:
        parts = [mine]
    out = np.full((n_w, n_c, n_c), np.nan + 0j)
    seen = np.zeros(n_w, dtype=bool)
    for idx, a in parts:
        for k, w in enumerate(idx):
            if seen[w]:
                raise RuntimeError(f"frequency {w} solved on two ranks")
            out[w] = a[k]
            seen[w] = True
    if not seen.all():
        raise RuntimeError("some frequencies were not solved by any rank")
    return out


def solve_sharded(solve, omegas, comps, rank: int, world: int, group=None) -> np.ndarray:
    """Run `solve(omegas_subset, comps) -> alpha [k, n_c, n_c]` on this rank's
    frequencies and gather the full alpha.  With the CUDA library `solve` is
    `lambda w, c: lrcc_solve(ctx, w, c)[0]`."""
    omegas = list(omegas)
    idx = partition(len(omegas), world, rank)
    n_c = len(comps)
    if idx:
        local = np.asarray(solve([omegas[i] for i in idx], comps))
    else:
        local = np.zeros((0, n_c, n_c), dtype=np.complex128)
    return gather_alpha(idx, local, len(omegas), n_c, group)
