"""Spreading independent q-points over ranks (one process per GPU).

Eq. (rpaE) sums independent q-point terms, so the ranks share no data while
they compute: each rank takes q-points round-robin and the only exchange is
the gather of the per-q energies at the end (N_q scalars).
"""
from __future__ import annotations


def qpoints_for_rank(n_q: int, rank: int, world: int) -> list[int]:
    """q indices of `rank` when n_q q-points are dealt round-robin over `world` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside world of %d" % (rank, world))
    return list(range(rank, n_q, world))


def gather_energies(local: dict, n_q: int, group=None) -> list:
    """Collect {iq: E_c} from every rank into a list indexed by q (all ranks get it)."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, dict(local), group=group)
    out = [None] * n_q
    for part in parts:
        for iq, ec in part.items():
            if out[iq] is not None:
                raise RuntimeError("q-point %d computed by two ranks" % iq)
            out[iq] = ec
    missing = [i for i, e in enumerate(out) if e is None]
    if missing:
        raise RuntimeError("q-points never computed: %s" % missing)
    return out
