"""The right-hand side split over the transfer momenta of one model, one shard per rank.

Loops, projections and products of a transfer momentum depend on that momentum alone; what couples the
momenta is the lattice Fourier transform of the exchange propagators to the bond classes (Sec. 3.3),
X(R'') = (1/Nq) sum_u e^{i u.R''} X(u).  Each rank holds the state rows of its own momenta, forms its part of
that sum, and one all-reduce over the ranks (2 ncls M^2 complex numbers: 2 x 25 x 324^2 x 16 B = 84 MB for the
t2g workload, 1.3 MB for the Rashba one) gives every rank the whole transform; each rank then finishes its own
rows.  This module holds the host side: the partition and the exchange.  The numbers come from a backend with
``shard_transform(state_local, q_list, mask)`` and ``shard_finish(T, state_local, q_list, xr, mask)``: a
``paper_1710_08830_gb300.api.Model`` (the library's CUDA kernels, NCCL for the exchange between GPUs).
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch


def partition(Nq: int, world: int, rank: int) -> np.ndarray:
    """The transfer momenta of one rank: a contiguous block of the mesh (q = qx Lq + qy), sizes differing by at
    most one between ranks."""
    if not (0 <= rank < world) or Nq < world:
        raise ValueError("need 0 <= rank < world <= Nq")
    lo = (Nq * rank) // world
    hi = (Nq * (rank + 1)) // world
    return np.arange(lo, hi, dtype=np.int32)


def _as_tensor(x) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)) if isinstance(x, np.ndarray) else x


def all_reduce_sum(x, group=None):
    """Sum of x over the ranks of the process group (complex values as pairs of reals); returns a tensor of the
    same kind as x (a numpy array comes back as a CPU tensor)."""
    import torch.distributed as dist
    t = _as_tensor(x).contiguous()
    if dist.is_available() and dist.is_initialized():
        r = torch.view_as_real(t) if t.is_complex() else t
        dist.all_reduce(r, op=dist.ReduceOp.SUM, group=group)
    return t


def sharded_rhs(backend, T: float, state_local, q_list: Sequence[int], group=None, mask: int = 3):
    """dX/dT of this rank's momenta q_list ([2][len(q_list)][M][M], list order) with the Fourier transform summed
    over all ranks of the group: this rank's part, one all-reduce, then the rank's own rows."""
    xr = backend.shard_transform(state_local, q_list, mask)
    xr = all_reduce_sum(xr, group)
    return backend.shard_finish(T, state_local, q_list, xr, mask)


def gather_rows(local, q_list, Nq: int, group=None) -> Optional[torch.Tensor]:
    """The full [2][Nq][M][M] array from every rank's rows (all-reduce of zero-padded copies); for checks."""
    t = _as_tensor(local)
    full = torch.zeros((2, Nq) + tuple(t.shape[2:]), dtype=t.dtype, device=t.device)
    full[:, torch.as_tensor(np.asarray(q_list, np.int64), device=t.device)] = t
    return all_reduce_sum(full, group)
