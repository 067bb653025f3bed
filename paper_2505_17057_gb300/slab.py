"""Slab decomposition of one periodic grid over ranks: y slabs in 2D, z slabs in 3D.

Rank r of R owns the rows (2D) or planes (3D) [lo_r, hi_r) of the slab axis and steps a local
grid of those rows plus T halo rows on each side.  The local grid is stepped as a periodic grid:
an output row depends on the rows within one row of it (every lattice here has |e_p| <= 1 per
axis), so after T steps the owned rows are exact and only the halo rows, whose neighbours wrapped
around the local grid, are wrong.  Every T steps the ranks exchange T rows with their
neighbours, periodic in the rank index: the first T owned rows go to the previous rank (they
become its upper halo), the last T owned rows to the next rank (its lower halo).  A three-level
scheme also needs level t - dt on the halo rows, so it exchanges both levels and takes T = 1.

This module is bookkeeping only (index ranges and the exchange itself); stepping the local grid
is the caller's: the library's solver on the GPU (bench.py --split slab), or any other stepper.
The exchange uses torch.distributed point-to-point operations, so it runs over NCCL with CUDA
tensors and over gloo with CPU tensors alike.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple


def partition(n: int, nranks: int) -> List[Tuple[int, int]]:
    """[lo, hi) of every rank: n rows split as evenly as possible, larger slabs first."""
    if nranks < 1 or n < nranks:
        raise ValueError("need at least one row per rank")
    base, extra = divmod(n, nranks)
    out, lo = [], 0
    for r in range(nranks):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


@dataclass
class Slab:
    rank: int
    nranks: int
    n: int          # global length of the slab axis
    halo: int       # halo rows per side (T)
    lo: int
    hi: int

    @property
    def rows(self) -> int:
        return self.hi - self.lo

    @property
    def local_rows(self) -> int:
        return self.rows + 2 * self.halo

    @property
    def prev(self) -> int:
        return (self.rank - 1) % self.nranks

    @property
    def next(self) -> int:
        return (self.rank + 1) % self.nranks

    def global_rows(self) -> List[int]:
        """Global row index of every local row (halo rows wrap periodically)."""
        return [(self.lo - self.halo + i) % self.n for i in range(self.local_rows)]


def make_slab(rank: int, nranks: int, n: int, halo: int) -> Slab:
    lo, hi = partition(n, nranks)[rank]
    if hi - lo < halo:
        raise ValueError("a slab must hold at least `halo` rows")
    return Slab(rank, nranks, n, halo, lo, hi)


def exchange(slab: Slab, send_lo: Sequence, send_hi: Sequence, recv_lo: Sequence, recv_hi: Sequence) -> None:
    """Swap halo rows with the neighbouring ranks.

    send_lo: tensors holding the first T owned rows (they go to the previous rank);
    send_hi: the last T owned rows (to the next rank);
    recv_lo: filled with the previous rank's last T owned rows (this rank's lower halo);
    recv_hi: filled with the next rank's first T owned rows (this rank's upper halo).
    One tensor per field (and level).  With one rank the halos are the rank's own rows."""
    if slab.nranks == 1:
        for d, s in zip(recv_lo, send_hi):
            d.copy_(s)
        for d, s in zip(recv_hi, send_lo):
            d.copy_(s)
        return
    import torch.distributed as dist
    ops = []
    # posting order is the same on every rank, so that with two ranks (prev == next) the two
    # messages of each direction match in order; tags tell them apart where the backend uses them
    for s, r in zip(send_lo, recv_hi):
        ops.append(dist.P2POp(dist.isend, s, slab.prev, tag=0))
        ops.append(dist.P2POp(dist.irecv, r, slab.next, tag=0))
    for s, r in zip(send_hi, recv_lo):
        ops.append(dist.P2POp(dist.isend, s, slab.next, tag=1))
        ops.append(dist.P2POp(dist.irecv, r, slab.prev, tag=1))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
