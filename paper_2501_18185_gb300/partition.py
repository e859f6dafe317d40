"""Row-partitioned sigma over several processes: cost-balanced row ranges and the
all-gather that merges them.

The paper distributes its work over MPI processes with the static data (integrals and
the basis) replicated on every process and the results merged at the end (Sec. 3.1, the
MPI dynamic scheduler: tasks need no communication apart from their scheduling and the
final merge).  Here the unit is a row of sigma = H c, which needs nothing from other rows:
- every rank holds the integrals and the whole determinant list (sci_set_integrals,
  sci_set_determinants), as the paper replicates its static data;
- the sorted rows are cut into one contiguous range per rank, balanced by the rows' cost
  (`balanced_ranges`, from the per-row connection counts of sci_row_costs);
- each rank computes its rows (sci_set_row_range, then sci_sigma);
- one all-gather of the row slices gives every rank the whole sigma (`gather_rows`), as a
  Davidson iteration needs it for its next projection.
The collective is torch.distributed's all-gather (NCCL on GPUs, on the process group's own
stream, ordered after the sigma kernels by torch; gloo on CPU for tests).  The library
itself has no collective in it.
"""
from __future__ import annotations

import math

import numpy as np


def row_weights(cost, overhead: float):
    """Modelled time of each row: its connected determinants (the off-diagonal elements it
    evaluates) plus a fixed `overhead` (the staging of the row's bucket entries and its
    accumulation, the same for every row of a space)."""
    return np.asarray(cost, dtype=np.float64) + float(overhead)


def balanced_ranges(weights, parts: int) -> list[tuple[int, int]]:
    """`parts` contiguous row ranges [b, e) that cover [0, M) in order, cut where the
    running sum of `weights` crosses k * total / parts (k = 1 .. parts - 1).  Each range
    then weighs at most total / parts plus the heaviest single row.  Ranges may be empty
    (more parts than rows, or zero weights at the end)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    w = np.asarray(weights, dtype=np.float64).reshape(-1)
    if np.any(w < 0) or not np.all(np.isfinite(w)):
        raise ValueError("weights must be finite and nonnegative")
    M = w.size
    csum = np.cumsum(w)
    total = float(csum[-1]) if M else 0.0
    cuts = [0]
    for k in range(1, parts):
        if total > 0:
            # first row index whose prefix sum reaches k * total / parts, cut after it
            c = int(np.searchsorted(csum, k * total / parts, side="left")) + 1
        else:
            c = (k * M) // parts
        cuts.append(min(max(c, cuts[-1]), M))
    cuts.append(M)
    return [(cuts[k], cuts[k + 1]) for k in range(parts)]


def rebalance(weights, ranges, times) -> list[tuple[int, int]]:
    """Re-cut the ranges after timing them once: within each range the measured time is
    spread over its rows in proportion to their weights (the weight model is trusted inside
    a range, its scale is not), and the rows are cut again by balanced_ranges.  This
    corrects costs the weights miss, such as the staging of the buckets a range touches,
    which grows for ranges of highly excited rows."""
    w = np.asarray(weights, dtype=np.float64).reshape(-1).copy()
    if len(times) != len(ranges):
        raise ValueError("one time per range")
    for (b, e), t in zip(ranges, times):
        s = float(w[b:e].sum())
        if e > b and s > 0:
            w[b:e] *= float(t) / s
    return balanced_ranges(w, len(ranges))


def gather_rows(S, ranges, group=None):
    """Merge the row slices of a row-partitioned sigma in place: rank r holds valid rows
    ranges[r] of S ([M] or [M, nvec] torch tensor, real or complex); afterwards every rank
    holds all rows.  One all_gather_into_tensor of equal-size chunks (the longest range,
    zero padded) over the process group; complex data travels as its real view."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if len(ranges) != world:
        raise ValueError(f"{len(ranges)} ranges for {world} ranks")
    R = torch.view_as_real(S) if S.is_complex() else S
    R2 = R.reshape(R.shape[0], -1)
    width = R2.shape[1]
    L = max((e - b for b, e in ranges), default=0)
    if L == 0:
        return S
    send = torch.zeros((L, width), dtype=R2.dtype, device=R2.device)
    b, e = ranges[rank]
    if e > b:
        send[: e - b] = R2[b:e]
    recv = torch.empty((world * L, width), dtype=R2.dtype, device=R2.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    for r, (b, e) in enumerate(ranges):
        if r != rank and e > b:
            R2[b:e] = recv[r * L: r * L + (e - b)]
    return S


class RowSplitSigma:
    """sigma = H c on one rank of a row partition: H (a sci.Hamiltonian holding the whole
    list) computes its range, then the slices are all-gathered.  `ranges` is the list of
    all ranks' ranges (from balanced_ranges), the same on every rank."""

    def __init__(self, H, ranges, rank: int, group=None):
        self.H, self.ranges, self.rank, self.group = H, list(ranges), int(rank), group
        b, e = self.ranges[self.rank]
        H.set_row_range(b, e)

    @classmethod
    def balanced(cls, H, world: int, rank: int, group=None):
        """Ranges balanced by the rows' connection counts plus the per-row overhead of the
        C(N, 2) (N-2)-hole keys a row emits."""
        cost = H.row_costs().cpu().numpy()
        N = H.n_electrons
        weights = row_weights(cost, math.comb(N, 2))
        rs = cls(H, balanced_ranges(weights, world), rank, group)
        rs.weights = weights
        return rs

    def rebalance(self, my_ms: float, weights):
        """Re-cut the ranges from every rank's measured sigma time (all-gathered, so every
        rank computes the same ranges) and set this rank's new range."""
        import torch
        import torch.distributed as dist

        world = dist.get_world_size(self.group)
        dev = self.H.device if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([float(my_ms)], dtype=torch.float64, device=dev)
        all_t = torch.empty(world, dtype=torch.float64, device=dev)
        dist.all_gather_into_tensor(all_t, t, group=self.group)
        self.ranges = rebalance(weights, self.ranges, all_t.cpu().numpy())
        b, e = self.ranges[self.rank]
        self.H.set_row_range(b, e)
        return self.ranges

    def __call__(self, C, out=None, prec=None):
        from . import sci

        S = self.H.sigma(C, out=out, prec=sci.SCI_PREC_F64 if prec is None else prec)
        return gather_rows(S, self.ranges, self.group)
