"""Multi-GPU decomposition (host logic).

Two ways the path shards:

* Independent snapshots or requests (the batch and serving workloads): each rank
  solves its own problems; no collective is needed.  ``replica_shard`` assigns items
  to ranks and ``weak_scaling_value`` turns per-rank times into the job's rate.
* One large grid split across GPUs: leaves are cut into contiguous bands of leaf rows,
  one band per rank.  A rank needs, besides its own data,
    - the source weights q of the leaf rows within Dmax rows of its band (near field),
    - at every level l the multipoles of the box rows within the largest |dy| of the
      interaction lists of its own box rows (multipole-to-local halo),
    - the multipoles of every box at the levels where one box spans more than one
      band (assembled by an all-reduce of the partial expansions; a few thousand boxes).
  ``GridPartition`` computes these sets and the point-to-point exchange plan.

Every box in this project has one GPU, so the large-grid split is exercised only by
CPU ranks (gloo) in the tests; nothing here launches device work.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# ------------------------------------------------------------------------ replicas
def replica_shard(n_items: int, rank: int, world: int) -> list:
    """Items (0..n_items-1) solved by ``rank``: round robin, so uneven sizes spread out."""
    return list(range(rank, n_items, world))


def weak_scaling_value(units_per_rank, seconds_per_rank) -> float:
    """Job rate: all units processed by all ranks divided by the slowest rank's time."""
    return float(np.sum(units_per_rank)) / float(np.max(seconds_per_rank))


# ------------------------------------------------------------- one grid, many GPUs
def leaf_row_bands(nL: int, world: int):
    """Contiguous leaf-row bands [r0, r1) of (nearly) equal size, one per rank."""
    edges = [(nL * r) // world for r in range(world + 1)]
    return [(edges[r], edges[r + 1]) for r in range(world)]


@dataclass
class GridPartition:
    nL: int                 # leaves per side
    world: int
    rank: int
    near: np.ndarray        # near-field leaf offsets (dx, dy), from pp_near_offsets
    m2l: list               # per child position, list entries (dx, dy, kind), from pp_m2l_entries

    @property
    def levels(self) -> int:
        return int(np.log2(self.nL))

    def band(self, rank=None):
        return leaf_row_bands(self.nL, self.world)[self.rank if rank is None else rank]

    def box_rows(self, level: int, rank=None):
        """Box rows [b0, b1) at ``level`` whose leaves lie in the rank's band, or None if
        some box of the band also holds leaves of another band (a shared level)."""
        r0, r1 = self.band(rank)
        sh = self.levels - level
        if r0 % (1 << sh) or r1 % (1 << sh):
            return None
        return r0 >> sh, r1 >> sh

    def shared_levels(self):
        """Levels whose boxes straddle bands: multipoles there come from an all-reduce."""
        return [l for l in range(self.levels + 1)
                if any(self.box_rows(l, r) is None for r in range(self.world))]

    def near_halo_rows(self):
        """Leaf rows of other ranks whose q this rank needs for its near field."""
        r0, r1 = self.band()
        dmax = int(np.max(np.abs(self.near[:, 1]))) if len(self.near) else 0
        rows = set(range(max(0, r0 - dmax), r0)) | set(range(r1, min(self.nL, r1 + dmax)))
        return sorted(rows)

    def m2l_halo_rows(self, level: int):
        """Source box rows of other ranks that this rank's targets at ``level`` need, as
        {source level: rows}: same-level entries read ``level``, parent-level entries read
        ``level - 1`` (only where the rank owns whole box rows; shared levels are
        all-reduced and need no halo)."""
        own = self.box_rows(level)
        if own is None:
            return {}
        shared = set(self.shared_levels())
        b0, b1 = own
        need = {level: set(), level - 1: set()}
        for c in range(4):
            cy = c >> 1
            for dx, dy, kind in self.m2l[c]:
                for by in range(b0 + ((cy - b0) % 2), b1, 2):  # target rows of parity cy
                    if kind == 0:
                        sl, sy = level, by + dy
                    else:
                        sl, sy = level - 1, (by >> 1) + dy
                    if not 0 <= sy < (1 << sl):
                        continue
                    if sl in shared:
                        continue  # a level that straddles some band: every rank holds it after the all-reduce
                    mine = self.box_rows(sl)
                    if mine is not None and mine[0] <= sy < mine[1]:
                        continue
                    need[sl].add(int(sy))
        return {k: sorted(v) for k, v in need.items() if v}

    def exchange_plan(self):
        """{(kind, level): {owner rank: [rows]}} that this rank receives point-to-point."""
        owner_leaf = np.zeros(self.nL, dtype=np.int64)
        for r, (a, b) in enumerate(leaf_row_bands(self.nL, self.world)):
            owner_leaf[a:b] = r
        plan = {}
        rows = self.near_halo_rows()
        plan[("q", self.levels)] = _group_by_owner(rows, lambda y: int(owner_leaf[y]))
        shared = set(self.shared_levels())
        need = {}
        for lev in range(2, self.levels + 1):
            if lev in shared:
                continue
            for sl, rows in self.m2l_halo_rows(lev).items():
                need.setdefault(sl, set()).update(rows)
        for sl, rows in sorted(need.items()):
            sh = self.levels - sl
            plan[("multipole", sl)] = _group_by_owner(sorted(rows), lambda y: int(owner_leaf[y << sh]))
        return plan


def _group_by_owner(rows, owner):
    out = {}
    for y in rows:
        out.setdefault(owner(y), []).append(y)
    return out
