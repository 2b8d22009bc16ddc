"""Admission policy of the serving loop (host logic only, no GPU needed).

Device memory counted against the HBM budget, per resident replica (one library handle of a
geometry with its own device input/output buffers): the radial tables, grid-brick neighbour
lists, atom-pair layout and workspace of the handle (gint_memory), plus D and H blocks, V and rho
on the grid and F.  A replica runs one job at a time.

Publication order (publish_order): in arrival order, a queued request is published when its
geometry has an idle replica left and no earlier request of the same geometry is still waiting;
requests of other geometries may overtake a waiting one (so one busy geometry does not hold up the
others), while each geometry's requests run in arrival order.  A geometry without a resident
replica gets one re-created, after evicting idle replicas least recently used first (Budget.plan);
a request that cannot fit even when every idle replica is evicted and nothing is on the GPU is
rejected.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Hashable, List, Optional, Sequence


@dataclasses.dataclass
class Resident:
    key: Hashable
    nbytes: int
    last_used: float
    busy: int = 0  # admitted requests of this geometry that have not completed


class Budget:
    """Accounting of resident handles + in-flight request buffers against a byte budget."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.resident: Dict[Hashable, Resident] = {}
        self.inflight = 0
        self.peak = 0

    @property
    def used(self) -> int:
        return self.inflight + sum(r.nbytes for r in self.resident.values())

    def plan(self, need: int, protect: Sequence[Hashable] = ()) -> Optional[List[Hashable]]:
        """Idle residents to evict (least recently used first) so that `need` more bytes fit;
        None if they cannot fit even after evicting every idle resident outside `protect`."""
        free = self.budget - self.used
        if need <= free:
            return []
        idle = sorted((r for r in self.resident.values() if r.busy == 0 and r.key not in protect),
                      key=lambda r: r.last_used)
        out = []
        for r in idle:
            out.append(r.key)
            free += r.nbytes
            if need <= free:
                return out
        return None

    def add_resident(self, key: Hashable, nbytes: int, now: float):
        self.resident[key] = Resident(key, int(nbytes), now)
        self.peak = max(self.peak, self.used)

    def evict(self, key: Hashable):
        self.resident.pop(key)

    def acquire(self, key: Hashable, nbytes: int):
        self.inflight += int(nbytes)
        self.resident[key].busy += 1
        self.peak = max(self.peak, self.used)

    def release(self, key: Hashable, nbytes: int, now: float):
        self.inflight -= int(nbytes)
        r = self.resident.get(key)
        if r is not None:
            r.busy -= 1
            r.last_used = now


def publish_order(pending_keys: Sequence[Hashable], idle: Dict[Hashable, int]) -> List[int]:
    """Indices (into the queue, in order) of the requests to publish now, given each geometry's
    count of idle replicas: per-geometry FIFO, other geometries may overtake."""
    left = dict(idle)
    blocked = set()
    out = []
    for i, k in enumerate(pending_keys):
        if k in blocked:
            continue
        if left.get(k, 0) > 0:
            left[k] -= 1
            out.append(i)
        else:
            blocked.add(k)
    return out
