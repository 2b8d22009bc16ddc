"""Admission policy of the serving loop (host logic only, no GPU needed).

Device memory counted against the HBM budget:
  * resident handles: per geometry, the radial tables, grid-brick neighbour lists, atom-pair
    layout and workspace of the library handle (gint_memory);
  * in-flight buffers: per admitted request, its device inputs and outputs (D and H blocks,
    V and rho on the grid, F).

A batch takes the queue's requests in arrival order (FIFO, no overtaking) while
  * it has fewer than ``max_batch`` requests,
  * the request's geometry is not already in the batch (one task per handle and launch),
  * the request's bytes (plus its handle's, if the handle is not resident) fit the budget after
    evicting idle resident handles, least recently used first (never one the batch uses).
The first request that does not fit ends the batch; it waits for memory that batches on the
GPU will release.  A request that cannot fit even when nothing else is admitted, nothing is on
the GPU and every idle handle is evicted is rejected.
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


@dataclasses.dataclass
class Plan:
    admit: List = dataclasses.field(default_factory=list)    # requests of the batch, in order
    reject: List = dataclasses.field(default_factory=list)   # requests that can never fit
    evict: List[Hashable] = dataclasses.field(default_factory=list)   # handles to free first
    create: List[Hashable] = dataclasses.field(default_factory=list)  # handles to (re)create

    @property
    def consumed(self) -> int:
        """Length of the queue prefix the plan takes (rejections come first, then admissions)."""
        return len(self.reject) + len(self.admit)


def select_batch(pending: Sequence, budget: Budget, max_batch: int, any_inflight: bool, now: float) -> Plan:
    """Plans the next batch from the FIFO `pending` (items with .key, .request_bytes and
    .handle_bytes) and applies it to `budget`: evictions, residents for created handles,
    in-flight bytes and busy counts of the admitted requests."""
    plan = Plan()
    keys = set()
    for r in pending:
        if len(plan.admit) >= max_batch or r.key in keys:
            break
        resident = r.key in budget.resident
        need = r.request_bytes + (0 if resident else r.handle_bytes)
        ev = budget.plan(need, tuple(keys) + (r.key,))
        if ev is None:
            if plan.admit or any_inflight:
                break
            plan.reject.append(r)
            continue
        for k in ev:
            budget.evict(k)
        plan.evict += ev
        if not resident:
            budget.add_resident(r.key, r.handle_bytes, now)
            plan.create.append(r.key)
        budget.acquire(r.key, r.request_bytes)
        keys.add(r.key)
        plan.admit.append(r)
    return plan
