"""Serving-loop admission policy (host logic, no GPU): FIFO batches under an HBM byte budget."""
import dataclasses
import random

from paper_2603_21835_gb300.admission import Budget, select_batch


@dataclasses.dataclass
class Req:
    key: int
    request_bytes: int
    handle_bytes: int
    rid: int = 0


def test_fifo_slots_and_one_request_per_geometry():
    b = Budget(10_000)
    for k in range(3):
        b.add_resident(k, 100, now=k)
    q = [Req(0, 10, 100, 0), Req(1, 10, 100, 1), Req(0, 10, 100, 2), Req(2, 10, 100, 3)]
    plan = select_batch(q, b, max_batch=8, any_inflight=False, now=10)
    assert [r.rid for r in plan.admit] == [0, 1]  # stops at the second request of geometry 0
    assert plan.consumed == 2 and not plan.evict and not plan.create
    assert b.inflight == 20 and b.resident[0].busy == 1 and b.resident[1].busy == 1
    plan = select_batch([Req(5, 1, 1, i) for i in range(4)], Budget(100), max_batch=1, any_inflight=False, now=0)
    assert len(plan.admit) == 1


def test_lru_eviction_of_idle_handles_only():
    b = Budget(1000)
    b.add_resident("a", 300, now=1.0)
    b.add_resident("b", 300, now=2.0)
    b.add_resident("c", 300, now=3.0)
    b.acquire("a", 50)  # "a" is busy: never evicted
    plan = select_batch([Req("d", 100, 300)], b, max_batch=4, any_inflight=True, now=5.0)
    # 950 bytes used; 400 needed: evict idle handles oldest first ("b", then "c"), never busy "a"
    assert plan.evict == ["b", "c"]
    assert "a" in b.resident and "d" in b.resident and plan.create == ["d"]
    assert b.used <= b.budget


def test_waits_for_inflight_memory_then_rejects_only_when_hopeless():
    b = Budget(1000)
    b.add_resident("x", 600, now=0.0)
    b.acquire("x", 300)  # a batch on the GPU holds 300 bytes
    big = Req("y", 200, 300)
    plan = select_batch([big], b, max_batch=4, any_inflight=True, now=1.0)
    assert not plan.admit and not plan.reject and plan.consumed == 0  # waits
    b.release("x", 300, now=2.0)
    plan = select_batch([big], b, max_batch=4, any_inflight=False, now=3.0)
    assert plan.admit == [big] and plan.evict == ["x"]
    hopeless = Req("z", 900, 200)
    b2 = Budget(1000)
    plan = select_batch([hopeless, Req("w", 10, 10)], b2, max_batch=4, any_inflight=False, now=0.0)
    assert plan.reject == [hopeless] and [r.key for r in plan.admit] == ["w"] and plan.consumed == 2


def test_random_stream_invariants():
    """Random arrivals and completions: the budget holds at every admission, requests leave the
    queue in arrival order, and every request is eventually served or rejected."""
    rng = random.Random(7)
    sizes = {k: (rng.randint(50, 400), rng.randint(100, 600)) for k in range(12)}
    b = Budget(2500)
    queue, onboard, served, rejected = [], [], [], []
    rid = 0
    t = 0.0
    order = []
    for step in range(4000):
        t += 1.0
        if rng.random() < 0.6 and rid < 600:
            k = rng.randrange(12)
            queue.append(Req(k, sizes[k][0], sizes[k][1], rid))
            rid += 1
        if onboard and rng.random() < 0.5:
            batch = onboard.pop(0)
            for r in batch:
                b.release(r.key, r.request_bytes, t)
                served.append(r.rid)
        if len(onboard) < 2 and queue:
            plan = select_batch(queue[:9], b, max_batch=8, any_inflight=bool(onboard), now=t)
            assert b.used <= b.budget
            assert all(b.resident[r.key].busy >= 1 for r in plan.admit)
            order += [r.rid for r in plan.reject + plan.admit]
            rejected += [r.rid for r in plan.reject]
            del queue[:plan.consumed]
            if plan.admit:
                onboard.append(plan.admit)
    while onboard:
        for r in onboard.pop(0):
            b.release(r.key, r.request_bytes, t)
            served.append(r.rid)
    assert order == sorted(order)  # FIFO
    assert sorted(served + rejected) == order
    assert not rejected  # every geometry fits on its own in this budget
    assert b.inflight == 0 and all(r.busy == 0 for r in b.resident.values())
