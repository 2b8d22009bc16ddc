"""Serving-loop admission policy (host logic, no GPU): the HBM byte budget of resident replicas and
the order in which queued requests are published to the device work queue."""
import random

from paper_2603_21835_gb300.admission import Budget, publish_order


def test_lru_eviction_of_idle_replicas_only():
    b = Budget(1000)
    b.add_resident("a", 300, now=1.0)
    b.add_resident("b", 300, now=2.0)
    b.add_resident("c", 300, now=3.0)
    b.acquire("a", 50)  # "a" is busy: never evicted
    # 950 bytes used; 400 more needed: evict idle replicas oldest first ("b", then "c"), never busy "a"
    assert b.plan(400) == ["b", "c"]
    assert b.plan(10_000) is None
    assert b.plan(40) == []
    for k in b.plan(400):
        b.evict(k)
    b.add_resident("d", 400, now=5.0)
    assert b.used <= b.budget and "a" in b.resident
    b.release("a", 50, now=6.0)
    assert b.resident["a"].busy == 0 and b.resident["a"].last_used == 6.0 and b.inflight == 0


def test_protected_replicas_are_not_evicted():
    b = Budget(600)
    b.add_resident("x", 300, now=0.0)
    b.add_resident("y", 300, now=1.0)
    assert b.plan(300, protect=("x",)) == ["y"]
    assert b.plan(600, protect=("x",)) is None


def test_publish_order_is_fifo_per_geometry_with_overtaking():
    keys = ["a", "a", "b", "c", "b", "a", "c"]
    # one idle replica each: the first request of every geometry goes
    assert publish_order(keys, {"a": 1, "b": 1, "c": 1}) == [0, 2, 3]
    # "a" busy: its requests wait in order, the others overtake them
    assert publish_order(keys, {"a": 0, "b": 2, "c": 1}) == [2, 3, 4]
    # two replicas of "a": its first two requests
    assert publish_order(keys, {"a": 2}) == [0, 1]
    assert publish_order([], {"a": 1}) == []


def test_random_stream_keeps_per_geometry_order():
    """Random arrivals and completions: every request is published once, in arrival order within
    its geometry, and never more jobs of a geometry than it has replicas."""
    rng = random.Random(7)
    reps = {k: rng.randint(1, 2) for k in range(6)}
    queue, running, published = [], [], []
    rid = 0
    for step in range(3000):
        if rng.random() < 0.6 and rid < 800:
            queue.append((rng.randrange(6), rid))
            rid += 1
        if running and rng.random() < 0.5:
            running.pop(rng.randrange(len(running)))
        busy = {k: sum(1 for kk, _ in running if kk == k) for k in reps}
        idle = {k: reps[k] - busy[k] for k in reps}
        idx = publish_order([k for k, _ in queue], idle)
        for i in idx:
            running.append(queue[i])
            published.append(queue[i])
        for i in reversed(idx):
            queue.pop(i)
        for k in reps:
            assert sum(1 for kk, _ in running if kk == k) <= reps[k]
    for k in reps:
        ids = [r for kk, r in published if kk == k]
        assert ids == sorted(ids)
    assert len({r for _, r in published}) == len(published)
