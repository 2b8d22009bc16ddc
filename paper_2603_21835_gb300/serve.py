"""Serving loop: continuous batching of grid-integration requests on one GPU.

A *session* is one geometry (cell, atoms, grid) registered with the server.  Its *replicas* are
library handles (radial tables, grid-brick neighbour lists, atom-pair layout, workspace) with their
own device input/output buffers; they stay resident between requests, so repeated requests on one
geometry pay for none of that set-up.  A *request* is (session, D blocks, V) and returns rho, the
local-H blocks and the local Pulay forces (the three passes of the paper's Sec. 3.3.1) as host
arrays.

The GPU side is the library's device work queue (gint_server_*): ONE resident launch of the brick
kernels drains a queue of jobs, and a job published while others are on the GPU starts as soon as
CTAs free up, in the same residency, its items interleaving with theirs.  The host side here (one
scheduler thread) decides what to publish:
  * requests wait in a FIFO queue; the scheduler publishes a request as soon as its session has an
    idle replica (a replica runs one job at a time: its workspace is the job's), overtaking earlier
    requests only of other sessions, so each session's requests run in arrival order;
  * publishing a request = copying D and V into the replica's device buffers (copy stream) and
    submitting the job; at most 64 jobs are in flight;
  * when a job's completion word arrives, its outputs are copied to pinned host memory and its
    future resolves; the replica is idle again.
Device memory is counted against the HBM budget per replica (gint_memory of the handle plus its
input/output buffers).  A session without a resident replica (evicted earlier) gets one re-created
when it is next needed: the queue is drained first (handle creation and release synchronise the
device), idle replicas are evicted least recently used first until it fits, and a request that
cannot fit even on an empty server fails with MemoryError.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future
from typing import Deque, Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import gint as G
from .admission import Budget, publish_order


# ----------------------------------------------------------------------------------------------
# Sessions, replicas, requests, results
# ----------------------------------------------------------------------------------------------
class Replica:
    """One resident handle of a session with its device buffers and pinned host outputs."""

    def __init__(self, session: "Session", index: int, device: torch.device):
        self.session, self.index = session, index
        self.g = G.Gint(session.system)
        s = session
        self.D = torch.empty(s.nblock, dtype=torch.float64, device=device)
        self.V = torch.empty(s.ngrid, dtype=torch.float64, device=device)
        self.rho = torch.empty(s.ngrid, dtype=torch.float64, device=device)
        self.H = torch.empty(s.nblock, dtype=torch.float64, device=device)
        self.F = torch.empty((s.natoms, 3), dtype=torch.float64, device=device)
        self.nbytes = self.g.memory() + s.request_bytes
        self.busy = False

    @property
    def key(self) -> Tuple[int, int]:
        return (self.session.key, self.index)

    def drop(self):
        self.g.close()
        self.D = self.V = self.rho = self.H = self.F = None


class Session:
    """A geometry registered with a server.  Layout arrays (pair list, block offsets, orbital
    offsets) stay on the host; replicas may be evicted and re-created (same layout)."""

    def __init__(self, server: "Server", key: int, system):
        self.server, self.key, self.system = server, key, system
        self.replicas: Dict[int, Replica] = {}
        g = G.Gint(system)
        self.nblock, self.ngrid, self.natoms, self.norb = g.nblock, g.ngrid, g.natoms, g.norb
        self.pair_IJ, self.pair_off, self.atom_off = g.pair_IJ, g.pair_off, g.atom_off
        self.W = g.stats()["W"]
        self.handle_bytes = g.memory()
        g.close()

    @property
    def request_bytes(self) -> int:
        """Device bytes of one replica's input/output buffers: D, H blocks; V, rho; F."""
        return 8 * (2 * self.nblock + 2 * self.ngrid + 3 * self.natoms)

    @property
    def replica_bytes(self) -> int:
        return self.handle_bytes + self.request_bytes

    def blocks_from_coefficients(self, C: np.ndarray) -> np.ndarray:
        """D = C C^T in this session's block layout (host, no dense D)."""
        out = np.empty(self.nblock, dtype=np.float64)
        ao = self.atom_off
        starts = np.searchsorted(self.pair_IJ[:, 0], np.arange(self.natoms + 1))
        for I in range(self.natoms):
            p0, p1 = starts[I], starts[I + 1]
            Js = self.pair_IJ[p0:p1, 1]
            rows = np.concatenate([np.arange(ao[J], ao[J + 1]) for J in Js])
            blk = C[ao[I]:ao[I + 1]] @ C[rows].T
            col = 0
            for q, J in enumerate(Js):
                nJ = ao[J + 1] - ao[J]
                out[self.pair_off[p0 + q]:self.pair_off[p0 + q + 1]] = blk[:, col:col + nJ].reshape(-1)
                col += nJ
        return out


@dataclasses.dataclass
class Result:
    rho: np.ndarray
    H: np.ndarray
    F: np.ndarray
    submit_t: float
    launch_t: float   # published to the device queue
    done_t: float
    concurrency: int  # jobs in flight (this one included) when it was published

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.done_t - self.submit_t)


@dataclasses.dataclass
class _Request:
    session: Session
    D: torch.Tensor  # pinned host
    V: torch.Tensor  # pinned host
    future: Future
    submit_t: float
    replica: Optional[Replica] = None
    ticket: int = -1
    launch_t: float = 0.0
    concurrency: int = 0
    copied: Optional[torch.cuda.Event] = None
    host: Tuple = ()  # pinned host outputs (the result's arrays: no copy on the host)


def _pinned(x) -> torch.Tensor:
    t = torch.as_tensor(x, dtype=torch.float64).reshape(-1)
    return t if t.is_pinned() else t.pin_memory()


# ----------------------------------------------------------------------------------------------
# Server
# ----------------------------------------------------------------------------------------------
class Server:
    """Continuous-batching gint server on one GPU (see the module docstring)."""

    def __init__(self, species: Sequence, budget_bytes: int, precision: int = G.F16X3, replicas: int = 1,
                 device: Optional[torch.device] = None, idle_s: float = 0.2, poll_s: float = 5e-5):
        self.species = list(species)
        self.precision = int(precision)
        self.replicas = max(1, int(replicas))
        self.device = torch.device(device if device is not None else "cuda")
        self.poll_s = poll_s
        self.budget = Budget(budget_bytes)
        self._sessions: Dict[int, Session] = {}
        self._queue: Deque[_Request] = collections.deque()  # guarded by _cv
        self._inflight: List[_Request] = []   # published jobs (scheduler thread only)
        self._draining: List[_Request] = []   # completed jobs whose outputs are being copied
        self._cv = threading.Condition(threading.Lock())
        self._state = threading.RLock()
        self._stop = False
        self._paused = False
        self._failed: Optional[BaseException] = None
        self.creations = 0  # replicas re-created after an eviction
        self.concurrency: List[int] = []  # jobs in flight at each publication
        self.errors: List[BaseException] = []
        with torch.cuda.device(self.device):
            self._copy = torch.cuda.Stream()
            self.queue = G.DeviceQueue(self.precision, forces=True, idle_s=idle_s)
        self._thread = threading.Thread(target=self._loop, name="gint-serve", daemon=True)
        self._thread.start()

    # -- client API
    def open(self, system) -> Session:
        """Registers a geometry (species indices refer to the server's species list) and makes its
        replicas resident now (counted against the budget; idle replicas may be evicted)."""
        names = [sp.name for sp in system.sp]
        lib = [sp.name for sp in self.species]
        if names != lib:
            raise ValueError(f"system species {names} differ from the server's list {lib}")
        with self._state:
            with torch.cuda.device(self.device):
                key = len(self._sessions)
                s = Session(self, key, system)
                self._sessions[key] = s
                for r in range(self.replicas):
                    self._make_replica(s, r, protect=())
        return s

    def submit(self, session: Session, D_blocks, V) -> Future:
        """Queues rho + H + F of `session` for D (blocks) and V (grid) given as host arrays or CPU
        tensors (pinned here if they are not); returns a Future[Result]."""
        t = time.perf_counter()
        D, Vp = _pinned(D_blocks), _pinned(V)
        if D.numel() != session.nblock or Vp.numel() != session.ngrid:
            raise ValueError("D or V does not match the session's layout")
        fut: Future = Future()
        with self._cv:
            if self._failed is not None:
                raise RuntimeError("server stopped after a device error") from self._failed
            if self._stop:
                raise RuntimeError("server is closed")
            self._queue.append(_Request(session, D, Vp, fut, t))
            self._cv.notify()
        return fut

    def pause(self):
        """Holds new publications (jobs already on the GPU complete); requests keep queuing."""
        with self._cv:
            self._paused = True

    def resume(self):
        with self._cv:
            self._paused = False
            self._cv.notify()

    def stats(self) -> dict:
        with self._state:
            q = self.queue.stats()
        c = np.asarray(self.concurrency) if self.concurrency else np.zeros(1)
        return dict(resident_launches=q["launches"], jobs=q["jobs"], mean_concurrency=float(c.mean()),
                    max_concurrency=int(c.max()))

    def close(self):
        with self._cv:
            self._paused = False
            self._stop = True
            self._cv.notify()
        self._thread.join()
        with self._state:
            self.queue.close()
            for s in self._sessions.values():
                for r in list(s.replicas.values()):
                    r.drop()
                s.replicas.clear()
            self._sessions.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- replicas and memory (scheduler thread, or open())
    def _make_replica(self, s: Session, index: int, protect) -> bool:
        """Evicts idle replicas (LRU) until one more of `s` fits, then creates it; False if it cannot
        fit.  Creating and releasing handles synchronise the device: the queue is drained first."""
        need = s.replica_bytes
        plan = self.budget.plan(need, protect)
        if plan is None:
            return False
        self.queue.stop()
        for key in plan:
            sk, ri = key
            self._sessions[sk].replicas.pop(ri).drop()
            self.budget.evict(key)
        r = Replica(s, index, self.device)
        s.replicas[index] = r
        self.budget.add_resident(r.key, r.nbytes, time.perf_counter())
        return True

    # -- scheduler (everything below runs on the scheduler thread)
    def _publish(self, req: _Request, r: Replica):
        req.replica = r
        r.busy = True
        now = time.perf_counter()
        with self._state:  # the queue and the budget are shared with open()
            self.budget.acquire(r.key, 0)
            with torch.cuda.device(self.device), torch.cuda.stream(self._copy):
                r.D.copy_(req.D, non_blocking=True)
                r.V.copy_(req.V, non_blocking=True)
            ticket = self.queue.submit(G.Task(r.g, r.D, r.V, rho=r.rho, H=r.H, F=r.F), stream=self._copy)
            if ticket is None:  # the queue's ring is full: try again later
                r.busy = False
                self.budget.release(r.key, 0, now)
                req.replica = None
                return False
        req.ticket, req.launch_t = ticket, now
        req.host = tuple(torch.empty(t.shape, dtype=torch.float64, pin_memory=True) for t in (r.rho, r.H, r.F))
        req.concurrency = len(self._inflight) + 1
        self.concurrency.append(req.concurrency)
        self._inflight.append(req)
        return True

    def _admit(self):
        """Publishes queued requests whose geometry has an idle replica (admission.publish_order),
        re-creating a replica first for a geometry that has none resident."""
        with self._cv:
            if self._paused:
                return
            pending = list(self._queue)
        if not pending:
            return
        taken = []
        for s in {req.session.key: req.session for req in pending}.values():
            if s.replicas:
                continue
            with self._state:  # evicted earlier: re-create one replica
                busy = tuple(x.key for ss in self._sessions.values() for x in ss.replicas.values() if x.busy)
                if self._make_replica(s, 0, protect=busy):
                    self.creations += 1
                elif not busy:
                    err = MemoryError(f"request needs {s.replica_bytes} device bytes; the budget is "
                                      f"{self.budget.budget}")
                    for req in pending:
                        if req.session is s:
                            req.future.set_exception(err)
                            taken.append(req)
        pending = [req for req in pending if req not in taken]
        idle = {s.key: [x for x in s.replicas.values() if not x.busy] for s in {r.session for r in pending}}
        for i in publish_order([req.session.key for req in pending], {k: len(v) for k, v in idle.items()}):
            req = pending[i]
            if not self._publish(req, idle[req.session.key].pop(0)):
                break  # the queue's ring is full
            taken.append(req)
        if taken:
            with self._cv:
                for req in taken:
                    self._queue.remove(req)

    def _collect(self):
        for req in list(self._inflight):
            with self._state:
                finished = self.queue.done(req.ticket)
            if finished:
                self._inflight.remove(req)
                r = req.replica
                with torch.cuda.device(self.device), torch.cuda.stream(self._copy):
                    for h, d in zip(req.host, (r.rho, r.H, r.F)):
                        h.copy_(d, non_blocking=True)
                    req.copied = torch.cuda.Event()
                    req.copied.record(self._copy)
                self._draining.append(req)
        for req in list(self._draining):
            if req.copied.query():
                self._draining.remove(req)
                r, s = req.replica, req.session
                done = time.perf_counter()
                try:
                    r.g.sync(stream=self._copy)  # the handle's device error word
                    rho, H, F = (x.numpy() for x in req.host)
                    req.future.set_result(Result(rho.reshape(s.system.grid), H, F, req.submit_t, req.launch_t, done,
                                                 req.concurrency))
                except BaseException as e:  # noqa: BLE001 - delivered to the caller's future
                    self.errors.append(e)
                    req.future.set_exception(e)
                r.busy = False
                with self._state:
                    self.budget.release(r.key, 0, done)

    def _loop(self):
        try:
            self._serve()
        except BaseException as e:  # noqa: BLE001 - e.g. a CUDA error: fail everything still pending
            self.errors.append(e)
            with self._cv:
                self._failed = e
                pending = list(self._queue)
                self._queue.clear()
            pending += self._inflight + self._draining
            self._inflight, self._draining = [], []
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(e)

    def _serve(self):
        while True:
            self._collect()
            with self._cv:
                if self._stop and not self._queue and not self._inflight and not self._draining:
                    return
                idle = not self._queue and not self._inflight and not self._draining
                if idle:
                    self._cv.wait(0.05)
                    continue
            self._admit()
            time.sleep(self.poll_s)


def percentiles(latencies_ms: Sequence[float]) -> Dict[str, float]:
    a = np.asarray(latencies_ms, dtype=np.float64)
    if a.size == 0:
        return dict(p50=float("nan"), p99=float("nan"), mean=float("nan"), max=float("nan"))
    return dict(p50=float(np.percentile(a, 50)), p99=float(np.percentile(a, 99)), mean=float(a.mean()),
                max=float(a.max()))
