"""Serving loop: continuous batching of grid-integration requests on one GPU.

A *session* is one geometry (cell, atoms, grid) registered with the server; its handle (radial
tables, grid-brick neighbour lists, atom-pair layout and workspace) stays resident on the device
between requests, so repeated requests on one geometry pay for none of that set-up.  A *request*
is (session, D blocks, V) and returns rho, the local-H blocks and the local Pulay forces (the
three passes of the paper's Sec. 3.3.1) as host arrays.

Scheduling (one scheduler thread):
  * requests wait in a FIFO queue; a batch takes queued requests in order while there is a free
    slot (at most ``max_batch`` systems, one request per session) and their device footprint fits
    the HBM budget, evicting idle resident handles (least recently used) when it would not;
  * up to ``depth`` batches are on the GPU at once: a request that arrives while a batch runs is
    admitted into the next one as soon as slots and memory allow, its inputs are copied on a
    side stream while the running batch computes, and its batch is queued behind it, so the
    device does not idle between batches;
  * each batch is ONE call of gint_run_batch: every system's density/force bricks and local-H
    bricks are items of one persistent launch (plus the per-batch preparation and H-reduction
    launches);
  * a batch's results are read back when its completion event fires and the futures resolve.

The budget counts resident handles (gint_memory) plus the device buffers of admitted requests
(D, V, rho, H, F).  A new geometry's handle is measured when it is created; until then its
footprint is unknown, so creation may exceed the budget by that one handle before idle handles
are evicted.  A request that cannot fit even in an empty server fails with MemoryError.
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
from .admission import Budget, select_batch


# ----------------------------------------------------------------------------------------------
# Sessions, requests, results
# ----------------------------------------------------------------------------------------------
class Session:
    """A geometry registered with a server.  Layout arrays (pair list, block offsets, orbital
    offsets) stay on the host; the handle may be evicted and re-created (same layout)."""

    def __init__(self, server: "Server", key: int, system):
        self.server, self.key, self.system = server, key, system
        self.g: Optional[G.Gint] = None
        self.handle_bytes = 0

    def _create(self):
        self.g = G.Gint(self.system)
        self.handle_bytes = self.g.memory()
        g = self.g
        self.nblock, self.ngrid, self.natoms, self.norb = g.nblock, g.ngrid, g.natoms, g.norb
        self.pair_IJ, self.pair_off, self.atom_off = g.pair_IJ, g.pair_off, g.atom_off
        st = g.stats()
        self.W = st["W"]

    def _drop(self):
        if self.g is not None:
            self.g.close()
            self.g = None

    @property
    def request_bytes(self) -> int:
        """Device bytes of one request's buffers: D, H blocks; V, rho; F."""
        return 8 * (2 * self.nblock + 2 * self.ngrid + 3 * self.natoms)

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
    launch_t: float
    done_t: float
    batch: int
    batch_size: int

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
    dev: Tuple = ()
    host_out: Tuple = ()

    @property
    def key(self) -> int:
        return self.session.key

    @property
    def request_bytes(self) -> int:
        return self.session.request_bytes

    @property
    def handle_bytes(self) -> int:
        return self.session.handle_bytes


@dataclasses.dataclass
class _Batch:
    index: int
    requests: List[_Request]
    event: torch.cuda.Event
    launch_t: float


def _pinned(x) -> torch.Tensor:
    t = torch.as_tensor(x, dtype=torch.float64).reshape(-1)
    return t if t.is_pinned() else t.pin_memory()


# ----------------------------------------------------------------------------------------------
# Server
# ----------------------------------------------------------------------------------------------
class Server:
    """Continuous-batching gint server on one GPU (see the module docstring)."""

    def __init__(self, species: Sequence, budget_bytes: int, precision: int = G.F16X3, max_batch: int = 32,
                 depth: int = 2, device: Optional[torch.device] = None, poll_s: float = 1e-4):
        self.species = list(species)
        self.precision = int(precision)
        self.max_batch = int(max_batch)
        self.depth = int(depth)
        self.device = torch.device(device if device is not None else "cuda")
        self.poll_s = poll_s
        self.budget = Budget(budget_bytes)
        self._sessions: Dict[int, Session] = {}
        self._queue: Deque[_Request] = collections.deque()  # guarded by _cv
        self._inflight: Deque[_Batch] = collections.deque()  # scheduler thread only
        self._cv = threading.Condition(threading.Lock())
        self._state = threading.RLock()  # budget and sessions (scheduler and open())
        self._stop = False
        self._failed: Optional[BaseException] = None  # a CUDA error: the context cannot be used any more
        self._paused = False
        self._nbatch = 0
        self.batch_sizes: List[int] = []
        self.creations = 0  # handles re-created after an eviction
        self.errors: List[BaseException] = []
        with torch.cuda.device(self.device):
            self._compute = torch.cuda.Stream()
            self._copy = torch.cuda.Stream()
            self._check = torch.cuda.Stream()
        self._thread = threading.Thread(target=self._loop, name="gint-serve", daemon=True)
        self._thread.start()

    # -- client API
    def open(self, system) -> Session:
        """Registers a geometry (species indices refer to the server's species list) and makes
        its handle resident now (counted against the budget; idle handles may be evicted)."""
        names = [sp.name for sp in system.sp]
        lib = [sp.name for sp in self.species]
        if names != lib:
            raise ValueError(f"system species {names} differ from the server's list {lib}")
        with self._state:
            key = len(self._sessions)
            s = Session(self, key, system)
            with torch.cuda.device(self.device):
                s._create()
            self._sessions[key] = s
            self.budget.add_resident(key, s.handle_bytes, time.perf_counter())
            self._evict_for(0, protect=(key,))
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
        """Holds new launches (batches already on the GPU complete); requests keep queuing."""
        with self._cv:
            self._paused = True

    def resume(self):
        with self._cv:
            self._paused = False
            self._cv.notify()

    def close(self):
        with self._cv:
            self._paused = False
            self._stop = True
            self._cv.notify()
        self._thread.join()
        with self._state:
            for s in self._sessions.values():
                s._drop()
            self._sessions.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scheduler (everything below runs on the scheduler thread)
    def _evict_for(self, need: int, protect=()) -> bool:
        plan = self.budget.plan(need, protect)
        if plan is None:
            return False
        for key in plan:
            self._sessions[key]._drop()
            self.budget.evict(key)
        return True

    def _admit(self) -> List[_Request]:
        """The next batch (FIFO prefix of the queue, see admission.select_batch)."""
        with self._cv:
            pending = [self._queue[i] for i in range(min(len(self._queue), self.max_batch + 1))]
        with self._state:
            plan = select_batch(pending, self.budget, self.max_batch, bool(self._inflight), time.perf_counter())
            for key in plan.evict:
                self._sessions[key]._drop()
            with torch.cuda.device(self.device):
                for key in plan.create:
                    self._sessions[key]._create()
                    self.creations += 1
        with self._cv:
            for _ in range(plan.consumed):
                self._queue.popleft()
        for r in plan.reject:
            r.future.set_exception(MemoryError(
                f"request needs {r.request_bytes + r.handle_bytes} device bytes; the budget is {self.budget.budget}"))
        return plan.admit

    def _launch(self, reqs: List[_Request]) -> _Batch:
        dev = self.device
        with torch.cuda.device(dev):
            with torch.cuda.stream(self._copy):
                for r in reqs:
                    s = r.session
                    Dd = torch.empty(s.nblock, dtype=torch.float64, device=dev)
                    Vd = torch.empty(s.ngrid, dtype=torch.float64, device=dev)
                    Dd.copy_(r.D, non_blocking=True)
                    Vd.copy_(r.V, non_blocking=True)
                    Dd.record_stream(self._compute)
                    Vd.record_stream(self._compute)
                    r.dev = (Dd, Vd)
                copied = torch.cuda.Event()
                copied.record(self._copy)
            self._compute.wait_event(copied)
            with torch.cuda.stream(self._compute):
                tasks = []
                for r in reqs:
                    s = r.session
                    rho = torch.empty(s.ngrid, dtype=torch.float64, device=dev)
                    H = torch.empty(s.nblock, dtype=torch.float64, device=dev)
                    F = torch.empty((s.natoms, 3), dtype=torch.float64, device=dev)
                    r.dev = r.dev + (rho, H, F)
                    tasks.append(G.Task(s.g, r.dev[0], r.dev[1], rho=rho, H=H, F=F))
                G.run_batch(tasks, self.precision, stream=self._compute)
                for r in reqs:
                    outs = r.dev[2:5]
                    r.host_out = tuple(torch.empty(d.shape, dtype=torch.float64, pin_memory=True) for d in outs)
                    for h, d in zip(r.host_out, outs):
                        h.copy_(d, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self._compute)
        b = _Batch(self._nbatch, reqs, ev, time.perf_counter())
        self._nbatch += 1
        self.batch_sizes.append(len(reqs))
        return b

    def _release(self, r: _Request, now: float):
        r.dev = ()
        with self._state:
            self.budget.release(r.key, r.request_bytes, now)

    def _finish(self, b: _Batch):
        done = time.perf_counter()
        for r in b.requests:
            s = r.session
            try:
                s.g.sync(stream=self._check)  # the handle's device error word (does not wait for later batches)
                rho, H, F = (x.numpy() for x in r.host_out)
                r.future.set_result(Result(rho.reshape(s.system.grid), H, F, r.submit_t, b.launch_t, done, b.index,
                                           len(b.requests)))
            except BaseException as e:  # noqa: BLE001 - delivered to the caller's future
                self.errors.append(e)
                r.future.set_exception(e)
            r.host_out = ()
            self._release(r, done)

    def _loop(self):
        try:
            self._serve()
        except BaseException as e:  # noqa: BLE001 - e.g. a CUDA error: fail everything still pending
            self.errors.append(e)
            with self._cv:
                self._failed = e
                pending = list(self._queue)
                self._queue.clear()
            for b in self._inflight:
                pending += b.requests
            self._inflight.clear()
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(e)

    def _serve(self):
        while True:
            while self._inflight and self._inflight[0].event.query():
                self._finish(self._inflight.popleft())
            with self._cv:
                if self._stop and not self._queue and not self._inflight:
                    return
                ready = bool(self._queue) and len(self._inflight) < self.depth and not self._paused
                if not ready:
                    self._cv.wait(self.poll_s if self._inflight else 0.05)
                    continue
            reqs = self._admit()
            if not reqs:
                time.sleep(self.poll_s)  # memory is held by batches on the GPU
                continue
            try:
                self._inflight.append(self._launch(reqs))
            except BaseException as e:  # noqa: BLE001 - fail this batch, keep serving
                self.errors.append(e)
                now = time.perf_counter()
                for r in reqs:
                    r.future.set_exception(e)
                    self._release(r, now)


def percentiles(latencies_ms: Sequence[float]) -> Dict[str, float]:
    a = np.asarray(latencies_ms, dtype=np.float64)
    if a.size == 0:
        return dict(p50=float("nan"), p99=float("nan"), mean=float("nan"), max=float("nan"))
    return dict(p50=float(np.percentile(a, 50)), p99=float(np.percentile(a, 99)), mean=float(a.mean()),
                max=float(a.max()))
