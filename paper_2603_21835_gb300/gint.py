"""ctypes binding of libgint (the C ABI declared in include/gint.h).

Argument marshalling only: every step of the density, local-Hamiltonian and force
passes runs in the CUDA library.  PyTorch provides device memory and streams.
Importing this module fails loudly if libgint.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgint.so")

FP64, FP32, F16X3, F16X1 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "f16x3": F16X3, "f16x1": F16X1}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgint.so is not built ({LIB_PATH}); run `python -m paper_2603_21835_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)


class GintError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.gint_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class _Radial(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("npts", ctypes.c_int), ("dr", ctypes.c_double), ("rc", ctypes.c_double),
                ("f", ctypes.c_void_p), ("df", ctypes.c_void_p)]


class _Species(ctypes.Structure):
    _fields_ = [("nradial", ctypes.c_int), ("radial", ctypes.POINTER(_Radial))]


class _Desc(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_double * 9), ("natoms", ctypes.c_int), ("pos", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("nspecies", ctypes.c_int), ("sp", ctypes.POINTER(_Species)),
                ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int), ("skin", ctypes.c_double)]


class _Task(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("D_blocks", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("H_blocks", ctypes.c_void_p), ("F", ctypes.c_void_p)]


_vp, _ll, _i, _d = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_double
_lib.gint_strerror.restype = ctypes.c_char_p
_lib.gint_strerror.argtypes = [_i]
_lib.gint_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_vp)]
_lib.gint_destroy.argtypes = [_vp]
_lib.gint_layout.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_ll)]
_lib.gint_pairs.argtypes = [_vp, _vp, _vp]
_lib.gint_stats.argtypes = [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_ll), ctypes.POINTER(_i),
                            ctypes.POINTER(_i)]
_lib.gint_set_positions.argtypes = [_vp, _vp, _vp]
_lib.gint_rho.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.gint_vlocal.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.gint_force.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp]
_lib.gint_grid_dot.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.gint_block_dot.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.gint_weight.restype = _d
_lib.gint_weight.argtypes = [_vp]
_lib.gint_sync.argtypes = [_vp, _vp]
_lib.gint_tc_selftest.argtypes = [_i, ctypes.POINTER(_d)]
_lib.gint_grid_dot_noalloc.argtypes = [_vp, _vp, _ll, _d, _vp, _vp]
_lib.gint_run_batch.argtypes = [ctypes.POINTER(_Task), _i, _i, _vp]
_lib.gint_run_batch_timed.argtypes = [ctypes.POINTER(_Task), _i, _i, _vp, _vp, _vp]
_lib.gint_memory.argtypes = [_vp, ctypes.POINTER(_ll)]
_lib.gint_set_reduction.argtypes = [_vp, _i]
_lib.gint_layout_R.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_ll), ctypes.POINTER(ctypes.POINTER(_i)),
                               ctypes.POINTER(ctypes.POINTER(_ll))]
_lib.gint_vlocal_R.argtypes = [_vp, _i, _vp, _vp, _vp]
_lib.gint_bloch.argtypes = [_vp, _vp, _i, _vp, _vp, _vp]
_lib.gint_set_projectors.argtypes = [_vp, _i, _vp]
_lib.gint_psibeta_layout.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_ll), ctypes.POINTER(ctypes.POINTER(_i)),
                                     ctypes.POINTER(ctypes.POINTER(_ll))]
_lib.gint_psibeta.argtypes = [_vp, _vp, _vp, _vp]
_lib.gint_cn_create.argtypes = [_i, _i, ctypes.POINTER(_vp)]
_lib.gint_cn_destroy.argtypes = [_vp]
_lib.gint_cn_step.argtypes = [_vp, _vp, _vp, _d, _vp, _vp, _vp]
_lib.gint_dm_build.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.gint_dm_build_f16x3.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.gint_cn_info.argtypes = [_vp, ctypes.POINTER(_i)]
_lib.gint_edm.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.gint_brick_lists.argtypes = [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll), _vp, _vp, _vp, _vp]
_lib.gint_server_create.argtypes = [_i, _i, _d, ctypes.POINTER(_vp)]
_lib.gint_server_submit.argtypes = [_vp, ctypes.POINTER(_Task), _vp, ctypes.POINTER(_ll)]
_lib.gint_server_test.argtypes = [_vp, _ll, ctypes.POINTER(_i)]
_lib.gint_server_stats.argtypes = [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]
_lib.gint_server_stop.argtypes = [_vp]
_lib.gint_server_destroy.argtypes = [_vp]
_lib.gint_orbitals.argtypes = [_vp, _i, _ll, _vp, _vp, _vp]

C_ABI_SYMBOLS = ("gint_create", "gint_destroy", "gint_layout", "gint_pairs", "gint_stats", "gint_set_positions",
                 "gint_rho", "gint_vlocal", "gint_force", "gint_grid_dot", "gint_block_dot", "gint_weight",
                 "gint_strerror", "gint_sync", "gint_tc_selftest", "gint_grid_dot_noalloc", "gint_run_batch",
                 "gint_run_batch_timed", "gint_memory", "gint_set_reduction", "gint_layout_R", "gint_vlocal_R", "gint_bloch",
                 "gint_set_projectors", "gint_psibeta_layout", "gint_psibeta", "gint_cn_create", "gint_cn_destroy",
                 "gint_cn_step", "gint_dm_build", "gint_dm_build_f16x3", "gint_cn_info", "gint_edm",
                 "gint_brick_lists", "gint_orbitals", "gint_server_create", "gint_server_submit", "gint_server_test",
                 "gint_server_stats", "gint_server_stop", "gint_server_destroy")


class CrankNicolson:
    """Density-matrix build and Crank-Nicolson steps for n x n matrices and nocc states on the current
    GPU (buffers held by the context).  States are rows of a complex128 [nocc, n] tensor."""

    def __init__(self, n: int, nocc: int):
        c = _vp()
        _check(_lib.gint_cn_create(int(n), int(nocc), ctypes.byref(c)), "gint_cn_create")
        self._c, self.n, self.nocc = c, int(n), int(nocc)

    def _cplx(self, psi: torch.Tensor):
        if psi.dtype != torch.complex128 or not psi.is_cuda or not psi.is_contiguous() or \
                tuple(psi.shape) != (self.nocc, self.n):
            raise ValueError(f"expected a contiguous CUDA complex128 tensor [{self.nocc}, {self.n}]")
        return ctypes.c_void_p(psi.data_ptr())

    def step(self, S: torch.Tensor, H: torch.Tensor, dt: float, psi: torch.Tensor,
             out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """(S + i dt/2 H)^{-1} (S - i dt/2 H) psi."""
        if out is None:
            out = torch.empty_like(psi)
        nn = self.n * self.n
        _check(_lib.gint_cn_step(self._c, _dptr(S, numel=nn), _dptr(H, numel=nn), float(dt), self._cplx(psi),
                                 self._cplx(out), _stream(stream)), "gint_cn_step")
        return out

    def density_matrix(self, psi: torch.Tensor, f: torch.Tensor, out: Optional[torch.Tensor] = None,
                       stream=None, precision: str = "fp64") -> torch.Tensor:
        """Re(psi^T diag(f) conj(psi)) as [n, n] float64 (rows of psi are the states); precision "fp64"
        (complex float64 GEMM) or "f16x3" (tensor cores, float16 three-term split)."""
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float64, device=psi.device)
        fn = {"fp64": _lib.gint_dm_build, "f16x3": _lib.gint_dm_build_f16x3}[precision]
        _check(fn(self._c, self._cplx(psi), _dptr(f, numel=self.nocc), _dptr(out, numel=self.n * self.n),
                  _stream(stream)), "gint_dm_build")
        return out

    def energy_density_matrix(self, S: torch.Tensor, H: torch.Tensor, D: torch.Tensor,
                              out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """(S^{-1} H D + D H S^{-1}) / 2 as [n, n] float64."""
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float64, device=S.device)
        nn = self.n * self.n
        _check(_lib.gint_edm(self._c, _dptr(S, numel=nn), _dptr(H, numel=nn), _dptr(D, numel=nn),
                             _dptr(out, numel=nn), _stream(stream)), "gint_edm")
        return out

    def info(self) -> int:
        i = _i()
        _check(_lib.gint_cn_info(self._c, ctypes.byref(i)), "gint_cn_info")
        return i.value

    def close(self):
        if self._c:
            _lib.gint_cn_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_selftest(n: int = 256) -> float:
    """Largest deviation of one tcgen05 f16 MMA (M=128, N=n, K=16, integer data) from exact,
    over the three shared-memory operand layouts the brick kernels use."""
    e = _d()
    _check(_lib.gint_tc_selftest(int(n), ctypes.byref(e)), "gint_tc_selftest")
    return e.value


def _check(code: int, where: str):
    if code != 0:
        raise GintError(code, where)


def _dptr(t: Optional[torch.Tensor], dtype=torch.float64, numel: Optional[int] = None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Task:
    """The passes of one system in a batch: outputs left as None are not computed (see gint_task)."""
    g: "Gint"
    D: Optional[torch.Tensor] = None     # D blocks [nblock]
    V: Optional[torch.Tensor] = None     # potential [ngrid]
    rho: Optional[torch.Tensor] = None   # out: density [ngrid]
    H: Optional[torch.Tensor] = None     # out: local-H blocks [nblock]
    F: Optional[torch.Tensor] = None     # out: forces [natoms, 3]


def run_batch(tasks: Sequence[Task], precision: int = F16X3, stream=None, kernel_events=None) -> None:
    """All tasks' bricks in one persistent launch (tensor-core precisions; up to 32 systems per
    launch), asynchronous on `stream`.  kernel_events: optional (start, stop) torch.cuda.Event
    pair recorded around the brick kernel(s) (they must have been recorded once before, so that
    the CUDA events exist)."""
    arr = (_Task * max(len(tasks), 1))()
    for i, t in enumerate(tasks):
        g = t.g
        arr[i] = _Task(g._h, _dptr(t.D, numel=g.nblock), _dptr(t.V, numel=g.ngrid), _dptr(t.rho, numel=g.ngrid),
                       _dptr(t.H, numel=g.nblock), _dptr(t.F, numel=3 * g.natoms))
    if kernel_events is None:
        _check(_lib.gint_run_batch(arr, len(tasks), int(precision), _stream(stream)), "gint_run_batch")
    else:
        e0, e1 = (ctypes.c_void_p(e.cuda_event) for e in kernel_events)
        if not e0.value or not e1.value:
            raise ValueError("kernel_events must have been recorded once (CUDA events are created lazily)")
        _check(_lib.gint_run_batch_timed(arr, len(tasks), int(precision), _stream(stream), e0, e1),
               "gint_run_batch_timed")


EBUSY = -9


class DeviceQueue:
    """The library's continuous-batching server (gint_server_*): one resident launch of the brick
    kernels drains a device work queue; jobs (Task) are published while it runs."""

    def __init__(self, precision: int = F16X3, forces: bool = True, idle_s: float = 0.2):
        q = _vp()
        _check(_lib.gint_server_create(int(precision), 1 if forces else 0, float(idle_s), ctypes.byref(q)),
               "gint_server_create")
        self._q = q

    def submit(self, t: Task, stream=None) -> Optional[int]:
        """Publishes the task (its D and V complete in order on `stream`); the ticket, or None when the
        queue is full or the task's handle has a job in flight (GINT_EBUSY)."""
        g = t.g
        arr = _Task(g._h, _dptr(t.D, numel=g.nblock), _dptr(t.V, numel=g.ngrid), _dptr(t.rho, numel=g.ngrid),
                    _dptr(t.H, numel=g.nblock), _dptr(t.F, numel=3 * g.natoms))
        tk = _ll()
        rc = _lib.gint_server_submit(self._q, ctypes.byref(arr), _stream(stream), ctypes.byref(tk))
        if rc == EBUSY:
            return None
        _check(rc, "gint_server_submit")
        return tk.value

    def done(self, ticket: int) -> bool:
        d = _i()
        _check(_lib.gint_server_test(self._q, int(ticket), ctypes.byref(d)), "gint_server_test")
        return bool(d.value)

    def stats(self) -> dict:
        la, jo = _ll(), _ll()
        _check(_lib.gint_server_stats(self._q, ctypes.byref(la), ctypes.byref(jo)), "gint_server_stats")
        return dict(launches=la.value, jobs=jo.value)

    def stop(self):
        _check(_lib.gint_server_stop(self._q), "gint_server_stop")

    def close(self):
        if getattr(self, "_q", None):
            _lib.gint_server_destroy(self._q)
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _species_array(species_list):
    """gint_species[] (and the arrays it points into, which must stay alive) from Species records."""
    keep, sp_arr = [], (_Species * len(species_list))()
    for s, sp in enumerate(species_list):
        arr = (_Radial * max(len(sp.radials), 1))()
        for k, r in enumerate(sp.radials):
            f = np.ascontiguousarray(r.f, dtype=np.float64)
            df = np.ascontiguousarray(r.df, dtype=np.float64)
            keep += [f, df]
            arr[k] = _Radial(int(r.l), int(f.shape[0]), float(r.dr), float(r.rc), f.ctypes.data, df.ctypes.data)
        keep.append(arr)
        sp_arr[s] = _Species(len(sp.radials), arr)
    return sp_arr, keep


class Gint:
    """One geometry (cell, atoms, species radial tables, grid) resident on the current GPU."""

    def __init__(self, system, skin: float = 0.0):
        sp_arr, rad_keep = _species_array(system.sp)
        pos = np.ascontiguousarray(system.pos, dtype=np.float64)
        spc = np.ascontiguousarray(system.species, dtype=np.int32)
        d = _Desc()
        d.cell[:] = [float(x) for x in np.asarray(system.cell, dtype=np.float64).reshape(-1)]
        d.natoms, d.pos, d.species = int(pos.shape[0]), pos.ctypes.data, spc.ctypes.data
        d.nspecies, d.sp = len(system.sp), sp_arr
        d.n1, d.n2, d.n3 = (int(x) for x in system.grid)
        d.skin = float(skin)
        h = ctypes.c_void_p()
        _check(_lib.gint_create(ctypes.byref(d), ctypes.byref(h)), "gint_create")
        self._h = h
        self.grid = tuple(int(x) for x in system.grid)
        self.ngrid = int(np.prod(self.grid))
        self.natoms = int(pos.shape[0])
        norb, npairs, nblock = _i(), _i(), _ll()
        _check(_lib.gint_layout(h, ctypes.byref(norb), ctypes.byref(npairs), ctypes.byref(nblock)), "gint_layout")
        self.norb, self.npairs, self.nblock = norb.value, npairs.value, nblock.value
        self.pair_IJ = np.zeros((self.npairs, 2), dtype=np.int32)
        self.pair_off = np.zeros(self.npairs + 1, dtype=np.int64)
        _check(_lib.gint_pairs(h, self.pair_IJ.ctypes.data, self.pair_off.ctypes.data), "gint_pairs")
        norbs = np.array([sum(2 * r.l + 1 for r in system.sp[s].radials) for s in system.species], dtype=np.int64)
        self.atom_norb = norbs
        self.atom_off = np.concatenate([[0], np.cumsum(norbs)]).astype(np.int64)
        self.weight = float(_lib.gint_weight(h))
        self._pos_host = pos.copy()
        self._pos_dev = None

    # -- bookkeeping
    def stats(self) -> dict:
        W, Wx, nb, mo, ma = _d(), _d(), _ll(), _i(), _i()
        _check(_lib.gint_stats(self._h, ctypes.byref(W), ctypes.byref(Wx), ctypes.byref(nb), ctypes.byref(mo),
                               ctypes.byref(ma)), "gint_stats")
        return dict(W=W.value, W_exec=Wx.value, nbricks=nb.value, max_brick_orb=mo.value, max_brick_atoms=ma.value)

    def brick_lists(self):
        """The grid-brick -> atom neighbour lists (host copies): b_off [nbricks + 1], slot_atom [nslots],
        slot_ent [nslots + 1], ent_pos [nentries, 3] (Cartesian tau_I + R of each entry)."""
        ns, ne = _ll(), _ll()
        _check(_lib.gint_brick_lists(self._h, ctypes.byref(ns), ctypes.byref(ne), None, None, None, None),
               "gint_brick_lists")
        nb = self.stats()["nbricks"]
        b_off = np.zeros(nb + 1, dtype=np.int64)
        atom = np.zeros(max(ns.value, 1), dtype=np.int32)
        ent = np.zeros(ns.value + 1, dtype=np.int64)
        epos = np.zeros((max(ne.value, 1), 3))
        _check(_lib.gint_brick_lists(self._h, ctypes.byref(ns), ctypes.byref(ne), b_off.ctypes.data, atom.ctypes.data,
                                     ent.ctypes.data, epos.ctypes.data), "gint_brick_lists")
        return b_off, atom[:ns.value], ent, epos[:ne.value]

    def orbitals(self, pts: np.ndarray, precision: int = FP64):
        """Periodised orbitals and gradients at the points [n, 3] by the kernels' evaluators (FP64 or
        F16X3): (phi [n, norb], grad [n, norb, 3])."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        phi = np.zeros((n, self.norb))
        grad = np.zeros((n, self.norb, 3))
        _check(_lib.gint_orbitals(self._h, int(precision), n, pts.ctypes.data, phi.ctypes.data, grad.ctypes.data),
               "gint_orbitals")
        return phi, grad

    def memory(self) -> int:
        """Device bytes held by the handle (tables, neighbour lists, workspace)."""
        b = _ll()
        _check(_lib.gint_memory(self._h, ctypes.byref(b)), "gint_memory")
        return b.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.gint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- compute (device tensors in, device tensors out)
    def rho(self, D_blocks: torch.Tensor, precision: int = FP64, out: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.grid, dtype=torch.float64, device=D_blocks.device)
        _check(_lib.gint_rho(self._h, int(precision), _dptr(D_blocks, numel=self.nblock),
                             _dptr(out, numel=self.ngrid), _stream(stream)), "gint_rho")
        return out

    def vlocal(self, V: torch.Tensor, precision: int = FP64, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.nblock, dtype=torch.float64, device=V.device)
        _check(_lib.gint_vlocal(self._h, int(precision), _dptr(V, numel=self.ngrid), _dptr(out, numel=self.nblock),
                                _stream(stream)), "gint_vlocal")
        return out

    def set_reduction(self, mode: str):
        """Cross-brick sums of the tensor-core local-H pass: "double-float" (default: float32 hi + lo
        pairs combined in float64) or "fp64" (every tile value added in float64)."""
        code = {"double-float": 0, "fp64": 1}[mode]
        _check(_lib.gint_set_reduction(self._h, code), "gint_set_reduction")

    def layout_R(self):
        """Keys of the local H per lattice vector (paper Sec. 2, H(R)): (keys [nkeys, 5] int32 rows
        (I, J, n1, n2, n3) with R = n1 a1 + n2 a2 + n3 a3, sorted; key_off [nkeys + 1] element offsets
        of the norb(I) x norb(J) row-major blocks).  Where some brick sees two images of one atom, the
        library computes H(R) on an unfolded twin of the handle (built here on first use)."""
        nk, nel = _i(), _ll()
        kp, op = ctypes.POINTER(_i)(), ctypes.POINTER(_ll)()
        _check(_lib.gint_layout_R(self._h, ctypes.byref(nk), ctypes.byref(nel), ctypes.byref(kp), ctypes.byref(op)),
               "gint_layout_R")
        keys = np.ctypeslib.as_array(kp, shape=(nk.value * 5,)).reshape(-1, 5).copy() if nk.value else \
            np.zeros((0, 5), np.int32)
        off = np.ctypeslib.as_array(op, shape=(nk.value + 1,)).copy()
        self.nblock_R = int(nel.value)
        return keys, off

    def vlocal_R(self, V: torch.Tensor, precision: int = F16X3, out: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
        """H(R) blocks (float64, device) in the layout of layout_R (tensor-core precisions)."""
        if not hasattr(self, "nblock_R"):
            self.layout_R()
        if out is None:
            out = torch.empty(self.nblock_R, dtype=torch.float64, device=V.device)
        _check(_lib.gint_vlocal_R(self._h, int(precision), _dptr(V, numel=self.ngrid),
                                  _dptr(out, numel=self.nblock_R), _stream(stream)), "gint_vlocal_R")
        return out

    def bloch(self, H_R: torch.Tensor, kfrac, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """H(k) = sum_R e^{ik.R} H(R) in the Gamma block layout (complex128, device); kfrac is one k
        ([3]) or several ([nk, 3]) in reciprocal-lattice units; the result is [nblock] or [nk, nblock]."""
        if not hasattr(self, "nblock_R"):
            self.layout_R()
        kf = np.ascontiguousarray(np.asarray(kfrac, dtype=np.float64))
        single = kf.ndim == 1
        kf = kf.reshape(-1, 3)
        nk = kf.shape[0]
        if out is None:
            out = torch.empty(nk * 2 * self.nblock, dtype=torch.float64, device=H_R.device)
        _check(_lib.gint_bloch(self._h, _dptr(H_R, numel=self.nblock_R), nk, kf.ctypes.data,
                               _dptr(out, numel=nk * 2 * self.nblock), _stream(stream)), "gint_bloch")
        z = torch.view_as_complex(out.view(nk, self.nblock, 2))
        return z[0] if single else z

    def set_projectors(self, species_list):
        """Nonlocal projector radials per species (Species records, same order as the system's)."""
        sp_arr, keep = _species_array(species_list)
        _check(_lib.gint_set_projectors(self._h, len(species_list), ctypes.cast(sp_arr, _vp)), "gint_set_projectors")
        n, ne = _i(), _ll()
        pp, op = ctypes.POINTER(_i)(), ctypes.POINTER(_ll)()
        _check(_lib.gint_psibeta_layout(self._h, ctypes.byref(n), ctypes.byref(ne), ctypes.byref(pp), ctypes.byref(op)),
               "gint_psibeta_layout")
        self.pb_pairs = np.ctypeslib.as_array(pp, shape=(2 * n.value,)).reshape(-1, 2).copy() if n.value else \
            np.zeros((0, 2), np.int32)
        self.pb_off = np.ctypeslib.as_array(op, shape=(n.value + 1,)).copy()
        self.pb_nelems = int(ne.value)

    def psibeta(self, A, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """<beta_{I j}| e^{-i A.r} |Phi_{J mu}> blocks (complex128, device) in the layout of
        set_projectors (pb_pairs, pb_off): pair p's block is nbeta(I) x norb(J) at pb_off[p]."""
        a = (ctypes.c_double * 3)(*[float(x) for x in A])
        if out is None:
            out = torch.empty(2 * self.pb_nelems, dtype=torch.float64, device="cuda")
        _check(_lib.gint_psibeta(self._h, a, _dptr(out, numel=2 * self.pb_nelems), _stream(stream)), "gint_psibeta")
        return torch.view_as_complex(out.view(self.pb_nelems, 2))

    def force(self, D_blocks: torch.Tensor, V: torch.Tensor, precision: int = FP64,
              out: Optional[torch.Tensor] = None, rho_out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.natoms, 3), dtype=torch.float64, device=V.device)
        _check(_lib.gint_force(self._h, int(precision), _dptr(D_blocks, numel=self.nblock),
                               _dptr(V, numel=self.ngrid), _dptr(out, numel=3 * self.natoms),
                               _dptr(rho_out, numel=self.ngrid) if rho_out is not None else None, _stream(stream)),
               "gint_force")
        return out

    def run(self, D_blocks: Optional[torch.Tensor], V: Optional[torch.Tensor], precision: int = F16X3,
            rho: Optional[torch.Tensor] = None, H: Optional[torch.Tensor] = None, F: Optional[torch.Tensor] = None,
            stream=None, kernel_events=None) -> None:
        """Several passes of this system in one call (with the tensor-core precisions the density
        or force bricks and the local-H bricks share one persistent launch)."""
        run_batch([Task(self, D_blocks, V, rho, H, F)], precision, stream, kernel_events)

    def grid_dot(self, V: Optional[torch.Tensor], rho: torch.Tensor, out: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=rho.device)
        _check(_lib.gint_grid_dot(self._h, _dptr(V, numel=self.ngrid) if V is not None else None,
                                  _dptr(rho, numel=self.ngrid), _dptr(out), _stream(stream)), "gint_grid_dot")
        return out

    def block_dot(self, A: torch.Tensor, B: torch.Tensor, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=A.device)
        _check(_lib.gint_block_dot(self._h, _dptr(A, numel=self.nblock), _dptr(B, numel=self.nblock), _dptr(out),
                                   _stream(stream)), "gint_block_dot")
        return out

    def sync(self, stream=None):
        """Waits for the stream; raises if a kernel recorded an error (e.g. a bounded wait timed out)."""
        _check(_lib.gint_sync(self._h, _stream(stream)), "gint_sync")

    def set_positions(self, pos: torch.Tensor, stream=None):
        """New positions (device float64 [natoms, 3]); neighbour lists are rebuilt on the device."""
        pos = pos.detach().contiguous()
        _check(_lib.gint_set_positions(self._h, _dptr(pos, numel=3 * self.natoms), _stream(stream)),
               "gint_set_positions")
        self._pos_dev = pos.clone()
        self.__dict__.pop("nblock_R", None)  # H(R) keys follow the new images

    def ensure_positions(self, pos: torch.Tensor, stream=None):
        """Rebuilds the neighbour lists only if pos differs from the current geometry."""
        if self._pos_dev is None:
            self._pos_dev = torch.from_numpy(self._pos_host).to(pos.device)
        if not torch.equal(self._pos_dev, pos.detach()):
            self.set_positions(pos, stream)

    # -- layout helpers (host, numpy): dense <-> atom-pair blocks
    def dense_to_blocks(self, M: np.ndarray) -> np.ndarray:
        out = np.empty(self.nblock, dtype=np.float64)
        ao = self.atom_off
        for p, (I, J) in enumerate(self.pair_IJ):
            out[self.pair_off[p]:self.pair_off[p + 1]] = M[ao[I]:ao[I + 1], ao[J]:ao[J + 1]].reshape(-1)
        return out

    def blocks_to_dense(self, blocks: np.ndarray) -> np.ndarray:
        M = np.zeros((self.norb, self.norb))
        ao = self.atom_off
        for p, (I, J) in enumerate(self.pair_IJ):
            nI, nJ = ao[I + 1] - ao[I], ao[J + 1] - ao[J]
            M[ao[I]:ao[I + 1], ao[J]:ao[J + 1]] = blocks[self.pair_off[p]:self.pair_off[p + 1]].reshape(nI, nJ)
        return M

    def blocks_from_coefficients(self, C: np.ndarray) -> np.ndarray:
        """D blocks of D = C C^T computed pair row by pair row (no dense D)."""
        out = np.empty(self.nblock, dtype=np.float64)
        ao = self.atom_off
        starts = np.searchsorted(self.pair_IJ[:, 0], np.arange(self.natoms + 1))
        for I in range(self.natoms):
            p0, p1 = starts[I], starts[I + 1]
            Js = self.pair_IJ[p0:p1, 1]
            rows = np.concatenate([np.arange(ao[J], ao[J + 1]) for J in Js])
            blk = C[ao[I]:ao[I + 1]] @ C[rows].T  # (nI, sum nJ)
            col = 0
            for q, J in enumerate(Js):
                nJ = ao[J + 1] - ao[J]
                out[self.pair_off[p0 + q]:self.pair_off[p0 + q + 1]] = blk[:, col:col + nJ].reshape(-1)
                col += nJ
        return out

    def block_index(self, I: int, J: int) -> int:
        lo = np.searchsorted(self.pair_IJ[:, 0], I)
        hi = np.searchsorted(self.pair_IJ[:, 0], I + 1)
        k = np.searchsorted(self.pair_IJ[lo:hi, 1], J)
        if k >= hi - lo or self.pair_IJ[lo + k, 1] != J:
            return -1
        return int(lo + k)
