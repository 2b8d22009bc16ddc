"""Python access to the FP64 CPU oracle (gint_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark use this module; the product path never imports it.  It
imports nothing from the CUDA library or its binding.  Systems are passed
duck-typed (``cell``, ``pos``, ``species``, ``sp[s].radials[k].{l, npts, dr,
rc, f, df, alpha}``, ``grid``); dense matrices only (no block layouts).

Every entry point follows the definitions of the paper's Sec. 3.3.1 (density,
local-potential matrix, local Pulay force) at the Gamma point; the C source
header lists the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gint_oracle.c")
_LIB = os.path.join(_HERE, "libgint_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libgint_oracle.so (gcc, -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Sys(ctypes.Structure):
    _fields_ = [
        ("cell", ctypes.c_double * 9),
        ("natoms", ctypes.c_int),
        ("pos", ctypes.c_void_p),
        ("species", ctypes.c_void_p),
        ("nspecies", ctypes.c_int),
        ("sp_rad_begin", ctypes.c_void_p),
        ("nrad", ctypes.c_int),
        ("rad_l", ctypes.c_void_p),
        ("rad_npts", ctypes.c_void_p),
        ("rad_dr", ctypes.c_void_p),
        ("rad_rc", ctypes.c_void_p),
        ("rad_off", ctypes.c_void_p),
        ("f", ctypes.c_void_p),
        ("df", ctypes.c_void_p),
        ("rad_alpha", ctypes.c_void_p),
        ("analytic", ctypes.c_int),
        ("n1", ctypes.c_int),
        ("n2", ctypes.c_int),
        ("n3", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Sys)
            vp, ll = ctypes.c_void_p, ctypes.c_longlong
            lib.orc_weight.restype = ctypes.c_double
            lib.orc_weight.argtypes = [P]
            lib.orc_norb.argtypes = [P]
            lib.orc_phi_points.argtypes = [P, ll, vp, vp, vp]
            lib.orc_rho.argtypes = [P, vp, ll, vp, vp]
            lib.orc_vlocal.argtypes = [P, vp, ll, vp, vp]
            lib.orc_vlocal_block.argtypes = [P, vp, ctypes.c_int, ctypes.c_int, vp]
            lib.orc_vlocal_block_R.argtypes = [P, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
            lib.orc_psibeta.argtypes = [P, P, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp,
                                        vp]
            lib.orc_force.argtypes = [P, vp, vp, ll, vp, vp, vp]
            lib.orc_count_pairs.argtypes = [P, ll, vp, vp, vp]
            lib.orc_num_threads.argtypes = []
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """FP64 oracle bound to one system.  ``analytic=True`` evaluates radials as
    r^l exp(-alpha r^2) (support r < rc) instead of the interpolated table."""

    def __init__(self, system, analytic: bool = False, rc_override: Optional[float] = None):
        self.lib = _load()
        sp = system.sp
        rad = [r for s in sp for r in s.radials]
        begin = np.zeros(len(sp) + 1, dtype=np.int32)
        for i, s in enumerate(sp):
            begin[i + 1] = begin[i] + len(s.radials)
        for s in sp:
            assert sum(2 * r.l + 1 for r in s.radials) <= 64 and all(r.l <= 2 for r in s.radials)
        self._keep = dict(
            pos=np.ascontiguousarray(system.pos, dtype=np.float64),
            species=np.ascontiguousarray(system.species, dtype=np.int32),
            begin=begin,
            l=np.array([r.l for r in rad], dtype=np.int32),
            npts=np.array([r.npts for r in rad], dtype=np.int32),
            dr=np.array([r.dr for r in rad], dtype=np.float64),
            rc=np.array([rc_override if rc_override is not None else r.rc for r in rad], dtype=np.float64),
            off=np.concatenate([[0], np.cumsum([r.npts for r in rad])[:-1]]).astype(np.int64),
            f=np.ascontiguousarray(np.concatenate([r.f for r in rad]), dtype=np.float64),
            df=np.ascontiguousarray(np.concatenate([r.df for r in rad]), dtype=np.float64),
            alpha=np.array([r.alpha for r in rad], dtype=np.float64),
        )
        k = self._keep
        s = _Sys()
        s.cell[:] = [float(x) for x in np.asarray(system.cell, dtype=np.float64).reshape(-1)]
        s.natoms = int(k["pos"].shape[0])
        s.pos, s.species = _ptr(k["pos"]), _ptr(k["species"])
        s.nspecies = len(sp)
        s.sp_rad_begin = _ptr(k["begin"])
        s.nrad = len(rad)
        s.rad_l, s.rad_npts, s.rad_dr, s.rad_rc = _ptr(k["l"]), _ptr(k["npts"]), _ptr(k["dr"]), _ptr(k["rc"])
        s.rad_off, s.f, s.df, s.rad_alpha = _ptr(k["off"]), _ptr(k["f"]), _ptr(k["df"]), _ptr(k["alpha"])
        s.analytic = 1 if analytic else 0
        s.n1, s.n2, s.n3 = (int(x) for x in system.grid)
        self.s = s
        self.grid = tuple(int(x) for x in system.grid)
        self.ngrid = int(np.prod(self.grid))
        self.natoms = s.natoms
        self.norb = int(self.lib.orc_norb(ctypes.byref(s)))

    # -- scalars
    def weight(self) -> float:
        return float(self.lib.orc_weight(ctypes.byref(self.s)))

    @staticmethod
    def num_threads() -> int:
        return int(_load().orc_num_threads())

    # -- orbitals
    def phi_points(self, pts: np.ndarray, grad: bool = True):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        phi = np.zeros((n, self.norb))
        g = np.zeros((n, self.norb, 3)) if grad else None
        self.lib.orc_phi_points(ctypes.byref(self.s), n, _ptr(pts), _ptr(phi), _ptr(g))
        return (phi, g) if grad else phi

    # -- passes
    def rho(self, D: np.ndarray, idx: Optional[np.ndarray] = None) -> np.ndarray:
        D = np.ascontiguousarray(D, dtype=np.float64)
        assert D.shape == (self.norb, self.norb)
        if idx is None:
            out = np.zeros(self.ngrid)
            self.lib.orc_rho(ctypes.byref(self.s), _ptr(D), 0, None, _ptr(out))
            return out.reshape(self.grid)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.zeros(idx.shape[0])
        self.lib.orc_rho(ctypes.byref(self.s), _ptr(D), idx.shape[0], _ptr(idx), _ptr(out))
        return out

    def vlocal(self, V: np.ndarray, idx: Optional[np.ndarray] = None) -> np.ndarray:
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        assert V.shape[0] == self.ngrid
        H = np.zeros((self.norb, self.norb))
        if idx is None:
            self.lib.orc_vlocal(ctypes.byref(self.s), _ptr(V), 0, None, _ptr(H))
        else:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            self.lib.orc_vlocal(ctypes.byref(self.s), _ptr(V), idx.shape[0], _ptr(idx), _ptr(H))
        return H

    def vlocal_block(self, V: np.ndarray, I: int, J: int) -> np.ndarray:
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        nI = self._norb_atom(I)
        nJ = self._norb_atom(J)
        out = np.zeros((nI, nJ))
        self.lib.orc_vlocal_block(ctypes.byref(self.s), _ptr(V), int(I), int(J), _ptr(out))
        return out

    def vlocal_block_R(self, V: np.ndarray, I: int, J: int, R) -> tuple:
        """H_IJ(R) for the listed lattice vectors R (integer triplets, units of the cell vectors):
        the local-H block between atom I at tau_I and atom J at tau_J + R (paper Sec. 2, H(R)).
        Returns (blocks [len(R), norb(I), norb(J)], missed): missed sums the absolute values of
        products that belong to an R outside the list (zero when the list is complete)."""
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        R = np.ascontiguousarray(np.asarray(R, dtype=np.int32).reshape(-1, 3))
        nI, nJ = self._norb_atom(I), self._norb_atom(J)
        out = np.zeros((R.shape[0], nI, nJ))
        missed = ctypes.c_double()
        self.lib.orc_vlocal_block_R(ctypes.byref(self.s), _ptr(V), int(I), int(J), int(R.shape[0]), _ptr(R),
                                    _ptr(out), ctypes.byref(missed))
        return out, missed.value

    def psibeta(self, projectors: "Oracle", A, I: int, J: int, radial, angular) -> np.ndarray:
        """Velocity-gauge projector overlaps (paper Sec. 3.3.2): [nbeta(I), norb(J)] complex,
        sum over the atom-centred grid around tau_I of beta_{I j}(x) e^{-i A.r} Phi_{J mu}(r), r = tau_I + x.
        ``projectors`` is an Oracle of the same cell and atoms whose radials are the projectors;
        ``radial`` = (nodes, weights) on [0, 1] (scaled to [0, rc_beta], times r^2); ``angular`` =
        [n, 4] points (x, y, z) and weights (summing to 4 pi)."""
        rt = np.ascontiguousarray(radial[0], dtype=np.float64)
        rw = np.ascontiguousarray(radial[1], dtype=np.float64)
        ang = np.ascontiguousarray(angular, dtype=np.float64).reshape(-1, 4)
        A = np.ascontiguousarray(A, dtype=np.float64).reshape(3)
        nb, no = projectors._norb_atom(I), self._norb_atom(J)
        out = np.zeros((nb, no, 2))
        self.lib.orc_psibeta(ctypes.byref(self.s), ctypes.byref(projectors.s), _ptr(A), int(I), int(J), rt.shape[0],
                             _ptr(rt), _ptr(rw), ang.shape[0], _ptr(ang), _ptr(out))
        return out[..., 0] + 1j * out[..., 1]

    def force(self, D: np.ndarray, V: np.ndarray, idx: Optional[np.ndarray] = None,
              atoms: Optional[np.ndarray] = None) -> np.ndarray:
        D = np.ascontiguousarray(D, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        F = np.zeros((self.natoms, 3))
        mask = None
        if atoms is not None:
            mask = np.zeros(self.natoms, dtype=np.int32)
            mask[np.asarray(atoms)] = 1
        if idx is None:
            self.lib.orc_force(ctypes.byref(self.s), _ptr(D), _ptr(V), 0, None, _ptr(mask), _ptr(F))
        else:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            self.lib.orc_force(ctypes.byref(self.s), _ptr(D), _ptr(V), idx.shape[0], _ptr(idx), _ptr(mask), _ptr(F))
        return F

    def energy(self, D: np.ndarray, V: np.ndarray) -> float:
        return float(self.weight() * np.dot(np.asarray(V).reshape(-1), self.rho(D).reshape(-1)))

    def count_pairs(self, idx: Optional[np.ndarray] = None):
        W = ctypes.c_double()
        sn = ctypes.c_double()
        if idx is None:
            self.lib.orc_count_pairs(ctypes.byref(self.s), 0, None, ctypes.byref(W), ctypes.byref(sn))
        else:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            self.lib.orc_count_pairs(ctypes.byref(self.s), idx.shape[0], _ptr(idx), ctypes.byref(W), ctypes.byref(sn))
        return W.value, sn.value

    def _norb_atom(self, a: int) -> int:
        sp = int(self._keep["species"][a])
        b = self._keep["begin"]
        return int(sum(2 * l + 1 for l in self._keep["l"][b[sp]:b[sp + 1]]))

    def atom_offsets(self) -> np.ndarray:
        n = [self._norb_atom(a) for a in range(self.natoms)]
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
