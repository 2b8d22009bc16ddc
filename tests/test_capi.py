"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
symbol include/gint.h declares, and rejects malformed descriptors before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_21835_gb300 import build as gbuild
from paper_2603_21835_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = gbuild.build()
    return ctypes.CDLL(path)


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gint_[A-Za-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert {"gint_create", "gint_rho", "gint_vlocal", "gint_force", "gint_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2603_21835_gb300 import gint

    assert set(gint.C_ABI_SYMBOLS) <= _declared_symbols()


def test_strerror_and_invalid_descriptors(lib):
    from paper_2603_21835_gb300 import gint as G

    lib.gint_strerror.restype = ctypes.c_char_p
    assert lib.gint_strerror(0) == b"success"
    assert b"invalid" in lib.gint_strerror(-1)
    w = inputs.si_workload((1, 1, 1), (8, 8, 8))
    sysm = w.system
    # NULL descriptor and NULL output
    h = ctypes.c_void_p()
    assert lib.gint_create(None, ctypes.byref(h)) == -1
    # species index out of range, bad l, empty grid: all rejected on the host
    bad = inputs.System(cell=sysm.cell, pos=sysm.pos, species=np.full(8, 3, np.int32), sp=sysm.sp, grid=(8, 8, 8))
    with pytest.raises(G.GintError) as e:
        G.Gint(bad)
    assert e.value.code == -1
    bad = inputs.System(cell=sysm.cell, pos=sysm.pos, species=sysm.species, sp=sysm.sp, grid=(0, 8, 8))
    with pytest.raises(G.GintError):
        G.Gint(bad)
    sp3 = inputs.Species("X", [inputs.make_radial(3, 0.5, 5.0)])
    bad = inputs.System(cell=sysm.cell, pos=sysm.pos[:1], species=np.zeros(1, np.int32), sp=[sp3], grid=(8, 8, 8))
    with pytest.raises(G.GintError):
        G.Gint(bad)
    sing = inputs.System(cell=np.zeros((3, 3)), pos=sysm.pos, species=sysm.species, sp=sysm.sp, grid=(8, 8, 8))
    with pytest.raises(G.GintError):
        G.Gint(sing)
    nanpos = sysm.pos.copy()
    nanpos[0, 0] = np.nan
    with pytest.raises(G.GintError):
        G.Gint(inputs.System(cell=sysm.cell, pos=nanpos, species=sysm.species, sp=sysm.sp, grid=(8, 8, 8)))


def test_entry_points_reject_null_arguments_on_the_host(lib):
    """NULL handles, contexts and buffers come back as GINT_EINVAL before any CUDA call."""
    EINVAL = -1
    i, ll = ctypes.c_int(), ctypes.c_longlong()
    assert lib.gint_layout_R(None, ctypes.byref(i), ctypes.byref(ll), None, None) == EINVAL
    assert lib.gint_vlocal_R(None, 2, None, None, None) == EINVAL
    assert lib.gint_bloch(None, None, 1, None, None, None) == EINVAL
    assert lib.gint_set_projectors(None, 1, None) == EINVAL
    assert lib.gint_psibeta_layout(None, ctypes.byref(i), ctypes.byref(ll), None, None) == EINVAL
    assert lib.gint_psibeta(None, None, None, None) == EINVAL
    c = ctypes.c_void_p()
    assert lib.gint_cn_create(0, 4, ctypes.byref(c)) == EINVAL
    assert lib.gint_cn_create(4, 0, ctypes.byref(c)) == EINVAL
    assert lib.gint_cn_create(4, 4, None) == EINVAL
    assert lib.gint_cn_step(None, None, None, ctypes.c_double(0.1), None, None, None) == EINVAL
    assert lib.gint_dm_build(None, None, None, None, None) == EINVAL
    assert lib.gint_dm_build_f16x3(None, None, None, None, None) == EINVAL
    assert lib.gint_edm(None, None, None, None, None, None) == EINVAL
    assert lib.gint_cn_info(None, ctypes.byref(i)) == EINVAL
    assert lib.gint_cn_destroy(None) == 0
    lib.gint_strerror.restype = ctypes.c_char_p
    msgs = {code: lib.gint_strerror(code) for code in range(-8, 1)}
    assert len(set(msgs.values())) == len(msgs) and all(msgs.values())
    assert lib.gint_strerror(-99) == b"unknown error"
