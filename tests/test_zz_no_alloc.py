"""The no-allocation dot product (gint_grid_dot_noalloc) against the handle-based gint_grid_dot.

gint_grid_dot_noalloc serves callers that cannot let a library allocate device memory (their
device memory is owned by their own pool allocator, or they run latency-critical loops that
cannot accept cudaMalloc's implicit synchronisation).  Its scratch is a fixed array inside the
library, so this file checks that it gives the same energy and electron count as the existing
entry point on two calls in a row (the array keeps the previous call's contents), and that a
size above its limit is rejected.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_grid_dot_noalloc_matches_handle_reduction():
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.si_workload((1, 1, 1), (32, 32, 40), seed=6, disp_sigma=0.05)
    g = G.Gint(w.system)
    Db = torch.from_numpy(g.dense_to_blocks(w.D)).cuda()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    rho = g.rho(Db, G.FP64).reshape(-1)
    stream = torch.cuda.current_stream()
    lib = G._lib
    for call in range(2):
        for vec in (V, None):
            ref = g.grid_dot(vec, rho)
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.gint_grid_dot_noalloc(ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(vec.data_ptr()) if vec is not None else None,
                                           rho.numel(), g.weight, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, G._lib.gint_strerror(rc)
            torch.cuda.synchronize()
            a, b = out.item(), ref.item()
            assert np.isfinite(a)
            assert abs(a - b) <= 1e-12 * abs(b), (call, vec is None, a, b)
    # beyond the scratch limit: rejected before any work
    too_many = 4096 * 65536 + 1
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.gint_grid_dot_noalloc(ctypes.c_void_p(rho.data_ptr()), None, too_many, 1.0,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -6
    g.close()
