"""The library's continuous-batching server (gint_server_*, DeviceQueue): one resident launch drains a
device work queue to which jobs are appended while it runs.

Checks: every job's rho and H are the same bits alone on the queue and in a mix (one owner brick per
grid point, the fixed-order reduction), F to 1e-12 Ha/Bohr (float64 atomics in another order); they
agree with the batched call on the same handle to the mixed-precision tolerance (the two kernels
compile the same brick code in different contexts, so float32 rounding may differ at a point whose
support test sits on the boundary) and with the oracle; a
job published while a large one is on the GPU completes in the same residency (one launch); the
kernel leaves when idle and the next submission relaunches it; a full ring or a busy handle is
refused with GINT_EBUSY, not queued behind the caller's back.
"""
import time

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    from paper_2603_21835_gb300 import gint as G

    return torch, G


def _case(G, torch, system, seed):
    V, C = inputs.serving_inputs(system, seed=seed)
    g = G.Gint(system)
    D = torch.from_numpy(g.blocks_from_coefficients(C)).cuda()
    Vd = torch.from_numpy(np.ascontiguousarray(V.reshape(-1))).cuda()
    return dict(g=g, D=D, V=Vd, C=C, Vh=V, system=system)


def _outputs(torch, c):
    g = c["g"]
    return (torch.empty(g.ngrid, dtype=torch.float64, device="cuda"),
            torch.empty(g.nblock, dtype=torch.float64, device="cuda"),
            torch.empty((g.natoms, 3), dtype=torch.float64, device="cuda"))


def _reference(G, torch, c):
    rho, H, F = _outputs(torch, c)
    G.run_batch([G.Task(c["g"], c["D"], c["V"], rho=rho, H=H, F=F)], G.F16X3)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), H.cpu().numpy(), F.cpu().numpy()


def _wait(q, tickets, timeout=60.0):
    t0 = time.time()
    pending = set(tickets)
    while pending:
        pending = {t for t in pending if not q.done(t)}
        assert time.time() - t0 < timeout, f"jobs {sorted(pending)} did not complete"
        time.sleep(0.0005)


def test_jobs_match_batched_calls_and_mid_residency_admission(mods):
    torch, G = mods
    lib = inputs.serving_library()
    pool = inputs.serving_pool()
    big = _case(G, torch, inputs.on_species(inputs.si_workload((3, 3, 3), (144, 144, 144), seed=3,
                                                                disp_sigma=0.05).system, lib), 11)
    smalls = [_case(G, torch, pool[i], 20 + i) for i in (0, 1, 10, 11)]  # two Si cells, two water clusters
    refs = [_reference(G, torch, c) for c in [big] + smalls]
    q = G.DeviceQueue(G.F16X3, forces=True, idle_s=0.5)
    alone = []
    for c in [big] + smalls:  # each job alone on the queue
        o = _outputs(torch, c)
        _wait(q, [q.submit(G.Task(c["g"], c["D"], c["V"], rho=o[0], H=o[1], F=o[2]))])
        alone.append(tuple(x.cpu().numpy() for x in o))
    q.stop()  # the next submission relaunches the resident kernel
    launches0 = q.stats()["launches"]
    outs = [_outputs(torch, c) for c in [big] + smalls]
    torch.cuda.synchronize()
    tickets = [q.submit(G.Task(big["g"], big["D"], big["V"], rho=outs[0][0], H=outs[0][1], F=outs[0][2]))]
    # published while the large job runs (it takes several ms): same residency
    for c, o in zip(smalls, outs[1:]):
        tk = q.submit(G.Task(c["g"], c["D"], c["V"], rho=o[0], H=o[1], F=o[2]))
        assert tk is not None
        tickets.append(tk)
    _wait(q, tickets)
    st = q.stats()
    assert st["launches"] == launches0 + 1 and st["jobs"] == 2 * len(tickets)  # one residency for the mix
    for (rho, H, F), (ra, Ha, Fa), (rr, Hr, Fr) in zip(outs, alone, refs):
        r, h, f = rho.cpu().numpy(), H.cpu().numpy(), F.cpu().numpy()
        assert np.array_equal(r, ra) and np.array_equal(h, Ha)
        assert np.abs(f - Fa).max() <= 1e-12
        assert np.abs(r - rr).max() <= 1e-6 * np.abs(rr).max() and np.abs(h - Hr).max() <= 1e-6 * np.abs(Hr).max()
        assert np.abs(f - Fr).max() <= 1e-5
    # against the oracle: one water cluster in full
    c, (rho, H, F) = smalls[2], outs[3]
    o = Oracle(c["system"])
    D = c["C"] @ c["C"].T
    rho_o, H_o, F_o = o.rho(D).reshape(-1), o.vlocal(c["Vh"]), o.force(D, c["Vh"])
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-6 * np.abs(rho_o).max()
    assert np.abs(c["g"].blocks_to_dense(H.cpu().numpy()) - H_o).max() <= 1e-6 * np.abs(H_o).max()
    assert np.abs(F.cpu().numpy() - F_o).max() <= 1e-5
    q.close()
    for cc in [big] + smalls:
        cc["g"].close()


def test_idle_exit_relaunch_and_busy(mods):
    torch, G = mods
    pool = inputs.serving_pool()
    c = _case(G, torch, pool[0], 5)
    ref = _reference(G, torch, c)
    q = G.DeviceQueue(G.F16X3, forces=True, idle_s=0.05)
    o = _outputs(torch, c)
    t1 = q.submit(G.Task(c["g"], c["D"], c["V"], rho=o[0], H=o[1], F=o[2]))
    # the same handle again while its job may be in flight: refused (None) until that job is done
    t2 = None
    t0 = time.time()
    while t2 is None:
        t2 = q.submit(G.Task(c["g"], c["D"], c["V"], rho=o[0], H=o[1], F=o[2]))
        assert t2 is not None or not q.done(t1) or time.time() - t0 < 60
    _wait(q, [t1, t2])
    time.sleep(0.3)  # the resident kernel leaves after 0.05 s without work
    t3 = q.submit(G.Task(c["g"], c["D"], c["V"], rho=o[0], H=o[1], F=o[2]))
    _wait(q, [t3])
    assert q.stats()["launches"] >= 2
    assert np.abs(o[0].cpu().numpy() - ref[0]).max() <= 1e-6 * np.abs(ref[0]).max()
    assert np.abs(o[1].cpu().numpy() - ref[1]).max() <= 1e-6 * np.abs(ref[1]).max()
    assert np.abs(o[2].cpu().numpy() - ref[2]).max() <= 1e-5
    q.stop()
    q.close()
    c["g"].close()
