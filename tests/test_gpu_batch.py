"""Batched launches (gint_run_batch): several systems' bricks in one persistent launch.

Every brick is computed the same way whatever else shares the launch, so a system's density and
local H are bitwise the same alone and in a mix; forces are reduced with float64 atomics whose
order varies, so they agree to rounding.  Each mixed result is also checked against the FP64
oracle at the path's tolerances (F16x3: 1e-6 max-norm relative for rho and H, 1e-5 Ha/Bohr for
forces; FP64: 1e-12).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


LIB = [inputs.si_species(), inputs.o_species(), inputs.h_species()]


def _systems():
    a = inputs.config_workload("si8_g48")
    b = inputs.h2o_workload(4, seed=3, box=20.0, grid=(96, 96, 96))
    c = inputs.si_workload((2, 1, 1), (96, 48, 48), seed=5, disp_sigma=0.05, name="si16")
    return [a, b, c]


class Sys:
    def __init__(self, w, G, torch):
        self.w = w
        self.system = inputs.on_species(w.system, LIB)
        self.g = G.Gint(self.system)
        self.D = torch.from_numpy(self.g.dense_to_blocks(w.D)).cuda()
        self.V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()

    def outputs(self, torch):
        g = self.g
        return (torch.empty(g.ngrid, dtype=torch.float64, device="cuda"),
                torch.empty(g.nblock, dtype=torch.float64, device="cuda"),
                torch.empty((g.natoms, 3), dtype=torch.float64, device="cuda"))


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2603_21835_gb300 import gint as G

    systems = [Sys(w, G, torch) for w in _systems()]
    refs = []
    for s in systems:
        o = Oracle(s.system)
        refs.append(dict(rho=o.rho(s.w.D).reshape(-1), H=s.g.dense_to_blocks(o.vlocal(s.w.V)), F=o.force(s.w.D, s.w.V)))
    return dict(torch=torch, G=G, systems=systems, refs=refs)


def _alone(env, prec):
    torch, G = env["torch"], env["G"]
    out = []
    for s in env["systems"]:
        rho, H, F = s.outputs(torch)
        s.g.run(s.D, s.V, prec, rho=rho, H=H, F=F)
        out.append((rho, H, F))
    torch.cuda.synchronize()
    for s in env["systems"]:
        s.g.sync()
    return [tuple(x.cpu().numpy() for x in o) for o in out]


def _mixed(env, prec, order):
    torch, G = env["torch"], env["G"]
    systems = env["systems"]
    outs = {i: systems[i].outputs(torch) for i in order}
    G.run_batch([G.Task(systems[i].g, systems[i].D, systems[i].V, *outs[i]) for i in order], prec)
    torch.cuda.synchronize()
    for s in systems:
        s.g.sync()
    return [tuple(x.cpu().numpy() for x in outs[i]) for i in range(len(systems))]


def test_mix_equals_alone_and_oracle(env):
    G = env["G"]
    alone = _alone(env, G.F16X3)
    mixed = _mixed(env, G.F16X3, [0, 1, 2])
    for i, (a, m, ref) in enumerate(zip(alone, mixed, env["refs"])):
        assert np.array_equal(a[0], m[0]), i  # rho: one owner brick per point
        assert np.array_equal(a[1], m[1]), i  # H: fixed-order reduction
        assert np.abs(a[2] - m[2]).max() <= 1e-12 * max(1.0, np.abs(a[2]).max()), i
        assert _rel(m[0], ref["rho"]) <= 1e-6, i
        assert _rel(m[1], ref["H"]) <= 1e-6, i
        assert np.abs(m[2] - ref["F"]).max() <= 1e-5, i


def test_mix_order_does_not_matter(env):
    G = env["G"]
    m1 = _mixed(env, G.F16X3, [0, 1, 2])
    m2 = _mixed(env, G.F16X3, [2, 0, 1])
    for a, b in zip(m1, m2):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fp64_batch_matches_oracle(env):
    G = env["G"]
    mixed = _mixed(env, G.FP64, [0, 1, 2])
    for m, ref in zip(mixed, env["refs"]):
        assert _rel(m[0], ref["rho"]) <= 1e-12
        assert _rel(m[1], ref["H"]) <= 1e-12
        assert np.abs(m[2] - ref["F"]).max() <= 1e-11 * max(1.0, np.abs(ref["F"]).max())


def test_partial_outputs(env):
    """Tasks asking for H only, rho only, or forces without rho, next to a full task."""
    torch, G = env["torch"], env["G"]
    s0, s1, s2 = env["systems"]
    full = _mixed(env, G.F16X3, [0, 1, 2])
    H1 = torch.empty(s1.g.nblock, dtype=torch.float64, device="cuda")
    rho2 = torch.empty(s2.g.ngrid, dtype=torch.float64, device="cuda")
    F0 = torch.empty((s0.g.natoms, 3), dtype=torch.float64, device="cuda")
    G.run_batch([G.Task(s0.g, s0.D, s0.V, F=F0), G.Task(s1.g, None, s1.V, H=H1), G.Task(s2.g, s2.D, None, rho=rho2)],
                G.F16X3)
    torch.cuda.synchronize()
    assert np.abs(F0.cpu().numpy() - full[0][2]).max() <= 1e-12 * max(1.0, np.abs(full[0][2]).max())
    assert np.array_equal(H1.cpu().numpy(), full[1][1])
    # rho from a density-only item (triangular chunks) vs the force item's full Y: rounding level
    assert _rel(rho2.cpu().numpy(), full[2][0]) <= 1e-6


def test_rejects_repeated_handle_and_other_species(env):
    torch, G = env["torch"], env["G"]
    s0 = env["systems"][0]
    rho, H, F = s0.outputs(torch)
    with pytest.raises(G.GintError) as e:
        G.run_batch([G.Task(s0.g, s0.D, s0.V, rho=rho), G.Task(s0.g, s0.D, s0.V, H=H)], G.F16X3)
    assert e.value.code == -1
    own = G.Gint(s0.w.system)  # species list [Si] only: different radial metadata
    D = torch.from_numpy(own.dense_to_blocks(s0.w.D)).cuda()
    rho2 = torch.empty(own.ngrid, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GintError) as e:
        G.run_batch([G.Task(s0.g, s0.D, s0.V, rho=rho), G.Task(own, D, s0.V, rho=rho2)], G.F16X3)
    assert e.value.code == -1
    with pytest.raises(G.GintError):
        G.run_batch([G.Task(s0.g, None, s0.V, rho=rho)], G.F16X3)  # density without D
    own.close()


def test_more_than_one_launch_group(env):
    """34 systems: two launch groups (32 + 2); each result equals the system alone."""
    torch, G = env["torch"], env["G"]
    w = inputs.si_workload((1, 1, 1), (24, 24, 24), seed=11, disp_sigma=0.05)
    system = inputs.on_species(w.system, LIB)
    gs = [G.Gint(system) for _ in range(34)]
    D = torch.from_numpy(gs[0].dense_to_blocks(w.D)).cuda()
    V0 = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    Vs = [V0 * (1.0 + 0.03 * k) for k in range(34)]
    outs = [(torch.empty(g.ngrid, dtype=torch.float64, device="cuda"),
             torch.empty(g.nblock, dtype=torch.float64, device="cuda")) for g in gs]
    G.run_batch([G.Task(g, D, V, rho=o[0], H=o[1]) for g, V, o in zip(gs, Vs, outs)], G.F16X3)
    torch.cuda.synchronize()
    for k in (0, 31, 32, 33):
        rho = torch.empty(gs[k].ngrid, dtype=torch.float64, device="cuda")
        H = torch.empty(gs[k].nblock, dtype=torch.float64, device="cuda")
        gs[k].run(D, Vs[k], G.F16X3, rho=rho, H=H)
        torch.cuda.synchronize()
        assert torch.equal(rho, outs[k][0]) and torch.equal(H, outs[k][1]), k
    for g in gs:
        g.sync()
        g.close()
