#!/usr/bin/env python
"""Benchmark: grid-integration throughput (density + local Hamiltonian) on one GB300.

One step = one density pass and one local-Hamiltonian pass over the whole grid of the
workload (inputs resident in HBM).  Work unit: ordered orbital pairs per grid point,
W = sum_g n_g^2 per pass, so one step is 2W pair updates; the metric is Gpt-pair/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f16x3|fp64|fp32|f16x1]
                  [--workload si512_g192|si64_g96|si8_g48] [--impl ours|reference]

The default workload is the 512-atom Si supercell (4x4x4, 6656 orbitals, 192^3 grid).  With the
tensor-core precisions both passes' bricks run in one persistent launch per step; the float64 GPU
path is timed on the same workload in the same run (fp64_gpu), and the line reports the ratio.
After the timed steps (rank 0, N = 1) a serving run submits a Poisson stream of density +
local-H + force requests over a mix of Si supercells (8-216 atoms) and water clusters (8-64
molecules) to the continuous-batching server and reports p50/p99 latency and throughput.

N > 1 runs N independent replicas (one per rank, launched by torch.distributed.run): the
path needs no exchange between GPUs; value is the total work of all ranks over the slowest
rank's time.  --impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gint Gpt-pair/s (rho+H_loc) mixed vs FP64 on GB300 at <=1e-6 rel err; p50/p99 ms"
UNIT = "Gpt-pair/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal float64 rate of GB300 (no fast float64 tensor path)
FP64_NOMINAL_TFLOPS = 1.25
FP32_SIMT_TFLOPS_PER_GHZ = 152 * 128 * 2 / 1e3  # 152 SMs x 128 FP32 lanes x 2 flops per clock
FP64_NOMINAL_TFLOPS = 1.25  # GB300 float64 (CUDA cores), nominal


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x3", choices=["f16x3", "fp64", "fp32", "f16x1"])
    ap.add_argument("--workload", default="si512_g192")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the float64 GPU comparator (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the serving run and the per-R, projector and Crank-Nicolson timings")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense propagation steps among the extras")
    ap.add_argument("--dense-only", action="store_true",
                    help="time only the dense steps (Crank-Nicolson, density matrices) at the workload's basis size")
    ap.add_argument("--serve-requests", type=int, default=256, help="Poisson serving run (0: skip)")
    ap.add_argument("--serve-load", type=float, default=0.75, help="arrival rate x mean service time alone")
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--serve-replicas", type=int, default=2,
                    help="resident handles per geometry (each runs one job at a time)")
    return ap.parse_args()


def profiled(workload: str, precision: str, source: str, key: str):
    """A figure (`key`) from a committed ncu summary under profiles/, if one was taken on this workload
    (None: any) and precision with the current source of the kernel (csrc/`source`); else None."""
    import glob
    import hashlib

    src = os.path.join(ROOT, "paper_2603_21835_gb300", "csrc", source)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        kv = {}
        with open(path) as f:
            for line in f:
                parts = line.strip().split(": ", 1)
                if len(parts) == 2 and parts[0] in ("workload", "precision", "kernel_source", "kernel_source_sha256", key):
                    kv[parts[0]] = parts[1].strip()
        if ((workload is None or kv.get("workload") == workload) and kv.get("precision") == precision
                and kv.get("kernel_source", "gint_tc.cu") == source
                and kv.get("kernel_source_sha256") == sha and key in kv):
            return float(kv[key]), os.path.relpath(path, ROOT)
    return None, None


def profiled_traffic(workload: str, precision: str):
    """DRAM bytes per launch of the brick kernel (ncu), if profiled with the current source."""
    v, path = profiled(workload, precision, "gint_tc.cu", "traffic_bytes_per_launch")
    return (int(v) if v is not None else None), path


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over all ranks (timings: the slowest rank sets the job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ oracle (CPU) baseline
# the oracle's region of a workload: the 512-atom case is checked on the grid sub-volume [0, n/2)^3
ORACLE_REGION = {"si512_g192": "sub-volume [0,96)^3 of the 192^3 grid"}


def oracle_region(workload_name: str, grid):
    """Grid indices the oracle baseline samples from (None: the whole grid)."""
    if workload_name not in ORACLE_REGION:
        return None
    n1, n2, n3 = grid
    i, j, k = np.meshgrid(np.arange(n1 // 2), np.arange(n2 // 2), np.arange(n3 // 2), indexing="ij")
    return ((i * n2 + j) * n3 + k).reshape(-1)


def oracle_sample(workload_name: str, target_s: float, seed: int = 7):
    """Times the FP64 oracle (rho + H over a random subset of grid points) on the host cores.
    Returns (Gpt-pair/s, threads, description)."""
    from oracle.oracle import Oracle
    from paper_2603_21835_gb300 import inputs

    w = inputs.config_workload(workload_name, dense_D=True)
    o = Oracle(w.system)
    rng = np.random.default_rng(seed)
    region = oracle_region(workload_name, o.grid)
    pool = region if region is not None else np.arange(o.ngrid)
    n = 4000
    while True:
        idx = np.sort(rng.choice(pool, min(n, pool.size), replace=False))
        t0 = time.perf_counter()
        o.rho(w.D, idx)
        o.vlocal(w.V, idx)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or n >= pool.size:
            break
        n = int(min(pool.size, n * max(2.0, 0.9 * target_s / max(dt, 1e-3))))
    n = idx.size
    Wsample, _ = o.count_pairs(idx)
    value = 2.0 * Wsample / dt / 1e9
    where = f"the {ORACLE_REGION[workload_name]}" if region is not None else "the grid"
    desc = (f"FP64 oracle rho + H_loc over {n} random grid points of {workload_name}, drawn from {where} "
            f"({n / o.ngrid:.3%} of the grid, 2W = {2 * Wsample:.3e} pair updates) in {dt:.1f} s; "
            f"no extrapolation")
    return value, Oracle.num_threads(), desc, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.oracle import build

    build()
    vals, cores, desc = [], None, ""
    per_step = max(5.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for k in range(args.warmup + args.steps):
        v, cores, desc, dt = oracle_sample(args.workload, per_step, seed=100 + k)
        if k >= args.warmup:
            vals.append((v, dt))
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([dt for _, dt in vals]) * 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64-cpu-oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
# kernels of ours per step (density + local-H passes; memsets are not kernels):
#   fp64: k_simt_rho, k_simt_vlocal;  fp32: k_to_f32, k_simt_rho, k_simt_vlocal;
#   f16x3 / f16x1: k_prep, k_prep_scales, k_build_tiles, k_tc_fused (both passes), k_h_reduce
KERNEL_LAUNCHES = {"fp64": 2, "fp32": 3, "f16x3": 5, "f16x1": 5}
TENSOR_PRECISIONS = ("f16x3", "f16x1")


def run_serving(args, prec, dev):
    """Continuous batching: rho + H + F requests over the serving mix (Si supercells and water
    clusters, half each), first one at a time (service times alone), then a Poisson stream at
    args.serve_load / (mean service time alone), then all at once (burst)."""
    import torch

    from paper_2603_21835_gb300 import inputs, serve

    pool = inputs.serving_pool()
    srv = serve.Server(inputs.serving_library(), budget_bytes=int(args.serve_budget_gb * (1 << 30)), precision=prec,
                       replicas=args.serve_replicas, device=dev)
    try:
        sessions = [srv.open(s) for s in pool]
        nvar = 4
        plan_idx = inputs.serving_requests(args.serve_requests, seed=1)
        cache = {}

        def req(i, k):
            if (i, k) not in cache:
                V, C = inputs.serving_inputs(pool[i], seed=100 * i + k)
                cache[(i, k)] = (torch.from_numpy(sessions[i].blocks_from_coefficients(C)).pin_memory(),
                                 torch.from_numpy(np.ascontiguousarray(V.reshape(-1))).pin_memory())
            return cache[(i, k)]

        plan = [(i, n % nvar) for n, i in enumerate(plan_idx)]
        for i, k in plan:
            req(i, k)
        # service time of each geometry alone (after one warm-up request each)
        alone = {}
        for rep in range(2):
            for i in range(len(pool)):
                r = srv.submit(sessions[i], *req(i, 0)).result(timeout=300)
                if rep == 1:
                    alone[i] = r.latency_ms
        mean_alone = float(np.mean([alone[i] for i, _ in plan]))
        rate = args.serve_load / (mean_alone * 1e-3)

        def run(gaps):
            nb0 = len(srv.concurrency)
            futs = []
            t0 = time.perf_counter()
            due = t0
            for (i, k), gap in zip(plan, gaps):
                due += gap
                while True:
                    dt = due - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 0.002))
                futs.append(srv.submit(sessions[i], *req(i, k)))
            res = [f.result(timeout=600) for f in futs]
            wall = max(r.done_t for r in res) - t0
            lat = serve.percentiles([r.latency_ms for r in res])
            conc = srv.concurrency[nb0:]
            pairs = sum(2.0 * sessions[i].W for i, _ in plan)
            return {"p50_ms": lat["p50"], "p99_ms": lat["p99"], "mean_ms": lat["mean"], "max_ms": lat["max"],
                    "throughput_req_s": len(plan) / wall, "throughput_gpt_pair_s": pairs / wall / 1e9,
                    "mean_jobs_in_flight_at_publication": float(np.mean(conc)), "max_jobs_in_flight": int(max(conc))}

        poisson = run(np.random.default_rng(1).exponential(1.0 / rate, len(plan)))
        burst = run(np.zeros(len(plan)))
        out = {
            "requests": len(plan), "outputs": "rho+H+F", "pool": [s.name for s in pool],
            "mix": "Si supercells and water clusters with probability 1/2 each (seed 1)",
            "mean_service_alone_ms": mean_alone,
            "arrivals": f"Poisson, rate = {args.serve_load:g} / mean service time alone",
            "rate_hz": rate, "poisson": poisson, "burst": burst,
            "p50_ms": poisson["p50_ms"], "p99_ms": poisson["p99_ms"],
            "throughput_note": "2W per request (rho + H pair updates); the force pass is extra work not counted",
            "replicas_per_geometry": args.serve_replicas,
            "budget_bytes": srv.budget.budget, "peak_bytes": srv.budget.peak, "errors": len(srv.errors),
            "resident_launches": srv.stats()["resident_launches"],
            "design": "device work queue: one resident launch drains jobs published while it runs",
        }
    finally:
        srv.close()
    return out


def run_per_R(g, V, prec, steps, stream, flush, hbm_gbs):
    """Local H per lattice vector, H_IJ(R), and its Bloch sum H(k) on the same workload (tensor-core
    precisions): mean times of gint_vlocal_R (the brick pass and the per-(I, J, R) reduction) and of
    gint_bloch (eight k points per pass), L2 flushed between steps."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    try:
        keys, _ = g.layout_R()
    except G.GintError as e:
        return {"unavailable": str(e)}
    HR = torch.empty(g.nblock_R, dtype=torch.float64, device=V.device)
    # eight k points of a 2 x 2 x 2 Monkhorst-Pack mesh share one pass over H(R)
    kf = [[(i + 0.5) / 2 - 0.5, (j + 0.5) / 2 - 0.5, (l + 0.5) / 2 - 0.5] for i in range(2) for j in range(2)
          for l in range(2)]
    Hk = torch.empty(len(kf) * 2 * g.nblock, dtype=torch.float64, device=V.device)
    for _ in range(3):
        g.vlocal_R(V, prec, out=HR, stream=stream)
        g.bloch(HR, kf, out=Hk, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tr, tb = [], []
    for k in range(steps):
        flush.fill_(float(k))
        ev[0].record(stream)
        g.vlocal_R(V, prec, out=HR, stream=stream)
        ev[1].record(stream)
        g.bloch(HR, kf, out=Hk, stream=stream)
        ev[2].record(stream)
        ev[2].synchronize()
        tr.append(ev[0].elapsed_time(ev[1]))
        tb.append(ev[1].elapsed_time(ev[2]))
    mr, mb = statistics.mean(tr), statistics.mean(tb)
    W = g.stats()["W"]
    bloch_bytes = 8 * (g.nblock_R + 2 * len(kf) * g.nblock)  # H(R) read once, each H(k) (complex) written once
    gbs = bloch_bytes / (mb * 1e-3) / 1e9
    return {"keys": int(len(keys)), "elements": int(g.nblock_R), "k_points": len(kf),
            "ms_vlocal_R": mr, "vlocal_R_gpt_pair_s": W / (mr * 1e-3) / 1e9,
            "ms_bloch": mb, "bloch_bytes": bloch_bytes, "bloch_gb_s": gbs,
            "bloch_frac_of_hbm": gbs / hbm_gbs if hbm_gbs else None}


def run_psibeta(g, system, steps, stream, workload):
    """Velocity-gauge projector overlaps <beta| e^{-i A.r} |Phi> (float64, spherical grids of 140 x 162
    points around every projector atom) for every (projector atom, orbital atom) pair of the workload:
    mean time of gint_psibeta with Si projectors (one s and one p channel)."""
    import torch

    from paper_2603_21835_gb300 import inputs

    if any(sp.name != "Si" for sp in system.sp):
        return None
    g.set_projectors([inputs.si_projectors()])
    A = (0.12, -0.07, 0.05)
    out = torch.empty(2 * g.pb_nelems, dtype=torch.float64, device="cuda")
    for _ in range(2):
        g.psibeta(A, out=out, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.psibeta(A, out=out, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    npairs = int(len(g.pb_pairs))
    points = npairs * 140 * 162
    # float64 roofline: the kernel's executed float64 flops per launch (2 DFMA + DADD + DMUL, counted by
    # ncu on this workload with the current source) over the CUDA-event time, against the nominal rate
    fl, src = profiled(workload, "f64", "gint_pb.cu", "fp64_flops_per_launch")
    roof = {"bound": "fp64", "kernel": "k_psibeta", "unit": "TFLOP/s", "peak": FP64_NOMINAL_TFLOPS,
            "peak_source": "nominal (none measured)", "flops_source": src,
            "achieved": None if fl is None else fl / (ms * 1e-3) / 1e12}
    roof["frac"] = None if fl is None else roof["achieved"] / FP64_NOMINAL_TFLOPS
    roof["fp64_pipe_active_ncu"] = profiled(workload, "f64", "gint_pb.cu", "fp64_pipe_active")[0]
    return {"pairs": npairs, "elements": int(g.pb_nelems), "ms": ms, "pairs_per_s": npairs / (ms * 1e-3),
            "grid_points_per_s": points / (ms * 1e-3), "precision": "f64", "roofline": roof,
            "quadrature": "140 Gauss-Legendre radial x 162-point degree-17 product angular rule"}


def run_cn(n, nocc, steps, stream):
    """Density-matrix build, one Crank-Nicolson step (float64 GEMMs and the complex symmetric L D L^T
    factorisation and solves, the library's own kernels) for an n x n basis and nocc states, and the
    energy-density matrix (real GEMM, L D L^T and solves): mean times over `steps` calls."""
    import numpy as np
    import torch

    from paper_2603_21835_gb300 import gint as G

    try:
        cn = G.CrankNicolson(n, nocc)
    except G.GintError as e:
        return {"unavailable": str(e)}
    rng = np.random.default_rng(0)
    S = torch.eye(n, dtype=torch.float64, device="cuda") + 1e-3 * torch.from_numpy(rng.normal(size=(n, n))).cuda()
    S = 0.5 * (S + S.T)
    H = torch.from_numpy(rng.normal(size=(n, n))).cuda()
    H = 0.5 * (H + H.T)
    psi = torch.from_numpy(rng.normal(size=(nocc, n)) + 1j * rng.normal(size=(nocc, n))).cuda()
    f = torch.full((nocc,), 2.0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(psi)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    cn.step(S, H, 0.05, psi, out=out, stream=stream)
    cn.density_matrix(out, f, out=D, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ts, td = [], []
    for _ in range(steps):
        ev[0].record(stream)
        cn.step(S, H, 0.05, psi, out=out, stream=stream)
        ev[1].record(stream)
        cn.density_matrix(out, f, out=D, stream=stream)
        ev[2].record(stream)
        ev[2].synchronize()
        ts.append(ev[0].elapsed_time(ev[1]))
        td.append(ev[1].elapsed_time(ev[2]))
    tt = []
    D16 = torch.empty_like(D)
    cn.density_matrix(psi, f, out=D16, stream=stream, precision="f16x3")
    for _ in range(max(steps, 5)):
        ev[0].record(stream)
        cn.density_matrix(psi, f, out=D16, stream=stream, precision="f16x3")
        ev[1].record(stream)
        ev[1].synchronize()
        tt.append(ev[0].elapsed_time(ev[1]))
    te = []
    E = torch.empty_like(D)
    cn.energy_density_matrix(S, H, D, out=E, stream=stream)
    for _ in range(steps):
        ev[0].record(stream)
        cn.energy_density_matrix(S, H, D, out=E, stream=stream)
        ev[1].record(stream)
        ev[1].synchronize()
        te.append(ev[0].elapsed_time(ev[1]))
    info = cn.info()
    cn.close()
    ms_s, ms_d, ms_e, ms_t = statistics.mean(ts), statistics.mean(td), statistics.mean(te), statistics.mean(tt)
    # tensor-core build: tiles I <= J of 128 x 128, K padded to 64, three float16 products per term
    T, kp = (n + 127) // 128, (2 * nocc + 63) // 64 * 64
    tc_flops = 3 * 2.0 * 128 * 128 * kp * (T * (T + 1) // 2)
    # float64 flops executed by the library's kernels: step = S psi (two real GEMMs, 4 n^2 nocc),
    # complex L D L^T (n^3 / 6 complex multiply-adds = 4/3 n^3), two triangular solves (8 n^2 nocc);
    # D = lower triangle of a real GEMM with K = 2 nocc (2 n^2 nocc); E = H D (2 n^3), real L D L^T
    # (n^3 / 3), solves with n right-hand sides (2 n^3)
    fl_step = 12.0 * n * n * nocc + 4.0 / 3.0 * n ** 3
    fl_d, fl_e = 2.0 * n * n * nocc, (4.0 + 1.0 / 3.0) * n ** 3
    step_tf, dm_tf, edm_tf = (fl / (ms * 1e-3) / 1e12 for fl, ms in ((fl_step, ms_s), (fl_d, ms_d), (fl_e, ms_e)))
    return {"n": n, "nocc": nocc, "ms_step": ms_s, "step_tflops": step_tf,
            "ms_density_matrix": ms_d, "dm_tflops": dm_tf,
            "ms_energy_density_matrix": ms_e, "edm_tflops": edm_tf,
            "fp64": {"kernels": "k_gemm, k_ldl_diag, k_trsv (hand-written float64 on the CUDA cores)",
                     "bound": "fp64", "peak_tflops": FP64_NOMINAL_TFLOPS, "peak_source": "nominal (none measured)",
                     "step_frac": step_tf / FP64_NOMINAL_TFLOPS, "dm_frac": dm_tf / FP64_NOMINAL_TFLOPS,
                     "edm_frac": edm_tf / FP64_NOMINAL_TFLOPS},
            "ms_density_matrix_f16x3": ms_t, "dm_f16x3_tflops_real_part": 4.0 * n * n * nocc / (ms_t * 1e-3) / 1e12,
            "dm_f16x3_tensor_tflops": tc_flops / (ms_t * 1e-3) / 1e12,
            "solver_info": info, "precision": "c128 / f64; f16x3 tensor-core D build"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2603_21835_gb300 import gint as G
    from paper_2603_21835_gb300 import inputs

    prec = G.PRECISIONS[args.precision]
    w = inputs.config_workload(args.workload, dense_D=False)
    g = G.Gint(w.system)
    if args.dense_only:
        n = g.norb
        g.close()
        cn = run_cn(n, 128 if n < 2048 else 1024, 3 if n < 2048 else 2, torch.cuda.current_stream())
        if rank == 0:
            print(json.dumps({"workload": args.workload, "crank_nicolson": cn}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    st = g.stats()
    W = st["W"]
    Db_host = g.blocks_from_coefficients(w.C)
    V_host = np.ascontiguousarray(w.V.reshape(-1))
    Db = torch.from_numpy(Db_host).to(dev)
    V = torch.from_numpy(V_host).to(dev)
    rho = torch.empty(g.grid, dtype=torch.float64, device=dev)
    H = torch.empty(g.nblock, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2
    tensor = args.precision in TENSOR_PRECISIONS

    def new_events(n):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:  # CUDA events are created on first record
            a.record(stream)
            b.record(stream)
        return evs

    def step(kev=None, rev=None, hev=None):
        """One step: density + local-H passes.  Tensor-core precisions: one call, both passes'
        bricks in one persistent launch (kev brackets that kernel); SIMT: two calls."""
        if tensor:
            g.run(Db, V, prec, rho=rho, H=H, kernel_events=kev)
        else:
            if rev:
                rev[0].record(stream)
            g.rho(Db, prec, out=rho)
            if rev:
                rev[1].record(stream)
                hev[0].record(stream)
            g.vlocal(V, prec, out=H)
            if hev:
                hev[1].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev, evk, evr, evh = (new_events(args.steps) for _ in range(4))
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(evk[k], evr[k], evh[k])
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    t_steps = [a.elapsed_time(b) for a, b in ev]
    # the passes one at a time, and the force pass (informational, outside the timed steps)
    t_rho, t_h, t_f = [], [], []
    F = torch.empty((g.natoms, 3), dtype=torch.float64, device=dev)
    for k in range(3):
        for fn, lst in ((lambda: g.rho(Db, prec, out=rho), t_rho), (lambda: g.vlocal(V, prec, out=H), t_h),
                        (lambda: g.force(Db, V, prec, out=F), t_f)):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            lst.append(a.elapsed_time(b))
    # the local-H pass alone with the strict float64 cross-brick reduction (every tile value added
    # in float64) instead of the default double-float sums
    t_h64 = []
    if tensor:
        g.set_reduction("fp64")
        for k in range(3):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.vlocal(V, prec, out=H)
            b.record(stream)
            torch.cuda.synchronize()
            t_h64.append(a.elapsed_time(b))
        g.set_reduction("double-float")
    # new positions (a molecular-dynamics step), on a second handle of the same system with a 0.5 Bohr
    # pair skin: neighbour lists rebuilt on the device, then the plan records only (moves of 1e-6 Bohr
    # keep every brick's atoms) or the whole tensor-core layout (moves of N(0, 0.02) Bohr change some
    # bricks' atom sets); host wall clock around the synchronous call
    t_pos = {}
    if not args.no_extras and tensor:
        try:
            gp = G.Gint(w.system, skin=0.5)
            pos0 = torch.from_numpy(np.ascontiguousarray(w.system.pos)).to(dev)
            for kind, sig in (("same_bricks", 1e-6), ("new_bricks", 0.02)):
                ts = []
                for k in range(3):
                    gen = torch.Generator(device="cpu").manual_seed(100 + k)
                    p2 = pos0 + sig * torch.randn(pos0.shape, generator=gen, dtype=torch.float64).to(dev)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    gp.set_positions(p2)
                    torch.cuda.synchronize()
                    ts.append(1e3 * (time.perf_counter() - t0))
                t_pos[kind] = statistics.median(ts)
            gp.close()
        except G.GintError as e:  # informational: the line is still printed
            t_pos = {"error": str(e)}
    ms_per_step = max_over_ranks(sum(t_steps), world, dev) / args.steps
    value = world * 2.0 * W / (ms_per_step * 1e-3) / 1e9

    # the float64 GPU path on the same workload and inputs (CUDA cores; the comparator of the
    # mixed-precision path), timed the same way: density + local-H passes, L2 flushed
    fp64_gpu = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        g.rho(Db, G.FP64, out=rho)
        g.vlocal(V, G.FP64, out=H)
        torch.cuda.synchronize()
        t64 = []
        for k in range(args.fp64_steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.rho(Db, G.FP64, out=rho)
            g.vlocal(V, G.FP64, out=H)
            b.record(stream)
            b.synchronize()
            t64.append(a.elapsed_time(b))
        ms64 = max_over_ranks(statistics.mean(t64), world, dev)
        v64 = world * 2.0 * W / (ms64 * 1e-3) / 1e9
        fp64_gpu = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
                    "kernels": "k_simt_rho, k_simt_vlocal (float64 CUDA cores)",
                    "mixed_over_fp64": value / v64}

    # roofline of the dominant kernel (per-launch mean over the timed region, CUDA events on its stream)
    peaks, peak_kind = load_peaks()
    if tensor:
        dom, tdom = "k_tc_fused (density + local-H bricks)", statistics.mean(a.elapsed_time(b) for a, b in evk)
        # 2 flops (one multiply-add) per ordered orbital pair per grid point per pass, both passes in
        # this launch; the kernels use the symmetry of D and H and execute about half of it
        flops = 4.0 * W
    else:
        mr = statistics.mean(a.elapsed_time(b) for a, b in evr)
        mh = statistics.mean(a.elapsed_time(b) for a, b in evh)
        dom, tdom = ("k_simt_rho", mr) if mr >= mh else ("k_simt_vlocal", mh)
        flops = 2.0 * W  # one pass per launch, 2 flops per ordered orbital pair per grid point
    if tensor:
        peak = peaks.get("bf16_tflops")
        bound, punit = "tensor", "TFLOP/s"
        pdesc = f"f16 dense = {peak_kind} bf16 burst (nominal f16 and bf16 dense rates are equal)"
    elif args.precision == "fp64":
        peak = FP64_NOMINAL_TFLOPS
        bound, punit, pdesc = "alu", "TFLOP/s", "fp64 nominal 1.25 TFLOP/s (GB300)"
    else:
        mhz = clocks.get("sm_mhz") or 2070.0
        peak = FP32_SIMT_TFLOPS_PER_GHZ * mhz / 1e3
        bound, punit, pdesc = "alu", "TFLOP/s", "fp32 SIMT 152 SMs x 128 lanes x 2 flops x sampled SM clock"
    achieved = flops / (tdom * 1e-3) / 1e12
    traffic, traffic_src = profiled_traffic(args.workload, args.precision) if tensor else (None, None)
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": punit,
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src, "peak_source": pdesc,
                "algorithmic_flops_per_launch": flops}

    # end to end through the public API: pinned host in, pinned host out, copies in the timed region
    e2e = None
    if not args.no_e2e:
        Dh = torch.from_numpy(Db_host).pin_memory()
        Vh = torch.from_numpy(V_host).pin_memory()
        rho_h = torch.empty(g.grid, dtype=torch.float64).pin_memory()
        H_h = torch.empty(g.nblock, dtype=torch.float64).pin_memory()
        Dd = torch.empty_like(Db)
        Vd = torch.empty_like(V)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        te = []
        for k in range(args.steps + 1):
            flush.fill_(float(k))
            e0.record(stream)
            Dd.copy_(Dh, non_blocking=True)
            Vd.copy_(Vh, non_blocking=True)
            if tensor:
                g.run(Dd, Vd, prec, rho=rho, H=H)
            else:
                g.rho(Dd, prec, out=rho)
                g.vlocal(Vd, prec, out=H)
            rho_h.copy_(rho, non_blocking=True)
            H_h.copy_(H, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                te.append(e0.elapsed_time(e1))
        ms_e2e = max_over_ranks(sum(te), world, dev) / len(te)
        e2e = {"value": world * 2.0 * W / (ms_e2e * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(Db.numel() * 8 + V.numel() * 8),
               "d2h_bytes_per_step": int(rho.numel() * 8 + H.numel() * 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, _ = oracle_sample(args.workload, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0 and not args.no_extras:
        serving = run_serving(args, prec, dev)

    per_R = None
    if rank == 0 and tensor and not args.no_extras:
        per_R = run_per_R(g, V, prec, args.steps, stream, flush, peaks.get("hbm_gbs"))

    psibeta = None
    if rank == 0 and tensor and not args.no_extras:
        psibeta = run_psibeta(g, w.system, 3, stream, args.workload)

    cn = None
    if rank == 0 and tensor and not args.no_extras and not args.no_dense:
        cn = run_cn(g.norb, 128 if g.norb < 2048 else 1024, 3 if g.norb < 2048 else 2, stream)

    launches = KERNEL_LAUNCHES.get(args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "f16x3": "f16x3+f64",
                                      "f16x1": "f16+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "natoms": g.natoms, "norb": g.norb, "grid": list(g.grid),
                   "precision": args.precision, "W_pairs_per_pass": W, "W_exec_padded": st["W_exec"],
                   "nbricks": st["nbricks"], "max_brick_orb": st["max_brick_orb"], "handle_bytes": g.memory(),
                   "l2": "flushed (256 MB write)",
                   "parallelism": f"replicas{world}"},
        "ms_kernel": tdom, "ms_rho_alone": statistics.mean(t_rho), "ms_vlocal_alone": statistics.mean(t_h),
        "ms_force_alone": statistics.mean(t_f),
        "ms_vlocal_alone_fp64_reduction": statistics.mean(t_h64) if t_h64 else None,
        "ms_set_positions": t_pos or None,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "fp64_gpu": fp64_gpu,
        "mixed_over_fp64": fp64_gpu["mixed_over_fp64"] if fp64_gpu else None,
        "gpu_launches": launches * args.steps, "serving": serving, "per_R": per_R, "psibeta": psibeta,
        "crank_nicolson": cn,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
