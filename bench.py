"""Benchmark of the Roe-AM SSP-RK3 step on GB300.

Default workload: a batch of 512 independent periodic 2D Euler grids with seeded sizes
from 32x32 to 512x256, free-stream Mach log-uniform in [0.001, 20] with Gaussian density
and pressure bumps, FP32 state and flux arithmetic, first-order Roe-AM, CFL 0.5, per-grid
dt; all grids advance in one persistent launch per Runge-Kutta stage, replayed from a
captured CUDA graph. Metric: cell-updates per second per RK stage (whole job).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch|warped-slabs]

With N > 1 every rank advances its own seeded batch (weak scaling, no data-path collective);
rank 0 prints one JSON line with the max-over-ranks time. Under torchrun the ranks come from
the environment (WORLD_SIZE must equal N); without it bench.py starts N ranks itself, one per
GPU, over NCCL. `--workload warped-slabs` times the 4096 x 4096 curvilinear workload split
into N row slabs, one per rank, with the ghost rows exchanged over NCCL in device memory
while each slab's interior is computed (strong scaling: the grid is fixed).
`--impl reference` times the CPU oracle (the FP64 C program under oracle/) on a bounded
sample of the same workload on this host's cores.
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

import workloads as W  # noqa: E402

METRIC = "Gcell-updates/s per RK stage"
UNIT = "Gcell-updates/s"
# Algorithmic HBM bytes per cell per RK stage in FP32 with each state read once per stage:
# stage 1 reads U^n and writes U1 (32 B); stages 2-3 read U^(k) and U^n and write (48 B).
BYTES_PER_CELL_STAGE = {32: (32 + 48 + 48) / 3.0, 64: 2 * (32 + 48 + 48) / 3.0}
WORKLOAD = ("batched FP32: 512 independent periodic 2D Euler grids, sizes U{32..512} x U{32..256} (seed 20171127), "
            "free-stream Mach 10^U(-3, log10 20) with Gaussian rho/p bumps of amplitude 0.1, first-order Roe-AM, "
            "SSP-RK3 at CFL 0.5 with per-grid dt, one persistent launch per stage, CUDA-graph replay")


def MEASURED_HBM():
    return peaks()[0]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ("paper_1711_09272_gb300/csrc/roeam_kernels.cuh", "paper_1711_09272_gb300/csrc/roeam_internal.h")


def kernel_hash() -> str:
    """Hash of the stage kernel's sources; ncu traffic figures are only reported for the kernel
    version they were measured on."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(name="stage_kernel_traffic.json"):
    """A committed ncu record of a stage kernel (profiles/<name>: the headline kernel's, or the
    reconstructing curvilinear kernel's), or None when it belongs to another kernel version."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    return d if d.get("kernel_hash") == kernel_hash() else None


def measured_traffic(ncells: int):
    """DRAM bytes per stage-kernel launch from the committed ncu record, scaled to this launch
    size, or None when the record belongs to another kernel version."""
    d = traffic_record()
    return None if d is None else d["dram_bytes_per_cell_per_launch"] * ncells


def issue_ceiling(sm_mhz, record="stage_kernel_traffic.json", bytes_per_cell=BYTES_PER_CELL_STAGE[32]):
    """Instruction-issue ceiling of a stage kernel from its committed ncu record: warp
    instructions per cell and stage (w) at the sampled SM clock, 4 issue slots per SM and cycle
    on 152 SMs: cells/s = 152 * 4 * f / w at 100 % issue, and at the issue rate ncu measured."""
    d = traffic_record(record)
    if d is None or not d.get("warp_inst_per_cell") or not sm_mhz:
        return None
    w = d["warp_inst_per_cell"]
    full = 152 * 4 * sm_mhz * 1e6 / w / 1e9
    act = d.get("issue_active_pct")
    return {"warp_inst_per_cell": w, "issue_active_pct": act, "gcell_at_full_issue": full,
            "gcell_at_measured_issue": None if act is None else full * act / 100.0,
            "hbm_frac_at_full_issue": full * bytes_per_cell / MEASURED_HBM()}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Every rank advances its own independent batch (weak scaling): seed of rank r."""
    return W.DEFAULT_SEED + rank


def reduce_max(value: float, world: int, device: str = "cuda") -> float:
    """Max over ranks of a per-rank time (the only collective of the benchmark)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: int, world: int, device: str = "cuda") -> int:
    """Sum over ranks of a per-rank count (the cells of every rank's batch; reporting only)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def weak_value(total_cells: int, steps: int, ms: float) -> float:
    """Whole-job Gcell-updates per second per RK stage: all ranks' cells (each rank its own
    batch) x 3 stages x steps over the slowest rank's time."""
    return total_cells * 3 * steps / (ms * 1e-3) / 1e9


def cpu_baseline(specs, states, steps: int = 1, budget_s: float = 20.0):
    """Times the FP64 C oracle (single thread, as it stands) on the first grids of the batch
    until `budget_s` is reached; returns (Gcell-updates/s per stage, sample description)."""
    import oracle
    cells, t_total, used = 0, 0.0, 0
    for spec, U in zip(specs, states):
        g = oracle.OracleGrid(spec)
        t0 = time.perf_counter()
        g.step(U, cfl=0.5, nsteps=steps)
        t_total += time.perf_counter() - t0
        cells += spec.ncells * 3 * steps
        used += 1
        if t_total > budget_s:
            break
    return cells / t_total / 1e9, f"first {used} of {len(specs)} grids of the same batch, {steps} SSP-RK3 step(s) each"


def time_single(P, torch, spec, U, prec, steps, cfl=0.5, dt_fixed=0.0, warmup=3):
    """Device time of `steps` steps of one grid; returns (ms per step, final state)."""
    stream = torch.cuda.current_stream()
    with P.Batch([spec], precision=prec, cuda_stream=stream.cuda_stream) as b:
        b.set_state(U, 0)
        b.step(cfl, dt_fixed=dt_fixed, nsteps=warmup)
        b.set_state(U, 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(cfl, dt_fixed=dt_fixed, nsteps=steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, b.get_state(0)


def precision_comparison(P, torch, n=1024, t_end=1.0):
    """FP32 vs FP64 on one grid at the same discretisation (isentropic vortex, first order,
    identical fixed time steps): speed and L2 density error against the exact solution."""
    spec, U = W.isentropic_vortex(n)
    with P.Batch([spec], precision=64) as b:
        b.set_state(U, 0)
        dt0 = b.step(0.5, nsteps=1, want_dt=True)[0]
    steps = int(np.ceil(t_end / dt0))
    dt = t_end / steps
    _, Ue = W.isentropic_vortex(n, t=t_end)
    out = {"workload": f"isentropic vortex {n}x{n} periodic, first order, t = {t_end}, {steps} steps of dt = {dt:.3e}"}
    for prec in (32, 64):
        ms, Uf = time_single(P, torch, spec, U, prec, steps, dt_fixed=dt)
        out[f"fp{prec}"] = {"gcell_updates_per_s_per_stage": spec.ncells * 3 / (ms * 1e-3) / 1e9,
                            "ms_per_step": ms, "l2_rho_error": float(np.sqrt(np.mean((Uf[0] - Ue[0]) ** 2)))}
    return out


def oracle_comparison(P):
    """Part of the CPU-baseline leg (the one place besides the reference arm where the bench runs
    the oracle): FP32 (and FP64) GPU results against the FP64 oracle: the per-step error relative to the
    step's increment on the low-Mach Gresho vortex (256 x 256, M = 0.01, MUSCL minmod: the
    increment is a small fraction of the state there), and the L2 state difference after N
    steps of independent trajectories from the same state (isentropic vortex 64 x 64, 100
    steps; Gresho vortex 256 x 256, 100 steps)."""
    import oracle
    out = {}
    spec, U = W.gresho(256, mach=0.01)
    for prec in (32, 64):
        with P.Batch([spec], precision=prec) as b:
            b.set_state(U, 0)
            U0 = b.get_state(0)
            b.step(0.5, nsteps=1)
            Ug = b.get_state(0)
        Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.5)
        d = np.abs(Ug - Uo).reshape(4, -1).max(axis=1)
        inc = np.abs(Uo - U0).reshape(4, -1).max(axis=1)
        scale = np.abs(Uo).reshape(4, -1).max(axis=1)
        out[f"gresho_256_one_step_fp{prec}"] = {"increment_rel_err": [float(x) for x in d / inc],
                                               "state_rel_err": [float(x) for x in d / scale],
                                               "increment_over_state": [float(x) for x in inc / scale]}
    for name, (spec, U), n, precs in (("vortex_64_100_steps", W.isentropic_vortex(64), 100, (32, 64)),
                                      ("gresho_256_100_steps", W.gresho(256, mach=0.01), 100, (32,))):
        for prec in precs:
            with P.Batch([spec], precision=prec) as b:
                b.set_state(U, 0)
                U0 = b.get_state(0)
                b.step(0.5, nsteps=n)
                Ug = b.get_state(0)
            Uo, _ = oracle.OracleGrid(spec).step(U0, cfl=0.5, nsteps=n)
            l2 = np.sqrt(((Ug - Uo) ** 2).reshape(4, -1).sum(axis=1) / (Uo ** 2).reshape(4, -1).sum(axis=1))
            out[f"{name}_fp{prec}_l2_vs_oracle"] = [float(x) for x in l2]
    return out


def warped_step_speed(P, torch, steps=20):
    """The large curvilinear FP32 workload (4096 x 4096 warped grid, Mach-3 step, MUSCL van
    Leer, solid block): device speed and its HBM fraction (50.67 algorithmic B/cell/stage)."""
    spec, U = W.warped_step(4096, 4096)
    ms, _ = time_single(P, torch, spec, U, 32, steps)
    v = spec.ncells * 3 / (ms * 1e-3) / 1e9
    peak, kind = peaks()
    rec = traffic_record("stage_kernel_curvilinear_record.json")
    return {"workload": "warped step 4096x4096 FP32, MUSCL van Leer, solid block, walls/inflow/outflow",
            "gcell_updates_per_s_per_stage": v, "ms_per_step": ms,
            "hbm_frac": v * (128.0 / 3 + 8) / peak, "peak_gbs": peak, "peak_kind": kind,
            "traffic_bytes_per_cell": None if rec is None else rec["dram_bytes_per_cell_per_launch"],
            "issue_ceiling": issue_ceiling(2070.0, "stage_kernel_curvilinear_record.json", 128.0 / 3 + 8)}


def cpu_baseline_curvilinear():
    """The FP64 CPU oracle, one thread, on the curvilinear workload (warped step, MUSCL van Leer,
    solid block) at 512 x 512 cells for one SSP-RK3 step: the CPU rate beside the 4096^2 line."""
    import oracle
    oracle.build()
    spec, U = W.warped_step(512, 512)
    t0 = time.perf_counter()
    oracle.OracleGrid(spec).step(U, cfl=0.5)
    t = time.perf_counter() - t0
    return {"value": spec.ncells * 3 / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one SSP-RK3 step of the warped-step workload at 512 x 512 cells, FP64 C oracle, one thread"}


def cpu_baseline_small_configs():
    """The FP64 CPU oracle, one thread, on the small paper-scale workloads of `small_configs`:
    ms per SSP-RK3 step (one step each, the same settings as the GPU measurement)."""
    import oracle
    oracle.build()
    cases = [("vortex_64_fp64", W.isentropic_vortex(64), dict()),
             ("gresho_256", W.gresho(256, mach=0.01), dict()),
             ("quirk_800x20", W.quirk(800, 20, eps_y=1e-6), dict(cfl=0.25)),
             ("cylinder_ogrid_100x72", W.cylinder_ogrid(mach=0.1), dict()),
             ("blunt_body_160x20", W.cylinder_blunt(), dict(dt_fixed=1e-5)),
             ("corner_400x400", W.supersonic_corner(400), dict(dt_fixed=2e-5)),
             ("wedge_dmr_800x200", W.wedge_dmr(800, 200), dict(dt_fixed=2e-5))]
    out = {}
    for name, (spec, U), kw in cases:
        g = oracle.OracleGrid(spec)
        t0 = time.perf_counter()
        g.step(U, **kw)
        out[name] = {"ms_per_step": (time.perf_counter() - t0) * 1e3, "cores": 1}
    return out


def three_d_speed(P, torch, n=256, nscal=1, steps=20):
    """The 3D path (include/roeam3.h): Taylor-Green vortex on n^3 cells, FP32, one passive
    scalar, first order. Algorithmic bytes per cell and stage: (5 + nscal) 4-byte variables read
    once and written once, plus the U^n read in stages 2-3, i.e. 8/3 x 4 (5 + nscal)."""
    spec, U = W.taylor_green3(n, mach=0.1, nscal=nscal)
    stream = torch.cuda.current_stream()
    with P.Batch3([spec], precision=32, cuda_stream=stream.cuda_stream) as b:
        b.set_state(U, 0)
        b.step(0.5, nsteps=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(0.5, nsteps=steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.check()
        ms = e0.elapsed_time(e1) / steps
    v = spec.ncells * 3 / (ms * 1e-3) / 1e9
    bpc = 8.0 / 3.0 * 4 * (5 + nscal)
    peak, kind = peaks()
    return {"workload": f"3D Taylor-Green vortex {n}^3 periodic, M = 0.1, {nscal} passive scalar(s), FP32, first order",
            "gcell_updates_per_s_per_stage": v, "ms_per_step": ms, "bytes_per_cell_stage": bpc,
            "hbm_frac": v * bpc / peak, "peak_gbs": peak, "peak_kind": kind}


def ablation_speed(P, torch, count=512, steps=50):
    """The ablation-variant kernels (every face on the scalar path) on the benchmark batch with
    the classical Roe flux (Eq. 7 with Eqs. 8-12), FP32, first order."""
    specs, states = W.batch(count)
    specs = [W.with_params(s, scheme=1) for s in specs]
    ncells = sum(s.ncells for s in specs)
    stream = torch.cuda.current_stream()
    with P.Batch(specs, precision=32, cuda_stream=stream.cuda_stream) as b:
        b.set_states(states)
        b.step(0.5, nsteps=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(0.5, nsteps=steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.check()
        ms = e0.elapsed_time(e1) / steps
    return {"workload": f"the {count}-grid batch with the classical Roe flux (ablation kernels), FP32, first order",
            "gcell_updates_per_s_per_stage": ncells * 3 / (ms * 1e-3) / 1e9, "ms_per_step": ms}


def small_configs(P, torch):
    """The small paper-scale workloads, reported for latency (too small to load the HBM): the
    64^2 isentropic vortex (FP64, 100 steps), the 256^2 Gresho vortex at M = 0.01 (MUSCL
    minmod, FP32 and FP64, 2000 steps), the 800 x 20 Quirk duct (FP32, CFL 0.25, 4000 steps) and
    the grids of Sections 7.3-7.6 (cylinder O-grid, blunt body, corner, wedge double-Mach
    reflection): device ms per step through graph replays."""
    out = {}
    spec, U = W.isentropic_vortex(64)
    out["vortex_64_fp64"] = {"ms_per_step": time_single(P, torch, spec, U, 64, 100)[0], "steps": 100}
    for prec in (32, 64):
        spec, U = W.gresho(256, mach=0.01)
        out[f"gresho_256_fp{prec}"] = {"ms_per_step": time_single(P, torch, spec, U, prec, 2000)[0], "steps": 2000}
    spec, U = W.quirk(800, 20, eps_y=1e-6)
    out["quirk_800x20_fp32"] = {"ms_per_step": time_single(P, torch, spec, U, 32, 4000, cfl=0.25)[0], "steps": 4000}
    # the Section 7.3-7.6 grids (FP32, first order; the hypersonic and shock cases at a fixed
    # small dt so that the impulsive start needs no CFL ramp)
    for name, (spec, U), steps, kw in (
            ("cylinder_ogrid_100x72_fp32", W.cylinder_ogrid(mach=0.1), 2000, dict()),
            ("blunt_body_160x20_fp32", W.cylinder_blunt(), 2000, dict(dt_fixed=1e-5)),
            ("corner_400x400_fp32", W.supersonic_corner(400), 500, dict(dt_fixed=2e-5)),
            ("wedge_dmr_800x200_fp32", W.wedge_dmr(800, 200), 500, dict(dt_fixed=2e-5))):
        ms = time_single(P, torch, spec, U, 32, steps, **kw)[0]
        out[name] = {"ms_per_step": ms, "steps": steps,
                     "gcell_updates_per_s_per_stage": spec.ncells * 3 / (ms * 1e-3) / 1e9}
    return out


def _oracle_worker(job):
    """One host process of the all-cores CPU baseline: steps grids w, w + P, w + 2P, ... of the
    seeded batch with the oracle for `budget` seconds of wall time; returns the cell-stages."""
    w, nproc, seed, ngrids, budget = job
    import oracle
    specs, states = W.batch(ngrids, seed=seed)
    cells, k = 0, w
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget:
        oracle.OracleGrid(specs[k]).step(states[k], cfl=0.5)
        cells += specs[k].ncells * 3
        k = (k + nproc) % ngrids
    return cells, time.perf_counter() - t0


def cpu_baseline_all_cores(seed: int, ngrids: int, budget_s: float):
    """The same oracle run as independent processes on every host core (the batch's grids are
    independent problems); returns (Gcell-updates/s per stage, cores)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    nproc = os.cpu_count() or 1
    import oracle
    oracle.build()
    # spawned workers (never forked from a process that has touched the GPU); the executor
    # fails loudly if a worker dies
    with ProcessPoolExecutor(nproc, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, [(w, nproc, seed, ngrids, budget_s) for w in range(nproc)], timeout=600))
    cells = sum(c for c, _ in res)
    wall = max(t for _, t in res)
    return cells / wall / 1e9, nproc


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    specs, states = W.batch(512, seed=W.DEFAULT_SEED)
    import oracle
    oracle.build()
    total_cells = 0
    times = []
    ncores = 1
    # each step: one SSP-RK3 step of consecutive grids of the batch for a bounded time, sized so
    # that the whole run stays within about two minutes
    budget = max(0.05, min(2.0, 120.0 / (args.steps + args.warmup)))
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cells = 0
        k = (it * 5) % len(specs)
        while time.perf_counter() - t0 < budget:
            s, U = specs[k], states[k]
            oracle.OracleGrid(s).step(U, cfl=0.5)
            cells += s.ncells * 3
            k = (k + 1) % len(specs)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            total_cells += cells
    value = total_cells / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "sample": f"each step: consecutive grids of the batch for {budget:.2f} s, one SSP-RK3 step each"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"FP64 C oracle, single thread, consecutive grids of the batch, {budget:.2f} s per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_1711_09272_gb300 as P

    prec = 32
    specs, states = W.batch(args.grids, seed=rank_seed(rank), recon=W.RECON_FIRST)
    ncells = sum(s.ncells for s in specs)
    stream = torch.cuda.current_stream()
    b = P.Batch(specs, precision=prec, device=local, cuda_stream=stream.cuda_stream)
    packed = np.concatenate([U.ravel() for U in states])
    b.set_state(packed, -1)

    tuned = None
    if args.tile_config is not None:
        b.set_tile_config(args.tile_config)
        tuned = {"chosen": args.tile_config, "fixed": True}
    elif not args.no_autotune:
        best, ms = b.autotune(0.5, 3)   # picks the work-unit shape; restores the state
        tuned = {"chosen": int(best), "ms_per_step": [round(float(x), 4) for x in ms]}
    # warm-up (also captures the graph of this (cfl, dt) pair)
    for _ in range(args.warmup):
        b.step(cfl=0.5, nsteps=1)
    b.step(cfl=0.5, nsteps=8)
    b.check()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region: K steps (graph replays + direct remainder)
    l0 = b.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        b.step(cfl=0.5, nsteps=args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = b.launches - l0
    b.check()
    ms = reduce_max(ms, world)
    total_cells = reduce_sum(ncells, world)
    value = weak_value(total_cells, args.steps, ms)

    # ---- per-launch duration of the stage kernel (events around single steps = 3 launches)
    per = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(cfl=0.5, nsteps=1)
        e1.record(stream)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1) / 3.0)
    launch_ms = statistics.median(per)
    peak, peak_kind = peaks()
    alg_bytes = BYTES_PER_CELL_STAGE[prec] * ncells
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers: single-precision host arrays
    # (the state is FP32, so float32 host arrays lose nothing), then float64 ones
    e2e = None
    if not args.no_e2e:
        e2e_steps = 5
        packed32 = packed.astype(np.float32)
        f_in = torch.from_numpy(packed32).pin_memory()
        f_out = torch.empty_like(f_in).pin_memory()
        P.roeam_step_host_f32(b.handle, 0.5, 0.0, 1, f_in, f_out)   # untimed: creates the pipeline streams
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            P.roeam_step_host_f32(b.handle, 0.5, 0.0, 1, f_in, f_out)
        f32_s = reduce_max((time.perf_counter() - t0) / e2e_steps, world)
        h_in = torch.from_numpy(packed).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        P.roeam_step_host(b.handle, 0.5, 0.0, 1, h_in, h_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            P.roeam_step_host(b.handle, 0.5, 0.0, 1, h_in, h_out)
        e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, world)
        # the same through three separate calls (copies not overlapped with the step)
        P.roeam_set_state(b.handle, -1, h_in)
        b.step(cfl=0.5, nsteps=1)
        P.roeam_get_state(b.handle, -1, h_out)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(e2e_steps):
            P.roeam_set_state(b.handle, -1, h_in)
            b.step(cfl=0.5, nsteps=1)
            P.roeam_get_state(b.handle, -1, h_out)
        sep_s = reduce_max((time.perf_counter() - t1) / e2e_steps, world)
        e2e = {"value": total_cells * 3 / f32_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": reduce_sum(packed32.nbytes, world),
               "d2h_bytes_per_step": reduce_sum(packed32.nbytes, world),
               "path": "roeam_step_host_f32(pinned float32 in, pinned float32 out, 1 step): chunked, copies "
                       "overlapped; the FP32 state loses nothing to float32 host arrays",
               "float64_host_arrays": {"value": total_cells * 3 / e2e_s / 1e9,
                                       "h2d_bytes_per_step": reduce_sum(packed.nbytes, world),
                                       "d2h_bytes_per_step": reduce_sum(packed.nbytes, world),
                                       "path": "roeam_step_host(pinned fp64 in, pinned fp64 out, 1 step)"},
               "separate_calls": {"value": total_cells * 3 / sep_s / 1e9,
                                  "path": "roeam_set_state + roeam_rk_step(1) + roeam_get_state (pinned fp64)"}}
        # a caller whose float64 state already lives on the GPU (device-pointer state I/O)
        d_in = h_in.to("cuda")
        d_out = torch.empty_like(d_in)
        b.set_state_device(d_in, -1, stream=stream.cuda_stream)
        b.step(cfl=0.5, nsteps=1)
        b.get_state_device(d_out, -1, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        ed0, ed1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ed0.record(stream)
        for _ in range(e2e_steps):
            b.set_state_device(d_in, -1, stream=stream.cuda_stream)
            b.step(cfl=0.5, nsteps=1)
            b.get_state_device(d_out, -1, stream=stream.cuda_stream)
        ed1.record(stream)
        torch.cuda.synchronize()
        dev_ms = reduce_max(ed0.elapsed_time(ed1) / e2e_steps, world)
        e2e["device_resident_fp64"] = {
            "value": total_cells * 3 / (dev_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": dev_ms,
            "path": "roeam_set_state_device + roeam_rk_step(1) + roeam_get_state_device (float64 CUDA tensors)"}
        del d_in, d_out

    line = None
    if rank == 0:
        cpu_v, cpu_sample, cpu_all = (None, None, None)
        vs_oracle = None
        curv_oracle = small_oracle = None
        if world == 1 and not args.no_cpu:
            cpu_v, cpu_sample = cpu_baseline(specs, states, steps=1, budget_s=args.cpu_budget)
            cpu_all = cpu_baseline_all_cores(rank_seed(rank), args.grids, args.cpu_budget)
            if not args.no_extra:
                vs_oracle = oracle_comparison(P)
                curv_oracle = cpu_baseline_curvilinear()
                small_oracle = cpu_baseline_small_configs()
        traffic = measured_traffic(ncells)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.grids == 512 else WORKLOAD.replace("512", str(args.grids), 1),
                       "grids_per_gpu": len(specs), "cells_per_gpu": ncells,
                       "recon": "first order", "cfl": 0.5, "autotune": tuned,
                       "l2": "inputs larger than L2 (3 state buffers of %.0f MB each)" % (16 * ncells / 1e6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "stage_kernel<float> (fused flux + residual + RK stage)",
                         "bytes_per_cell_stage": BYTES_PER_CELL_STAGE[prec], "launch_ms": launch_ms,
                         "limiter": "instruction issue, not HBM: DRAM traffic equals the algorithmic bytes while "
                                    "issue is the binding resource (issue_ceiling); see the ncu summary of this "
                                    "kernel"},
            "cpu_baseline": None if cpu_v is None else {
                "value": cpu_all[0], "unit": UNIT, "cores": cpu_all[1], "kind": "oracle",
                "sample": f"FP64 C oracle as independent processes, one per core, each stepping its share of "
                          f"the same batch's grids for {args.cpu_budget:.0f} s",
                "single_core": {"value": cpu_v, "cores": 1, "sample": cpu_sample},
                "curvilinear_single_core": curv_oracle,
                "small_configs_single_core": small_oracle,
                "gpu_vs_oracle": vs_oracle},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        line["roofline"]["issue_ceiling"] = issue_ceiling(line["clocks"].get("sm_mhz") or 2070.0)
        if world == 1 and not args.no_extra:
            line["precision_comparison"] = precision_comparison(P, torch)
            line["curvilinear"] = warped_step_speed(P, torch)
            line["three_d"] = three_d_speed(P, torch)
            line["ablation_roe"] = ablation_speed(P, torch)
            line["small_configs"] = small_configs(P, torch)
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_warped_slabs(args):
    """The 4096 x 4096 warped step in row slabs over the ranks (strong scaling)."""
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_1711_09272_gb300 as P  # noqa: F401
    from paper_1711_09272_gb300.slab import DistExchange, LocalExchange, SlabStepper
    spec, U = W.warped_step(4096, 4096)
    ex = DistExchange(torch, device=f"cuda:{local}") if world > 1 else LocalExchange()
    st = SlabStepper(spec, world, [rank], ex, precision=32, device=local, overlap=True)
    st.set_state(U)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        st.step(0.5)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    h = st.handles[rank]
    l0 = h.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        st.step(0.5, nsteps=args.steps)
        ev1.record(stream)
        barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), world)
    launches = h.launches - l0
    h.check()
    value = spec.ncells * 3 * args.steps / (ms * 1e-3) / 1e9
    j0, j1 = st.slabs[rank][1]
    if rank == 0:
        peak, peak_kind = peaks()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "warped step 4096x4096 FP32 (MUSCL van Leer, solid block, walls/inflow/"
                                       "outflow) in %d row slabs, one per GPU; ghost rows over NCCL in device "
                                       "memory, overlapped with each slab's interior" % world,
                           "rows_per_slab": j1 - j0, "cells": spec.ncells,
                           "exchange_bytes_per_stage_per_side": 2 * 4 * 4 * spec.ni},
                "roofline": {"bound": "hbm", "achieved": value * (128.0 / 3 + 8), "peak": peak, "unit": "GB/s",
                             "frac": value * (128.0 / 3 + 8) / (peak * world), "traffic": None,
                             "peak_kind": peak_kind, "bytes_per_cell_stage": 128.0 / 3 + 8},
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    st.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _spawned_rank(local, n, port, argv):
    """One rank started by bench.py itself (no torchrun): the environment torchrun would set."""
    os.environ.update(RANK=str(local), LOCAL_RANK=str(local), WORLD_SIZE=str(n), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.argv = [sys.argv[0]] + argv
    rc = main()
    if rc:
        raise SystemExit(rc)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--grids", type=int, default=512, help="grids in the batch (512 is the benchmark workload)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default work-unit shape")
    ap.add_argument("--tile-config", type=int, default=None, help="use this work-unit shape (profiling runs)")
    ap.add_argument("--no-extra", action="store_true", help="skip the FP32/FP64 and curvilinear side measurements")
    ap.add_argument("--only", choices=["three_d", "ablation_roe", "curvilinear", "small_configs",
                                       "precision_comparison"],
                    help="run one side measurement alone and print its JSON (profiling runs)")
    ap.add_argument("--n3", type=int, default=256, help="cells per side of the 3D side measurement")
    ap.add_argument("--workload", default="batch", choices=["batch", "warped-slabs"],
                    help="batch: the 512-grid benchmark (weak scaling); warped-slabs: the 4096^2 warped step in "
                         "row slabs over the GPUs (strong scaling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    env_world = os.environ.get("WORLD_SIZE")
    if env_world is not None and int(env_world) != args.gpus:
        print(f"bench.py: WORLD_SIZE={env_world} but --gpus {args.gpus}", file=sys.stderr)
        return 2
    if env_world is None and args.gpus > 1:
        # no launcher: start one rank per GPU here (rank 0 prints the line)
        import socket

        import torch
        import torch.multiprocessing as mp
        if torch.cuda.device_count() < args.gpus:
            print(f"bench.py: --gpus {args.gpus} but {torch.cuda.device_count()} GPU(s) visible", file=sys.stderr)
            return 2
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        mp.spawn(_spawned_rank, args=(args.gpus, port, sys.argv[1:]), nprocs=args.gpus, join=True)
        return 0
    if args.workload == "warped-slabs" and args.impl == "ours":
        return run_warped_slabs(args)
    if args.only:
        import torch
        import paper_1711_09272_gb300 as P
        P.load_library()
        fn = {"three_d": lambda: three_d_speed(P, torch, n=args.n3),
              "ablation_roe": lambda: ablation_speed(P, torch),
              "curvilinear": lambda: warped_step_speed(P, torch),
              "small_configs": lambda: small_configs(P, torch),
              "precision_comparison": lambda: precision_comparison(P, torch)}[args.only]
        print(json.dumps({args.only: fn()}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
