"""Throughput benchmark of the coupled ADR lattice (species MLUPS and the HBM
roofline fraction of the fused 3-species stream-collide kernel).

Workload: the large membrane lattice, 16384 x 4096 nodes (67.1M), 2000 seeded
R = 8 fibers in four membranes with alternating A->B / B->C catalysts,
Pe = 50, Da = 0.5, species A, B, C.  Set-up (untimed): raster, upload, flow
(D2Q9 BGK, fixed step count).  One benchmark step = 100 ADR time steps of all
three species, the last two of which also record the concentration change,
followed by the outflux reduction and the efficiency read back to the host:
one pass of the whole hot path.  The population state (14.5 GB in FP32) is
far larger than L2, so no flush is needed between steps.  The flow is solved
once in FP64 and cast to float for the float precisions.

The line is the --precision run (FP32 by default).  On one GPU it also
carries, unless --no-extra: the other two precisions timed the same way
(fewer steps; their own roofline and clocks; the FP64 step's roofline is
its FP64 arithmetic against the FMA rate measured on the same GPU by
lbm_fp64_fma_tflops); an efficiency check at equal step counts, FP32 and
FP16 storage against FP64 on the full lattice (outfluxes on the first
fiber-free plane behind the first (A->B) membrane, and the share of B in the
lattice); and a steady-state check of the outlet efficiency of Eq. (A-B) on
the two-membrane cascade lattice (2048 x 512, Da = 1, Pe = 10): FP64 to a
per-step residual of 1e-9, FP32 to 1e-6, and FP32 and FP16 storage at
FP64's step count.  On the full lattice the C front needs of order 10^5
steps to reach the second membrane, far beyond the bench's time, so the
cascade's non-zero efficiency is checked on the smaller lattice.  Last, the
Pe x Da sweep record: the 64-instance sweep (61 with k < 1), every instance
2000 steps in every precision, one lbm_adr_solve per instance in FP64 and
FP32 against one batch in FP32 and FP16 storage (solves/s and the largest
efficiency difference to FP64 at equal step counts).

python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f16dev|f64]
python bench.py --impl reference ...   # the FP64 CPU oracle on host cores
Under torchrun each rank solves its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CHUNK = 100          # ADR time steps per benchmark step
SPECIES = 3
METRIC = "species MLUPS (ADR, 3 species)"
UNIT = "MLUPS"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lbm", choices=["lbm", "reference"])
    ap.add_argument("--precision", default="f32",
                    choices=["f32", "f16dev", "f64"])
    ap.add_argument("--flow-steps", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--nx", type=int, default=16384)
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--fibers-per-band", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the other precisions' records and the "
                         "equal-step efficiency check")
    ap.add_argument("--extra-steps", type=int, default=5,
                    help="timed bench steps of each other precision")
    ap.add_argument("--eps-steps", type=int, default=3000,
                    help="ADR steps of the equal-step efficiency check")
    ap.add_argument("--workload", default="large",
                    choices=["large", "sweep", "adjoint", "series",
                             "cascade", "noflow", "adjoint-check"],
                    help="large: the 67M-node membrane (default line); "
                         "sweep: the 64-instance Pe x Da sweep, batched "
                         "FP32 / FP16 against unbatched FP64 (solves/s); "
                         "adjoint: discrete-adjoint iterations on the "
                         "67M-node membrane (f32 or f64); series: the "
                         "paper's 2D experiment series (isolated fiber, "
                         "fiber pairs, side-by-side fiber against Pe), "
                         "batched, to steady state; cascade: the "
                         "two-membrane cascade (2048x512) at Da = 1 and "
                         "Pe = 1, 10, 100 to steady state in FP64 and "
                         "FP32; noflow: the pure-diffusion cascade of "
                         "Sec. IV.B (periodic 300x300 box, fiber pair and "
                         "side-by-side fiber, Da = 150 and 1.5)")
    ap.add_argument("--adjoint-iters", type=int, default=200)
    ap.add_argument("--sweep-instances", type=int, default=64)
    ap.add_argument("--sweep-first", type=int, default=0,
                    help="steady sweep: index of the first instance")
    ap.add_argument("--sweep-max-steps", type=int, default=5000)
    ap.add_argument("--sweep-tol", type=float, default=0.0,
                    help="residual tolerance of the sweep solves; 0 (default) "
                         "runs every instance exactly --sweep-max-steps "
                         "steps in every precision")
    ap.add_argument("--sweep-flow-steps", type=int, default=3000)
    ap.add_argument("--sweep-mode", default="fixed", choices=["fixed", "steady"],
                    help="fixed: every instance a fixed step count in every "
                         "precision; steady: every instance to its steady "
                         "state (residual and efficiency tests)")
    ap.add_argument("--fd-steps", type=int, default=400000,
                    help="adjoint-check: steps of each perturbed solve "
                         "after the base state")
    ap.add_argument("--fd-every", type=int, default=50000,
                    help="adjoint-check: record the difference quotient "
                         "every this many steps (0: only at the end)")
    ap.add_argument("--fd-fibers", default="",
                    help="adjoint-check: comma-separated fiber indices "
                         "instead of 16 random ones")
    ap.add_argument("--cascade-pe", default="1,10,100")
    ap.add_argument("--sweep-check-steps", type=int, default=2000,
                    help="steps per instance of the Pe x Da sweep record in "
                         "the default line (0: left out)")
    ap.add_argument("--cascade-check-pe", type=float, default=10.0,
                    help="Pe of the two-membrane cascade steady-state check "
                         "in the default line (0: left out)")
    ap.add_argument("--cascade-max-steps", type=int, default=3000000)
    return ap.parse_args()


def _workload(a, seed=0):
    from paper_2109_04455_gb300 import inputs
    return inputs.large_membrane(seed=seed, nx=a.nx, ny=a.ny,
                                 per_band=a.fibers_per_band)


def _config(a, w):
    return {"workload": f"{w.name}: {w.nx}x{w.ny} D2Q9 channel, "
                        f"{w.fibers.shape[0]} R=8 fibers in 4 membranes, "
                        f"species A,B,C, Pe={w.pe:g}, Da={w.da1:g}",
            "nx": w.nx, "ny": w.ny, "species": SPECIES,
            "precision": a.precision, "adr_steps_per_step": CHUNK,
            "flow_steps": a.flow_steps,
            "l2": "inputs larger than L2 (population state >> 129 MB)",
            "parallelism": f"replica per GPU x{a.gpus}"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _loop(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.index),
                     f"--query-gpu={self.Q}", "--format=csv,noheader,nounits"],
                    capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
# algorithmic double flops of one FP64 interior node update with the E table:
# per species 8 additions for C and, per population, C E_i - g and
# g + omega (...) as two FMAs (4 flops)
FP64_FLOPS_PER_NODE = SPECIES * (8 + 9 * 4)


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "f32": ("lbm_kernels.cuh", "lbm_launch_impl.cuh", "kernels_f32.cu"),
    "f16dev": ("lbm_kernels.cuh", "lbm_launch_impl.cuh", "lbm_f16.cuh",
               "kernels_f16dev.cu"),
    "f64": ("lbm_kernels.cuh", "lbm_launch_impl.cuh", "kernels_f64.cu"),
}


def _kernel_source_hash(precision: str):
    """Hash of the sources the precision's step kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2109_04455_gb300", "csrc")
    for f in KERNEL_SOURCES[precision]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(precision: str, units_per_launch: int):
    """DRAM bytes per launch of the ADR step kernel from the committed ncu
    summary, scaled to this launch by fluid nodes; None if the kernel source
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"adr_step_{precision}_ncu.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    try:
        if kv.get("kernel_source_hash") != _kernel_source_hash(precision):
            return None
        per_unit = float(kv["dram_bytes_per_fluid_node"])
        return per_unit * units_per_launch
    except (KeyError, ValueError):
        return None


def _algorithmic_bytes(geom, w, precision):
    """Bytes one ADR step must move: per fluid node 3 species x 9
    populations read + written, the velocity (2 values) and the link word
    (half storage: also each species' half reference, read + written; FP64:
    the nine equilibrium factors instead of the velocity); per solid node
    its link word; the rates of each catalytic link (two doubles)."""
    import numpy as np
    import torch
    es = {"f32": 4, "f16dev": 2, "f64": 8}[precision]
    ue = 8 if precision == "f64" else 4
    n_nodes = geom.nx_pad * geom.ny
    n_solid = geom.n_solid + (geom.nx_pad - geom.nx) * geom.ny
    n_fluid = n_nodes - n_solid
    links = geom.ws[:4 * n_nodes].view(torch.int32).cpu().numpy().view(np.uint32)
    fl = links[links != 0xFFFFFFFF]
    ncat = 0
    for j in range(8):
        ncat += int((((fl >> (4 * j)) & 0xF) == 3).sum())
    per_fluid = SPECIES * 9 * 2 * es + 2 * ue + 4
    if precision == "f16dev":
        per_fluid += SPECIES * 2 * 2   # per-node half reference, read + written
    if precision == "f64":
        per_fluid += 9 * 8 - 2 * ue    # the E_i(u) table is read instead of u
    total = n_fluid * per_fluid + n_solid * 4 + ncat * 16
    return total, n_fluid, per_fluid


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (replicas: no data-path collective)
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, device=None) -> float:
    """Slowest rank's value (the job is done when the last replica is)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or \
            dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, elapsed_s: float,
                   scale: float = 1e-6) -> float:
    """Whole-job rate: units of every rank over the slowest rank's time."""
    return units_per_rank * world / elapsed_s * scale


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def _oracle_sample(w, steps, nxs=1024, nys=512, x0=1536):
    """Crop of the workload (x in [x0, x0+nxs), y in [0, nys)) with the fibers
    that touch it; returns a callable that runs ``steps`` oracle ADR steps
    and the species-node updates it performs."""
    import numpy as np

    import oracle
    fib = w.fibers.copy()
    fib[:, 0] -= x0
    keep = ((fib[:, 0] + fib[:, 2] >= 0) & (fib[:, 0] - fib[:, 2] < nxs) &
            (fib[:, 1] + fib[:, 2] >= 0) & (fib[:, 1] - fib[:, 2] < nys))
    fib = fib[keep]
    solid, kab, kbc = oracle.raster(nxs, nys, fib, w.k1, w.k2)
    _, ux, uy, _ = oracle.flow_run(solid, w.tau_flow, w.u0, 20)
    prob = oracle.ADRProblem(solid, kab, kbc, ux, uy, [w.tau_c] * SPECIES,
                             list(w.c_in))
    state = {"g": prob.init()}

    def run():
        prob.steps(state["g"], steps)
    desc = (f"x in [{x0},{x0 + nxs}) x y in [0,{nys}) crop of the workload "
            f"({int(keep.sum())} fibers), {SPECIES} species, {steps} ADR "
            f"steps per sample, FP64 oracle, {oracle.num_threads()} OpenMP "
            "threads over lattice rows")
    return run, SPECIES * nxs * nys * steps, desc


def _oracle_threads():
    import oracle
    return oracle.num_threads()


def cpu_baseline(w, target_s=12.0):
    run, units, desc = _oracle_sample(w, 5)
    t = time.perf_counter()
    run()
    dt = time.perf_counter() - t
    reps = max(1, int(target_s / max(dt, 1e-3)))
    t = time.perf_counter()
    for _ in range(reps):
        run()
    dt = time.perf_counter() - t
    import oracle
    return {"value": units * reps / dt / 1e6, "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{desc}; {reps} samples, {dt:.1f} s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(a)
    run, units, desc = _oracle_sample(w, 5)
    for _ in range(a.warmup):
        run()
    t = time.perf_counter()
    for _ in range(a.steps):
        run()
    dt = time.perf_counter() - t
    value = units * a.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": _config(a, w),
            "cpu_baseline": {"value": value, "unit": UNIT,
                             "cores": _oracle_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def _gpu_index(dev):
    gpu_index = dev.index
    try:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            gpu_index = int(vis.split(",")[dev.index])
    except ValueError:
        pass
    return gpu_index


def _measure(precision, geom, w, u, steps, warmup, dev, world, fp64_peak):
    """Time `steps` bench steps (CHUNK ADR steps each, the last two checked,
    then the outflux and the efficiency read back) of one precision after
    `warmup` untimed ones.  Returns the record (throughput, the roofline of
    the step kernel, clocks, launches) and the solver."""
    import torch

    from paper_2109_04455_gb300 import lbm
    prec = lbm.PRECISIONS[precision]
    prm = lbm.adr_params(SPECIES, w.tau_c, w.c_in, precision=prec)
    solver = lbm.ADRSolver(geom, prm, u).init()
    stream = torch.cuda.current_stream()

    def bench_step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        solver.run(CHUNK - 2, check=False)
        if evs is not None:
            evs[1].record(stream)
        return solver.run(2)

    info = None
    for _ in range(warmup):
        info = bench_step()
    ev_plain = [(torch.cuda.Event(enable_timing=True),
                 torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(_gpu_index(dev)) as clk:
        t0.record(stream)
        for k in range(steps):
            info = bench_step(ev_plain[k])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    elapsed = max_over_ranks(t0.elapsed_time(t1) * 1e-3, dev)
    plain_s = sum(e0.elapsed_time(e1) for e0, e1 in ev_plain) * 1e-3
    # per ADR step the bulk kernel and (when the lattice has boundary nodes)
    # the boundary-node kernel; per bench step the two-level partial-sum
    # reduce (2 launches) and the outflux kernel
    lw = geom.ws[:4 * geom.nx_pad * geom.ny].view(torch.int32).cpu().numpy()
    has_bnd = bool(((lw != 0) & (lw != -1)).any())
    launches_per_step = CHUNK * (2 if has_bnd else 1) + 3
    updates = SPECIES * w.nx * w.ny * CHUNK * steps
    value = job_throughput(updates, world, elapsed)
    alg_bytes, n_fluid, per_fluid = _algorithmic_bytes(geom, w, precision)
    step_launch_s = plain_s / ((CHUNK - 2) * steps)
    achieved = alg_bytes / step_launch_s / 1e9
    peak, peak_kind = _peak_hbm()
    traffic = _ncu_traffic(precision, n_fluid)
    kernel = ("adr_bulk_quad_kernel<3 species> (f16dev, plain steps)"
              if precision == "f16dev" else
              f"adr_bulk_kernel<{precision},3 species,step>")
    if precision != "f64":
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} (copy bandwidth)"}
    else:
        tf = FP64_FLOPS_PER_NODE * n_fluid / step_launch_s / 1e12
        roof = {"bound": "alu", "achieved": tf, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": tf / fp64_peak,
                "peak_kind": "measured: lbm_fp64_fma_tflops (independent "
                             "FP64 FMA chains on this GPU, this run)",
                "hbm_gbs": achieved, "hbm_frac": achieved / peak}
    roof.update({"traffic": traffic, "kernel": kernel,
                 "algorithmic_bytes_per_launch": alg_bytes,
                 "bytes_per_fluid_node": per_fluid, "fluid_nodes": n_fluid,
                 "avg_launch_ms": step_launch_s * 1e3})
    rec = {"value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": elapsed / steps * 1e3,
           "dtype": {"f32": "f32", "f16dev": "f16-storage/f32-compute",
                     "f64": "f64"}[precision],
           "roofline": roof, "clocks": clk.summary(),
           "gpu_launches": launches_per_step * steps,
           "eps": info["eps"], "adr_residual": info["residual"]}
    return rec, solver, bench_step


def _eps_check(geom, w, u64, steps, plane, dev):
    """FP32 and FP16 storage against FP64 on the full lattice at equal step
    counts from the same start on the same FP64 flow: outfluxes on a plane
    just behind the first (A->B) membrane, and the lattice's amount of each
    species.  Reports each precision's fluxes, the A->B efficiency
    N_B / (N_A + N_B) on that plane, the cascade efficiency of Eq. (A-B)
    (N_C / sum N), the share of B in the lattice's species (the conversion
    so far) and the differences to FP64."""
    import torch

    from paper_2109_04455_gb300 import lbm
    out = {"plane": plane, "steps": steps,
           "flow": "FP64 (cast to float for FP32 / FP16)"}
    ref = None
    for name in ("f64", "f32", "f16dev"):
        prec = lbm.PRECISIONS[name]
        prm = lbm.adr_params(SPECIES, w.tau_c, w.c_in, precision=prec,
                             max_steps=steps, x_plane=plane)
        _, info = lbm.lbm_adr_solve(geom, prm, u64 if name == "f64"
                                    else u64.float(), want_conc=False)
        torch.cuda.empty_cache()
        f, m = info["flux"], info["mass"]
        rec = {"flux": f, "eps_ab": f[1] / (f[0] + f[1]),
               "eps": info["eps"], "c_min": info["c_min"], "mass": m,
               "conversion_b": m[1] / sum(m)}
        if ref is None:
            ref = rec
        else:
            rec["eps_ab_err_vs_f64"] = abs(rec["eps_ab"] - ref["eps_ab"])
            rec["eps_err_vs_f64"] = abs(rec["eps"] - ref["eps"])
            rec["conversion_b_err_vs_f64"] = abs(rec["conversion_b"]
                                                 - ref["conversion_b"])
            rec["flux_rel_err_vs_f64"] = max(
                abs(a - b) / abs(ref["flux"][0]) for a, b in zip(f, ref["flux"]))
        out[name] = rec
    return out


def run_gpu(a):
    import torch
    import torch.distributed as dist

    from paper_2109_04455_gb300 import lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = _workload(a, seed=rank)

    # ---- set-up (untimed): raster, upload, flow (FP64: one velocity field
    # for every precision, cast to float for the float paths)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload(dev)
    stream = torch.cuda.current_stream()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    f0.record(stream)
    u64, finfo = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, a.flow_steps,
                                    precision=lbm.LBM_F64)
    f1.record(stream)
    torch.cuda.synchronize()
    flow_ms = f0.elapsed_time(f1)
    flow_mlups = w.nx * w.ny * a.flow_steps / (flow_ms * 1e-3) / 1e6
    fp64_peak = lbm.lbm_fp64_fma_tflops()

    def vel(precision):
        return u64 if precision == "f64" else u64.float()

    main, solver, bench_step = _measure(a.precision, geom, w,
                                        vel(a.precision), a.steps, a.warmup,
                                        dev, world, fp64_peak)

    # ---- end to end through the public API with host buffers
    u = solver.u
    ws_host = torch.empty(geom.ws.numel(), dtype=torch.uint8, pin_memory=True)
    ws_host.copy_(geom.ws)
    u_host = torch.empty(u.shape, dtype=u.dtype, pin_memory=True)
    u_host.copy_(u)
    h2d = ws_host.numel() + u_host.numel() * u_host.element_size()
    d2h = 24 * 8
    e2e_steps = max(1, a.e2e_steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    ev_copy = [(torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    e0.record(stream)
    for k in range(e2e_steps):
        ev_copy[k][0].record(stream)
        geom.ws.copy_(ws_host, non_blocking=True)
        u.copy_(u_host, non_blocking=True)
        ev_copy[k][1].record(stream)
        bench_step()          # ends with the D2H read of flux / eps
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dev)
    h2d_ms = sum(c0.elapsed_time(c1) for c0, c1 in ev_copy) / e2e_steps
    e2e_value = job_throughput(SPECIES * w.nx * w.ny * CHUNK * e2e_steps,
                               world, e2e_s)
    solver.close()
    del solver, bench_step
    torch.cuda.empty_cache()

    # ---- the other precisions (timed the same way, fewer steps) and the
    # efficiency check at equal step counts (one GPU only)
    others, eps_check, cascade, sweep = {}, None, None, None
    if world == 1 and not a.no_extra:
        # each record is optional: one that fails is reported in its place
        # (its error text), and the headline record above still prints
        def guarded(fn):
            try:
                return fn()
            except Exception as e:   # noqa: BLE001 (reported, not hidden)
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
                return {"error": f"{type(e).__name__}: {e}"}

        def other(name):
            rec, sv, _ = _measure(name, geom, w, vel(name), a.extra_steps, 3,
                                  dev, world, fp64_peak)
            sv.close()
            torch.cuda.empty_cache()
            return rec

        for name in ("f32", "f16dev", "f64"):
            if name != a.precision:
                others[name] = guarded(lambda: other(name))
        # the first fiber-free column behind the first (A->B) membrane
        # (fiber surfaces end at x = 2 W / 9): B made by the band's last
        # fibers crosses it within these steps
        plane = int(math.ceil(2.0 * w.nx / 9.0)) + 1
        eps_check = guarded(lambda: _eps_check(geom, w, u64, a.eps_steps,
                                               plane, dev))
        if a.cascade_check_pe > 0:
            cascade = guarded(lambda: cascade_rows([a.cascade_check_pe],
                                                   a.cascade_max_steps))
        if a.sweep_check_steps > 0:
            sweep = guarded(lambda: sweep_record(
                a.sweep_instances, a.sweep_check_steps, a.sweep_flow_steps,
                0.0))

    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": main["dtype"],
            "data": "synthetic (seeded fiber geometry)",
            "config": _config(a, w),
            "roofline": main["roofline"],
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_s / e2e_steps * 1e3,
                    "h2d_ms_per_step": h2d_ms},
            "gpu_launches": main["gpu_launches"],
            "clocks": main["clocks"],
            "flow": {"mlups": flow_mlups, "steps": a.flow_steps,
                     "precision": "f64", "residual": finfo["residual"]},
            "eps": main["eps"], "adr_residual": main["adr_residual"],
            "fp64_fma_tflops_measured": fp64_peak,
        }
        if others:
            line["other_precisions"] = others
        if eps_check:
            line["eps_check"] = eps_check
        if cascade:
            line["cascade_check"] = cascade
        if sweep:
            line["sweep"] = sweep
        if not a.no_cpu_baseline and world == 1:
            try:
                line["cpu_baseline"] = cpu_baseline(w)
            except Exception as e:   # noqa: BLE001 (reported, not hidden)
                line["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Pe x Da sweep: batched reduced precision against unbatched FP64
# ---------------------------------------------------------------------------
def run_sweep_steady(a):
    """The Pe x Da sweep to steady state.  Untimed: each instance's flow in
    FP64 to a per-step residual of 1e-8.  Timed (CUDA events): every
    instance's ADR solve to its steady state, judged by the per-step
    residual and by the efficiency test (eps_tol: Aitken's extrapolation of
    the last three checks, every 1000 steps): FP64 one lbm_adr_solve per
    instance (residual 1e-9, eps settled to 1e-7: the reference), FP32 the
    same way and in one batch (residual 1e-6, eps 1e-5), FP16 storage in one
    batch (residual 1e-5, above its stochastic-rounding floor; eps 1e-5).
    Reports solves/s, steps, and the largest |eps - eps_FP64| of each."""
    import torch

    from paper_2109_04455_gb300 import inputs, lbm
    torch.cuda.set_device(0)
    ws_all = [inputs.sweep_instance(i) for i in
              range(a.sweep_first, a.sweep_first + a.sweep_instances)]
    ws = [w for w in ws_all if max(w.k1, w.k2) < 1.0]
    geoms, u64 = [], []
    t0 = time.perf_counter()
    flow_steps = 0
    for w in ws:
        g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
        u, fi = lbm.lbm_flow_solve(g, w.tau_flow, w.u0, 1000000, tol=1e-8,
                                   check_every=1000, precision=lbm.LBM_F64)
        flow_steps += fi["steps"]
        geoms.append(g)
        u64.append(u)
    flow_s = time.perf_counter() - t0
    u32 = [u.float() for u in u64]
    cap, check = a.sweep_max_steps, 1000

    def params(prec, tol, eps_tol):
        return [lbm.adr_params(3, w.tau_c, precision=prec, max_steps=cap,
                               tol=tol, eps_tol=eps_tol, check_every=check)
                for w in ws]

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record()
        out = fn()
        ev1.record()
        torch.cuda.synchronize()
        return out, ev0.elapsed_time(ev1) * 1e-3

    def one(g, p, u):
        # a lattice that goes unstable is reported in its row, not raised
        try:
            return lbm.lbm_adr_solve(g, p, u, want_conc=False)[1]
        except lbm.LBMError as e:
            return {"eps": float("nan"), "steps": p.max_steps,
                    "converged": 0, "status": str(e)}

    res = {}
    ref, t64 = timed(lambda: [one(g, p, u) for g, p, u in zip(
        geoms, params(lbm.LBM_F64, 1e-9, 1e-7), u64)])
    res["f64_unbatched"] = (ref, t64)
    print(json.dumps({"phase": "f64_unbatched", "seconds": t64,
                      "flow_seconds_untimed": flow_s,
                      "steps": sum(r["steps"] for r in ref)}), flush=True)
    r32, t32 = timed(lambda: [one(g, p, u) for g, p, u in zip(
        geoms, params(lbm.LBM_F32, 1e-6, 1e-5), u32)])
    print(json.dumps({"phase": "f32_unbatched", "seconds": t32}), flush=True)
    res["f32_unbatched"] = (r32, t32)
    for name, prec, tol in (("f32_batched", lbm.LBM_F32, 1e-6),
                            ("f16dev_batched", lbm.LBM_F16DEV, 1e-5)):
        b = lbm.Batch(geoms, params(prec, tol, 1e-5), u32)
        b.tune()
        infos, t = timed(lambda: b.solve())
        b.close()
        res[name] = (infos, t)
    out = {"metric": "Pe x Da sweep solves/s to steady state (ADR, 3 species)",
           "unit": "solves/s", "higher_is_better": True,
           "instances": len(ws), "left_out_k_ge_1": len(ws_all) - len(ws),
           "nodes": sum(w.nx * w.ny for w in ws), "step_cap": cap,
           "check_every": check, "flow": {"steps": flow_steps,
                                          "seconds_untimed": flow_s}}
    for name, (infos, t) in res.items():
        errs = [abs(i["eps"] - r["eps"]) for i, r in zip(infos, ref)
                if math.isfinite(i["eps"]) and math.isfinite(r["eps"])]
        out[name] = {"solves_per_s": len(ws) / t, "seconds": t,
                     "speedup_vs_f64": t64 / t,
                     "converged": sum(bool(i["converged"]) for i in infos),
                     "steps": sum(i["steps"] for i in infos),
                     "max_abs_eps_err_vs_f64": max(errs) if errs else None,
                     "instances_compared": len(errs),
                     "instances_over_1e-3": sum(e > 1e-3 for e in errs)}
    out["per_instance"] = [
        {"pe": round(w.pe, 4), "da": round(w.da1, 4), "nx": w.nx, "ny": w.ny,
         "eps_f64": r["eps"], "steps_f64": r["steps"],
         "err_f32": abs(res["f32_batched"][0][k]["eps"] - r["eps"]),
         "err_f16": abs(res["f16dev_batched"][0][k]["eps"] - r["eps"]),
         "steps_f32": res["f32_batched"][0][k]["steps"],
         "steps_f16": res["f16dev_batched"][0][k]["steps"]}
        for k, (w, r) in enumerate(zip(ws, ref))]
    print(json.dumps(out), flush=True)


def run_sweep(a):
    """The Pe x Da sweep at fixed step counts (see sweep_record)."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(sweep_record(a.sweep_instances, a.sweep_max_steps,
                                  a.sweep_flow_steps, a.sweep_tol)), flush=True)


def sweep_record(n_instances, max_steps, flow_steps, sweep_tol):
    """The first n_instances seeded lattices of the sweep (Pe =
    logspace(-1,2,8) x Da = logspace(-2,2,8), widths 512..2048, heights
    256..512), each with its own flow (FP64, flow_steps steps, untimed).
    Timed: the ADR solves of all instances.  sweep_tol <= 0: every instance
    runs exactly max_steps steps in every precision, so the efficiencies
    are compared at equal step counts (a per-step residual of 1e-6 is no
    steady state on these lattices, and stopping there leaves the
    efficiency off by up to 1e-2); otherwise each solve stops at that
    residual (FP64 at 1e-3 of it).  Batched (one lbm_batch for all, FP32
    and FP16 storage) against one lbm_adr_solve per instance in FP64 and in
    FP32.  Returns solves/s and the largest efficiency difference to
    FP64."""
    import torch

    from paper_2109_04455_gb300 import inputs, lbm
    ws_all = [inputs.sweep_instance(i) for i in range(n_instances)]
    # the explicit Dawson source needs k < 1 per step (k = 1 empties A in one
    # step); the (Pe, Da) pairs with k = Da D / R^2 >= 1 are left out
    ws = [w for w in ws_all if max(w.k1, w.k2) < 1.0]
    geoms, u64 = [], []
    for w in ws:
        g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
        u, _ = lbm.lbm_flow_solve(g, w.tau_flow, w.u0, flow_steps,
                                  precision=lbm.LBM_F64)
        geoms.append(g)
        u64.append(u)
    nodes = sum(w.nx * w.ny for w in ws)
    check = 500
    cap = max_steps

    def params(prec, tol):
        return [lbm.adr_params(3, w.tau_c, precision=prec, max_steps=cap,
                               tol=tol, check_every=check) for w in ws]

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    # unbatched FP64
    p64 = params(lbm.LBM_F64, sweep_tol * 1e-3)
    torch.cuda.synchronize()
    ev0.record()
    ref = [lbm.lbm_adr_solve(g, p, u, want_conc=False)[1]
           for g, p, u in zip(geoms, p64, u64)]
    ev1.record()
    torch.cuda.synchronize()
    t64 = ev0.elapsed_time(ev1) * 1e-3
    out = {"metric": "Pe x Da sweep solves/s (ADR, 3 species)",
           "mode": ("fixed step count" if sweep_tol <= 0 else
                    f"to a residual of {sweep_tol:g}"),
           "unit": "solves/s", "higher_is_better": True,
           "instances": len(ws),
           "left_out_k_ge_1": len(ws_all) - len(ws),
           "nodes": nodes, "step_cap": cap,
           "check_every": check,
           "f64_unbatched": {"solves_per_s": len(ws) / t64, "seconds": t64,
                             "converged": sum(r["converged"] for r in ref),
                             "steps": sum(r["steps"] for r in ref)}}
    u32 = [u.float() for u in u64]
    # unbatched FP32: the gain of batching alone, at the same precision
    p32 = params(lbm.LBM_F32, sweep_tol)
    torch.cuda.synchronize()
    ev0.record()
    ref32 = [lbm.lbm_adr_solve(g, p, u, want_conc=False)[1]
             for g, p, u in zip(geoms, p32, u32)]
    ev1.record()
    torch.cuda.synchronize()
    t32 = ev0.elapsed_time(ev1) * 1e-3
    out["f32_unbatched"] = {"solves_per_s": len(ws) / t32, "seconds": t32,
                            "speedup_vs_f64": t64 / t32,
                            "steps": sum(r["steps"] for r in ref32)}
    # with a tolerance: FP64 to tol * 1e-3, FP32 to tol, FP16 (stochastic
    # rounding: a per-step residual floor of a few 1e-6) to max(tol, 1e-5)
    tols = {lbm.LBM_F32: sweep_tol,
            lbm.LBM_F16DEV: max(sweep_tol, 1e-5) if sweep_tol > 0 else 0.0}
    for name, prec in (("f32_batched", lbm.LBM_F32),
                       ("f16dev_batched", lbm.LBM_F16DEV)):
        tol = tols[prec]
        b = lbm.Batch(geoms, params(prec, tol), u32)
        tile, grid = b.tune()
        torch.cuda.synchronize()
        ev0.record()
        infos = b.solve()
        ev1.record()
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) * 1e-3
        de = max(abs(i["eps"] - r["eps"]) for i, r in zip(infos, ref))
        out[name] = {"solves_per_s": len(ws) / t, "seconds": t, "tol": tol,
                     "speedup_vs_f64": t64 / t,
                     "speedup_vs_f32_unbatched": t32 / t,
                     "max_abs_eps_err_vs_f64": de,
                     "converged": sum(i["converged"] for i in infos),
                     "steps": sum(i["steps"] for i in infos),
                     "tile": tile, "grid": grid}
        b.close()
    for g in geoms:
        g.close()
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# discrete adjoint on the large lattice
# ---------------------------------------------------------------------------
def run_adjoint(a):
    """Adjoint iterations nu <- K^T (P^T nu + l) on the large membrane.
    Untimed: flow, and a few hundred forward steps (the adjoint linearises
    around the forward's last checked state).  Timed with CUDA events:
    lbm_adr_adjoint with a fixed iteration count (tol = 0), which also
    zeroes its outputs and runs the rate-gradient kernel once at the end.
    Reports adjoint species MLUPS of whole calls of 2N iterations, and the
    HBM roofline of one adjoint iteration (time of a 2N-iteration call less
    that of an N-iteration call, over N), whose algorithmic bytes per fluid
    node equal the forward step's (the gather of 27 values, 27 stores, u
    and the link word)."""
    import torch

    from paper_2109_04455_gb300 import lbm
    torch.cuda.set_device(0)
    if a.precision == "f16dev":
        raise SystemExit("the adjoint runs in f32 or f64")
    prec = lbm.PRECISIONS[a.precision]
    w = _workload(a)
    geom = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(geom, w.tau_flow, w.u0, a.flow_steps,
                              precision=lbm.LBM_F64 if prec == lbm.LBM_F64
                              else lbm.LBM_F32)
    # flux plane 8 nodes behind the first (A->B) membrane: the adjoint
    # starts there and runs upstream at the flow speed, so within the timed
    # iterations it reaches that membrane's last fibers and the gradient is
    # not zero (at the outlet, 1800 nodes behind the last membrane, it would
    # need ~55000 iterations)
    plane = int(round(2 * w.nx / 9.0)) + 8
    prm = lbm.adr_params(SPECIES, w.tau_c, w.c_in, precision=prec,
                         x_plane=plane)
    sv = lbm.ADRSolver(geom, prm, u).init()
    sv.run(CHUNK - 2, check=False)
    sv.run(2)
    nfib = w.fibers.shape[0]
    n_it = max(2, a.adjoint_iters)
    for _ in range(max(1, a.warmup)):
        sv.adjoint(20, tol=0.0, check_every=20, nfibers=nfib)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)

    def timed(n):
        ev0.record()
        out = sv.adjoint(n, tol=0.0, check_every=n, nfibers=nfib)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) * 1e-3, out

    t1s, t2s = [], []
    with ClockSampler(0) as clk:
        for _ in range(a.steps):
            t1s.append(timed(n_it)[0])
            t2, (_, _, dw, info) = timed(2 * n_it)
            t2s.append(t2)
    t = sum(t2s) / len(t2s)
    alg_bytes, n_fluid, per_fluid = _algorithmic_bytes(geom, w, a.precision)
    # per iteration: the difference of the two call lengths, free of the
    # fixed per-call work (workspace zeroing, fiber-id upload, gradients)
    per_it = (t - sum(t1s) / len(t1s)) / n_it
    n_it = 2 * n_it
    achieved = alg_bytes / per_it / 1e9
    peak, peak_kind = _peak_hbm()
    line = {"metric": "adjoint species MLUPS (ADR, 3 species)",
            "value": SPECIES * w.nx * w.ny * n_it / t / 1e6, "unit": UNIT,
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True,
            "dtype": a.precision, "data": "synthetic (seeded fiber geometry)",
            "config": dict(_config(a, w), adjoint_iters_per_step=n_it),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None,
                         "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "kernel": f"adj_kernel<{a.precision},3 species>",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "bytes_per_fluid_node": per_fluid,
                         "avg_iteration_ms": per_it * 1e3},
            "clocks": clk.summary(),
            "eps": info["eps"], "flux_plane": plane,
            "flux": info["flux"],
            "dw_abs_max": float(dw.abs().max().item()),
            "dw_nonzero_fibers": int((dw != 0).sum().item())}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the paper's 2D experiment series
# ---------------------------------------------------------------------------
def run_series(a):
    """Isolated A->B fiber (Da = 150, 1.5), A->B->C fiber pairs at xi = 2,
    20, 100, the side-by-side fiber (Da = 150), and membranes of six fibers
    (three seeds; A->B at Da = 150, 1.5 and the A->B->C pair of membranes
    at Da = 150), Pe = 1..30 where k < 1 and tau_c >= 0.52: 110 lattices
    of 300x300 and 1000x300.  Untimed: one FP64 flow per geometry.  Timed
    on the host clock (the solves end synchronised): the launch-shape tuning
    and the batched ADR solves (two batches, 2 and 3 species) to a per-step
    residual of 2e-7 (FP32's floor at tau_c = 0.525 is ~1.1e-7) or the
    300000-step cap.  Reports solves/s, and per lattice the efficiency, the
    collision-zone model's value and the production rate."""
    import torch

    from paper_2109_04455_gb300 import lbm, series
    torch.cuda.set_device(0)
    prec = lbm.PRECISIONS[a.precision]
    items = series.workloads()
    flows = series.solve_flows(items)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows, shapes = series.run(items, flows, precision=prec, tol=2e-7,
                              max_steps=300000)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    # efficiency against Da at Pe = 1, 7, 20 (Fig. singleAB_Da), and at
    # Pe = 7 with the node-wise reaction as well (Fig. node_vs_pop)
    da_items = series.da_workloads()
    da_rows, _ = series.run(da_items, flows, precision=prec, tol=2e-7,
                            max_steps=300000)
    pe7 = [it for it in da_items if it[1].pe == 7.0]
    nw_rows, _ = series.run(pe7, flows, precision=prec, tol=2e-7,
                            max_steps=300000, flags=lbm.LBM_ADR_NODEWISE)
    for r in da_rows:
        r["series"] = "eps_vs_da"
    for r in nw_rows:
        r["series"] = "eps_vs_da_nodewise"
    out = {"metric": "paper 2D series solves/s (ADR to steady state)",
           "value": len(rows) / t, "unit": "solves/s",
           "higher_is_better": True, "seconds": t, "dtype": a.precision,
           "lattices": len(rows),
           "nodes": sum(r["nx"] * r["ny"] for r in rows),
           "converged": sum(r["converged"] for r in rows),
           "steps": sum(r["steps"] for r in rows),
           "launch_shapes": shapes,
           "timing": "host clock around the batched solves, tuning included",
           "rows": [{k: (round(v, 8) if isinstance(v, float) else v)
                     for k, v in r.items() if k != "flux"}
                    for r in rows + da_rows + nw_rows]}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# the two-membrane cascade to steady state
# ---------------------------------------------------------------------------
def run_cascade(a):
    """Two-membrane cascade lattice (2048 x 512, 40 + 40 R = 8 fibers,
    seed 0), Da1 = Da2 = 1, per Pe of --cascade-pe (see cascade_rows)."""
    import torch
    torch.cuda.set_device(0)
    cascade_rows([float(v) for v in a.cascade_pe.split(",")],
                 a.cascade_max_steps, verbose=True)


def cascade_rows(pes, max_steps, verbose=False):
    """The two-membrane cascade lattice per Pe: FP64 ADR to a per-step
    residual of 1e-9 and FP32 to 1e-6 (checked every 1000 steps); then FP32
    and FP16-deviation storage run exactly FP64's step count, so that their
    efficiencies are compared with FP64's at equal steps.  Untimed: the
    FP64 flow to a per-step residual of 1e-9 (shared by every Pe, since u0
    is fixed and Pe only sets D).  Timed with CUDA events: each solve.
    Returns per Pe and precision the steps, seconds, the outlet efficiency
    of Eq. (A-B) on x = nx - 3, its difference to FP64, the outflux shares
    and the most negative concentration met at the last check."""
    import torch

    from paper_2109_04455_gb300 import inputs, lbm
    w0 = inputs.two_membrane_cascade(seed=0, pe=pes[0])
    geom = lbm.Geometry(w0.nx, w0.ny, w0.fibers, w0.k1, w0.k2)
    geom.upload()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(
        enable_timing=True)
    ev0.record()
    u64, finfo = lbm.lbm_flow_solve(geom, w0.tau_flow, w0.u0, 1000000,
                                    tol=1e-9, check_every=1000,
                                    precision=lbm.LBM_F64)
    ev1.record()
    torch.cuda.synchronize()
    out = {"metric": "two-membrane cascade steady solves (ADR, 3 species)",
           "unit": "s", "lattice": f"{w0.nx}x{w0.ny}",
           "fibers": int(w0.fibers.shape[0]),
           "flow": {"steps": finfo["steps"], "residual": finfo["residual"],
                    "converged": finfo["converged"],
                    "seconds": ev0.elapsed_time(ev1) * 1e-3},
           "runs": []}
    u32 = u64.float()

    def solve(w, prec, tol, steps):
        g = lbm.Geometry(w.nx, w.ny, w.fibers, w.k1, w.k2).upload()
        prm = lbm.adr_params(3, w.tau_c, precision=prec, max_steps=steps,
                             tol=tol, check_every=1000)
        torch.cuda.synchronize()
        ev0.record()
        try:
            _, info = lbm.lbm_adr_solve(g, prm, u64 if prec == lbm.LBM_F64
                                        else u32, want_conc=False)
            status = "ok" if info["converged"] or tol <= 0 else "not converged"
        except lbm.LBMError as e:
            info, status = {"steps": None, "eps": None, "flux": [None] * 3,
                            "residual": None, "c_min": [None] * 3}, str(e)
        ev1.record()
        torch.cuda.synchronize()
        fl = info["flux"]
        tot = sum(fl) if None not in fl else None
        return {"steps": info["steps"], "residual": info["residual"],
                "eps": info["eps"], "status": status,
                "flux_share": [f / tot for f in fl] if tot else None,
                "c_min": info["c_min"],
                "seconds": ev0.elapsed_time(ev1) * 1e-3}

    for pe in pes:
        w = inputs.two_membrane_cascade(seed=0, pe=pe)
        row = {"pe": pe, "tau_c": w.tau_c, "k1": w.k1, "k2": w.k2}
        r64 = solve(w, lbm.LBM_F64, 1e-9, max_steps)
        row["f64_to_1e-9"] = r64
        row["f32_to_1e-6"] = solve(w, lbm.LBM_F32, 1e-6, max_steps)
        if r64["steps"]:
            for name, prec in (("f32_equal_steps", lbm.LBM_F32),
                               ("f16dev_equal_steps", lbm.LBM_F16DEV)):
                row[name] = solve(w, prec, 0.0, r64["steps"])
            for k in ("f32_to_1e-6", "f32_equal_steps", "f16dev_equal_steps"):
                if row[k]["eps"] is not None and r64["eps"] is not None:
                    row[k]["eps_err_vs_f64"] = abs(row[k]["eps"] - r64["eps"])
        out["runs"].append(row)
        if verbose:
            print(json.dumps(row), flush=True)
    if verbose:
        print(json.dumps(out), flush=True)
    return out


# ---------------------------------------------------------------------------
# the pure-diffusion cascade (Sec. IV.B)
# ---------------------------------------------------------------------------
def run_noflow(a, steps=200000, every=1000):
    """Totals of A, B and C over time in the periodic 300 x 300 box without
    flow (Figs. noflow, noflow_k001): the A->B / B->C fiber pair (R = 5,
    surfaces 100 apart) and the side-by-side fiber (R = 10), Da = 150 and
    1.5, FP64.  Reports the curves at a few times and the time at which
    half of the initial A has become C."""
    import torch

    from paper_2109_04455_gb300 import lbm, series
    torch.cuda.set_device(0)
    rows = []
    t_all = time.perf_counter()
    for da in (150.0, 1.5):
        for kind in ("pair", "side_by_side"):
            t0 = time.perf_counter()
            out = series.noflow_cascade(kind, da, steps=steps, every=every,
                                        precision=lbm.LBM_F64)
            dt = time.perf_counter() - t0
            t = out["t"]
            half = next((tt for tt, c in zip(t, out["C"]) if c >= 0.5), None)
            pick = [i for i, tt in enumerate(t)
                    if tt in (1000, 5000, 20000, 50000, 100000, 200000)]
            rows.append({"kind": kind, "da": da, "k1": out["k1"],
                         "k2": out["k2"], "tau": out["tau_c"], "seconds": dt,
                         "t_half_C": half,
                         "curve": {str(t[i]): [round(out["A"][i], 6),
                                               round(out["B"][i], 6),
                                               round(out["C"][i], 6)]
                                   for i in pick}})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": "pure-diffusion cascade (periodic box)",
                      "steps": steps, "seconds": time.perf_counter() - t_all,
                      "rows": rows}), flush=True)


# ---------------------------------------------------------------------------
# the adjoint on the two-membrane cascade, fiber by fiber
# ---------------------------------------------------------------------------
def run_adjoint_check(a):
    """The adjoint check of the two-membrane cascade lattice (2048 x 512,
    80 fibers, seed 0, Pe = 10, Da1 = Da2 = 1, relaxed weights 0.9 on the
    A->B fibers and 0.1 on the B->C fibers).  FP64: steady state to a
    per-step residual of 1e-13 and the adjoint to 1e-13.  FP32 populations
    (FP64 sums): steady state to 1e-7 and the adjoint at FP64's iteration
    count.  Then for each of 16 random fibers the central difference with
    h = 1e-4 of two FP64 solves warm-started from the base state, each run
    a fixed --fd-steps steps (a solve stopped by the per-step residual
    leaves ~1e-3 of so small a perturbation unrelaxed).  The response to a
    fiber's weight first has to travel to the outlet, so the quotient
    converges slowly at first: for the slowest fibers of this lattice it
    is still 2.5e-2 short after 150000 steps, 1.2e-3 after 200000 and
    within 1e-6 after 300000.  Reports per fiber the difference quotient
    every --fd-every steps, its Aitken limit, the FP64 and FP32 adjoint
    values and their relative differences."""
    import numpy as np
    import torch

    from paper_2109_04455_gb300 import inputs, lbm
    torch.cuda.set_device(0)
    t_all = time.perf_counter()
    w = inputs.two_membrane_cascade(seed=0, pe=10.0)
    fib = w.fibers.copy()
    fib[:, 5] = np.where(fib[:, 3] == 1, 0.9, 0.1)
    nf = fib.shape[0]
    g0 = lbm.Geometry(w.nx, w.ny, fib, w.k1, w.k2).upload()
    u, _ = lbm.lbm_flow_solve(g0, w.tau_flow, w.u0, 400000, tol=1e-10,
                              check_every=1000, precision=lbm.LBM_F64)

    def solver(fb, prec, uu):
        g = lbm.Geometry(w.nx, w.ny, fb, w.k1, w.k2).upload()
        return g, lbm.ADRSolver(g, lbm.adr_params(3, w.tau_c,
                                                  precision=prec), uu).init()

    g, sv = solver(fib, lbm.LBM_F64, u)
    base_info = sv.solve(1e-13, 1000, 2000000)
    base = sv.state_save()
    _, _, dw, ainfo = sv.adjoint(2000000, tol=1e-13, check_every=1000,
                                 nfibers=nf)
    dw = dw.cpu().numpy()
    g32, sv32 = solver(fib, lbm.LBM_F32, u.float())
    sv32.solve(1e-7, 1000, 2000000)
    _, _, dw32, _ = sv32.adjoint(ainfo["steps"], tol=0.0,
                                 check_every=ainfo["steps"], nfibers=nf)
    dw32 = dw32.cpu().numpy()
    rng = np.random.default_rng(4)
    pick = rng.choice(nf, 16, replace=False)
    if a.fd_fibers:
        pick = [int(v) for v in a.fd_fibers.split(",")]
    h = 1e-4
    every = a.fd_every if a.fd_every > 0 else a.fd_steps
    marks = list(range(every, a.fd_steps + 1, every))
    rows = []
    for f in pick:
        e = []
        for sgn in (1.0, -1.0):
            fb = fib.copy()
            fb[f, 5] += sgn * h
            gg, sp = solver(fb, lbm.LBM_F64, u)
            sp.state_load(base)
            seq, done = [], 0
            for m in marks:
                seq.append(sp.run(m - done)["eps"])
                done = m
            e.append(seq)
            sp.close()
        # the difference quotient after each mark of steps past the base
        # state, and Aitken's extrapolation of its last three values (the
        # limit of a sequence that approaches it geometrically)
        q = [(p_ - m_) / (2 * h) for p_, m_ in zip(e[0], e[1])]
        fd = q[-1]
        fd_lim = None
        if len(q) >= 3:
            d1, d2 = q[-1] - q[-2], q[-2] - q[-3]
            fd_lim = q[-1] - d1 * d1 / (d1 - d2) if d1 != d2 else q[-1]
        rows.append({"fiber": int(f), "cat": int(fib[f, 3]), "fd": fd,
                     "fd_by_steps": dict(zip(marks, q)), "fd_aitken": fd_lim,
                     "adjoint_f64": float(dw[f]), "adjoint_f32": float(dw32[f]),
                     "rel_f64_vs_fd": (float(dw[f]) - fd) / fd,
                     "rel_f64_vs_fd_aitken": (None if fd_lim is None else
                                              (float(dw[f]) - fd_lim) / fd_lim),
                     "rel_f32_vs_fd": (float(dw32[f]) - fd) / fd,
                     "rel_f32_vs_f64": (float(dw32[f]) - float(dw[f]))
                     / float(dw[f])})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({
        "metric": "adjoint check, two-membrane cascade (2048x512, Pe 10, Da 1)",
        "base": {"steps": base_info["steps"], "residual": base_info["residual"],
                 "eps": base_info["eps"]},
        "adjoint_f64": {"iterations": ainfo["steps"],
                        "residual": ainfo["residual"]},
        "f32_vs_f64_rel_l2": float(np.linalg.norm(dw32 - dw) /
                                   np.linalg.norm(dw)),
        "h": h, "fd_steps": a.fd_steps,
        "max_rel_f64_vs_fd": max(abs(r["rel_f64_vs_fd"]) for r in rows),
        "max_rel_f32_vs_fd": max(abs(r["rel_f32_vs_fd"]) for r in rows),
        "max_rel_f32_vs_f64": max(abs(r["rel_f32_vs_f64"]) for r in rows),
        "seconds": time.perf_counter() - t_all, "rows": rows}), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "sweep":
        if a.sweep_mode == "steady":
            run_sweep_steady(a)
        else:
            run_sweep(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    elif a.workload == "series":
        run_series(a)
    elif a.workload == "cascade":
        run_cascade(a)
    elif a.workload == "noflow":
        run_noflow(a)
    elif a.workload == "adjoint-check":
        run_adjoint_check(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
