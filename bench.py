"""Benchmark of the fused peridynamic step (bond updates per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload beam|plate|bar] [--precision 32|64]

Default workload: the notched three-point-bend beam, 300 x 58 x 58 = 1,009,200
nodes, delta = pi dx, 117.7M directed bonds, per-bond critical stretch, FP32
bulk arithmetic.  A step is one pass of the whole method over the model (one
fused kernel launch).  Inputs are resident in HBM when the timed region starts.
The beam is a regular lattice, so its step runs the stencil kernel, whose
per-step footprint (about 120 MB of node state) fits in L2: every step is timed
alone with CUDA events, and a 516 MB write followed by a read of it between
the timed intervals flushes L2.  Rank 0 prints one JSON line.

Under torchrun (N > 1) every rank advances its own replica of the workload
(the method has no exchange step on one model: replicas only, weak scaling);
the time is the maximum over ranks and the value counts all ranks' bonds.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the host cores, on a row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

import workloads  # noqa: E402

# Algorithmic bytes of one step (what the method must move, padding excluded):
# per directed bond a 4-byte neighbour id and one state bit; per node (FP32 bulk)
# position+weight 16 B read, FP64 displacement 24 B read + 24 B written, FP32
# velocity 12 B read + 12 B written, damage 4 B written, BC class 1 B.
BYTES_PER_BOND = 4.125
BYTES_PER_NODE = {32: 93.0, 64: 136.0}
# The FP64 step is bound by GB300's FP64 arithmetic, not by HBM.  Algorithmic
# FP64 work per bond (Eqs. 4-5 as written): xi, eta, y (9), |xi|^2 and |y|^2
# (10), two square roots and the stretch's division (3), c V s / |y| (3), the
# force accumulation (6 as 3 fused multiply-adds) = 31 flops, counting a square
# root or a division as one.  Peak: FP64 fused multiply-add throughput measured
# on a GB300 of this pool with a plain dependent-chain probe, 1.20 TFLOP/s
# (nominal 1.25).
FP64_FLOPS_PER_BOND = 31.0
FP64_PEAK_TFLOPS = 1.20
# Ordinary state-based step, both loops: the dilation loop (xi, eta, y 9; |y|^2
# 5; root 1; e 1; |xi| e V and the sum 3 = 19) and the force loop (y 9; |y|^2
# 5; root 1; e 1; t_ij 5; t_ji 8; the sum, V / |y| 3; accumulation 6 = 38):
# 57 flops per bond.
OSB_FLOPS_PER_BOND = 57.0
# The double-word step (precision 48) is bound by the FP32 pipe.  FP32
# operations per bond of its arithmetic (pd_step_dw.cu, uniform weights; an add,
# multiply or fused multiply-add each counted once): xi 2, eta 8, y 8 and
# 2 xi + eta 8 and their product 4 per component (90); the sum num 16; L^2 and
# |y|^2 12; the refined 1/|y| seed 4, |y| 5, 1/|y| 3; den 12; the quotient 10;
# s / |y| 4; the force term and its double-word accumulation 12 per component
# (36) = 192, plus two hardware reciprocal(-square-root) seeds.  Peak: FP32 FMA
# lane rate measured by a probe on this machine's GB300, 35.1 T/s (70.2 TFLOP/s
# counting an FMA as two).
DW_FP32_OPS_PER_BOND = 192.0
# per-node weights (batches): the coefficient times w_j (4) and the weight sum (8)
DW_FP32_OPS_PER_BOND_NODE_W = DW_FP32_OPS_PER_BOND + 12.0
# double-word state-based step (pd_step_osb_dw.cu), both loops: the bond's
# stretch, y and 1/|y| (152) in each; the dilation term and its sum (20); the
# force scalar (36), s V / |y| (8) and the force and its sum (36) = 404
DW_OSB_FP32_OPS_PER_BOND = 404.0
FP32_PEAK_TOPS = 35.1
# per node: the double-word record 64 B read + 64 B written, the FP64 record
# (x, w copied, u) 56 B read + 56 B written, FP64 velocity 24 + 24 B, damage
# 8 B, wsum_inv 8 B, BC class 1 B; per bond 8 B of double-word |xi| on top
BYTES_PER_NODE[48] = 305.0
DW_BYTES_PER_BOND = BYTES_PER_BOND + 8.0
STEP_SRC = {32: ["pd_step_f32.cu"], 64: ["pd_step_f64.cu"], 48: ["pd_step_dw.cu"],
            "lat": ["pd_step_f32_lat.cu"], "lat_tma": ["pd_step_f32_lat_tma.cu", "pd_step_f32_lat.cu"]}
STEP_TAG = {32: "f32", 64: "f64", 48: "dw", "lat": "f32_lat", "lat_tma": "f32_lat_tma"}
TMA_BOX = ["16x2x8", "8x4x8", "32x2x4"]  # pd_config.lat_variant 2, 3, 4
# Device memory one FP32 lattice step touches per node: FP64 displacement 24 B
# read + 24 B written (double-buffered), the published record 16 B read + 16 B
# written, velocity 12 B, bond flags 16 B, BC class 4 B, inverse weight sum 4 B,
# damage 4 B; the state-based step adds its published record {h, A} 16 B, its
# per-node coefficients 16 B, B 4 B and theta 4 B.
LAT_FOOTPRINT_PER_NODE = 120.0
LAT_OSB_FOOTPRINT_PER_NODE = LAT_FOOTPRINT_PER_NODE + 2 * 16.0 + 8.0
L2_BYTES = 129e6
# the L2 flush between timed steps: a write, then a read, of four times the L2
FLUSH_BYTES = int(4 * L2_BYTES)


def step_footprint(n_nodes, n_bonds, precision, lattice, osb=False):
    """Bytes of device memory one step touches (node state, and the family where
    the kernel streams one)."""
    if lattice:
        return n_nodes * (LAT_OSB_FOOTPRINT_PER_NODE if osb else LAT_FOOTPRINT_PER_NODE)
    per_bond = DW_BYTES_PER_BOND if precision == 48 else BYTES_PER_BOND
    return n_bonds * per_bond + n_nodes * BYTES_PER_NODE[precision]


def l2_flush_buffer(torch, device):
    return torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)


def flush_l2(torch, flush):
    """Write the flush buffer (four times L2), then read it back: the L2 then holds
    none of the step's data and no dirty lines whose write-back the next step
    would pay for."""
    flush.zero_()
    flush.view(torch.int32).max()


def timed_steps_flushed(torch, stream, m, steps, flush):
    """`steps` steps, each timed alone with CUDA events on the launching stream,
    with an L2 flush (flush_l2) between the timed intervals; returns the
    summed device time in ms.  A device-side sleep first lets the host queue the
    steps ahead of the device, so that no interval holds host launch latency."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(4_000_000)
        for e0, e1 in ev:
            flush_l2(torch, flush)
            e0.record(stream)
            m.step(1)
            e1.record(stream)
        ev[-1][1].synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev)


def l2_flush(torch, stream, flush):
    """One L2 flush on `stream`, waited for (before a timed leg)."""
    with torch.cuda.stream(stream):
        flush_l2(torch, flush)
    stream.synchronize()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="beam",
                   choices=["beam", "plate", "bar", "batch", "adjoint"])
    p.add_argument("--integrator", default="ec", choices=["ec", "vv"],
                   help="damped Euler-Cromer (default) or damped velocity-Verlet")
    p.add_argument("--ramp-steps", type=int, default=0,
                   help="smooth start of the displacement loading over this many steps")
    p.add_argument("--kr", type=float, default=0.0,
                   help="bilinear softening with s_0 = s_c / kr (0: the PMB law)")
    p.add_argument("--state-based", type=float, default=None, metavar="NU",
                   help="ordinary state-based linear solid with Poisson's ratio NU (FP64)")
    p.add_argument("--fd-directions", type=int, default=32)
    p.add_argument("--checkpoint-every", type=int, default=45)
    p.add_argument("--precision", type=int, default=32, choices=[32, 64, 48],
                   help="32: FP32 bonds; 64: FP64; 48: FP64-grade double-word FP32 bonds")
    p.add_argument("--shape", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                   help="lattice dimensions of the beam, plate or bar (default: the workload's)")
    p.add_argument("--graph-steps", type=int, default=50)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default stencil variant and launch shape on lattice models")
    p.add_argument("--no-outer", action="store_true",
                   help="leave out the batch and adjoint sub-objects of the default line")
    return p.parse_args()


def make_workload(name, shape=None):
    if name == "beam":
        if shape is None:
            return workloads.notched_beam()
        return workloads.notched_beam(*shape, length=shape[0] / 600.0)  # the beam's spacing
    if name == "plate":
        return workloads.plate() if shape is None else workloads.plate(*shape)
    return workloads.tensile_bar() if shape is None else workloads.tensile_bar(*shape)


def describe(w, n_bonds, precision, integrator="ec", lattice=None):
    osb = getattr(w, "state_based", None) is not None
    return {
        "integrator": {"ec": "damped Euler-Cromer", "vv": "damped velocity-Verlet"}[integrator],
        "ramp_steps": int(getattr(w, "ramp_steps", 0)),
        "bond_law": ("ordinary state-based linear solid, K = %.3g, G = %.3g" % w.state_based
                     if getattr(w, "state_based", None) is not None
                     else "PMB" if not getattr(w, "kr", 0.0)
                     else f"bilinear softening, s_0 = s_c / {w.kr:g}"),
        "workload": f"{w.name}: {w.n:,} nodes, {n_bonds:,} directed bonds, "
                    f"delta = {w.horizon / w.dx:.4g} dx, "
                    + ("per-bond s_c ~ U[9e-5, 1.1e-4)" if w.sc_hash else f"s_c = {w.sc:g}"),
        "precision": {32: "fp32 bonds, fp64 displacement (lattice stencil kernel)" if lattice
                      else "fp32 bonds, float-float (48-bit) displacement", 64: "fp64",
                      48: "fp64-grade: double-word fp32 bonds, fp64 node state"}[precision],
        "n_nodes": w.n,
        "n_bonds": int(n_bonds),
        "l2_policy": (f"L2 flushed between timed steps: a {FLUSH_BYTES / 1e6:.0f} MB write, then "
                      f"a read of it, on the launching stream between per-step CUDA-event "
                      f"intervals (step "
                      f"footprint {step_footprint(w.n, n_bonds, precision, lattice, osb) / 1e6:.0f}"
                      f" MB, L2 {L2_BYTES / 1e6:.0f} MB)"),
    }


# --------------------------------------------------------------------------- peaks, clocks
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        picked = [l for t, l in self.lines if (t0 is None or t >= t0) and (t1 is None or t <= t1)]
        if not picked:  # timed region shorter than one sample period: nearest samples
            picked = [l for _, l in self.lines[-3:]]
        for line in picked:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- multi-rank
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    group = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        group = dist
    return world, rank, local, group


def barrier(group, device_sync):
    if device_sync is not None:
        device_sync()
    if group is not None:
        group.barrier()


def aggregate_max(value: float, group) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a group)."""
    if group is None:
        return value
    import torch
    dev = "cuda" if group.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    group.all_reduce(t, op=group.ReduceOp.MAX)
    return float(t.item())


def whole_job(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


# --------------------------------------------------------------------------- traffic
def profiled_traffic(precision, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (matched by hash); else None.  precision: 32, 64, 48, or
    "lat" for the FP32 regular-lattice stencil kernel."""
    h = hashlib.sha256()
    for name in STEP_SRC[precision]:
        h.update(open(os.path.join(ROOT, "paper_2105_04150_gb300", "csrc", name), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"step_{STEP_TAG[precision]}_{workload}_traffic.txt")
    try:
        kv = dict(l.split(None, 1) for l in open(path) if l.strip() and not l.startswith("#"))
        if kv.get("kernel_source_sha256_16", "").strip() == sha:
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------- oracle timing
def oracle_sample(w, c, budget_s, steps=None, warmup=0):
    """Time the FP64 oracle step on a row sample of the workload (host cores)."""
    import oracle
    off_all = None
    rng = np.random.default_rng(0)
    if getattr(w, "state_based", None) is not None:
        # the state-based step reads every node's dilation: whole steps only
        off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
        m = oracle.Model.from_workload(w, off, idx, c=c)
        u, v = workloads.random_state(w.n, 1, 1e-9, 1e-4)
        mu = m.fresh_bonds()
        t = time.perf_counter()
        m.step(0, u, v, mu)
        t1 = time.perf_counter() - t
        n_steps = int(max(1, min(steps if steps is not None else 5, budget_s / max(t1, 1e-9))))
        t = time.perf_counter()
        for k in range(n_steps):
            m.step(1 + k, u, v, mu)
        el = time.perf_counter() - t
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        return {
            "value": m.nbonds * n_steps / el, "unit": "bond updates/s", "cores": cores,
            "kind": "oracle", "seconds": el, "steps": n_steps, "n_bonds_total": m.nbonds,
            "sample": f"{n_steps} oracle FP64 state-based steps over all {w.n:,} rows "
                      f"({m.nbonds:,} bonds) of the same workload, OpenMP on {cores} host threads",
        }
    # estimate the full-step cost from a 2% row sample
    probe_rows = np.sort(rng.choice(w.n, max(1, w.n // 50), replace=False))
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array(), rows=probe_rows)
    m = oracle.Model.from_workload(w, off, idx, c=c, rows=probe_rows)
    u, v = workloads.random_state(w.n, 1, 1e-9, 1e-4)
    t = time.perf_counter()
    m.step(0, u, v, m.fresh_bonds())
    t_probe = time.perf_counter() - t
    per_bond = t_probe / max(1, m.nbonds)
    n_steps = steps if steps is not None else 5
    bonds_budget = budget_s / max(per_bond, 1e-12) / max(1, n_steps)
    frac = min(1.0, bonds_budget / max(1, w.n * (m.nbonds / len(probe_rows))))
    rows = np.sort(rng.choice(w.n, max(1, int(frac * w.n)), replace=False)) if frac < 1 else None
    off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array(), rows=rows)
    m = oracle.Model.from_workload(w, off, idx, c=c, rows=rows)
    mu = m.fresh_bonds()
    for _ in range(warmup):
        m.step(0, u, v, mu)
    t = time.perf_counter()
    for k in range(n_steps):
        m.step(k, u, v, mu)
    el = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "value": m.nbonds * n_steps / el, "unit": "bond updates/s", "cores": cores,
        "kind": "oracle", "seconds": el, "steps": n_steps,
        "n_bonds_total": m.nbonds if rows is None else None,
        "sample": f"{n_steps} oracle FP64 steps over {m.nrows:,} of {w.n:,} rows "
                  f"({m.nbonds:,} bonds each) of the same workload, OpenMP on {cores} host threads",
    }


def run_reference(args):
    world, rank, local, group = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.workload, args.shape)
    w.ramp_steps = args.ramp_steps
    w.kr = args.kr
    if args.state_based is not None:
        nu = args.state_based
        w.state_based = (w.bulk_modulus, 3 * w.bulk_modulus * (1 - 2 * nu) / (2 * (1 + nu)))
    c = oracle.micromodulus(w.bulk_modulus, w.horizon)
    # each timed step is a row sample sized so the whole run takes about a minute
    budget = float(os.environ.get("BENCH_REFERENCE_BUDGET_S", "60"))
    res = oracle_sample(w, c, budget_s=budget, steps=args.steps, warmup=args.warmup)
    # the workload's directed bonds, for the same config object as our arm's
    n_bonds = res["n_bonds_total"]
    if n_bonds is None:
        n_bonds = 0
        for lo in range(0, w.n, 1 << 20):
            rows = np.arange(lo, min(w.n, lo + (1 << 20)))
            off, _ = oracle.cut_family(w.coords, w.horizon, w.cuts_array(), rows=rows)
            n_bonds += int(off[-1])
    line = {
        "impl": "reference", "metric": "bond updates/s", "value": res["value"],
        "unit": "bond updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["seconds"] * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        # the same config object as our arm (whose beam, plate and bar are lattice models)
        "config": describe(w, n_bonds, args.precision, args.integrator,
                           args.precision == 32 and args.integrator == "ec" and not args.ramp_steps
                           and not args.kr and args.state_based is None),
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": "bond updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    world, rank, local, group = dist_setup(args)
    import paper_2105_04150_gb300 as pdgb
    pdgb.lib()
    torch.cuda.set_device(local)
    dev_sync = torch.cuda.synchronize
    w = make_workload(args.workload, args.shape)
    w.ramp_steps = args.ramp_steps
    w.kr = args.kr
    if args.state_based is not None:
        nu = args.state_based
        w.state_based = (w.bulk_modulus, 3 * w.bulk_modulus * (1 - 2 * nu) / (2 * (1 + nu)))
    c = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    stream = torch.cuda.Stream(device=local)
    G = max(0, min(args.graph_steps, args.steps))
    m = pdgb.Model.from_workload(w, precision=args.precision, c=c, graph_steps=G,
                                 stream=stream.cuda_stream, device=local,
                                 integrator=1 if args.integrator == "vv" else 0)
    info = m.info()
    n_bonds = info["n_bonds"]
    # the FP32 step on a regular lattice runs the stencil kernel (FP64 displacement)
    lat = args.precision == 32 and info["layout"] == pdgb.PD_LAYOUT_LATTICE
    # lattice models: the autotuner picks the stencil step's variant (records
    # through L1, or staged in shared memory by TMA per box) and launch shape
    tuned = None
    if lat and not args.no_autotune:
        block, bps = m.autotune(10)
        info = m.info()
        tuned = {"block_threads": block, "blocks_per_sm": bps,
                 "lat_variant": info["lat_variant"], "step_registers": info["step_registers"]}
    tma = lat and info["lat_variant"] >= 2
    # warm-up: W steps (also captures the graph)
    m.step(args.warmup)
    m.sync()
    barrier(group, dev_sync)
    flush = l2_flush_buffer(torch, local)
    with ClockSampler(local) as clk:
        time.sleep(0.5)  # let the sampler start
        barrier(group, dev_sync)
        t_on = time.time()
        ms = timed_steps_flushed(torch, stream, m, args.steps, flush)
        t_off = time.time()
        barrier(group, dev_sync)
        time.sleep(0.25)
    m.sync()
    ms_max = aggregate_max(ms, group)
    # each timed interval: the step's kernels (two passes for the state-based
    # model) and, except on lattice models (whose step kernel advances the step
    # counter itself when launched directly), the step-counter advance
    launches = args.steps * ((2 if args.state_based is not None else 1) + (0 if lat else 1))
    # context: the same number of steps back to back in CUDA graphs of G steps,
    # with no flush between them
    unflushed = None
    if G > 0:
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.step(args.steps)
            e1.record(stream)
            e1.synchronize()
        unflushed = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "graph_steps": G,
                     "note": "the same steps replayed back to back in CUDA graphs, "
                             "no L2 flush between them (context, not the line's value)"}

    # end to end through the public API with pinned host buffers: every step uploads
    # the state (u, v), advances one step and reads the new state back.
    e2e = None
    if not args.no_e2e:
        uh = torch.empty((w.n, 3), dtype=torch.float64).pin_memory()
        vh = torch.empty((w.n, 3), dtype=torch.float64).pin_memory()
        pdgb.pd_get_state(m.h, uh, vh)
        k_e2e = max(3, min(args.steps, 50))
        for _ in range(2):
            pdgb.pd_set_state(m.h, uh, vh)
            m.step(1)
            pdgb.pd_get_state(m.h, uh, vh)
        barrier(group, dev_sync)
        t = time.perf_counter()
        for _ in range(k_e2e):
            pdgb.pd_set_state(m.h, uh, vh)
            m.step(1)
            pdgb.pd_get_state(m.h, uh, vh)
        dev_sync()
        el = aggregate_max(time.perf_counter() - t, group)
        e2e = {"value": whole_job(n_bonds * k_e2e, el * 1e3, world), "unit": "bond updates/s",
               "h2d_bytes_per_step": 2 * uh.numel() * 8, "d2h_bytes_per_step": 2 * uh.numel() * 8,
               "steps": k_e2e}
    m.close()

    if rank != 0:
        barrier(group, None)
        return
    ms_step = ms_max / args.steps
    value = whole_job(n_bonds * args.steps, ms_max, world)
    # softening adds the per-bond integrity read every step (FP32 4 B, FP64 8 B)
    per_bond = BYTES_PER_BOND + ((4.0 if args.precision == 32 else 8.0) if args.kr else 0.0)
    if args.precision == 48:
        per_bond = DW_BYTES_PER_BOND + (8.0 if args.kr else 0.0)
    osb = args.state_based is not None
    alg_bytes = n_bonds * per_bond + w.n * BYTES_PER_NODE[args.precision]
    if osb and args.precision == 32:
        # two passes over the family (ids and flags twice), and per node the
        # weighted volume, dilation and (alpha', beta') besides the step's node data
        alg_bytes = n_bonds * 2 * BYTES_PER_BOND + w.n * (BYTES_PER_NODE[32] + 16)
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (ms_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": None if (args.kr or osb)
                else profiled_traffic(("lat_tma" if tma else "lat") if lat else args.precision,
                                      args.workload),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": alg_bytes,
                "kernel": ("k_osb_lat_dilation + k_osb_lat_force" if lat
                           else "k_osb32_dilation + k_osb32_force") if osb
                else (f"k_step_f32_lat_tma (box {TMA_BOX[info['lat_variant'] - 2]}, z y x)" if tma
                      else "k_step_f32_lat") if lat else f"k_step_f{args.precision}"}
    if lat:
        roofline["note"] = ("algorithmic bytes of the stored-family step (4.125 B per directed "
                            "bond, 93 B per node); the lattice stencil kernel reads no neighbour "
                            "ids, so its DRAM traffic is below them")
    if args.precision == 64:
        fpb = OSB_FLOPS_PER_BOND if args.state_based is not None else FP64_FLOPS_PER_BOND
        tf = fpb * n_bonds / (ms_step * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS,
                    "traffic": None if args.state_based is not None
                    else profiled_traffic(64, args.workload),
                    "peak_source": "FP64 FMA throughput measured by a probe on this pool's GB300 "
                                   "(nominal 1.25 TFLOP/s)",
                    "algorithmic_flops_per_bond": fpb,
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak},
                    "kernel": "k_osb_dilation + k_osb_force" if args.state_based is not None
                    else "k_step_f64"}
    if args.precision == 48:
        ops = DW_OSB_FP32_OPS_PER_BOND if osb else DW_FP32_OPS_PER_BOND
        f64 = OSB_FLOPS_PER_BOND if osb else FP64_FLOPS_PER_BOND
        tops = ops * n_bonds / (ms_step * 1e-3) / 1e12
        tf64 = f64 * n_bonds / (ms_step * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": tops, "peak": FP32_PEAK_TOPS, "unit": "TFLOP/s",
                    "frac": tops / FP32_PEAK_TOPS,
                    "traffic": None if osb else profiled_traffic(48, args.workload),
                    "peak_source": "FP32 operations (add, multiply or fma each counted once) "
                                   "against the FP32 FMA lane rate measured by a probe on this "
                                   "pool's GB300 (70.2 TFLOP/s counting an FMA as two)",
                    "algorithmic_flops_per_bond": ops,
                    "fp64_equivalent": {"achieved": tf64, "peak": FP64_PEAK_TFLOPS,
                                        "unit": "TFLOP/s", "frac": tf64 / FP64_PEAK_TFLOPS,
                                        "flops_per_bond": f64},
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak},
                    "kernel": "k_osb_dw_dilation + k_osb_dw_force" if osb else "k_step_dw"}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cb = oracle_sample(w, oracle.micromodulus(w.bulk_modulus, w.horizon), budget_s=15.0)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # the same oracle on one host thread (a smaller sample of the same workload)
        oracle.set_threads(1)
        c1 = oracle_sample(w, oracle.micromodulus(w.bulk_modulus, w.horizon), budget_s=5.0)
        oracle.set_threads(os.cpu_count() or 1)
        cpu["single_thread"] = {"value": c1["value"], "unit": c1["unit"], "cores": 1,
                                "sample": c1["sample"].replace(f"on {c1['cores']} host threads",
                                                               "on 1 host thread")}
    line = {
        "metric": "bond updates/s", "value": value, "unit": "bond updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "time_steps_per_s": 1e3 / ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {32: "f32", 64: "f64", 48: "f32 double-word"}[args.precision],
        "data": "synthetic", "config": describe(w, n_bonds, args.precision, args.integrator, lat),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(t_on, t_off),
    }
    if unflushed is not None:
        line["unflushed_graph_replay"] = unflushed
    if tuned is not None:
        line["autotuned_launch"] = tuned
    if world == 1 and not args.no_outer and args.workload == "beam":
        # the outer-loop forms, measured in the same process: the batched UQ sweep
        # (256 instances) and the sensitivity plate's adjoint (2000 steps,
        # checkpoints every 45; central differences on a few directions and the
        # oracle's reverse mode over a bounded number of steps)
        b = measure_batch(args, max(10, min(args.steps, 200)), 5, False, False)
        line["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "instance_steps_per_s",
                                           "loop", "batched_over_loop",
                                           "loop_single_model_kernels", "roofline", "config",
                                           "gpu_launches", "clocks")}
        a = measure_adjoint(args, 2000, 45, 4, 1, not args.no_cpu_baseline)
        line["adjoint"] = {k: a[k] for k in ("value", "unit", "dtype", "config", "gradient_ms",
                                             "gradient_parts_ms", "forward_ms",
                                             "adjoint_over_forward", "bonds_broken", "fd",
                                             "oracle_check", "gpu_launches", "clocks")}
    print(json.dumps(line), flush=True)
    if group is not None:
        group.barrier()


def run_batch(args):
    """256 independent bars and notched beams (2k-60k nodes, per-instance K and s_c):
    one batch handle (one fused launch per step, graph-captured, autotuned launch
    shape) against per-instance loops captured in one CUDA graph."""
    print(json.dumps(measure_batch(args, args.steps, args.warmup, not args.no_cpu_baseline,
                                   not args.no_e2e)), flush=True)


def loop_graph_ms(pdgb, torch, ws, precision, general, stream, G, reps):
    """The per-instance loop: one handle per instance, every instance stepped G
    times per replay (G step launches and one counter advance each), all of them
    captured in one CUDA graph; ms per step of all instances."""
    hs = [pdgb.Model.from_workload(w, precision=precision, graph_steps=0,
                                   stream=stream.cuda_stream, general=general) for w in ws]
    layouts = sorted({m.info()["layout"] for m in hs})
    for m in hs:
        m.step(2)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for m in hs:
            pdgb.pd_step(m.h, G)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):  # replays go to the current stream
        g.replay()  # warm-up replay
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1) / (reps * G)
    del g
    for m in hs:
        m.close()
    return ms, layouts


def measure_batch(args, steps, warmup, with_cpu, with_e2e):
    import torch
    import paper_2105_04150_gb300 as pdgb
    torch.cuda.set_device(0)
    ws = workloads.batch_instances()
    stream = torch.cuda.Stream()
    G = max(1, min(args.graph_steps, steps))
    bm = pdgb.Model.batch(ws, precision=args.precision, graph_steps=G, stream=stream.cuda_stream)
    n_bonds = bm.info()["n_bonds"]
    # FP32 batches of lattice models (these bars and beams) run the stencil kernel
    lat = bm.info()["layout"] == pdgb.PD_LAYOUT_LATTICE
    block, bps = bm.autotune(10)
    bm.step(warmup)
    bm.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        time.sleep(0.5)
        t_on = time.time()
        e0.record(stream)
        bm.step(steps)
        e1.record(stream)
        e1.synchronize()
        t_off = time.time()
    bm.sync()
    ms_b = e0.elapsed_time(e1) / steps
    n_nodes = sum(w.n for w in ws)
    # end to end through the public API: pinned host u and v of all instances in
    # and out every step
    e2e = None
    if with_e2e:
        uh = torch.empty((n_nodes, 3), dtype=torch.float64).pin_memory()
        vh = torch.empty((n_nodes, 3), dtype=torch.float64).pin_memory()
        pdgb.pd_get_state(bm.h, uh, vh)
        k_e2e = max(3, min(steps, 50))
        for _ in range(2):
            pdgb.pd_set_state(bm.h, uh, vh)
            bm.step(1)
            pdgb.pd_get_state(bm.h, uh, vh)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(k_e2e):
            pdgb.pd_set_state(bm.h, uh, vh)
            bm.step(1)
            pdgb.pd_get_state(bm.h, uh, vh)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        e2e = {"value": n_bonds * k_e2e / el, "unit": "bond updates/s",
               "h2d_bytes_per_step": 2 * uh.numel() * 8, "d2h_bytes_per_step": 2 * uh.numel() * 8,
               "steps": k_e2e}
    bm.close()
    n_inst = len(ws)
    # the per-instance loops, each captured in one CUDA graph of GL steps: the
    # batch's own (general) step kernel, and each instance's best single-model step
    # (FP32 bars and beams alone are lattice models: the stencil kernel)
    GL = 10
    reps = max(1, min(steps, 20) // GL)
    ms_l, lay_l = loop_graph_ms(pdgb, torch, ws, args.precision, True, stream, GL, reps)
    ms_ll, lay_ll = loop_graph_ms(pdgb, torch, ws, args.precision, False, stream, GL, reps)
    # roofline: the step's algorithmic bytes over all instances (FP32, FP64), or
    # the double-word step's FP32 operations
    per_bond = DW_BYTES_PER_BOND if args.precision == 48 else BYTES_PER_BOND
    alg_bytes = n_bonds * per_bond + n_nodes * BYTES_PER_NODE[args.precision]
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (ms_b * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic("lat", "batch") if lat else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "kernel": "k_step_f32_lat (batch)" if lat
                else f"k_step_{STEP_TAG[args.precision]} (batch)"}
    if lat:
        roofline["note"] = ("algorithmic bytes of the stored-family step; the lattice stencil "
                            "kernel reads no neighbour ids")
    if args.precision == 48:
        tops = DW_FP32_OPS_PER_BOND_NODE_W * n_bonds / (ms_b * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": tops, "peak": FP32_PEAK_TOPS,
                    "unit": "TFLOP/s", "frac": tops / FP32_PEAK_TOPS, "traffic": None,
                    "peak_source": "FP32 operations against the measured FP32 FMA lane rate",
                    "algorithmic_flops_per_bond": DW_FP32_OPS_PER_BOND_NODE_W,
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak},
                    "kernel": "k_step_dw (batch, per-node weights)"}
    # the oracle over whole instances, in order, for about 10 s of host time
    cpu = None
    if with_cpu:
        import oracle
        oracle.build()
        done_bonds, el, used = 0, 0.0, 0
        for w in ws:
            off, idx = oracle.cut_family(w.coords, w.horizon, w.cuts_array())
            om = oracle.Model.from_workload(w, off, idx,
                                            c=oracle.micromodulus(w.bulk_modulus, w.horizon))
            u, v = np.zeros((w.n, 3)), np.zeros((w.n, 3))
            mu = om.fresh_bonds()
            t = time.perf_counter()
            for k in range(5):
                om.step(k, u, v, mu)
            el += time.perf_counter() - t
            done_bonds += 5 * om.nbonds
            used += 1
            if el > 10.0:
                break
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": done_bonds / el, "unit": "bond updates/s", "cores": cores,
               "kind": "oracle",
               "sample": f"5 oracle FP64 steps of each of the first {used} instances "
                         f"(the per-instance loop), OpenMP on {cores} host threads"}
    loop_launches = n_inst + n_inst / GL  # per step: a step kernel per instance, an advance per graph
    return {
        "metric": "bond updates/s", "value": n_bonds / (ms_b * 1e-3), "unit": "bond updates/s",
        "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms_b,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {32: "f32", 64: "f64", 48: "f32 double-word"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"batch of {n_inst} bars and notched beams, "
                               f"{n_nodes:,} nodes, {n_bonds:,} directed bonds",
                   "layout": "lattice stencil kernel" if lat else "sliced ELL",
                   "autotuned_launch": {"block_threads": block, "blocks_per_sm": bps},
                   "l2_policy": f"inputs larger than L2 (step footprint "
                                f"{step_footprint(n_nodes, n_bonds, args.precision, lat) / 1e6:.0f}"
                                f" MB over all instances, L2 {L2_BYTES / 1e6:.0f} MB)"},
        "instance_steps_per_s": n_inst / (ms_b * 1e-3),
        "loop": {"ms_per_step": ms_l, "instance_steps_per_s": n_inst / (ms_l * 1e-3),
                 "launches_per_step": loop_launches, "graph_steps": GL, "steps": reps * GL,
                 "kernel": "the batch's general step kernel, one handle per instance",
                 "layouts": lay_l},
        "batched_over_loop": ms_l / ms_b,
        "loop_single_model_kernels": {
            "ms_per_step": ms_ll, "instance_steps_per_s": n_inst / (ms_ll * 1e-3),
            "launches_per_step": loop_launches, "graph_steps": GL, "steps": reps * GL,
            "kernel": "each instance's own best step (regular-lattice stencil kernel)",
            "layouts": lay_ll, "batched_over_loop": ms_ll / ms_b},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": steps + steps // G + (1 if steps % G else 0),
        "clocks": clk.summary(t_on, t_off),
    }


def cmod_loss(u, above, below):
    """L = CMOD^2 with CMOD = mean u_y above the slit - mean u_y below, at the mouth;
    returns L and dL/du (n x 3)."""
    cmod = u[above, 1].mean() - u[below, 1].mean()
    g = np.zeros_like(u)
    g[above, 1] = 2.0 * cmod / len(above)
    g[below, 1] = -2.0 * cmod / len(below)
    return cmod * cmod, g


def run_adjoint(args):
    """Gradient of the squared crack-mouth opening after N steps of the pre-cracked
    100k-node plate with respect to every directed bond's stiffness (a 10 %
    random field) and the edge load: checkpointed forward + reverse sweep (FP64),
    against the plain forward run, central differences on random directions and
    the oracle's reverse mode on a bounded number of steps."""
    print(json.dumps(measure_adjoint(args, args.steps, args.checkpoint_every, args.fd_directions,
                                     args.warmup, not args.no_cpu_baseline)), flush=True)


def measure_adjoint(args, N, C, fd_directions, warmup, with_cpu):
    import torch
    import paper_2105_04150_gb300 as pdgb
    torch.cuda.set_device(0)
    w = workloads.sensitivity_plate(steps=N)
    c0 = pdgb.pd_micromodulus(w.bulk_modulus, w.horizon)
    stream = torch.cuda.Stream()
    G = max(1, min(args.graph_steps, N))
    prec = 48 if args.precision == 48 else 64  # the adjoint is FP64 or FP64-grade double-word
    vv = args.integrator == "vv"
    m = pdgb.Model.from_workload(w, precision=prec, c=c0, graph_steps=G, stream=stream.cuda_stream,
                                 integrator=pdgb.PD_INTEGRATOR_VV if vv else pdgb.PD_INTEGRATOR_EC)
    off, idx = m.family()
    n_bonds = len(idx)
    cb = workloads.bond_stiffness_grf(w, off, idx, c0)
    rev = workloads.reverse_bond(w.n, off, idx)
    above, below = workloads.mouth_nodes(w)
    zero = np.zeros((w.n, 3))

    def forward_loss(c_bond, load, steps=N):
        m.set_params(c0, w.sc, load, w.disp_rate, c_bond)
        m.set_state(zero, zero, step=0)
        m.step(steps)
        return cmod_loss(m.state()[0], above, below)[0]

    def gradient(c_bond, load, steps=N, ck=C, times=None, flush=None):
        m.set_params(c0, w.sc, load, w.disp_rate, c_bond)
        m.set_state(zero, zero, step=0)
        m.sync()
        if flush is not None:
            l2_flush(torch, stream, flush)
        t0 = time.perf_counter()
        pdgb.pd_adjoint_forward(m.h, steps, ck)
        L, g = cmod_loss(m.state()[0], above, below)
        t1 = time.perf_counter()
        gc, gl, _, _ = pdgb.pd_adjoint_backward(m.h, g)
        m.sync()
        t2 = time.perf_counter()
        if times is not None:
            times.update(forward_ms=(t1 - t0) * 1e3, backward_ms=(t2 - t1) * 1e3)
        return L, gc, gl

    for _ in range(max(1, min(warmup, 3))):
        forward_loss(cb, w.load)
        gradient(cb, w.load)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    flush = l2_flush_buffer(torch, 0)
    with ClockSampler(0) as clk:
        time.sleep(0.5)
        t_on = time.time()
        m.set_params(c0, w.sc, w.load, w.disp_rate, cb)
        m.set_state(zero, zero, step=0)
        m.sync()
        l2_flush(torch, stream, flush)
        e0.record(stream)
        m.step(N)
        e1.record(stream)
        e1.synchronize()
        ms_fwd = e0.elapsed_time(e1)
        parts = {}
        L0, gc, gl = gradient(cb, w.load, times=parts, flush=flush)
        ms_grad = parts["forward_ms"] + parts["backward_ms"]
        t_off = time.time()
    broken = int((m.bonds() == 0).sum())

    # central differences on random directions in (c_bond, load)
    rng = np.random.default_rng(2105041506)
    h = 1e-3  # of a direction whose per-bond entries are 0.1 c0: relative changes ~1e-4
    worst = 0.0
    for _ in range(fd_directions):
        r = rng.standard_normal(n_bonds)
        dc = 0.5 * (r + r[rev]) * 0.1 * c0
        dl = rng.standard_normal() * 0.1 * w.load
        fd = (forward_loss(cb + h * dc, w.load + h * dl)
              - forward_loss(cb - h * dc, w.load - h * dl)) / (2 * h)
        ana = float(gc @ dc) + gl * dl
        worst = max(worst, abs(fd - ana) / abs(ana))

    cpu, oracle_check = None, None
    if with_cpu:
        import oracle
        oracle.build()
        om = oracle.Model.from_workload(w, off, idx, c=c0, c_bond=cb)
        u1, v1 = zero.copy(), zero.copy()
        t = time.perf_counter()
        om.step(0, u1, v1, om.fresh_bonds())
        per_step = time.perf_counter() - t
        S = int(max(2, min(N, 15.0 / (3.0 * per_step))))
        _, gS, _ = gradient(cb, w.load, steps=S, ck=min(C, S))
        uS, vS = zero.copy(), zero.copy()
        if vv:
            om.run_vv(0, S, uS, vS, zero.copy(), om.fresh_bonds(), init=True)
        else:
            om.run(0, S, uS, vS, om.fresh_bonds())
        _, g_u = cmod_loss(uS, above, below)
        t = time.perf_counter()
        gc_o, gl_o, _, _ = oracle.adjoint(om, 0, S, zero, zero, om.fresh_bonds(), g_u, None,
                                          integrator="vv" if vv else "ec")
        el = time.perf_counter() - t
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": n_bonds * S / el, "unit": "bond updates/s", "cores": cores,
               "kind": "oracle",
               "sample": f"oracle FP64 reverse mode (all states stored, "
                         f"{'velocity-Verlet' if vv else 'Euler-Cromer'}) over {S} steps of the "
                         f"full plate, {n_bonds:,} bonds, OpenMP on {cores} host threads"}
        oracle_check = {"steps": S, "checkpoint_every": min(C, S),
                        "dL_dc_max_rel_err": float(np.abs(gS - gc_o).max() / np.abs(gc_o).max())}
    m.close()
    nck = -(-N // C)
    launches = (N + 2 * nck + 1) + (5 * N - 2 * nck + 9)
    if prec == 48:  # double-word records again per recomputed segment and at the end,
        launches += nck + 2  # and the gradient merge
    if vv:  # the force pass that forms the full-step velocity the loss reads with u^N
        launches += 1
    return {
        "metric": "bond updates/s", "value": n_bonds * N / (ms_grad * 1e-3),
        "unit": "bond updates/s", "n_gpus": 1, "steps": N, "warmup": warmup,
        "ms_per_step": ms_grad / N, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == 64 else "f32 double-word",
        "data": "synthetic",
        "config": {"workload": f"{w.name}: {w.n:,} nodes, {n_bonds:,} directed bonds, "
                               f"gradient of CMOD^2 after {N} steps w.r.t. per-bond stiffness "
                               f"and edge load, checkpoint every {C} steps",
                   "integrator": "damped velocity-Verlet" if vv else "damped Euler-Cromer",
                   "load": w.load,
                   "l2_policy": "L2 flushed before each timed leg (the forward run and the "
                                "gradient); within a trajectory the plate's state stays in L2, "
                                "in both legs alike"},
        "gradient_ms": ms_grad, "gradient_parts_ms": parts, "forward_ms": ms_fwd,
        "adjoint_over_forward": ms_grad / ms_fwd, "bonds_broken": broken,
        "loss": L0, "dL_dload": gl,
        "fd": {"directions": fd_directions, "h_rel": h, "max_rel_err": worst},
        "oracle_check": oracle_check, "cpu_baseline": cpu,
        "e2e": {"value": n_bonds * N / (ms_grad * 1e-3), "unit": "bond updates/s",
                "h2d_bytes_per_step": 2 * 24 * w.n / N, "d2h_bytes_per_step": (24 * w.n * 3 +
                                                                             8 * n_bonds) / N},
        "gpu_launches": launches, "clocks": clk.summary(t_on, t_off),
    }


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
