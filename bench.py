#!/usr/bin/env python3
"""Benchmark of the PDG hot path: kinetic DOF-updates/s, FP64 against the mixed-precision
form, as a fraction of the roofline, with the batched and serving forms beside it.

Default workload (one GPU): 3-D compressible Euler (gamma = 1.4) through the vectorial
D3Q6 kinetic model (30 populations), periodic unit cube, 32^3 macrocells x 4^3 subcells,
DG degree 2 (3 GL points per cell and axis: 384^3 points, 1,698,693,120 kinetic DOF,
13.6 GB of FP64 state), theta = 1/2, omega = 2, dt = h / lambda, lambda = 5; seeded
smooth density and velocity fields, pressure 1.  One benchmark step = one palindromic
step M2(dt) = T(dt/2) C(dt) T(dt/2) over the whole state.  DOF-update = one population
value at one GL point advanced through one full step.  The state is larger than L2, so
no L2 flush is needed between steps.

Output: ONE JSON line (rank 0).
  value       FP64, state resident in HBM, K steps between CUDA events on the context
              stream, no per-kernel timing inside that region;
  roofline    the dominant kernel, from a second K-step run with per-kernel CUDA events;
  mixed       the double-float form (FP32-pair state and arithmetic), timed the same way,
              with its error against the FP64 run;
  e2e         the same metric through the C ABI with host buffers (pdg_set_w from pinned
              host memory, pdg_step, pdg_get_w to host) inside the timed region; the
              median of three such runs;
  cpu_baseline  the FP64 oracle on every host core (one replica of a bounded sample per
              core), measured, not scaled;
  batched / serving  the batched form (256 shallow-water meshes) and the serving form
              (Poisson stream, continuous batching, p50/p99 and a sweep of arrival rates),
              on the default workload only (--no-forms skips them).

`--impl reference` times the FP64 CPU oracle (the only reference this method has: the
paper ships no code) on a bounded sample of the same workload, one replica per host core.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling, no
collective on the data path); value = sum over ranks / max time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "kinetic DOF-updates/s"
UNIT = "DOF-updates/s"

# Algorithmic per-unit figures of the dominant kernel (the last-axis pass:
# T(dt/2), collision, T(dt/2)), counted from the operations each step must do:
#   bytes: every population of every point read once and written once = 16 B per DOF.
#   flops per transported DOF per sub-step (degree d, n = d+1): E row (n FMA) + inflow
#     term (1 FMA) + per cell the z combination (2 flops) -> 2n + 2 + 2/n flops.
#   collision flops per point (shallow water): see collision_flops().


def transport_flops_per_dof(n):
    return 2.0 * n + 2.0 + 2.0 / n


def collision_flops_sw():
    # moments 12 adds->9 adds; 1/h (1 div), u, v (2 mul), p = 0.5 g h h (2 mul), 4 flux
    # products (2 FMA + 2 mul = 6 flops); c0 w_k (3 mul); per population fma + mul + add (4 flops) x 12
    return 9 + 1 + 2 + 2 + 6 + 3 + 4 * 12 + 9  # = 80


def diag_flops_per_dof(n):
    """D2Q9 diagonal transport, per DOF (n^2 nodes per cell): the dense Binv row (n^2 FMA),
    r = f/theta (1 mul), the -c1 f term (1 FMA), the face injections and the two
    published faces (4n FMA per cell)."""
    return 2.0 * n * n + 1.0 + 2.0 + 8.0 / n


def corner_flops_per_dof(n):
    """D3Q15 / D3Q27 corner transport, per DOF (n^3 nodes per cell): the dense Binv row
    (n^3 FMA), r = f/theta (1 mul), the -c1 f term (1 FMA), the three face injections and
    the three published faces (6 n^2 FMA per cell)."""
    return 2.0 * n ** 3 + 1.0 + 2.0 + 12.0 / n


def lattice_xi_x(kind):
    """x components of the unit lattice velocities in the population orders of pdg.h."""
    if kind == "isothermal_d2q9":
        return [0, 1, 0, -1, 0, 1, -1, -1, 1]
    axis = [0, 1, -1, 0, 0, 0, 0]
    edges = [1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0]     # planes xy, xz (x first), yz
    corners = [1, -1, -1, 1, 1, -1, -1, 1]
    return {"isothermal_d3q19": axis + edges, "isothermal_d3q15": axis + corners,
            "isothermal_d3q27": axis + edges + corners}[kind]


def collision_flops(kind, dim):
    """Algorithmic flops of the collision at one point (FMA = 2)."""
    nv = 2 * dim
    if kind == "isothermal_d2q9":
        # rho, j_x, j_y (18 adds); 1/rho; s_x, s_y (4 mul); |s|^2/6 and base (4); the four
        # quadratic bases (4 x 3); s_x + s_y, s_y - s_x (2); nine e_i (8 adds); W_i rho (3 mul);
        # relaxation (9 x 3)
        return 18 + 1 + 4 + 4 + 12 + 2 + 8 + 3 + 27
    if kind == "isothermal_d3q19":
        # rho, j (18 + 3 x 9 adds); 1/rho; s (6 mul); base (6); axis bases (3 x 3) and the
        # 12 e_i (2 x 6 adds); plane sums (6) and bases (6 x 3), 12 e_i; W_i rho (3 mul);
        # relaxation (19 x 3)
        return 45 + 1 + 6 + 6 + 9 + 6 + 6 + 18 + 12 + 3 + 57
    if kind in ("isothermal_d3q15", "isothermal_d3q27"):
        # moments (q - 1 adds for rho; each j_a sums 2 axis, 8 corner and (D3Q27) 8 edge
        # populations); 1/rho; s (6); base (6); axis factors (3 x 3); D3Q27 edges as in
        # D3Q19 (6 x 3 + 12); corner sums t (8), q (4 x 3), e (8); W_i rho (4 mul);
        # relaxation (q x 3)
        q = 27 if kind == "isothermal_d3q27" else 15
        edges = 30 if q == 27 else 0
        j_adds = 3 * (17 if q == 27 else 9)
        return (q - 1) + j_adds + 1 + 6 + 6 + 9 + edges + 8 + 12 + 8 + 4 + 3 * q
    if kind == "shallow_water":
        return collision_flops_sw()
    if kind == "advection":
        return (nv - 1) + 4 * nv
    m = dim + 2
    # moments; 1/rho; velocities; kinetic energy; pressure; per axis D momentum fluxes
    # (one FMA, D-1 products) and the energy flux; c0 w_k per axis; 2 FMA per population
    return m * (nv - 1) + 1 + dim + 2 * dim + 3 + dim * (2 + (dim - 1) + 2) + dim * m + 4 * m * nv


# DRAM bytes (read + write) of one launch of the dominant kernel, from the ncu captures
# summarised under profiles/: (workload, kernel kind, precision, lines per block) -> bytes.
# Lines per block (the first number of the line-pass launch shape, which sets how much of a
# block's lines stays in L2 between the operations of a pass) or None for the diagonal /
# corner passes (shape chosen by the host planner).  Only kernels that have not changed
# since their capture are listed; the others report null.  The last-axis passes are those of
# the schedule with the collision after the composed pair of half steps ([T T, C]).  The
# Euler D3Q6 figure was captured at 192^3 points (1.7 GB state, larger than L2) and scaled by
# the 8 times more points of a 384^3 launch (profiles/pass_kernel_fp64_euler_d3q6_384cube.md);
# the shallow-water one at the workload's own size.
TRAFFIC = {("shallow_water_d2q4_64x64x8x8_d3", 1, "fp64", 16): 1192.8e6,
           ("isothermal_d2q9_64x64x8x8_d3", 3, "fp64", None): 279.29e6,
           ("euler_d3q6_32c3x4c3_d2", 1, "fp64", 16): 8 * 4385.8e6}

SOURCES = {"gravity": dict(gravity=(0.0, -1.0)),
           "penalization": dict(K_s=300.0, kappa=40.0, x_c=(0.25, 0.5), w_s=(1.0, 0.0, 0.0)),
           "both": dict(gravity=(0.0, -1.0), K_s=300.0, kappa=40.0, x_c=(0.25, 0.5), w_s=(1.0, 0.0, 0.0))}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", default="euler",
                    choices=["shallow_water", "advection", "euler", "d2q9", "d3q19", "d3q15", "d3q27", "batched",
                             "serving"])
    ap.add_argument("--requests", type=int, default=1000,
                    help="serving: requests in the Poisson stream at --rate")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--chunk", type=int, default=10)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--impl", default="pdg", choices=["pdg", "reference"])
    ap.add_argument("--source", default="none", choices=["none", "gravity", "penalization", "both"],
                    help="d2q9 workload: source stages S(dt/2) C S(dt/2) (gravity g = -1 e_y; "
                         "penalisation K_s = 300, kappa = 40 at (0.25, 0.5), w_s = (1, 0, 0))")
    ap.add_argument("--scheme", default="M2", choices=["M2", "M2_collapsed", "M2_kin", "M4_kin"])
    ap.add_argument("--inflow-x", action="store_true",
                    help="x axis with inflow boundaries (f^b = f^eq of the initial state at the faces)")
    ap.add_argument("--cfl", type=float, default=None,
                    help="Courant number of dt = cfl h / lambda instead of the workload's (M4_kin needs "
                         "moderate values: its middle sub-step runs backwards)")
    ap.add_argument("--n-macro", type=int, default=None,
                    help="macrocells per axis instead of the workload's (a smaller case of the same "
                         "workload, e.g. for profiler captures)")
    ap.add_argument("--graph", action="store_true",
                    help="time pdg_step replaying a captured CUDA graph (PDG_OPT_GRAPH); the roofline "
                         "and kernel figures come from a run with direct launches")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=None,
                    help="oracle steps per core in cpu_baseline (default: about 10 s of work)")
    ap.add_argument("--cpu-cores", type=int, default=None,
                    help="oracle replicas in cpu_baseline / --impl reference (default: every host core)")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the batched and serving sub-objects")
    ap.add_argument("--sweep-requests", type=int, default=100,
                    help="serving: requests per arrival rate of the latency sweep (0: no sweep)")
    ap.add_argument("--serial", action="store_true",
                    help="serving: also time every request alone (serial FIFO baseline; as long as the stream)")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured FP64 / FP32 multiply-add throughput and HBM copy rate, and exit")
    ap.add_argument("--no-mixed", action="store_true", help="skip the double-float measurement")
    ap.add_argument("--shapes", default=None,
                    help="fixed launch shapes 'lpb,nseg,ngroup/lpb,nseg,ngroup' for the transport and "
                         "last-axis passes instead of autotuning (reproduces a timed configuration)")
    ap.add_argument("--tc-layers", type=int, default=2, choices=[1, 2],
                    help="tensor-core corner pass: box layers swept together (PDG_OPT_TC_LAYERS)")
    ap.add_argument("--corner-sweep", type=int, default=1, choices=[0, 1],
                    help="corner pass of D3Q15 / D3Q27: 1 hyperplanes, 0 boxes (PDG_OPT_CORNER_SWEEP)")
    ap.add_argument("--resident", type=int, default=0,
                    help="1: line passes run the line-resident kernel (PDG_OPT_RESIDENT)")
    ap.add_argument("--caxis", type=int, default=-1,
                    help="axis whose pass carries the collision (PDG_OPT_COLLISION_AXIS; -1 = last)")
    ap.add_argument("--rshapes", default=None,
                    help="line-resident launch shapes 'lpb,nseg,ngroup/lpb,nseg,ngroup' (kinds 7 / 8)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df32", "tf32", "tf32_df"],
                    help="precision of the headline run (profiling of the other forms; tf32 / tf32_df: the "
                         "tensor-core cell inverse of the D3Q15 / D3Q27 corner sweeps)")
    return ap.parse_args()


def aggregate_ranks(ms_local, units_local):
    """Whole-job figures of a replica run: the slowest rank's time and the sum of the
    units all ranks processed (torch.distributed all_reduce, any backend)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), float(units_local)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[6 + k].lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# Oracle sample of each workload for the CPU timings: macrocells per axis (the subcells and
# the degree stay the workload's).  About 0.3 s per oracle step on one core.
ORACLE_SAMPLE_MACRO = {2: 8, 3: 4}

_REPLICA = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_1702_00169_gb300 import workloads as W
from oracle import models as OM, scheme as OS
from oracle.dg import CartesianMesh
cfg = W.CONFIGS[{name!r}]
cfg = cfg.scaled(n_macro=tuple(min({nm}, x) for x in cfg.n_macro))
mesh = CartesianMesh(cfg.dim, cfg.ncells, cfg.order, lengths=cfg.lengths[:cfg.dim])
kind = {{"advection": OM.ADVECTION, "shallow_water": OM.SHALLOW_WATER, "euler": OM.EULER,
        "isothermal_d2q9": OM.ISOTHERMAL_D2Q9, "isothermal_d3q19": OM.ISOTHERMAL_D3Q19,
        "isothermal_d3q15": OM.ISOTHERMAL_D3Q15, "isothermal_d3q27": OM.ISOTHERMAL_D3Q27}}[cfg.kind]
model = OM.Model(kind, cfg.dim, cfg.lam, a=cfg.a[:cfg.dim], gravity=cfg.gravity, gamma=cfg.gamma)
w0 = W.initial_w(cfg, [mesh.coords1d(a) for a in range(cfg.dim)])
tr = OS.Transporter(mesh, model, theta=cfg.theta, method="bloch")
f = OS.initial_state(model, w0)
for _ in range({warmup}):
    f = OS.m2_step(f, tr, model, cfg.dt, cfg.omega)
print("READY", flush=True)
sys.stdin.readline()
t0 = time.time()
for _ in range({steps}):
    f = OS.m2_step(f, tr, model, cfg.dt, cfg.omega)
t1 = time.time()
print(json.dumps({{"t0": t0, "t1": t1, "dofs": cfg.dofs, "finite": bool(np.all(np.isfinite(f))),
                  "mesh": "%s macrocells x %s subcells, d=%d" % (
                      "x".join(map(str, cfg.n_macro)), "x".join(map(str, cfg.n_sub)), cfg.order)}}))
"""


def oracle_replicas(cfg_name, dim, steps, warmup, cores=None):
    """Time the FP64 oracle on every host core: one process per core, each advancing its own
    copy of a bounded sample of the workload (macrocells per axis capped at
    ORACLE_SAMPLE_MACRO[dim]) through `warmup` untimed and `steps` timed M2 steps.  The timed
    steps start together (every process reports after its warm-up and waits for a common go);
    the wall time runs from the first start to the last process's end.  Returns the measured figures
    of that sample (nothing is scaled to the full workload)."""
    cores = cores or host_cores()
    nm = ORACLE_SAMPLE_MACRO.get(dim, 4)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = _REPLICA.format(root=ROOT, name=cfg_name, nm=nm, warmup=warmup, steps=steps)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(cores)]
    for p in procs:            # every replica has set up and warmed up
        p.stdout.readline()
    for p in procs:            # common start
        try:
            p.stdin.write("go\n")
            p.stdin.flush()
        except OSError:
            pass
    outs = []
    err = None
    for p in procs:
        try:
            o, e = p.communicate(timeout=1800)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        if p.returncode != 0:
            err = (e or "")[-500:]
            continue
        outs.append(json.loads(o.strip().splitlines()[-1]))
    if not outs or err:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": err or "no output"}
    t0 = min(d["t0"] for d in outs)
    t1 = max(d["t1"] for d in outs)
    wall = t1 - t0
    dofs = outs[0]["dofs"]
    late = max(d["t0"] for d in outs) - t0
    return {"value": len(outs) * dofs * steps / wall, "unit": UNIT, "cores": len(outs), "kind": "oracle",
            "ms_per_step": 1e3 * wall / steps, "seconds": wall, "steps": steps, "sample_dofs": dofs,
            "start_spread_s": late, "finite": all(d["finite"] for d in outs),
            "sample": (f"FP64 numpy oracle (Bloch/FFT transport), {len(outs)} processes (one per host core), each "
                       f"advancing its own copy of the workload's model on {outs[0]['mesh']} ({dofs} DOF) through "
                       f"{steps} timed M2 steps after {warmup} untimed; wall time {wall:.1f} s from the common "
                       f"start to the last process's end; value = {len(outs)} x {dofs} x {steps} / wall")}


def cpu_baseline(cfg_name, dim, steps=None, cores=None):
    """The oracle on all host cores, about 10 s of work per core (see oracle_replicas)."""
    if steps is None:
        steps = 30 if dim == 3 else 20
    return oracle_replicas(cfg_name, dim, steps, 1, cores)


def run_reference(args, cfg, base_name):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # each reference step = one M2 step of the oracle on the bounded sample, on every core
    res = oracle_replicas(base_name, cfg.dim, max(1, args.steps), max(1, args.warmup), args.cpu_cores)
    value = res.get("value")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res.get("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg.name, "reference": "FP64 CPU oracle (the paper ships no code)",
                       "sample": res.get("sample"), "sample_dofs": res.get("sample_dofs"),
                       "ms_per_step": "measured wall time per M2 step of the sample on all cores (not scaled)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res.get("cores"), "kind": "oracle",
                             "sample": res.get("sample")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if res.get("error"):
        line["error"] = res["error"]
    print(json.dumps(line), flush=True)


def measure_peaks(stream=None):
    """Measured FP64 / FP32 multiply-add throughput (pdg_measure_fma_peak) and a device copy
    rate (read + write bytes of a 4 GiB torch copy, best of 5)."""
    import torch
    from paper_1702_00169_gb300 import pdg
    out = {}
    try:
        out["fp64_tflops"] = pdg.measure_fma_peak(True, stream)[0]
        out["fp32_tflops"] = pdg.measure_fma_peak(False, stream)[0]
    except Exception as e:  # noqa: BLE001 - reported in the line
        out["error"] = str(e)
    a = torch.empty(1 << 29, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1.0)
    best = 1e30
    for _ in range(6):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    out["copy_gbs"] = 2.0 * a.numel() * 8 / (best * 1e-3) / 1e9
    del a, b
    torch.cuda.empty_cache()
    return out


def bench_batched(args):
    """256 independent shallow-water meshes (8..96 macrocells per axis x 4x4 subcells,
    degrees 1-4, per-instance dt at CFL 1) advanced by persistent batched launches replayed
    from a CUDA graph, FP64 and double-float; compared with the same instances stepped one
    by one through pdg_step, each with its own autotuned launch shapes and its K-step CUDA
    graph replayed, so that the ratio measures batching alone.  Returns a dict."""
    import torch
    from paper_1702_00169_gb300 import pdg
    from paper_1702_00169_gb300 import workloads as W
    K = args.steps if args.steps is not None else 20
    insts = W.batched_instances()
    stream = torch.cuda.Stream()
    dts = [c.dt for c in insts]
    dofs = sum(c.dofs for c in insts)
    w0s = []

    def make(precision):
        sol = []
        for i, c in enumerate(insts):
            sv = pdg.solver_for(c, stream=stream.cuda_stream, precision=precision)
            if len(w0s) <= i:
                w0s.append(np.ascontiguousarray(W.initial_w(c, [sv.points(a) for a in range(c.dim)]).reshape(-1)))
            sv.set_w(w0s[i])
            sol.append(sv)
        return sol, pdg.Batch(sol, stream=stream.cuda_stream)

    def timed(b, with_clocks):
        t0 = time.perf_counter()
        if not args.no_autotune:
            b.autotune(dts, reps=2)
        tune = time.perf_counter() - t0
        b.step(dts, K, use_graph=True)          # warm-up (captures the graph)
        torch.cuda.synchronize()
        sampler = ClockSampler(str(torch.cuda.get_device_properties(0).uuid)) if with_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.4)
        b.step(dts, K, use_graph=True)          # timed: graph replay
        ms, launches = b.elapsed()
        return ms, launches, tune, (sampler.stop() if sampler else None)

    # mixed-precision variant first (double-float state and arithmetic), then FP64
    sol_d, b_d = make("df32")
    ms_d, _, _, _ = timed(b_d, False)
    w_d = [sv.get_w() for sv in sol_d[:16]]
    b_d.close()
    for sv in sol_d:
        sv.close()
    sol, b = make("fp64")
    ms, launches, tune_s, clocks = timed(b, True)
    err_d = float(np.sqrt(sum(np.sum((sv.get_w() - wd) ** 2) for sv, wd in zip(sol[:16], w_d))
                          / sum(np.sum(sv.get_w() ** 2) for sv in sol[:16])))
    finite = all(bool(np.all(np.isfinite(sv.get_w()))) for sv in sol[:8])
    b.close()
    # the same instances one by one: autotuned shapes, a captured K-step graph each (untimed
    # set-up), then the K-step replays of all instances back to back between two events
    t0 = time.perf_counter()
    for sv, dt in zip(sol, dts):
        if not args.no_autotune:
            sv.autotune(dt, reps=1)
        sv.set_option(pdg.PDG_OPT_GRAPH, 1)
        sv.step(dt, K)
    tune_serial = time.perf_counter() - t0
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for sv, dt in zip(sol, dts):
        sv.step(dt, K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_serial = ev0.elapsed_time(ev1)
    for sv in sol:
        sv.close()
    return {"value": dofs * K / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms, "steps": K, "dtype": "f64",
            "config": {"workload": "batched_shallow_water_256", "instances": len(insts), "dof": dofs,
                       "mesh": "M x M macrocells, M ~ U{8..96}, 4x4 subcells, d ~ U{1..4} (seed 4)",
                       "dt": "per instance, CFL 1", "graph": True, "autotuned": not args.no_autotune,
                       "autotune_s": tune_s, "l2": "18 GB state >> L2"},
            "gpu_launches": launches, "clocks": clocks,
            "one_by_one": {"value": dofs * K / (ms_serial * 1e-3), "ms": ms_serial, "setup_s": tune_serial,
                           "note": "each instance alone through pdg_step: its own autotuned shapes, its K-step "
                                   "CUDA graph replayed, instances back to back"},
            "speedup_vs_one_by_one": ms_serial / ms, "state_finite": finite,
            "mixed": {"precision": "df32", "value": dofs * K / (ms_d * 1e-3), "speedup_vs_fp64": ms / ms_d,
                      "rel_l2_w_vs_fp64": err_d, "note": "same batch, double-float state and arithmetic; error over "
                                                         "the first 16 instances after warm-up + K steps"}}


def _serve_stream(reqs, args, stream, with_clocks=False):
    """Serve one request stream [(t_arrival, cfg, nsteps)] through a fresh pdg server with
    continuous batching (arrivals follow their times on the server clock).  Latency =
    completion - arrival, queue wait = admission - arrival."""
    import queue
    import torch
    from paper_1702_00169_gb300 import pdg
    from paper_1702_00169_gb300 import workloads as W

    def coords(cfg):
        # GL coordinates from the library's own quadrature (a throw-away context)
        sv = pdg.Solver(cfg.dim, cfg.n_macro, cfg.n_sub, cfg.order)
        sv.set_model(cfg.kind, cfg.lam, a=cfg.a, gravity=cfg.gravity)
        c = [sv.points(a) for a in range(cfg.dim)]
        sv.close()
        return c

    inputs = queue.Queue(maxsize=32)

    def producer():
        for t, cfg, ns in reqs:
            inputs.put((t, cfg, ns, W.initial_w(cfg, coords(cfg)).reshape(-1)))

    th = threading.Thread(target=producer, daemon=True)
    srv = pdg.Server(int(args.budget_gb * 2 ** 30), chunk_steps=args.chunk, stream=stream.cuda_stream)
    # warm-up: one small solve
    wcfg = W.SW_D2Q4.scaled(n_macro=(4, 4), n_sub=(4, 4))
    srv.submit(wcfg, W.initial_w(wcfg, coords(wcfg)), 3)
    while srv.pending()[1] or srv.pending()[0]:
        srv.iterate()
    srv.poll()
    th.start()
    t0 = srv.now()
    lat, work, ids = [], {}, {}
    nxt = None
    submitted = 0
    sampler = ClockSampler(str(torch.cuda.get_device_properties(0).uuid)) if with_clocks else None
    if sampler:
        sampler.start()
    while len(lat) < len(reqs):
        now = srv.now() - t0
        while submitted < len(reqs):
            if nxt is None:
                try:
                    nxt = inputs.get(timeout=0.001 if srv.pending()[1] else 0.05)
                except queue.Empty:
                    break
            t, cfg, ns, w0 = nxt
            if t > now:
                break
            rid = srv.submit(cfg, w0, ns, t_arrival=t0 + t)
            ids[rid] = cfg
            work[rid] = cfg.dofs * ns
            submitted += 1
            nxt = None
        nw, nr = srv.pending()
        if nr or nw:
            srv.iterate()
        else:
            time.sleep(0.0005)
        for rid, ta, tb, tc in srv.poll():
            lat.append((tc - ta, tb - ta, rid))
            srv.result(rid, ids[rid].m * ids[rid].npoints)
    makespan = srv.now() - t0
    clocks = sampler.stop() if sampler else None
    st = srv.stats()
    srv.close()
    th.join(timeout=5)
    total = sum(work.values())
    L = np.array([x[0] for x in lat])
    Q = np.array([x[1] for x in lat])
    return {"requests": len(reqs), "value": total / makespan, "makespan_s": makespan, "dof_updates": total,
            "latency_s": {"p50": float(np.percentile(L, 50)), "p99": float(np.percentile(L, 99)),
                          "mean": float(L.mean()), "queue_p50": float(np.percentile(Q, 50)),
                          "queue_p99": float(np.percentile(Q, 99))},
            "offered_dof_updates_per_s": total / max(1e-9, reqs[-1][0]), "server": st, "clocks": clocks}


def bench_serving(args, serial=False):
    """Poisson stream of 2-D advection / shallow-water solves served with continuous
    batching under a device-memory budget (the stream at --rate, default 1000 requests at
    200 req/s), then a sweep of arrival rates on the first --sweep-requests requests of the
    same stream (rates at 1/4, 1/2, 3/4, 1 and 5/4 of the capacity the first run measured), and
    the highest swept rate whose p99 latency stays within twice the p99 at the lowest rate.
    serial: also time every request alone through pdg_step (single-server FIFO on the same
    arrivals).  Returns a dict."""
    import torch
    from paper_1702_00169_gb300 import pdg
    from paper_1702_00169_gb300 import workloads as W
    stream = torch.cuda.Stream()
    reqs = W.serving_requests(n=args.requests, rate=args.rate)
    main = _serve_stream(reqs, args, stream, with_clocks=True)
    out = {"value": main["value"], "unit": UNIT, "dtype": "f64",
           "config": {"workload": "serving_poisson", "requests": len(reqs), "rate_req_s": args.rate,
                      "budget_gb": args.budget_gb, "chunk_steps": args.chunk,
                      "mix": "50/50 advection D2Q4 / shallow water D2Q4, M ~ U{16..128} macrocells, 4x4 subcells, "
                             "d ~ U{1..4}, steps log-uniform [10, 1000] (seed 5)"},
           "stream": main}
    if args.sweep_requests > 0:
        sub = W.serving_requests(n=args.sweep_requests, rate=1.0)
        mean_work = float(np.mean([c.dofs * ns for _, c, ns in sub]))
        cap = main["value"] / mean_work          # requests per second the server sustained
        sweep = []
        for frac in (0.25, 0.5, 0.75, 1.0, 1.25):
            r = frac * cap
            res = _serve_stream(W.serving_requests(n=args.sweep_requests, rate=r), args, stream)
            sweep.append({"rate_req_s": r, "fraction_of_capacity": frac, "value": res["value"],
                          "p50_s": res["latency_s"]["p50"], "p99_s": res["latency_s"]["p99"],
                          "queue_p99_s": res["latency_s"]["queue_p99"], "makespan_s": res["makespan_s"]})
        bound = 2.0 * sweep[0]["p99_s"]
        ok = [x["rate_req_s"] for x in sweep if x["p99_s"] <= bound]
        out["rate_sweep"] = {"requests_per_rate": args.sweep_requests, "capacity_req_s": cap,
                             "mean_dof_updates_per_request": mean_work, "points": sweep,
                             "p99_bound_s": bound,
                             "max_rate_bounded_p99_req_s": max(ok) if ok else None,
                             "criterion": "highest swept rate whose p99 latency is at most twice the p99 at "
                                          "1/4 of the capacity (where requests rarely queue)"}
    if serial:
        service = []
        for t, cfg, ns in reqs:
            sv = pdg.solver_for(cfg, stream=stream.cuda_stream)
            sv.set_w(np.ascontiguousarray(W.initial_w(cfg, [sv.points(a) for a in range(cfg.dim)]).reshape(-1)))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.step(cfg.dt, ns)
            e1.record(stream)
            e1.synchronize()
            service.append(e0.elapsed_time(e1) * 1e-3)
            sv.close()
        tdone, sl = 0.0, []
        for (t, cfg, ns), sv_t in zip(reqs, service):
            tdone = max(t, tdone) + sv_t
            sl.append(tdone - t)
        sl = np.array(sl)
        out["serial"] = {"value": main["dof_updates"] / float(np.sum(service)),
                         "latency_p50_s": float(np.percentile(sl, 50)),
                         "latency_p99_s": float(np.percentile(sl, 99)),
                         "note": "each request alone through pdg_step (plain FP64, heuristic shapes), single-server "
                                 "FIFO on the same arrivals"}
    return out


def _line_for_form(args, sub, workload):
    """A standalone JSON line for --workload batched / serving."""
    steps = sub.get("steps", sub.get("config", {}).get("requests"))
    line = {"metric": METRIC, "value": sub["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": steps if workload == "batched" else 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    line.update(sub)
    if workload == "batched":
        line["ms_per_step"] = sub["ms_per_call"] / sub["steps"]
    else:
        line["ms_per_step"] = 1e3 * sub["stream"]["makespan_s"] / sub["config"]["requests"]
        line["clocks"] = sub["stream"]["clocks"]
    return line


def main():
    args = parse_args()
    from paper_1702_00169_gb300 import workloads as W
    cfg = {"advection": W.ADVECTION_D2Q4, "shallow_water": W.SW_D2Q4, "euler": W.EULER_D3Q6, "d2q9": W.D2Q9_ISO,
           "d3q19": W.D3Q19_ISO, "d3q15": W.D3Q15_ISO, "d3q27": W.D3Q27_ISO}.get(args.workload, W.EULER_D3Q6)
    base_name = cfg.name   # the oracle's sample is drawn from the named workload
    if args.cfl:
        import dataclasses
        cfg = dataclasses.replace(cfg, cfl=args.cfl)
    if args.n_macro:
        cfg = cfg.scaled(n_macro=(args.n_macro,) * cfg.dim,
                         name=f"{cfg.name}_n{args.n_macro}" if args.n_macro != cfg.n_macro[0] else cfg.name)
    if args.source != "none" and cfg.kind != "isothermal_d2q9":
        raise SystemExit("--source: sources run on the D2Q9 workload (--workload d2q9)")
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 20
        if args.warmup is None:
            args.warmup = 3
        run_reference(args, cfg, base_name)
        return
    if args.peaks:
        import torch
        torch.cuda.set_device(0)
        pk = measure_peaks()
        nominal = torch.cuda.get_device_properties(0).multi_processor_count * 2 * 2 * 2070e6 / 1e12
        print(json.dumps({"peaks": pk, "fp64_nominal_tflops_at_2070mhz": nominal}), flush=True)
        return
    if args.workload in ("batched", "serving"):
        sub = bench_batched(args) if args.workload == "batched" else bench_serving(args, serial=True)
        print(json.dumps(_line_for_form(args, sub, args.workload)), flush=True)
        return
    if args.steps is None:
        args.steps = {"euler": 20, "advection": 1000, "d2q9": 100, "d3q19": 10, "d3q15": 4,
                      "d3q27": 4}.get(args.workload, 1000)
    if args.warmup is None:
        args.warmup = {"euler": 3, "d2q9": 5, "d3q19": 3, "d3q15": 3, "d3q27": 3}.get(args.workload, 20)

    import torch
    ws, rank, local = dist_env()
    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1702_00169_gb300 import pdg

    stream = torch.cuda.Stream()
    periodic = [True] * cfg.dim
    if args.inflow_x:
        periodic[0] = False

    def solver(precision):
        sv = pdg.Solver(cfg.dim, cfg.n_macro, cfg.n_sub, cfg.order, lengths=cfg.lengths[:cfg.dim],
                        stream=stream.cuda_stream, periodic=periodic)
        sv.set_model(cfg.kind, cfg.lam, a=cfg.a, gravity=cfg.gravity, gamma=cfg.gamma, omega=cfg.omega,
                     theta=cfg.theta, scheme=args.scheme, precision=pdg.PRECISION[precision])
        if args.source != "none":
            sv.set_source(**SOURCES[args.source])
        if precision in ("tf32", "tf32_df"):
            sv.set_option(pdg.PDG_OPT_TC_LAYERS, args.tc_layers)
        if not args.corner_sweep:
            sv.set_option(pdg.PDG_OPT_CORNER_SWEEP, 0)
        if args.resident:
            sv.set_option(pdg.PDG_OPT_RESIDENT, 1)
        if args.caxis >= 0:
            sv.set_option(pdg.PDG_OPT_COLLISION_AXIS, args.caxis)
        if args.rshapes:
            for kind, sh in enumerate(args.rshapes.split("/")):
                sv.set_launch(7 + kind, *[int(x) for x in sh.split(",")])
        return sv

    s = solver(args.precision)
    info = s.info()
    coords = [s.points(a) for a in range(cfg.dim)]
    w0 = np.ascontiguousarray(W.initial_w(cfg, coords).reshape(-1))
    w0_dev = torch.from_numpy(w0).cuda()
    fb = None
    if args.inflow_x:
        # inflow data: the initial equilibrium populations at the two x faces
        s.set_w(w0_dev)
        f0 = s.get_f().reshape((cfg.groups, cfg.nv) + tuple(reversed(cfg.npoints_axis)))
        if cfg.kind.startswith("isothermal"):
            # the populations entering through the low x face (xi_x > 0) and the high x face
            # (xi_x < 0), in population order, at that face's points
            sx = lattice_xi_x(cfg.kind)
            lo = [i for i in range(cfg.nv) if sx[i] > 0]
            hi = [i for i in range(cfg.nv) if sx[i] < 0]
            fb = np.ascontiguousarray(np.stack([f0[0, lo, ..., 0].reshape(len(lo), -1),
                                                f0[0, hi, ..., -1].reshape(len(hi), -1)]))
        else:
            fb = np.ascontiguousarray(np.stack([f0[:, 0, ..., 0].reshape(cfg.m, -1),
                                                f0[:, 1, ..., -1].reshape(cfg.m, -1)]))
        del f0
    torch.cuda.synchronize()
    dev_uuid = None
    try:
        dev_uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def timed_run(sv, per_kernel=False, graph=False):
        """W untimed steps, then K steps between CUDA events on the context stream, with
        clock sampling around them.  per_kernel: CUDA events around every launch as well
        (the roofline run; the headline run has none).  graph: the K steps replay a CUDA
        graph captured by one untimed run of K steps."""
        sv.set_w(w0_dev)
        if fb is not None:
            sv.set_inflow(0, fb)
        if not getattr(sv, "_bench_tuned", False) and not graph:
            if args.shapes:
                for kind, sh in enumerate(args.shapes.split("/")):
                    sv.set_launch(kind, *[int(x) for x in sh.split(",")])
            elif not args.no_autotune:
                sv.autotune(cfg.dt, reps=3)     # launch shapes picked on a scratch copy (untimed)
            sv._bench_tuned = True
        sv.step(cfg.dt, args.warmup)
        if graph:
            sv.set_option(pdg.PDG_OPT_GRAPH, 1)
            sv.step(cfg.dt, args.steps)     # capture (and run) the K-step graph, untimed
        sv.synchronize()
        sampler = ClockSampler(dev_uuid)
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.4)
        if per_kernel:
            sv.timing_enable(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sv.step(cfg.dt, args.steps)
        ev1.record(stream)
        sv.synchronize()
        torch.cuda.synchronize()
        clk = sampler.stop()
        barrier()
        launches, kms = sv.timing_read() if per_kernel else ([0] * 5, [0.0] * 5)
        sv.timing_enable(False)
        if graph:
            sv.set_option(pdg.PDG_OPT_GRAPH, 0)
        return ev0.elapsed_time(ev1), launches, kms, clk

    n = cfg.order + 1
    P = info.npoints
    F = info.nfields
    q9 = cfg.kind == "isothermal_d2q9"
    lattice = cfg.kind.startswith("isothermal")
    pops_line = 2 if lattice else F // cfg.dim     # populations transported by one line pass

    def dominant(kms):
        """Kernel kind with the largest share of the timed region (0, 1, 3 or 4)."""
        return max((0, 1, 3, 4), key=lambda k: kms[k])

    def kernel_work(kind):
        """(algorithmic bytes, algorithmic flops) of one launch of a kernel kind."""
        if kind == 3:   # one launch = one plane orientation, four populations
            return 16.0 * 4 * P, 4 * P * diag_flops_per_dof(n)
        if kind == 4:   # one launch = the eight corner populations
            return 16.0 * 8 * P, 8 * P * corner_flops_per_dof(n)
        if kind == 1:
            return 16.0 * F * P, 2 * pops_line * P * transport_flops_per_dof(n) + P * collision_flops(cfg.kind, cfg.dim)
        return 16.0 * pops_line * P, 2 * pops_line * P * transport_flops_per_dof(n)

    dofs = cfg.dofs
    # ---- FP64 (or --precision), state resident in HBM: headline, then per-kernel timing ----
    ms, _, _, clocks = timed_run(s)
    w_end = s.get_w()
    finite = bool(np.all(np.isfinite(w_end)))
    ms_k, launches, kms, clocks_k = timed_run(s, per_kernel=True)
    graph_run = None
    if args.graph:
        ms_g, _, _, clocks_g = timed_run(s, graph=True)
        graph_run = {"ms_per_step_direct": ms / args.steps,
                     "note": "one CUDA graph of K steps replayed; bitwise the direct launches (tests/test_gpu_graph.py)"}
        ms, clocks = ms_g, clocks_g
    shape0, shape1 = s.get_launch(0), s.get_launch(1)
    s_shape = {0: shape0, 1: shape1}
    ms_max, units = aggregate_ranks(ms, dofs * args.steps)
    value = units / (ms_max * 1e-3)

    # ---- the same run in double-float precision (FP32-pair state and arithmetic) ----
    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        s.close()                       # one state at a time on the device
        s = None
        sd = solver("df32")
        ms_d, _, _, clocks_d = timed_run(sd)
        w_end_d = sd.get_w()
        _, launches_d, kms_d, _ = timed_run(sd, per_kernel=True)
        sd.close()
        k_d = dominant(kms_d)
        avg_d = kms_d[k_d] / max(1, launches_d[k_d])
        bytes_d = kernel_work(k_d)[0]
        ms_d_max, units_d = aggregate_ranks(ms_d, dofs * args.steps)
        mixed = {"precision": "df32 (FP32-pair state and double-word arithmetic on the FP32 pipes)",
                 "value": units_d / (ms_d_max * 1e-3),
                 "ms_per_step": ms_d_max / args.steps,
                 "speedup_vs_fp64": ms_max / ms_d_max,
                 "rel_l2_w_vs_fp64_after_steps": float(np.linalg.norm(w_end_d - w_end) / np.linalg.norm(w_end)),
                 "steps_compared": args.warmup + args.steps,
                 "dominant_kernel_avg_ms": avg_d,
                 "hbm_achieved_gbs": bytes_d / (avg_d * 1e-3) / 1e9, "clocks": clocks_d,
                 "kernels": {name: {"launches": int(launches_d[k]), "avg_ms": kms_d[k] / launches_d[k],
                                    "share": kms_d[k] / max(1e-12, sum(kms_d))}
                             for k, name in ((0, "transport pass"), (1, "last-axis pass"), (2, "state kernels"),
                                             (3, "diagonal pass"), (4, "corner pass")) if launches_d[k]},
                 "gpu_launches": int(sum(launches_d))}
        del w_end_d

    # ---- the tensor-core forms of the corner sweep (D3Q15 / D3Q27), FP64 state ----
    tensor_core = None
    if cfg.kind in ("isothermal_d3q15", "isothermal_d3q27") and args.precision == "fp64" and not args.no_mixed:
        if s is not None:
            s.close()
            s = None
        tensor_core = {}
        k4_fp64 = kms[4] / max(1, launches[4])
        for prec in ("tf32", "tf32_df"):
            st_ = solver(prec)
            ms_t, _, _, clocks_t = timed_run(st_)
            w_end_t = st_.get_w()
            _, launches_t, kms_t, _ = timed_run(st_, per_kernel=True)
            st_.close()
            avg4 = kms_t[4] / max(1, launches_t[4])
            ms_t_max, units_t = aggregate_ranks(ms_t, dofs * args.steps)
            tensor_core[prec] = {
                "precision": ("split-TF32 cell inverse on the tensor cores (tcgen05), one refinement with the "
                              "residual in " + ("FP64" if prec == "tf32" else "double-float") + "; FP64 state; " +
                              ("batches of 128 hyperplane cells per product (degree <= 2)" if args.corner_sweep
                               else "box anti-diagonals per product")),
                "value": units_t / (ms_t_max * 1e-3), "ms_per_step": ms_t_max / args.steps,
                "speedup_vs_fp64": ms_max / ms_t_max,
                "rel_l2_w_vs_fp64_after_steps": float(np.linalg.norm(w_end_t - w_end) / np.linalg.norm(w_end)),
                "corner_pass_avg_ms": avg4, "corner_pass_avg_ms_fp64": k4_fp64,
                "corner_pass_speedup": k4_fp64 / avg4 if avg4 else None,
                "corner_pass_algorithmic_tflops": kernel_work(4)[1] / (avg4 * 1e-3) / 1e12 if avg4 else None,
                "clocks": clocks_t}
            del w_end_t
        if mixed is not None:
            tensor_core["df32_corner_pass_avg_ms"] = mixed["kernels"].get("corner pass", {}).get("avg_ms")

    # ---- end-to-end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        if s is not None:
            s.close()
            s = None
        del w0_dev
        torch.cuda.empty_cache()
        w_host = torch.from_numpy(w0).pin_memory()
        w_out = torch.empty_like(w_host).pin_memory()
        s2 = solver("fp64")
        s2.set_w(w_host)
        if fb is not None:
            s2.set_inflow(0, fb)
        if args.shapes or not args.no_autotune:
            for kind in (0, 1):
                s2.set_launch(kind, *s_shape[kind])
        s2.step(cfg.dt, 2)
        s2.get_w(w_out)
        # three timed runs, the median reported: a host-to-device copy from pinned memory
        # occasionally runs at a fraction of its usual rate on a shared host
        runs = []
        for _ in range(3):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2.set_w(w_host)
            s2.step(cfg.dt, args.steps)
            s2.get_w(w_out)
            t1 = time.perf_counter()
            runs.append(t1 - t0)
        el_max, units_e2e = aggregate_ranks(sorted(runs)[1], dofs * args.steps)
        s2.close()
        nbytes = w0.nbytes
        e2e = {"value": units_e2e / el_max, "unit": UNIT,
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
               "runs_s": [round(r, 4) for r in runs],
               "note": "one pdg_set_w (pinned host) + pdg_step(K) + pdg_get_w (pinned host) per timed run; "
                       "bytes amortised over K; median of three runs"}
        del w_host, w_out
    if s is not None:
        s.close()

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (from the per-kernel CUDA-event run) ----
    kinds = {0: "transport pass (composed T T on the populations of the other axes)",
             1: "last-axis pass (T, collision, T)",
             3: "diagonal transport pass (4 populations of one plane, tiled 2-D wavefront)",
             4: ("corner transport pass (8 populations, cell hyperplanes of the whole mesh, cooperative launch)"
                 if args.corner_sweep else "corner transport pass (8 populations, boxes swept as layer-by-layer wavefronts)")}
    k_dom = dominant(kms)
    avg_ms = kms[k_dom] / max(1, launches[k_dom])
    bytes_launch, flops_launch = kernel_work(k_dom)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = clocks_k.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    measured = measure_peaks(stream.cuda_stream)
    # FP64 pipe: 2 DFMA per SM per clock (GB300 nominal 1.26 TFLOP/s at 2.07 GHz)
    fp64_peak_tflops = n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12
    achieved_tflops = flops_launch / (avg_ms * 1e-3) / 1e12
    achieved_gbs = bytes_launch / (avg_ms * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": achieved_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
            "frac": achieved_tflops / fp64_peak_tflops,
            "peak_measured": measured.get("fp64_tflops"),
            "frac_of_measured": (achieved_tflops / measured["fp64_tflops"]) if measured.get("fp64_tflops") else None,
            "traffic": (TRAFFIC.get((cfg.name, k_dom, args.precision,
                                     s_shape[k_dom][0] if k_dom in (0, 1) else None))
                        if args.source == "none" else None),
            "kernel": kinds[k_dom], "avg_launch_ms": avg_ms, "launches": launches[k_dom],
            "algorithmic_flops_per_launch": flops_launch, "algorithmic_bytes_per_launch": bytes_launch,
            "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak, "hbm_frac": achieved_gbs / hbm_peak,
            "timing_run": "a second K-step run with CUDA events around every launch (the headline run has none)",
            "peak_note": (f"peak = {n_sm} SMs x 2 DFMA/clk x 2 flop x median SM clock under load (nominal); "
                          "peak_measured = pdg_measure_fma_peak (FP64 FMA chains on every SM), of measured"
                          + ("; double-float run: the algorithmic flops are FP64-equivalent operations "
                             "executed as double-word FP32 arithmetic, so the FP64 pipe is not its bound"
                             if args.precision == "df32" else ""))}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(base_name, cfg.dim, args.cpu_sample_steps, args.cpu_cores)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32x2",
            "data": "synthetic",
            "config": {"workload": cfg.name,
                       "model": ("isothermal Euler via D2Q9 (9 populations, 4 diagonal)" if q9 else
                                 "isothermal Euler via D3Q19 (19 populations, 12 edge)"
                                 if cfg.kind == "isothermal_d3q19" else
                                 "isothermal Euler via D3Q15 (15 populations, 8 corner)"
                                 if cfg.kind == "isothermal_d3q15" else
                                 "isothermal Euler via D3Q27 (27 populations, 12 edge, 8 corner)" if lattice else
                                 f"{cfg.kind} via vectorial D{cfg.dim}Q{2 * cfg.dim} ({cfg.nfields} populations)"),
                       "mesh": (f"{'x'.join(map(str, cfg.n_macro))} macrocells x {'x'.join(map(str, cfg.n_sub))} "
                                f"subcells, d={cfg.order}, {'x'.join(map(str, cfg.npoints_axis))} GL points, periodic"),
                       "dof": dofs, "scheme": args.scheme, "theta": cfg.theta, "omega": cfg.omega,
                       "source": (f"M2^s: S(dt/2) C S(dt/2), {args.source} {SOURCES[args.source]}"
                                  if args.source != "none" else "none"),
                       "boundaries": "x: inflow (f^b = initial equilibrium), others periodic" if args.inflow_x
                       else "periodic",
                       "dt": cfg.dt, "lambda": cfg.lam, "precision": args.precision.upper(),
                       "l2": (f"state {cfg.dofs * 8 / 1e6:.0f} MB > 126 MB L2: inputs larger than L2, no flush"
                              if cfg.dofs * 8 > 126e6 else
                              f"state {cfg.dofs * 8 / 1e6:.1f} MB fits in L2: L2-resident (small parity workload)"),
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                       "collision_axis": args.caxis if args.caxis >= 0 else cfg.dim - 1,
                       "line_resident": bool(args.resident),
                       "corner_sweep": "hyperplanes" if args.corner_sweep else "boxes",
                       "launch_shapes": {"autotuned": not args.no_autotune and not args.shapes,
                                         "transport_pass": list(shape0),
                                         "last_axis_pass": list(shape1)}},
            "gpu_launches": int(sum(launches)),
            "kernels": {name: {"launches": int(launches[k]), "avg_ms": kms[k] / launches[k],
                               "share": kms[k] / max(1e-12, sum(kms))}
                        for k, name in ((0, "transport pass"), (1, "last-axis pass"), (2, "state kernels"),
                                        (3, "diagonal pass"), (4, "corner pass")) if launches[k]},
            "per_kernel_run_ms_per_step": ms_k / args.steps,
            "roofline": roof, "clocks": clocks, "peaks_measured": measured,
            "e2e": e2e, "cpu_baseline": cpu, "mixed": mixed, "state_finite": finite}
    if tensor_core:
        line["tensor_core"] = tensor_core
    if graph_run:
        line["graph_replay"] = graph_run
    if args.workload == "euler" and not args.no_forms and ws == 1 and not (args.n_macro or args.cfl):
        line["batched"] = bench_batched(args)
        line["serving"] = bench_serving(args, serial=args.serial)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
