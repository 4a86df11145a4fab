"""Benchmark of the FFT-PIM apply on GB300 (one JSON line on rank 0).

Workload: 2D-periodic (x, y) Helmholtz with a Bloch phase shift, cell
1 x 1 x 0.5, k = 2 pi 0.8, k0 = (0.3k, 0.1k, 0), N = 262144 points (half
uniform, half on a sphere of radius 0.2 at the cell centre), complex64
sources CN(0, 1), near grid 128 x 128 x 64, p = 4, FP32 bulk with FP64 far
series, far grid sum and near-pair correction (values computed in FP64; per
row the entries above 2^-10 of its largest stored as an FP32 head and a bf16
tail and summed in double-float, the others as complex64 summed in FP32).  A step is one forward apply plus one adjoint apply (every row
of the hot path).  Metric: Mpts/s per apply (fwd+adjoint) = 2 N / t_step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (test infrastructure, the
reference arm of this method) on a bounded sample of rows of the same
workload.  Multi-GPU: the apply does not shard; N independent replicas
(weak scaling).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT-PIM Mpts/s per apply (fwd+adjoint) at stated rel-L2 vs FP64; % HBM peak"
UNIT = "Mpts/s"
WORKLOAD = "helmholtz2d_262k"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "gather_correct_helmholtz2d_262k.md")
GOLDEN_ROWS = os.path.join(ROOT, "tests", "golden", "helmholtz2d_262k_ewald_rows.txt")


def golden_rows():
    """(rows, values) of the committed Ewald ground truth of the 262k workload."""
    try:
        d = np.loadtxt(GOLDEN_ROWS, comments="#")
        return d[:, 0].astype(np.int64), d[:, 1] + 1j * d[:, 2]
    except OSError:
        return None, None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(name=WORKLOAD):
    from paper_2312_02376_gb300 import inputs
    if name == "helmholtz2d_65k":   # the same recipe at a quarter of the points and half the grid per axis
        return inputs.helmholtz2d(N=65536, n=(64, 64, 32))
    return inputs.helmholtz2d()


def dist_init(n_gpus, backend="nccl"):
    """Ranks from the launcher's environment; one process group over all
    ranks for the barrier and the max of the step times (replicas: no
    collective on the data path)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend, init_method="env://")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    """The maximum of x over the ranks (the slowest replica sets the time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(n_points, world, ms_step):
    """Whole-job Mpts/s of a step of one forward and one adjoint apply on
    every replica."""
    return 2.0 * n_points * world / (ms_step * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "pim_clocks_%d.csv" % os.getpid())
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


VALUE_BYTES = {0: 16, 1: 16, 2: 8, 3: 8}   # per correction value, by pim_corr_mode


def gather_bytes(info, N, G, nf3, fp64=False, nbig=0):
    """Algorithmic bytes of one gather + correction launch: the correction
    value (16 B FP64 or double-float, 8 B FP32 or compact, plus a 4 B tail
    for the nbig compact entries summed in double-float) and a 4 B column per
    entry; per point the stencil start, local coordinates, permutation,
    sorted source and output (and the compact row split); the near grid
    once.  (The far interpolation is a separate kernel on the far stream.)"""
    compact = int(info.corr_mode) == 3
    per_nnz = VALUE_BYTES[int(info.corr_mode)] + 4
    c, r = (16, 8) if fp64 else (8, 4)        # complex and real element sizes
    per_point = 4 + 3 * r + 4 + c + c + (4 if compact else 0)
    return info.nnz * per_nnz + 4 * nbig + (N + 1) * 8 + N * per_point + G * c


def gather_source_hash():
    """First 16 hex digits of the SHA-256 of the gather kernel's sources
    (the kernel, the Lagrange helpers it inlines and the shared header)."""
    csrc = os.path.join(ROOT, "paper_2312_02376_gb300", "csrc")
    hs = hashlib.sha256()
    for f in ("gather.cuh", "lagrange.cuh", "pim_internal.cuh"):
        hs.update(open(os.path.join(csrc, f), "rb").read())
    return hs.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per launch of the gather kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        txt = open(PROFILE_SUMMARY).read()
        h = gather_source_hash()
        m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
        t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        if m and t and m.group(1) == h:
            return float(t.group(1))
    except OSError:
        pass
    return None


def run_gpu(args):
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import pim

    rank, world = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    W = workload(args.workload)
    if args.corr_radius is not None:
        W.b = args.corr_radius
    fp64 = args.precision == "fp64"
    cdt = torch.complex128 if fp64 else torch.complex64
    plan = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=args.precision, b=W.b,
                    nf=W.nf, pf=W.pf, corr_mode=pim.PIM_CORR_FP64 if fp64 else pim.PIM_CORR_COMPACT)
    plan.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    info = plan.info()
    q = torch.tensor(W.q, dtype=cdt, device="cuda")
    u = torch.empty_like(q)
    w = torch.empty_like(q)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        pim.pim_apply(plan._h, q, u, 1, stream)
        pim.pim_apply_adjoint(plan._h, u, w, 1, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = plan.info().launches
    plan.set_profiling(True)
    clk = ClockSampler(local)
    times = []
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    stage_ms, napplies = plan.stage_times()
    plan.set_profiling(False)
    # accuracy of this configuration against the Ewald ground truth
    err_truth = None
    rows, ref = golden_rows()
    if rows is not None and args.workload == WORKLOAD:
        uu = u.cpu().numpy()[rows]
        err_truth = float(np.linalg.norm(uu - ref) / np.linalg.norm(ref))
    launches = plan.info().launches - launches0
    ms_step = allmax(float(np.mean(times)), world)
    value = replica_value(W.N, world, ms_step)

    # end to end through the C ABI with pinned host buffers (copies timed)
    qh = torch.tensor(W.q, dtype=cdt).pin_memory()
    uh = torch.empty_like(qh).pin_memory()
    wh = torch.empty_like(qh).pin_memory()
    for _ in range(2):
        pim.pim_apply(plan._h, qh, uh, 1, stream)
        pim.pim_apply_adjoint(plan._h, uh, wh, 1, stream)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        pim.pim_apply(plan._h, qh, uh, 1, stream)
        pim.pim_apply_adjoint(plan._h, uh, wh, 1, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = allmax(1e3 * float(np.mean(e2e_t)), world)
    e2e_val = 2.0 * W.N * world / (e2e_ms * 1e-3) / 1e6
    elem = 16 if fp64 else 8
    result = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        G = int(np.prod(W.n))
        nf3 = int(np.prod(W.nf))
        nbig = int(plan.debug(7).astype(np.int64).sum()) if int(info.corr_mode) == 3 else 0
        gb = gather_bytes(info, W.N, G, nf3, fp64, nbig)
        g_ms = stage_ms["gather_correct"] / max(1, napplies)
        achieved = gb / (g_ms * 1e-3) / 1e9
        apply_ms = stage_ms["apply"] / max(1, napplies)
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if fp64 else "c64+f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": W.N, "grid": list(W.n), "p": W.p, "near_layers": W.layers,
                       "corr_radius_steps": W.b, "far_grid": list(W.nf), "far_p": W.pf, "nnz": int(info.nnz),
                       "nnz_double_float": nbig if int(info.corr_mode) == 3 else None,
                       "precision": "FP64 throughout" if fp64 else
                                    "complex64 bulk, FP64 far series/grid sum, correction values computed "
                                    "in FP64; per row the entries above 2^-10 of its largest as FP32 head + "
                                    "bf16 tail summed in double-float, the rest complex64 summed in FP32 "
                                    "(every stored value within 2^-33 of the row's largest)",
                       "rel_l2_vs_ewald_ground_truth": err_truth,
                       "ground_truth_rows": 16,
                       "l2": "256 MB buffer written between timed steps", "parallelism": "replicas"},
            "roofline": {"bound": "hbm", "kernel": "gather_kernel (near gather + CSR correction)",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "traffic": None if fp64 else profile_traffic(), "algorithmic_bytes_per_launch": gb,
                         "kernel_ms": round(g_ms, 4)},
            "stages_ms_per_apply": {k: round(v / max(1, napplies), 4) for k, v in stage_ms.items()},
            "apply_ms": round(apply_ms, 4),
            "e2e": {"value": round(e2e_val, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * W.N * elem,
                    "d2h_bytes_per_step": 2 * W.N * elem},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
    plan.close()
    return rank, world, result


_ORACLE_TIMER = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import pim as opim
from paper_2312_02376_gb300 import inputs
W = inputs.helmholtz2d()
P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf, pf=W.pf)
t0 = time.perf_counter()
pl = opim.Plan(P, W.points)
tplan = time.perf_counter() - t0
q = W.q.astype(np.complex128)
t0 = time.perf_counter()
state = pl.rows_prepare(q)
tshared = time.perf_counter() - t0
rng = np.random.default_rng(0)
times = []
for i in range(%d):
    rows = rng.choice(W.N, %d, replace=False)
    t0 = time.perf_counter()
    pl.rows_from(state, rows)
    times.append(time.perf_counter() - t0)
print(json.dumps({"rows": %d, "seconds": times, "shared_seconds": tshared, "plan_seconds": tplan, "N": W.N}))
"""


def oracle_timer(nsteps, rows):
    """Runs the FP64 oracle, as it stands, in one single-threaded subprocess:
    its tables once (not timed), the part of an apply shared by all rows once
    (timed), then `nsteps` samples of `rows` sampled rows (timed each).
    Returns the parsed result, or None and the error text."""
    code = _ORACLE_TIMER % (ROOT, nsteps, rows, rows)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return None, r.stderr[-300:]
    return json.loads(r.stdout.strip().splitlines()[-1]), ""


def oracle_rate(d, per_row_seconds):
    """Mpts/s of a whole oracle apply of the workload: the shared part once
    plus N rows at the sampled per-row cost."""
    return d["N"] / (d["shared_seconds"] + d["N"] * per_row_seconds) / 1e6


def cpu_baseline(rows=8):
    """The oracle on a bounded sample of the same workload (forward apply),
    single-threaded: the shared part and `rows` sampled rows."""
    d, err = oracle_timer(1, rows)
    if d is None:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + err}
    t = d["seconds"][0]
    return {"value": oracle_rate(d, t / d["rows"]), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s forward apply: shared part (spreads, far grid sum) %.1f s once + %d sampled rows in "
                      "%.1f s, rate = N / (shared + N x per-row); oracle tables %.1f s not counted"
                      % (WORKLOAD, d["shared_seconds"], d["rows"], t, d["plan_seconds"])}


def run_reference(args):
    """The reference arm: there is no reference implementation, so the FP64
    oracle is timed on the host: per step one sampled row of the same
    workload, after the oracle's tables (not timed) and the part of the apply
    shared by all rows (timed once, counted in the rate)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d, err = oracle_timer(args.warmup + args.steps, 1)
    if d is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + err.replace("\n", " ")}))
        return
    ts = d["seconds"][args.warmup:]
    per_row = float(np.mean(ts))
    value = oracle_rate(d, per_row)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * per_row, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "per step: 1 sampled row of the forward apply (FP64 oracle, 1 thread); "
                                      "shared part %.1f s once; rate = N / (shared + N x mean row time); "
                                      "oracle tables %.1f s not timed" % (d["shared_seconds"], d["plan_seconds"])},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """16 point sets x 64 right-hand sides, one captured graph per direction."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import inputs, pim
    torch.cuda.set_device(0)
    sets = inputs.helmholtz1d_batch()
    plans, qs, us, ws = [], [], [], []
    t0 = time.perf_counter()
    for W in sets:
        pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision="fp32", b=W.b, pf=W.pf,
                      corr_mode=pim.PIM_CORR_COMPACT)
        pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
        plans.append(pl)
        qs.append(torch.tensor(W.q, device="cuda"))
        us.append(torch.empty_like(qs[-1]))
        ws.append(torch.empty_like(qs[-1]))
    t_plan = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    R = sets[0].nrhs

    def step():
        pim.pim_apply_batched(plans, qs, us, R, False, stream)
        pim.pim_apply_batched(plans, us, ws, R, True, stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    clk = ClockSampler(0)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = clk.stop()
    ms = float(np.mean(times))
    NT = sum(W.N for W in sets)
    nnz = sum(pl.info().nnz for pl in plans)
    out = {"metric": METRIC, "value": round(2.0 * NT * R / (ms * 1e-3) / 1e6, 3), "unit": "Mpts/s (x RHS)",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
           "data": "synthetic",
           "config": {"workload": "helmholtz1d_batch", "sets": len(sets), "N_total": NT, "nrhs": R,
                      "nnz_total": int(nnz), "corr_radius_steps": sets[0].b, "set_points_s": round(t_plan, 1),
                      "graph": "one captured graph per direction, replayed"},
           "clocks": clocks}
    for pl in plans:
        pl.close()
    return out


def run_coulomb_grad(args):
    """Differentiated 3D Coulomb, N = 1e6, 256^3, FP32 bulk: forward,
    adjoint and position gradient per step."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import inputs, pim
    torch.cuda.set_device(0)
    W = inputs.coulomb3d_big()
    t0 = time.perf_counter()
    pl = pim.Plan(W.D, W.pdims, 0.0, W.k0, W.n, p=W.p, layers=W.layers, precision="fp32", b=W.b, nf=W.nf,
                  pf=W.pf, corr_mode=pim.PIM_CORR_COMPACT, with_gradient=True)
    pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    t_plan = time.perf_counter() - t0
    q = torch.tensor(W.q, device="cuda")
    u = torch.empty_like(q)
    w = torch.empty_like(q)
    gx = torch.empty((W.N, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        pim.pim_apply(pl._h, q, u, 1, stream)
        pim.pim_apply_adjoint(pl._h, u, w, 1, stream)
        pim.pim_position_grad_reuse(pl._h, q, u, gx, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pl.set_profiling(True)
    clk = ClockSampler(0)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = clk.stop()
    stage_ms, nap = pl.stage_times()
    ms = float(np.mean(times))
    out = {"metric": METRIC, "value": round(2.0 * W.N / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "coulomb3d_1m", "N": W.N, "grid": list(W.n), "nnz": int(pl.info().nnz),
                      "corr_radius_steps": W.b,
                      "step": "forward + adjoint + position gradient (on the grid potentials the two applies kept)",
                      "set_points_s": round(t_plan, 1)},
           "stages_ms_per_apply": {k: round(v / max(1, nap), 4) for k, v in stage_ms.items()},
           "clocks": clocks}
    pl.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "helmholtz2d_65k", "helmholtz1d_batch", "coulomb3d_1m"],
                    help="helmholtz2d_65k: the same recipe, smaller, for profiler captures; "
                         "helmholtz1d_batch: 16 sets x 64 right-hand sides, batched graph; "
                         "coulomb3d_1m: forward + adjoint + position gradient")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp64: the plain FP64 apply of the same workload, for comparison with the FP32-bulk path")
    ap.add_argument("--corr-radius", type=int, default=None,
                    help="override the correction radius of the helmholtz2d workloads (for profiler captures "
                         "of the stages that do not depend on it; the line then states the radius used)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "helmholtz1d_batch":
        print(json.dumps(run_batch(args)))
        return
    if args.workload == "coulomb3d_1m":
        print(json.dumps(run_coulomb_grad(args)))
        return
    rank, world, result = run_gpu(args)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline()
        print(json.dumps(result))


if __name__ == "__main__":
    main()
