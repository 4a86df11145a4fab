"""Benchmark of the FFT-PIM apply on GB300 (one JSON line on rank 0).

Default workload (helmholtz3d_16m): 3D-periodic Helmholtz with a Bloch phase
shift, unit cube, k = 2 pi 2, k0 = (0.2k, 0.2k, 0), N = 1.6e7 points (3/4
uniform, 1/4 on 8 sphere surfaces of radius 0.05), complex64 sources CN(0, 1),
near grid 512^3, p = 4, correction radius 5 steps, far grid 20^3; FP32 bulk
(spread, FFT, gather, list-free exact and grid sums) with the far series and
far grid sum in FP64 and the stored correction values computed in FP64.  A
step is one forward apply plus one adjoint apply (every row of the hot path).
Metric: Mpts/s per apply (fwd+adjoint) = 2 N / t_step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Other workloads: helmholtz2d_262k (2D-periodic Helmholtz + Bloch, N = 262144,
128 x 128 x 64), helmholtz3d_4m and helmholtz2d_65k (the same recipes,
smaller, for profiler captures), helmholtz1d_batch (16 sets x 64 right-hand
sides, batched graph), coulomb3d_1m (forward + adjoint + position gradient).
--impl reference times the FP64 CPU oracle (test infrastructure, the
reference arm of this method) on a bounded sample of rows.  Multi-GPU: the
apply does not shard; N independent replicas (weak scaling).
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
WORKLOAD = "helmholtz3d_16m"
GOLDEN = {"helmholtz3d_16m": "helmholtz3d_16m_ewald_rows.txt", "helmholtz2d_262k": "helmholtz2d_262k_ewald_rows.txt"}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "gather_correct_helmholtz2d_262k.md")
# the oracle's sample for each workload: the workload itself where its rows
# take seconds, else the same recipe at a size whose near table fits the host
ORACLE_SAMPLE = {"helmholtz3d_16m": "helmholtz3d_250k", "helmholtz3d_4m": "helmholtz3d_250k",
                 "helmholtz2d_262k": "helmholtz2d_262k", "helmholtz2d_65k": "helmholtz2d_65k"}


def golden_rows(name):
    """(rows, values) of the committed Ewald ground truth of a workload, or
    (None, None)."""
    try:
        d = np.loadtxt(os.path.join(ROOT, "tests", "golden", GOLDEN[name]), comments="#")
        return d[:, 0].astype(np.int64), d[:, 1] + 1j * d[:, 2]
    except (OSError, KeyError):
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
    if name == "helmholtz3d_16m":
        return inputs.helmholtz3d()
    if name == "helmholtz3d_4m":    # the same recipe on 256^3: the same points per box on the spheres
        return inputs.helmholtz3d(N=4_000_000, n=256)
    if name == "helmholtz3d_spheres_1m":  # the sphere points alone on 256^3: the same points per sphere box
        return inputs.helmholtz3d(N=1_000_000, n=256, uniform=0.0)
    if name == "helmholtz3d_250k":  # the same recipe on 128^3
        return inputs.helmholtz3d(N=250_000, n=128)
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
CORR_MODES = {"fp64": 0, "double_float": 1, "fp32": 2, "compact": 3}
CORR_TEXT = {
    0: "stored correction values FP64, summed in FP64",
    1: "stored correction values FP64 split into two FP32 words per component, summed in double-float",
    2: "stored correction values rounded to complex64 after the FP64 cancellation, summed in FP32",
    3: "stored correction values computed in FP64, per row the entries above 2^-10 of its largest as FP32 "
       "head + bf16 tail summed in double-float, the rest complex64 summed in FP32",
}


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


def nextpow2(x):
    v = 1
    while v < x:
        v *= 2
    return v


def fft_geometry(W):
    """Padded FFT lengths (the next power of two >= 2 n - 1 per axis, every
    axis zero-padded) and the stored spectrum's extent (L/2 + 1 along the
    axes where the near kernel is even: open, or periodic without a phase
    shift; L otherwise)."""
    L = [nextpow2(2 * n - 1) for n in W.n]
    S = [L[d] // 2 + 1 if (d not in W.pdims or W.k0[d] == 0) else L[d] for d in range(3)]
    return L, S


def stage_bytes(W, info, fp64=False, nbig=0):
    """Algorithmic HBM bytes of one apply's main-stream stages (one right-hand
    side): what each stage must read and write at least once.
      permute         q in, permutation, sorted sources out
      spread          per point stencil start, local coordinates and sorted
                      source; the near grid written once (box moments, which
                      stay in L2, not counted)
      fft             the five passes: x (n0 n1 n2 in, L0 n1 n2 out), y (L0 n1 n2
                      in, L0 L1 n2 out), z with the spectrum (L0 L1 n2 in and
                      out, the stored spectrum in), inverse y and inverse x (the
                      mirror images of y and x)
      gather_correct  gather_bytes()"""
    c, r = (16, 8) if fp64 else (8, 4)
    N = W.N
    G = int(np.prod(W.n))
    (L0, L1, _), S = fft_geometry(W)
    n0, n1, n2 = W.n
    xb = (n0 * n1 * n2 + L0 * n1 * n2) * c
    yb = (L0 * n1 * n2 + L0 * L1 * n2) * c
    zb = (2 * L0 * L1 * n2 + int(np.prod(S))) * c
    return {"permute": N * (2 * c + 4), "spread": N * (4 + 3 * r + c) + G * c, "fft": 2 * xb + 2 * yb + zb,
            "gather_correct": gather_bytes(info, N, G, int(np.prod(W.nf)), fp64, nbig)}


def hbm_table(W, info, per, peak, fp64=False, nbig=0):
    """Per stage and for the whole apply: algorithmic bytes over the CUDA-event
    time, as a fraction of the measured HBM peak.  The whole-apply figure
    divides the main-stream stages' bytes by the apply's duration (every
    stage included, the list-free ones and the far part's join too)."""
    sb = stage_bytes(W, info, fp64, nbig)
    out = {}
    for k, b in sb.items():
        ms = per.get(k, 0.0)
        if ms > 0:
            out[k] = {"bytes": int(b), "ms": round(ms, 4), "GBs": round(b / (ms * 1e-3) / 1e9, 1),
                      "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}
    tot = sum(sb.values())
    ams = per.get("apply", 0.0)
    if ams > 0:
        out["whole_apply"] = {"bytes": int(tot), "ms": round(ams, 4), "GBs": round(tot / (ams * 1e-3) / 1e9, 1),
                              "frac": round(tot / (ams * 1e-3) / 1e9 / peak, 4)}
    return out


def library_fft_alone_ms(W, fp64, reps=10):
    """The library's FFT stage (five pruned passes and the spectrum) on its
    own: a plan with the workload's grids and 1000 uniform points (no
    list-free boxes, so nothing runs beside it), CUDA-event stage timers."""
    import torch
    from paper_2312_02376_gb300 import pim
    prec = "fp64" if fp64 else "fp32"
    pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=prec, b=W.b, nf=W.nf, pf=W.pf)
    rng = np.random.default_rng(5)
    pl.set_points(torch.tensor(rng.random((1000, 3)) * np.asarray(W.D), dtype=torch.float64, device="cuda"))
    q = torch.tensor(rng.standard_normal(1000) + 1j * rng.standard_normal(1000),
                     dtype=torch.complex128 if fp64 else torch.complex64, device="cuda")
    for _ in range(3):
        pl.apply(q)
    torch.cuda.synchronize()
    pl.set_profiling(True)
    for _ in range(reps):
        pl.apply(q)
    st, n = pl.stage_times()
    pl.set_profiling(False)
    pl.close()
    return st["fft"] / max(1, n)


def cufft_comparison(W, fp64, ours_fft_ms, reps=10):
    """cuFFT (torch.fft) on the same padded grid: forward 3D transform, the
    product with a stored spectrum of the full padded size, inverse 3D
    transform, timed with CUDA events on the current stream.  cuFFT
    transforms every padded line (no pruning of the zero half on input or of
    the discarded half on output), so this is the unpruned convolution the
    library's five passes replace."""
    import torch
    L, _ = fft_geometry(W)
    dt = torch.complex128 if fp64 else torch.complex64
    shape = (L[2], L[1], L[0])
    x = torch.zeros(shape, dtype=dt, device="cuda")
    x[: W.n[2], : W.n[1], : W.n[0]] = 1.0
    spec = torch.ones(shape, dtype=dt, device="cuda")
    ts = []
    for it in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        y = torch.fft.ifftn(torch.fft.fftn(x) * spec)
        e1.record()
        e1.synchronize()
        if it >= 2:
            ts.append(e0.elapsed_time(e1))
    del x, spec, y
    torch.cuda.empty_cache()
    ms = float(np.mean(ts))
    alone = library_fft_alone_ms(W, fp64)
    return {"padded_grid": [L[0], L[1], L[2]], "cufft_fwd_mul_inv_ms": round(ms, 4),
            "library_fft_alone_ms": round(alone, 4), "speedup": round(ms / alone, 2),
            "library_fft_stage_in_apply_ms": round(ours_fft_ms, 4),
            "note": "torch.fft.fftn / ifftn (cuFFT), unpruned, against the library's FFT stage alone (same grids, "
                    "1000 points); in the timed apply other streams run beside the FFT stage; both timed after "
                    "the bench's timed region"}


# algorithmic FP32 operations of one exact-kernel pair (list-free boxes): the
# difference vector (3), its square norm (5), 1/r (1), the cos and sinc
# polynomials in r^2 (2 x 2 (NT - 1)), their product with 1/r (1) and the
# complex multiply-add with the source (8)
def lf_pair_flops(nterm):
    return 18 + 4 * (nterm - 1)


def lf_nterm(W):
    """Terms of the exact kernel's polynomials, chosen as the library does
    for the region's largest k r (truncation below 1.5e-8)."""
    R = W.b + 1
    h = np.asarray(W.D, np.float64) / (np.asarray(W.n) - 1)
    x = W.k * np.sqrt(np.sum(((R + 1) * h) ** 2))
    term = 1.0
    for t in range(1, 9):
        term *= x * x / ((2.0 * t - 1.0) * (2.0 * t))
        if term < 1.5e-8:
            return max(t, 2)
    return 0


def tc_roofline(W, info, ms):
    """The list-free grid part's matrix product on the tensor cores: executed
    TF32 operations per launch (three products, hi.hi + hi.lo + lo.hi, of the
    256 x 2 KP operator by 2 KP x boxes: 6 x 256 x 2 KP per box; KP = E^3
    padded to 32, E = 2 (b + 1) + 2 floor(p/2) + p + 1) against the TF32 peak
    derived from the measured sustained bf16 GEMM rate x the nominal
    TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s); also the useful complex work
    (125 x E^3 complex multiply-adds, 8 operations each, per box)."""
    E = 2 * (W.b + 1) + 2 * (W.p // 2) + W.p + 1
    KP = (E ** 3 + 31) // 32 * 32
    boxes = int(info.lf_tc_boxes)
    fl = 6.0 * 256 * 2 * KP * boxes
    useful = 8.0 * (W.p + 1) ** 3 * E ** 3 * boxes
    pk = measured_peaks_all()
    peak = pk.get("bf16_tflops_sustained", 1700.0) * 1.1 / 2.25
    ach = fl / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "lf_tc_gemm_kernel (list-free grid part: tcgen05 kind::tf32, 3 TF32 products "
                                        "per FP32 product)",
            "achieved": round(ach, 1), "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "peak_kind": "measured sustained bf16 x 1.1/2.25 (nominal TF32 / bf16)", "traffic": None,
            "executed_flops_per_launch": fl, "useful_complex_flops_per_launch": useful, "boxes": boxes,
            "kernel_ms": round(ms, 4)}


def measured_peaks_all():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def fp32_alu_peak():
    """FP32 FLOP/s of the chip's CUDA cores: 152 SMs x 128 FP32 lanes x 2 (FMA)
    x the maximum SM clock (2070 MHz)."""
    return 152 * 128 * 2 * 2.070e9


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
    cmode = pim.PIM_CORR_FP64 if fp64 else CORR_MODES[args.corr_mode or "compact"]
    plan = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=args.precision, b=W.b,
                    nf=W.nf, pf=W.pf, corr_mode=cmode, listfree=args.listfree)
    t0 = time.perf_counter()
    plan.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    t_points = time.perf_counter() - t0
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
    # accuracy of this configuration against the Ewald ground truth (the
    # forward apply of the last step)
    err_truth = None
    rows, ref = golden_rows(args.workload)
    if rows is not None and args.corr_radius is None:
        pim.pim_apply(plan._h, q, u, 1, stream)
        torch.cuda.synchronize()
        uu = u[torch.tensor(rows, device="cuda")].cpu().numpy()
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
        per = {k: v / max(1, napplies) for k, v in stage_ms.items()}
        gb = gather_bytes(info, W.N, G, nf3, fp64, nbig)
        g_ms = per["gather_correct"]
        hbm = {"bound": "hbm", "kernel": "gather_kernel (near gather + stored-list correction)",
               "achieved": round(gb / (g_ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
               "frac": round(gb / (g_ms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
               "traffic": None if fp64 or args.workload != "helmholtz2d_262k" or int(info.corr_mode) != 3
               else profile_traffic(),
               "algorithmic_bytes_per_launch": gb, "kernel_ms": round(g_ms, 4)}
        rooflines = [hbm]
        if info.lf_pairs > 0 and not fp64:
            nt = lf_nterm(W)
            fl = info.lf_pairs * lf_pair_flops(nt if nt else 8)
            x_ms = per["lf_exact"]
            apk = fp32_alu_peak()
            rooflines.append({"bound": "alu", "kernel": "lf_exact_f32 (list-free boxes: exact kernel over the "
                                                        "region's dense boxes)",
                              "achieved": round(fl / (x_ms * 1e-3) / 1e12, 2), "peak": round(apk / 1e12, 1),
                              "unit": "TFLOP/s", "frac": round(fl / (x_ms * 1e-3) / apk, 4),
                              "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz",
                              "traffic": None, "algorithmic_flops_per_launch": fl,
                              "pairs_per_launch": int(info.lf_pairs), "flops_per_pair": lf_pair_flops(nt if nt else 8),
                              "kernel_ms": round(x_ms, 4)})
        if int(getattr(info, "lf_tc_boxes", 0)) > 0 and per.get("lf_tc_gemm", 0) > 0:
            rooflines.append(tc_roofline(W, info, per["lf_tc_gemm"]))
        # the dominant kernel of the modelled ones first
        rooflines.sort(key=lambda r: -r["kernel_ms"])
        apply_ms = per["apply"]
        stages_hbm = hbm_table(W, info, per, peak, fp64, nbig)
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if fp64 else "c64+f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": W.N, "grid": list(W.n), "p": W.p, "near_layers": W.layers,
                       "corr_radius_steps": W.b, "far_grid": list(W.nf), "far_p": W.pf, "nnz_stored": int(info.nnz),
                       "nnz_double_float": nbig if int(info.corr_mode) == 3 else None,
                       "listfree_boxes": int(info.lf_boxes), "listfree_points": int(info.lf_points),
                       "listfree_pairs": int(info.lf_pairs),
                       "precision": "FP64 throughout" if fp64 else
                                    "complex64 bulk (spread, FFT, gather, list-free exact and grid sums in FP32), "
                                    "FP64 far series and far grid sum; " + CORR_TEXT[int(info.corr_mode)],
                       "corr_mode": [k for k, v in CORR_MODES.items() if v == int(info.corr_mode)][0],
                       "rel_l2_vs_ewald_ground_truth": err_truth,
                       "ground_truth_rows": None if rows is None else int(len(rows)),
                       "set_points_s": round(t_points, 1),
                       "l2": "inputs larger than L2; a 256 MB buffer is also written between timed steps",
                       "parallelism": "replicas"},
            "roofline": rooflines[0],
            "roofline_other": rooflines[1:],
            "stages_ms_per_apply": {k: round(v, 4) for k, v in per.items()},
            "stages_hbm_per_apply": stages_hbm,
            "apply_ms": round(apply_ms, 4),
            "e2e": {"value": round(e2e_val, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * W.N * elem,
                    "d2h_bytes_per_step": 2 * W.N * elem},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
    plan.close()
    if rank == 0 and args.cufft:
        result["cufft_comparison"] = cufft_comparison(W, fp64, per["fft"])
    return rank, world, result


_ORACLE_TIMER = r"""
import os, sys, time, json
import multiprocessing as mp
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import pim as opim
import bench
W = bench.workload(%(name)r)
P = opim.Params(D=W.D, pdims=W.pdims, k=W.k, k0=W.k0, n=W.n, p=W.p, layers=W.layers, b=W.b, nf=W.nf, pf=W.pf)
t0 = time.perf_counter()
pl = opim.Plan(P, W.points)
tplan = time.perf_counter() - t0
q = W.q.astype(np.complex128)
t0 = time.perf_counter()
state = pl.rows_prepare(q)
tshared = time.perf_counter() - t0
rng = np.random.default_rng(0)
cores = %(cores)d
def rows_time(rows):
    t0 = time.perf_counter()
    pl.rows_from(state, rows)
    return time.perf_counter() - t0
times = []
# no GPU in this process: the pool may fork
with mp.get_context("fork").Pool(cores) as pool:
    for i in range(%(nsteps)d):
        rows = rng.choice(W.N, %(rows)d * cores, replace=False)
        t0 = time.perf_counter()
        pool.map(rows_time, [rows[c::cores] for c in range(cores)])
        times.append(time.perf_counter() - t0)
print(json.dumps({"rows": %(rows)d * cores, "seconds": times, "shared_seconds": tshared, "plan_seconds": tplan,
                  "N": W.N, "cores": cores, "name": %(name)r}))
"""


def oracle_timer(name, nsteps, rows_per_core, cores):
    """Runs the FP64 oracle, as it stands, in a subprocess without a GPU: its
    tables once (not timed), the part of an apply shared by all rows once
    (timed, one core), then `nsteps` samples of rows_per_core sampled rows on
    each of `cores` worker processes (wall time of each sample).  Returns the
    parsed result, or None and the error text."""
    code = _ORACLE_TIMER % {"root": ROOT, "name": name, "nsteps": nsteps, "rows": rows_per_core, "cores": cores}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        return None, r.stderr[-300:]
    return json.loads(r.stdout.strip().splitlines()[-1]), ""


def oracle_rate(d, sample_seconds):
    """Mpts/s of a whole oracle apply of the sampled workload: the shared part
    once plus N rows at the sampled rate (rows done in parallel)."""
    return d["N"] / (d["shared_seconds"] + d["N"] * sample_seconds / d["rows"]) / 1e6


def cpu_baseline(name, rows_per_core=2):
    """The oracle on a bounded sample, on all host cores (forward apply)."""
    cores = os.cpu_count() or 1
    sample = ORACLE_SAMPLE.get(name, name)
    d, err = oracle_timer(sample, 1, rows_per_core, cores)
    if d is None:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": "failed: " + err}
    t = d["seconds"][0]
    return {"value": oracle_rate(d, t), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s forward apply (the oracle's sample of %s): shared part (spreads, far grid sum) %.1f s "
                      "once on one core + %d sampled rows in %.1f s on %d processes, rate = N / (shared + N x "
                      "row time); oracle tables %.1f s not counted"
                      % (sample, name, d["shared_seconds"], d["rows"], t, cores, d["plan_seconds"])}


def run_reference(args):
    """The reference arm: there is no reference implementation, so the FP64
    oracle is timed on the host cores: per step a sample of rows of the
    workload (or, where its rows take minutes, of the same recipe at a
    smaller size), after the oracle's tables (not timed) and the part of the
    apply shared by all rows (timed once, counted in the rate)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample = ORACLE_SAMPLE.get(args.workload, args.workload)
    d, err = oracle_timer(sample, args.warmup + args.steps, 1, cores)
    if d is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + err.replace("\n", " ")}))
        return
    ts = d["seconds"][args.warmup:]
    per_sample = float(np.mean(ts))
    value = oracle_rate(d, per_sample)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * per_sample, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "oracle_sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "per step: %d sampled rows of the %s forward apply (FP64 oracle, one row per "
                                      "process); shared part %.1f s once; rate = N / (shared + N x row time); "
                                      "oracle tables %.1f s not timed"
                                      % (d["rows"], sample, d["shared_seconds"], d["plan_seconds"])},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def corr_multi_bytes(info, N, nrhs, fp64=False, nbig=0):
    """Algorithmic bytes of one multi-RHS correction launch: the list once
    (value and column per entry, the bf16 tails of the double-float entries),
    per point its row pointer, row split and permutation; the sorted sources
    of all right-hand sides read once and the output read and written once."""
    c = 16 if fp64 else 8
    per_nnz = VALUE_BYTES[int(info.corr_mode)] + 4
    return info.nnz * per_nnz + 4 * nbig + (N + 1) * 8 + N * 8 + 3 * N * nrhs * c


def run_batch(args):
    """16 point sets x 64 right-hand sides, one captured graph per direction.
    --precision fp64: the plain FP64 apply of the same sets (FP64 plans and
    correction values, each set applied in turn through pim_apply, no graph)."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import inputs, pim
    torch.cuda.set_device(0)
    fp64 = args.precision == "fp64"
    sets = inputs.helmholtz1d_batch()
    plans, qs, us, ws = [], [], [], []
    t0 = time.perf_counter()
    for W in sets:
        pl = pim.Plan(W.D, W.pdims, W.k, W.k0, W.n, p=W.p, layers=W.layers, precision=args.precision, b=W.b,
                      nf=W.nf, pf=W.pf, corr_mode=pim.PIM_CORR_FP64 if fp64 else pim.PIM_CORR_COMPACT)
        pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
        plans.append(pl)
        qs.append(torch.tensor(W.q, dtype=torch.complex128 if fp64 else torch.complex64, device="cuda"))
        us.append(torch.empty_like(qs[-1]))
        ws.append(torch.empty_like(qs[-1]))
    t_plan = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    R = sets[0].nrhs

    def step():
        if fp64:
            for pl, q, u, w in zip(plans, qs, us, ws):
                pim.pim_apply(pl._h, q, u, R, stream)
            for pl, q, u, w in zip(plans, qs, us, ws):
                pim.pim_apply_adjoint(pl._h, u, w, R, stream)
        else:
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

    # kernels per step: the graph replays the launches of one direct forward
    # and one direct adjoint call per set (the same capture), counted by the plans
    l0 = sum(pl.info().launches for pl in plans)
    with torch.cuda.stream(stream):
        for pl, q, u, w in zip(plans, qs, us, ws):
            pim.pim_apply(pl._h, q, u, R, stream)
            pim.pim_apply_adjoint(pl._h, u, w, R, stream)
    stream.synchronize()
    launches = sum(pl.info().launches for pl in plans) - l0

    # stage times of direct calls (one forward and one adjoint per set), for
    # the multi-RHS correction's roofline and the per-RHS near paths' share
    peak, peak_kind = measured_peaks()
    stage_tot = {}
    corr_bytes = 0
    for pl, q, u, w, W in zip(plans, qs, us, ws, sets):
        pl.set_profiling(True)
        pim.pim_apply(pl._h, q, u, R, stream)
        pim.pim_apply_adjoint(pl._h, u, w, R, stream)
        st, _ = pl.stage_times()
        pl.set_profiling(False)
        for k, v in st.items():
            stage_tot[k] = stage_tot.get(k, 0.0) + v
        info = pl.info()
        nbig = int(pl.debug(7).astype(np.int64).sum()) if int(info.corr_mode) == 3 else 0
        corr_bytes += 2 * corr_multi_bytes(info, W.N, R, fp64, nbig)
    cm_ms = stage_tot.get("corr_multi", 0.0)
    roofline = {"bound": "hbm", "kernel": "corr_multi_kernel (stored-list correction of all 64 right-hand sides, "
                                          "one launch per set and direction)",
                "achieved": round(corr_bytes / (cm_ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                "frac": round(corr_bytes / (cm_ms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
                "traffic": None, "algorithmic_bytes_per_step": int(corr_bytes), "kernel_ms_per_step": round(cm_ms, 3),
                "note": "launches timed with CUDA events in direct (ungraphed) calls of the same plans"}

    # end to end: every set's sources copied in from pinned host memory, both
    # graphs, the adjoint's output copied back, inside the timed region
    qh = [q.cpu().pin_memory() for q in qs]
    wh = [torch.empty_like(h).pin_memory() for h in qh]

    def e2e_step():
        with torch.cuda.stream(stream):
            for h, q in zip(qh, qs):
                q.copy_(h, non_blocking=True)
        step()
        with torch.cuda.stream(stream):
            for h, w in zip(wh, ws):
                h.copy_(w, non_blocking=True)
        stream.synchronize()

    e2e_step()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    io_bytes = sum(h.numel() * h.element_size() for h in qh)
    unit = "Mpts/s (x RHS)"
    out = {"metric": METRIC, "value": round(2.0 * NT * R / (ms * 1e-3) / 1e6, 3), "unit": unit,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "c128" if fp64 else "c64+f64", "data": "synthetic",
           "config": {"workload": "helmholtz1d_batch", "sets": len(sets), "N_total": NT, "nrhs": R,
                      "nnz_total": int(nnz), "corr_radius_steps": sets[0].b, "far_grid": list(sets[0].nf),
                      "set_points_s": round(t_plan, 1),
                      "form": ("plain FP64: FP64 plans and correction values, pim_apply per set, no graph" if fp64
                               else "FP32 bulk, compact correction rows; one captured graph per direction, "
                                    "replayed"),
                      "l2": "inputs larger than L2 (64 right-hand sides of 1.6e6 points, 0.8 GB per direction)"},
           "roofline": roofline,
           "stage_ms_per_step_direct": {k: round(v, 3) for k, v in stage_tot.items()},
           "e2e": {"value": round(2.0 * NT * R / (e2e_ms * 1e-3) / 1e6, 3), "unit": unit,
                   "h2d_bytes_per_step": int(io_bytes), "d2h_bytes_per_step": int(io_bytes)},
           "gpu_launches": int(launches) * args.steps,
           "clocks": clocks}
    for pl in plans:
        pl.close()
    return out


def grad_bytes(info, N, G, fp64=False, nbig=0):
    """Algorithmic bytes of one position-gradient launch on the kept grid
    potentials: per entry the column and the three derivative values (FP64
    or double-float: 48 B; compact rows: the 24 B of FP32 heads, 24 B more for
    the leading entries summed in double-float); per point the stencil start,
    local coordinates, permutation, q, g and the FP64 gradient out; the near
    grid potentials of q and g once (the far ones are small)."""
    c, r = (16, 8) if fp64 else (8, 4)
    compact = int(info.corr_mode) == 3
    per_nnz = 4 + (24 if compact else 48)
    return info.nnz * per_nnz + 24 * nbig + (N + 1) * 8 + N * (4 + 3 * r + 4 + 2 * c + 24) + 2 * G * c


def run_coulomb_grad(args):
    """Differentiated 3D Coulomb, N = 1e6, 256^3, FP32 bulk: forward,
    adjoint and position gradient per step (the gradient on the grid
    potentials the two applies kept).  --precision fp64: the plain FP64
    form (FP64 plan and values; the full pim_position_grad, which recomputes
    both grid potentials)."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import inputs, pim
    torch.cuda.set_device(0)
    fp64 = args.precision == "fp64"
    W = inputs.coulomb3d_big()
    t0 = time.perf_counter()
    pl = pim.Plan(W.D, W.pdims, 0.0, W.k0, W.n, p=W.p, layers=W.layers, precision=args.precision, b=W.b, nf=W.nf,
                  pf=W.pf, corr_mode=pim.PIM_CORR_FP64 if fp64 else pim.PIM_CORR_COMPACT, with_gradient=True)
    pl.set_points(torch.tensor(W.points, dtype=torch.float64, device="cuda"))
    t_plan = time.perf_counter() - t0
    rdt = torch.float64 if fp64 else torch.float32
    q = torch.tensor(W.q, dtype=rdt, device="cuda")
    u = torch.empty_like(q)
    w = torch.empty_like(q)
    gx = torch.empty((W.N, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    gev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
    gms = []

    def step(timed_grad=False):
        pim.pim_apply(pl._h, q, u, 1, stream)
        pim.pim_apply_adjoint(pl._h, u, w, 1, stream)
        if timed_grad:
            gev[0].record(stream)
        if fp64:
            pim.pim_position_grad(pl._h, q, u, gx, 1, stream)
        else:
            pim.pim_position_grad_reuse(pl._h, q, u, gx, stream)
        if timed_grad:
            gev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = pl.info().launches
    pl.set_profiling(True)
    clk = ClockSampler(0)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(timed_grad=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        gms.append(gev[0].elapsed_time(gev[1]))
    clocks = clk.stop()
    stage_ms, nap = pl.stage_times()
    pl.set_profiling(False)
    launches = pl.info().launches - launches0
    ms = float(np.mean(times))
    info = pl.info()
    per = {k: v / max(1, nap) for k, v in stage_ms.items()}
    peak, peak_kind = measured_peaks()
    nbig = int(pl.debug(7).astype(np.int64).sum()) if int(info.corr_mode) == 3 else 0
    G = int(np.prod(W.n))
    gb = gather_bytes(info, W.N, G, int(np.prod(W.nf)), fp64, nbig)
    grb = grad_bytes(info, W.N, G, fp64, nbig)
    g_ms = float(np.mean(gms))
    rooflines = [
        {"bound": "hbm", "kernel": "gather_kernel (near gather + stored-list correction), per apply",
         "achieved": round(gb / (per["gather_correct"] * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
         "frac": round(gb / (per["gather_correct"] * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
         "traffic": None, "algorithmic_bytes_per_launch": int(gb), "kernel_ms": round(per["gather_correct"], 4)},
        {"bound": "hbm", "kernel": ("position gradient, full (recomputes both grid potentials)" if fp64 else
                                    "grad_kernel (position gradient on the kept grid potentials)"),
         "achieved": round(grb / (g_ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
         "frac": round(grb / (g_ms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind, "traffic": None,
         "algorithmic_bytes_per_launch": int(grb), "kernel_ms": round(g_ms, 4)}]
    rooflines.sort(key=lambda r: -r["kernel_ms"])

    # end to end: q in from pinned host memory, the step, u and the gradient out
    qh = q.cpu().pin_memory()
    uh = torch.empty_like(qh).pin_memory()
    gh = torch.empty((W.N, 3), dtype=torch.float64).pin_memory()

    def e2e_step():
        q.copy_(qh, non_blocking=True)
        step()
        uh.copy_(u, non_blocking=True)
        gh.copy_(gx, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    rb = q.element_size()
    out = {"metric": METRIC, "value": round(2.0 * W.N / (ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32+f64", "data": "synthetic",
           "config": {"workload": "coulomb3d_1m", "N": W.N, "grid": list(W.n), "nnz": int(info.nnz),
                      "corr_radius_steps": W.b,
                      "step": ("forward + adjoint + full position gradient (plain FP64)" if fp64 else
                               "forward + adjoint + position gradient (on the grid potentials the two applies "
                               "kept)"),
                      "set_points_s": round(t_plan, 1),
                      "l2": "inputs, list and grids larger than L2"},
           "roofline": rooflines[0], "roofline_other": rooflines[1:],
           "stages_ms_per_apply": {k: round(v, 4) for k, v in per.items()},
           "grad_ms": round(g_ms, 4),
           "e2e": {"value": round(2.0 * W.N / (e2e_ms * 1e-3) / 1e6, 3), "unit": UNIT,
                   "h2d_bytes_per_step": W.N * rb, "d2h_bytes_per_step": W.N * rb + W.N * 24},
           "gpu_launches": int(launches),
           "clocks": clocks}
    pl.close()
    return out


TIMING_WORKLOADS = ("coulomb3d_4k", "helmholtz2d_262k", "helmholtz1d_batch", "coulomb3d_1m", "helmholtz3d_16m")


def timing_sets(name):
    """The point sets of a workload for the timing report, and whether its
    plans store the position derivatives (the differentiated 3D Coulomb)."""
    from paper_2312_02376_gb300 import inputs
    if name == "coulomb3d_4k":
        return [inputs.coulomb3d()], False
    if name == "helmholtz1d_batch":
        return inputs.helmholtz1d_batch(), False
    if name == "coulomb3d_1m":
        return [inputs.coulomb3d_big()], True
    return [workload(name)], False


def run_timing_report(args):
    """Pre-processing against execution, and the cost of periodicity (the
    paper's Sec. 4.2 comparison), for each workload named in
    --timing-workloads: the wall time of pim_plan_create and pim_set_points
    and the CUDA-event time of a forward and an adjoint apply (all right-hand
    sides; summed over the point sets of the batched workload, applied one
    set at a time); then the same points and grid with no periodic axis and
    no phase shift (no far zone, one image), the apply's time and the
    periodic overhead t_periodic / t_open - 1.  Each workload in its own
    precision (FP64 for the 4096-point Coulomb set); real data where k and
    k0 vanish."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import pim
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    names = [x for x in args.timing_workloads.split(",") if x]
    rows = []
    for name in names:
        sets, grad = timing_sets(name)
        res = {"workload": name, "N": int(sum(W.N for W in sets)), "sets": len(sets), "nrhs": sets[0].nrhs,
               "precision": sets[0].precision, "grid": list(sets[0].n) if len(sets) == 1 else None}
        try:
            for label in ("periodic", "open"):
                tot = {"plan_create_s": 0.0, "plan_ms_library": 0.0, "set_points_s": 0.0, "points_ms_library": 0.0,
                       "apply_fwd_adj_ms": 0.0, "nnz": 0, "listfree_pairs": 0}
                for W in sets:
                    pdims, k0 = (W.pdims, W.k0) if label == "periodic" else ((), (0.0, 0.0, 0.0))
                    fp64 = W.precision == "fp64"
                    real = W.k == 0 and not any(k0)
                    t0 = time.perf_counter()
                    pl = pim.Plan(W.D, pdims, W.k, k0, W.n, p=W.p, layers=W.layers, precision=W.precision, b=W.b,
                                  nf=W.nf if pdims else None, pf=W.pf,
                                  corr_mode=pim.PIM_CORR_FP64 if fp64 else pim.PIM_CORR_COMPACT, with_gradient=grad)
                    torch.cuda.synchronize()
                    t_create = time.perf_counter() - t0
                    xyz = torch.tensor(W.points, dtype=torch.float64, device="cuda")
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    pl.set_points(xyz)
                    torch.cuda.synchronize()
                    t_points = time.perf_counter() - t0
                    if real:
                        q = torch.tensor(np.real(W.q), dtype=torch.float64 if fp64 else torch.float32, device="cuda")
                    else:
                        q = torch.tensor(W.q, dtype=torch.complex128 if fp64 else torch.complex64, device="cuda")
                    R = 1 if q.dim() == 1 else int(q.shape[1])
                    u = torch.empty_like(q)
                    w = torch.empty_like(q)
                    for _ in range(3):
                        pim.pim_apply(pl._h, q, u, R, stream)
                        pim.pim_apply_adjoint(pl._h, u, w, R, stream)
                    ts = []
                    for _ in range(max(3, args.steps)):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        pim.pim_apply(pl._h, q, u, R, stream)
                        pim.pim_apply_adjoint(pl._h, u, w, R, stream)
                        e1.record(stream)
                        e1.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    if pl.device_status() != pim.PIM_OK:
                        raise RuntimeError("device status %d" % pl.device_status())
                    info = pl.info()
                    tot["plan_create_s"] += t_create
                    tot["plan_ms_library"] += info.plan_ms
                    tot["set_points_s"] += t_points
                    tot["points_ms_library"] += info.points_ms
                    tot["apply_fwd_adj_ms"] += float(np.mean(ts))
                    tot["nnz"] += int(info.nnz)
                    tot["listfree_pairs"] += int(info.lf_pairs)
                    pl.close()
                    del xyz, q, u, w
                    torch.cuda.empty_cache()
                res[label] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in tot.items()}
            res["periodic_overhead"] = round(res["periodic"]["apply_fwd_adj_ms"] / res["open"]["apply_fwd_adj_ms"] - 1,
                                             4)
        except Exception as e:  # one workload's failure is reported in its row; the others still run
            res["error"] = "%s: %s" % (type(e).__name__, e)
            torch.cuda.empty_cache()
        rows.append(res)
    return {"report": "pre-processing vs execution; periodic vs open", "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "helmholtz3d_4m", "helmholtz3d_spheres_1m", "helmholtz3d_250k", "helmholtz2d_262k",
                             "helmholtz2d_65k",
                             "helmholtz1d_batch", "coulomb3d_1m"],
                    help="helmholtz3d_4m / _250k, helmholtz2d_65k: the same recipes, smaller, for profiler "
                         "captures; helmholtz3d_spheres_1m: the sphere points alone on 256^3 (list-free kernel "
                         "captures); helmholtz1d_batch: 16 sets x 64 right-hand sides, batched graph; "
                         "coulomb3d_1m: forward + adjoint + position gradient")
    ap.add_argument("--listfree", type=int, default=None,
                    help="pim_options.corr_listfree (default: the library's; 0 stores every correction)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp64: the plain FP64 apply of the same workload, for comparison with the FP32-bulk path")
    ap.add_argument("--cufft", action="store_true",
                    help="also time cuFFT (torch.fft) on the same padded grid after the timed region")
    ap.add_argument("--report", default=None, choices=["timing"],
                    help="timing: plan and set-points times beside the apply, and the periodic overhead, "
                         "for the workloads of --timing-workloads; prints its own JSON line")
    ap.add_argument("--timing-workloads", default=",".join(TIMING_WORKLOADS),
                    help="comma-separated workloads of --report timing (default: all five)")
    ap.add_argument("--corr-mode", default=None, choices=list(CORR_MODES),
                    help="pim_corr_mode of the FP32 plan's stored correction values (default compact); fp64, "
                         "double_float and fp32 for comparison with the default")
    ap.add_argument("--corr-radius", type=int, default=None,
                    help="override the correction radius of the helmholtz2d workloads (for profiler captures "
                         "of the stages that do not depend on it; the line then states the radius used)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.report == "timing":
        print(json.dumps(run_timing_report(args)))
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
            result["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(result))


if __name__ == "__main__":
    main()
