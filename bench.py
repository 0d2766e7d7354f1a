#!/usr/bin/env python3
"""Benchmark: non-uniform points/s of one NU-ASM_2 solve on GB300.

Workload (synthetic, seeded): uniform 1024 x 1024 source at 8 um holding a
binary-amplitude random-phase pattern, zero-padded to 2048^2; 1,048,576
destination points whose local pitch grades from 4 um at the centre to 16 um
at the edge (radial warp, +-0.3 local-pitch jitter); lambda = 532 nm,
z = 20 cm, off-axis offset (1 mm, 0); complex64 data with FP64-derived phase.

A step is one full solve (column FFT, fused row pass with deconvolution and
transfer function, folded column inverse FFT, tile interpolation) on inputs
already resident in HBM.  L2 (129 MB) is flushed by writing a 256 MB buffer
before every step; each step is timed with CUDA events on the solve's stream
and `value` = points x steps / summed step time (max over ranks).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (weak scaling,
no data-path collective).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "non-uniform points/s per NUASM solve at rel-L2≤1e-5 vs FP64; served p50/p99"
UNIT = "points/s"
WORKLOAD = "nuasm2_graded_n1024_m1048576_lambda532nm_z20cm_o1mm"
CPU_SAMPLE_POINTS = 16384
FLUSH_BYTES = 256 << 20
E2E_LANES = 3   # plans rotating in the pipelined end-to-end measurement
L2_BYTES = 129e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload():
    from paper_1308_6644_gb300 import workloads as WL
    return WL.nuasm2_graded(seed=1002, n=1024, pitch=8e-6)


def reduce_over_ranks(total_ms: float, points: float, device) -> tuple[float, float]:
    """Replicas only: the job time is the slowest rank's time (MAX) and the job
    processed every rank's points (SUM).  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, points
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([points], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="nuasm_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            self._discard()

    def _discard(self):
        try:
            self.fh.close()
        except Exception:
            pass
        if self.path and os.path.exists(self.path):
            os.remove(self.path)

    def stop(self) -> dict | None:
        if self.proc is None:
            self._discard()
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [s.strip() for s in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.remove(self.path)
        note = None
        if not sm:
            # timed region shorter than the sampling interval: one query right at its end
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=10).stdout
                f = [s.strip() for s in out.split(",")]
                sm, smax = [float(f[1])], [float(f[2])]
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
                note = "one sample at the end of the timed region (shorter than the 100 ms interval)"
            except Exception:
                return None
        rec = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
               "samples": len(sm)}
        if note:
            rec["note"] = note
        return rec


# ---------------------------------------------------------------- roofline bookkeeping
def stage_bytes(info: dict, m: int, type_: int = 2, eb: int = 8) -> dict:
    """Algorithmic HBM bytes per launch of each stage, the pruned chain's
    figures: each grid input read once and each grid output written once
    (eb = 8 B per complex64 value, 16 per complex128), and per non-uniform
    point its value (eb) plus a 12-byte sorted record (two fractional offsets
    and the packed cell; 20 B per point in complex64).  Plan-owned tables
    (the transfer function's phase-factor table the row passes read, this
    library's 16-byte record format, the halo duplicates of the tiles) are
    not algorithmic bytes; see plan_table_bytes."""
    n, np_, W = info["n"], info["n_pad"], info["window"]
    pt = eb + 12
    if type_ == 1:
        return {
            "spread": pt * m + eb * W * W,
            "col_fwd_fold": eb * (W * W + np_ * W),
            "row_t1": eb * (np_ * W + np_ * n),
            "col_inv": eb * (np_ * n + n * n),
        }
    return {
        "col_fwd": eb * (n * n + np_ * n),
        "row_t2": eb * (np_ * n + np_ * W),
        "col_inv_fold": eb * (np_ * W + W * W),
        "interp": eb * W * W + pt * m,
    }


def plan_table_bytes(info: dict, type_: int = 2, eb: int = 8) -> dict:
    """Bytes of plan-owned tables a stage reads on top of its algorithmic
    bytes: the row pass's non-separable phase-factor table (E over the |k|
    quadrant, or type 2's rows with the per-column factor folded in), and the
    gridding stages' records beyond 12 B per point (16 B / 24 B records, halo
    duplicates)."""
    np_ = info["n_pad"]
    tables = info.get("phase_table_bytes", 0)
    equad = (np_ // 2 + 1) * (np_ // 2 + 2) * eb if tables else 0
    etab2 = tables - equad
    rb = 16 if eb == 8 else 24
    extra_rec = rb * info["records"] - 12 * info["points"]
    if type_ == 1:
        return {"row_t1": equad, "spread": extra_rec + eb * (info["records"] - info["points"])}
    return {"row_t2": etab2 if etab2 > 0 else equad, "interp": (rb - 12) * info["points"]}


# FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64: the part's nominal rate
ALU_PEAK_TFLOPS = {False: 152 * 128 * 2 * 2.07e9 / 1e12, True: 1.25}
# FP64 gridding in double-float arithmetic: one double-float multiply-add (2 flops) takes
# 12 FP32-pipe instructions (product with its FMA error term, two-sum, carries)
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12


def stage_flops(info: dict, m: int, type_: int = 2, f64: bool = False) -> dict:
    """Algorithmic flops per launch of each stage: 5 L log2 L per L-point
    complex FFT, one complex multiply (6 flops) per kept mode for the
    transfer function, and per gridding point or record the Horner taps
    (2 axes x w taps x d FMA, d = the tap polynomials' degree: w + 1 in FP32,
    13 in FP64) plus w^2 complex-by-real MACs."""
    n, np_, W, w = info["n"], info["n_pad"], info["window"], info["kernel_width"]
    fft = 5.0 * np_ * np.log2(np_)
    d = 13 if f64 else w + 1
    taps = 2 * 2 * w * d + 4 * w * w + 4 * w
    if type_ == 1:
        return {"spread": taps * info["records"], "col_fwd_fold": 2 * W * fft,
                "row_t1": 3 * np_ * fft + 6.0 * np_ * np_, "col_inv": n * fft}
    return {"col_fwd": n * fft, "row_t2": 3 * np_ * fft + 6.0 * np_ * np_, "col_inv_fold": 2 * W * fft,
            "interp": taps * m}


def kernel_of_stage(stage: str, info: dict, f64: bool) -> str:
    """Name of the kernel a stage launches for this geometry (as ncu lists it)."""
    lognp = int(np.log2(info["n_pad"]))
    v, s = ("double2", "double") if f64 else ("float2", "float")
    rv = "dfc" if f64 and lognp >= 9 else v   # FP64 FFT passes from N' = 512 up: double-float
    w = info["kernel_width"]
    if f64:
        tap = f"double, {w}, true" if w in (11, 13) else f"double, {8 if w <= 8 else (16 if w <= 16 else 26)}, false"
    else:
        tap = f"float, {w}, true" if 4 <= w <= 8 else f"float, {16 if w <= 16 else 26}, false"
    tma = not f64 and 512 <= info["n_pad"] <= 4096          # folded column passes
    tma_wide = not f64 and info["n_pad"] == 4096              # unfolded ones too
    tile = info.get("tile", 64)
    interp = f"interp_kernel<{tap}>"
    if f64 and info.get("double_float"):
        interp = f"interp_df_kernel<{w}>"
    if f64 and info.get("double_float"):
        spread = f"spread_df_kernel<{w}>"
    elif f64:
        spread = f"spread_private_kernel<{tap}>" if tile <= 16 else f"spread_kernel<{tap}>"
    elif tile <= 32:
        spread = f"spread_private_kernel<{tap}>"
    else:
        spread = (f"spread_fixed_kernel<{w}, true, 2>" if 4 <= w <= 8 else
                  f"spread_fixed_kernel<{16 if w <= 16 else 26}, false, 2>")
    return {"col_fwd": f"col_tma_kernel<{lognp}, 2>" if tma_wide else f"col_kernel<{rv}, {lognp}, 2>",
            "row_t2": f"row_t2_kernel<{rv}, {lognp}>",
            "col_inv_fold": f"col_tma_kernel<{lognp}, 3>" if tma else f"col_kernel<{rv}, {lognp}, 3>",
            "interp": interp, "spread": spread,
            "col_fwd_fold": f"col_tma_kernel<{lognp}, 0>" if tma else f"col_kernel<{rv}, {lognp}, 0>",
            "row_t1": f"row_t1_kernel<{rv}, {lognp}>",
            "col_inv": f"col_tma_kernel<{lognp}, 1>" if tma_wide else f"col_kernel<{rv}, {lognp}, 1>"}[stage]


_FFT_SOURCES = ["passes.cuh", "fft_engine.cuh", "tma.cuh", "dfloat.cuh"]
STAGE_SOURCES = {"col_fwd": _FFT_SOURCES, "row_t2": _FFT_SOURCES, "col_inv_fold": _FFT_SOURCES,
                 "col_fwd_fold": _FFT_SOURCES, "row_t1": _FFT_SOURCES, "col_inv": _FFT_SOURCES,
                 "interp": ["gridding.cu"], "spread": ["gridding.cu"]}


def source_hash(stage: str) -> str:
    """Hash of the sources a stage's kernel is compiled from (traffic figures
    taken with ncu are reported only while this matches)."""
    h = hashlib.sha256()
    for f in STAGE_SOURCES[stage] + ["common.cuh"]:
        with open(os.path.join(ROOT, "paper_1308_6644_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record(stage: str, workload: str = "nuasm2"):
    """The committed ncu counters of a stage's kernel (profiles/traffic.json),
    if they were taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except Exception:
        return None
    rec = t.get(stage if workload == "nuasm2" else f"{workload}:{stage}")
    if not rec or rec.get("source_hash") != source_hash(stage):
        return None
    return rec


def measured_traffic(stage: str, workload: str = "nuasm2"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    rec = ncu_record(stage, workload)
    return None if rec is None else rec.get("dram_bytes_per_launch")


def ncu_limiter(stage: str, workload: str = "nuasm2"):
    """Issue-slot and pipe utilisation of a stage's kernel from the committed
    ncu capture (fractions of the kernel's cycles), or None."""
    rec = ncu_record(stage, workload)
    if rec is None:
        return None
    keys = {"issue_active": "issue_active_pct", "fma_pipe": "fma_pipe_pct", "lsu_pipe": "lsu_pipe_pct",
            "shared_pipe": "shared_pipe_pct", "dram_throughput": "dram_throughput_pct"}
    out = {k: round(rec[v] / 100.0, 3) for k, v in keys.items() if v in rec}
    return out or None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(wl, n_sample: int, rng_seed: int = 5):
    """Time the FP64 oracle on a bounded sample: the full spectrum G(k) H(k)
    (separable DFT matrix products) plus the direct NUFFT_2 sum at n_sample
    points; returns timings and the sampled outputs."""
    import oracle as O
    rng = np.random.default_rng(rng_seed)
    idx = np.sort(rng.choice(wl.m, n_sample, replace=False))
    n, n_pad = wl.n, 2 * wl.n
    u1 = wl.values.astype(np.complex64).astype(np.complex128)
    t0 = time.perf_counter()
    g = O.uniform_dft(u1, n_pad)
    h = O.asm_transfer(n, n_pad, wl.pitch, wl.lam, wl.z, wl.ox, wl.oy)
    a = g * h / float(n_pad) ** 2
    t1 = time.perf_counter()
    v = O.nudft_type2(a, wl.x[idx] / wl.pitch, wl.y[idx] / wl.pitch, n_pad)
    t2 = time.perf_counter()
    return idx, v, t1 - t0, t2 - t1


def cpu_baseline(wl, n_sample: int = CPU_SAMPLE_POINTS):
    idx, v, t_spec, t_pts = oracle_sample(wl, n_sample)
    full = t_spec + t_pts * wl.m / n_sample
    rec = {"value": wl.m / full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"FP64 direct NUDFT oracle: full spectrum ({t_spec:.2f} s) + {n_sample} of "
                      f"{wl.m} destination points ({t_pts:.2f} s), extrapolated to all points")}
    return rec, idx, v


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if ws > 1 and rank != 0:
        return 0
    wl = _workload()
    n_sample = 4096
    for _ in range(args.warmup):
        oracle_sample(wl, n_sample)
    times = []
    for _ in range(args.steps):
        _, _, t_spec, t_pts = oracle_sample(wl, n_sample)
        times.append(t_spec + t_pts * wl.m / n_sample)
    tot = float(sum(times))
    value = wl.m * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": wl.n, "n_pad": 2 * wl.n, "points": wl.m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: full spectrum + {n_sample} destination points, "
                                       f"extrapolated to {wl.m} points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
SINGLE = {
    # key: (generator, precision, workload label)
    "nuasm2": (lambda W: W.nuasm2_graded(seed=1002, n=1024, pitch=8e-6), "f32", WORKLOAD),
    "c1": (lambda W: W.nuasm1_small(1001), "f64", "nuasm1_n64_m4864_dense_core_lambda633nm_z5cm"),
    # the paper's own NU-ASM_1 experiment geometry (context for its CPU timing)
    "paper1": (lambda W: W.paper_experiment(1006), "f32", "nuasm1_paper_n256_m65536_quadrant_pitch_lambda500nm_z8mm"),
    "paper1f64": (lambda W: W.paper_experiment(1006), "f64",
                  "nuasm1_paper_n256_m65536_quadrant_pitch_lambda500nm_z8mm"),
    "c3t1": (lambda W: W.fresnel_clustered(1003, type_=1), "f32", "nufre1_n2048_m4194304_clusters_lambda633nm_z1m"),
    "c3t2": (lambda W: W.fresnel_clustered(1003, type_=2), "f32", "nufre2_n2048_m4194304_clusters_lambda633nm_z1m"),
    "c3t1f64": (lambda W: W.fresnel_clustered(1003, type_=1), "f64",
                "nufre1_n2048_m4194304_clusters_lambda633nm_z1m"),
    "c3t2f64": (lambda W: W.fresnel_clustered(1003, type_=2), "f64",
                "nufre2_n2048_m4194304_clusters_lambda633nm_z1m"),
}


def oracle_sample_type1(wl, n_points: int, rng_seed: int = 5):
    """Time the FP64 oracle's direct NUFFT_1 (every mode) for a sample of the
    points; the cost is linear in the point count."""
    import oracle as O
    rng = np.random.default_rng(rng_seed)
    idx = np.sort(rng.choice(wl.m, n_points, replace=False))
    c = np.asarray(wl.values).reshape(-1)[idx].astype(np.complex128)
    t0 = time.perf_counter()
    O.nudft_type1(wl.x[idx] / wl.pitch, wl.y[idx] / wl.pitch, c, 2 * wl.n)
    return time.perf_counter() - t0


def cpu_baseline_single(wl, prec: str):
    """The oracle on a bounded sample of a single-solve workload (see the
    `sample` string of the returned record)."""
    import oracle as O
    if wl.type == 2 and wl.kind == "asm" and wl.n <= 1024:
        return cpu_baseline(wl)
    if wl.type == 2:
        rng = np.random.default_rng(5)
        n_pad = 2 * wl.n
        a = rng.normal(size=(n_pad, n_pad)) + 1j * rng.normal(size=(n_pad, n_pad))
        idx = np.sort(rng.choice(wl.m, 256, replace=False))
        t0 = time.perf_counter()
        O.nudft_type2(a, wl.x[idx] / wl.pitch, wl.y[idx] / wl.pitch, n_pad)
        t = (time.perf_counter() - t0) * wl.m / 256
        return ({"value": wl.m / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                 "sample": f"FP64 direct NUFFT_2 at 256 of {wl.m} points, extrapolated (the spectrum's "
                           f"dense-DFT cost at N' = {n_pad} is left out, so this overstates the oracle)"},
                None, None)
    n_pts = wl.m if wl.m <= 8192 else 256
    t = oracle_sample_type1(wl, n_pts) * wl.m / n_pts
    what = "every point" if n_pts == wl.m else f"{n_pts} of {wl.m} points, extrapolated"
    return ({"value": wl.m / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"FP64 direct NUFFT_1 over all {(2 * wl.n) ** 2} modes for {what} (the inverse DFT "
                       "to the plane is left out, so this overstates the oracle)"}, None, None)


def run_ours(args):
    import torch
    from paper_1308_6644_gb300 import workloads as WL

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1308_6644_gb300 import _build
    _build.build()
    import paper_1308_6644_gb300 as P

    make, prec, label = SINGLE[args.workload]
    wl = make(WL)
    f64 = prec == "f64"
    cdt, tdt, eb = (np.complex128, torch.complex128, 16) if f64 else (np.complex64, torch.complex64, 8)
    params = P.make_params(wl.n, wl.pitch, wl.lam, wl.z, ox=wl.ox, oy=wl.oy, kind=wl.kind, prec=prec,
                           kernel=args.kernel, tol=args.tol)
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(wl.x).to(dev)
    y = torch.from_numpy(wl.y).to(dev)
    wts = None if wl.weights is None else torch.from_numpy(np.asarray(wl.weights, np.float64)).to(dev)
    tuned = None
    if args.autotune:
        params, tuned_ms = P.nuasm_autotune(params, x, y, wl.type, stream=stream)
        tuned = {"tile": params.tile, "interp_chunk": params.interp_chunk, "spread_chunk": params.spread_chunk,
                 "solve_ms": round(tuned_ms, 4)}
    t_plan0 = time.perf_counter()
    plan = P.nuasm_plan(params, x, y, wts, stream=stream)
    plan_s = time.perf_counter() - t_plan0
    info = plan.info()
    n_out = wl.n * wl.n if wl.type == 1 else wl.m
    inp = torch.from_numpy(np.ascontiguousarray(np.asarray(wl.values).astype(cdt).reshape(-1))).to(dev)
    out = torch.empty(n_out, dtype=tdt, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if wl.kind == "asm":
        execute = P.nuasm1_execute if wl.type == 1 else P.nuasm2_execute
    else:
        def execute(pl, i, o, stream=None):
            return P.nufresnel_execute(pl, wl.type, i, o, stream=stream)

    def solve():
        execute(plan, inp, out, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        solve()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        solve()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    total_ms = float(step_ms.sum())
    total_ms, points = reduce_over_ranks(total_ms, float(wl.m * args.steps), dev)
    value = points / (total_ms * 1e-3)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    h_in = inp.cpu().pin_memory()
    h_out = torch.empty(n_out, dtype=tdt).pin_memory()
    for _ in range(2):
        execute(plan, h_in, h_out, stream=stream)
    torch.cuda.synchronize()
    e2e_ms = []
    aux_steps = min(args.steps, 200)
    for k in range(aux_steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        execute(plan, h_in, h_out, stream=stream)
        e.record(stream)
        e.synchronize()
        e2e_ms.append(s.elapsed_time(e))
    e2e_serial = wl.m / (np.mean(e2e_ms) * 1e-3)

    # pipelined: three plans on three streams and steps rotating over them, so
    # one step's host copies overlap the others' kernels; every step copies its
    # input in and reads its result back.  Where the other plans' steps stream
    # more than twice the 129 MB L2 through the cache before a plan's data
    # recurs, no flush is needed; smaller workloads flush L2 before every step.
    ws_bytes = sum(stage_bytes(info, wl.m, wl.type, eb).values())
    e2e_flush = e2e_needs_flush(ws_bytes)
    lanes = [(plan, stream, h_in, h_out)]
    for _ in range(E2E_LANES - 1):
        lanes.append((P.nuasm_plan(params, x, y, wts, stream=stream), torch.cuda.Stream(dev),
                      inp.cpu().pin_memory(), torch.empty(n_out, dtype=tdt).pin_memory()))
    for pl, st, hi, ho in lanes:
        execute(pl, hi, ho, stream=st)
    torch.cuda.synchronize()
    t_a, t_b = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    t_a.record(stream)
    for _, st, _, _ in lanes[1:]:
        st.wait_event(t_a)
    for k in range(aux_steps):
        pl, st, hi, ho = lanes[k % E2E_LANES]
        if e2e_flush:
            with torch.cuda.stream(st):
                flush.zero_()
        execute(pl, hi, ho, stream=st)
    for _, st, _, _ in lanes[1:]:
        t_j = torch.cuda.Event()
        t_j.record(st)
        stream.wait_event(t_j)
    t_b.record(stream)
    t_b.synchronize()
    e2e_value = wl.m * aux_steps / (t_a.elapsed_time(t_b) * 1e-3)
    for pl, _, _, _ in lanes[1:]:
        pl.destroy()

    # per-stage times for the roofline (separate pass, events on the solve stream)
    P.nuasm_profile_enable(plan, True)
    P.nuasm_profile_read(plan)
    for _ in range(aux_steps):
        flush.zero_()
        solve()
    torch.cuda.synchronize()
    prof = P.nuasm_profile_read(plan)
    P.nuasm_profile_enable(plan, False)
    sbytes = stage_bytes(info, wl.m, wl.type, eb)
    tbytes = plan_table_bytes(info, wl.type, eb)
    sflops = stage_flops(info, wl.m, wl.type, f64)
    peak, peak_kind = hbm_peak()
    def alu_peak_of(stage):
        """The arithmetic roof of a stage: FP32, FP64, or double-float for FP64 gridding on the FP32 pipe."""
        kname = kernel_of_stage(stage, info, f64)
        if f64 and ("_df_" in kname or "<dfc" in kname):
            return DF_PEAK_TFLOPS
        return ALU_PEAK_TFLOPS[f64]

    stages = {}
    for name, b in sbytes.items():
        ms, cnt = prof[name]
        if cnt:
            avg = ms / cnt
            alu_peak = alu_peak_of(name)
            gbs, tfs = b / (avg * 1e-3) / 1e9, sflops[name] / (avg * 1e-3) / 1e12
            # the binding roof: the one this stage's algorithmic work takes longest on
            bound = "alu" if sflops[name] / (alu_peak * 1e12) > b / (peak * 1e9) else "hbm"
            stages[name] = {"ms": avg, "gbs": gbs, "tfs": tfs, "bound": bound, "hbm_frac": gbs / peak,
                            "alu_frac": tfs / alu_peak,
                            "frac": (tfs / alu_peak) if bound == "alu" else (gbs / peak)}
    dom = max(stages, key=lambda s: stages[s]["ms"])
    d = stages[dom]
    if d["bound"] == "alu":
        dom_peak = alu_peak_of(dom)
        roofline = {"bound": "alu", "achieved": d["tfs"], "peak": dom_peak, "unit": "TFLOP/s", "frac": d["frac"],
                    "peak_source": ("double-float on the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz / 12 "
                                    "instructions per 2-flop multiply-add" if dom_peak == DF_PEAK_TFLOPS else
                                    "FP64 nominal rate" if f64 else
                                    "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz")}
    else:
        roofline = {"bound": "hbm", "achieved": d["gbs"], "peak": peak, "unit": "GB/s", "frac": d["frac"],
                    "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                    if peak_kind == "measured" else "fallback 6.8 TB/s"}

    def stage_rec(k, v):
        r = {"ms": round(v["ms"], 5), "GB/s": round(v["gbs"], 1), "TFLOP/s": round(v["tfs"], 2),
             "bound": v["bound"], "frac": round(v["frac"], 3), "hbm_frac": round(v["hbm_frac"], 3),
             "alu_frac": round(v["alu_frac"], 3), "algorithmic_bytes": int(sbytes[k])}
        if tbytes.get(k):
            r["plan_table_bytes"] = int(tbytes[k])
        lim = ncu_limiter(k, args.workload)
        if lim:
            r["ncu"] = lim
        return r

    roofline.update({"traffic": measured_traffic(dom, args.workload), "kernel": kernel_of_stage(dom, info, f64),
                     "algorithmic_bytes": int(sbytes[dom]), "algorithmic_flops": float(sflops[dom]),
                     "hbm_frac": round(d["hbm_frac"], 4), "alu_frac": round(d["alu_frac"], 4),
                     "bytes_model": "grid values read and written once (8 B complex64) + 20 B per point "
                                    "(value + 12-byte record); plan tables excluded",
                     "stages": {k: stage_rec(k, v) for k, v in stages.items()}})
    lim = ncu_limiter(dom, args.workload)
    if lim:
        roofline["ncu_limiter"] = lim

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("df64" if info.get("double_float") or info["n_pad"] >= 512 else "f64") if f64 else prec,
            "data": "synthetic",
            "config": {"workload": label, "n": wl.n, "n_pad": info["n_pad"], "points": wl.m,
                       "kernel": args.kernel, "tol": params.tol or (1e-12 if f64 else 1e-6),
                       "kernel_width": info["kernel_width"], "tile": info["tile"],
                       "precision": ("complex128 data; double-float (pairs of FP32) arithmetic in the gridding "
                                     "and the FFT passes from N' = 512 up, FP64 elsewhere" if f64
                                     else "complex64 + FP64-derived phase"),
                       "l2": "flushed (256 MB write) before every step", "plan_s": round(plan_s, 3),
                       "autotuned": tuned,
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h_in.numel() * eb),
                    "d2h_bytes_per_step": int(h_out.numel() * eb),
                    "how": f"host buffers through nuasm*_execute; {E2E_LANES} plans on {E2E_LANES} streams, steps "
                           "rotating (one step's copies overlap the others' kernels, and steps on different streams "
                           "fill each other's last kernel waves, so this rate can exceed the one-solve-at-a-time "
                           "device rate); " +
                           ("L2 flushed before every step" if e2e_flush else
                            f"L2 not flushed: a plan's ~{ws_bytes / 1e6:.0f} MB of step traffic recurs only after "
                            f"the other plans' ~{(E2E_LANES - 1) * ws_bytes / 1e6:.0f} MB (L2 129 MB)") +
                           "; serial_value: one plan, L2 flushed before every step",
                    "serial_value": e2e_serial},
            "gpu_launches": 4 * args.steps,
            "roofline": roofline,
            "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rec, idx, ref = cpu_baseline_single(wl, prec)
        line["cpu_baseline"] = rec
        if ref is not None:
            got = out.cpu().numpy()[idx]
            line["rel_l2_vs_fp64_sample"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        elif args.workload == "c1":
            import oracle as O
            want = O.nuasm1(wl.x, wl.y, np.asarray(wl.values).astype(cdt).astype(np.complex128),
                            dict(n=wl.n, pitch=wl.pitch, lam=wl.lam, z=wl.z)).reshape(-1)
            line["rel_l2_vs_fp64"] = float(O.rel_l2(out.cpu().numpy(), want))
    plan.destroy()
    del flush, h_in, h_out
    if rank == 0 and ws == 1 and args.workload == "nuasm2" and args.served_requests > 0:
        # the served form on a bounded trace (continuous batching over resident
        # point sets) beside the plain one-plane-per-call path on the same requests
        torch.cuda.synchronize()
        r = serve_session(P, local, args.served_requests, args.served_sets, args.slots, 12, 24, clocks=False)
        line["served"] = {k: r[k] for k in (
            "requests", "sets", "slots", "failed", "arrival_rate_per_s", "p50_ms", "p99_ms",
            "served_points_per_s", "plain_points_per_s", "served_over_plain", "plain_resident_points_per_s",
            "served_over_plain_resident", "plain", "plain_resident", "inputs")}
        line["served"]["workload"] = (f"Poisson arrivals of {r['requests']} requests over {r['sets']} resident point "
                                      "sets (N 1024-4096, 0.9M-10M points), type 1/2, z and lambda per request")
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batched planes
def e2e_needs_flush(step_bytes: float, lanes: int = E2E_LANES) -> bool:
    """Whether the pipelined end-to-end loop must flush L2 before every step:
    yes unless the other lanes' steps stream more than twice the L2 through
    the cache before a lane's data recurs."""
    return (lanes - 1) * step_bytes < 2 * L2_BYTES


def _timed_steps(fn, steps, stream, flush):
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        fn()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])


def run_batch(args):
    """64 mixed planes (N in {256..2048}, types 1/2 interleaved, z in [1, 50] cm,
    lambda in {450, 532, 633} nm, M/N^2 log-uniform in [1/4, 4]) recorded into
    one CUDA graph over `lanes` streams, against the same planes issued one
    execute call per plane on one stream."""
    import torch
    from paper_1308_6644_gb300 import workloads as WL
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1308_6644_gb300 import _build
    _build.build()
    import paper_1308_6644_gb300 as P
    stream = torch.cuda.current_stream(dev)
    planes, items, total_m, in_bytes, out_bytes = [], [], 0, 0, 0
    tiles = {}
    for i in range(args.planes):
        wl = WL.mixed_plane(1004, i)
        params = P.make_params(wl.n, wl.pitch, wl.lam, wl.z, kind="asm", prec="f32")
        xd, yd = torch.from_numpy(wl.x).to(dev), torch.from_numpy(wl.y).to(dev)
        if args.autotune:
            params, _ = P.nuasm_autotune(params, xd, yd, wl.type, stream=stream)
        plan = P.nuasm_plan(params, xd, yd, stream=stream)
        t_used = plan.info()["tile"]
        tiles[t_used] = tiles.get(t_used, 0) + 1
        del xd, yd
        inp = torch.from_numpy(np.ascontiguousarray(wl.values.astype(np.complex64).reshape(-1))).to(dev)
        out = torch.empty(wl.n * wl.n if wl.type == 1 else wl.m, dtype=torch.complex64, device=dev)
        planes.append((plan, wl.type, inp, out))
        items.append((plan, wl.type, inp, out))
        total_m += wl.m
        in_bytes += inp.numel() * 8
        out_bytes += out.numel() * 8
    batch = P.nuasm_batch_create(items, lanes=args.lanes)
    lanes, kernels = batch.info()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def plain():
        for plan, t, inp, out in planes:
            (P.nuasm1_execute if t == 1 else P.nuasm2_execute)(plan, inp, out, stream=stream)

    # the planes whose every kernel launches at least a full wave of CTAs over the
    # GPU (N >= 1024: >= 1024 rows / columns per pass, >= 1089 tiles); running the
    # others side by side with them can hide at most the others' time
    large = [it for it in planes if it[0].n >= 1024]

    def plain_large():
        for plan, t, inp, out in large:
            (P.nuasm1_execute if t == 1 else P.nuasm2_execute)(plan, inp, out, stream=stream)

    def batched():
        batch.execute(stream)

    for _ in range(args.warmup):
        flush.zero_()
        plain()
        batched()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    b_ms = _timed_steps(batched, args.steps, stream, flush)
    clk = clocks.stop()
    p_ms = _timed_steps(plain, max(3, min(args.steps, 20)), stream, flush)
    pl_ms = _timed_steps(plain_large, max(3, min(args.steps, 20)), stream, flush)
    total_ms, points = reduce_over_ranks(float(b_ms.sum()), float(total_m * args.steps), dev)
    value = points / (total_ms * 1e-3)
    plain_value = total_m / (float(p_ms.mean()) * 1e-3)

    # end to end: pinned host inputs copied in, the graph, outputs copied back, every step
    h_in = [inp.cpu().pin_memory() for _, _, inp, _ in planes]
    h_out = [torch.empty(out.shape, dtype=out.dtype).pin_memory() for _, _, _, out in planes]

    def e2e_step():
        for h, (_, _, inp, _) in zip(h_in, planes):
            inp.copy_(h, non_blocking=True)
        batch.execute(stream)
        for h, (_, _, _, out) in zip(h_out, planes):
            h.copy_(out, non_blocking=True)

    e_ms = _timed_steps(e2e_step, max(3, min(args.steps, 20)), stream, flush)
    alg = 0
    for plan, t, inp, out in planes:
        info = plan.info()
        n, np_, W = info["n"], info["n_pad"], info["window"]
        alg += 8 * (n * n + 2 * np_ * n + 2 * np_ * W + W * W) + 24 * info["points"]
    peak, peak_kind = hbm_peak()
    ach = alg / (float(b_ms.mean()) * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"mixed{args.planes}_planes_n256-2048_types1+2", "planes": args.planes,
                       "points_per_step": total_m, "lanes": lanes, "graph_kernels": kernels,
                       "tiles": ("autotuned per plane (tile side and split chunks): " if args.autotune
                                 else "library rule: ") +
                       ", ".join(f"T={k} x{v}" for k, v in sorted(tiles.items())),
                       "plain_points_per_s": plain_value, "batched_over_plain": value / plain_value,
                       "plain": "one execute call per plane, back to back on one stream",
                       "large_planes": len(large),
                       "plain_ms_all": float(p_ms.mean()), "plain_ms_large_planes_only": float(pl_ms.mean()),
                       "batched_over_plain_bound": float(p_ms.mean() / pl_ms.mean()),
                       "bound": "plain time of all planes / plain time of the N >= 1024 planes alone: the gain "
                                "batching could reach if every smaller plane ran for free beside them",
                       "l2": "flushed (256 MB write) before every step", "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": float(np.percentile(b_ms, 50)), "p99": float(np.percentile(b_ms, 99))},
            "e2e": {"value": total_m / (float(e_ms.mean()) * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes},
            "gpu_launches": kernels * args.steps,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "kernel": "whole batch graph (every kernel of every plane)",
                         "peak_source": f"{peak_kind} copy bandwidth"},
            "clocks": clk}
    batch.destroy()
    for plan, *_ in planes:
        plan.destroy()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- serving loop
def serve_session(P, local: int, n_requests: int, n_sets: int, slots: int, plain_requests: int,
                  resident_requests: int, clocks=True) -> dict:
    """Poisson arrivals of requests over resident point sets (N in
    {512..4096}, up to 16M points), each with its own wavelength, distance and
    type, served with continuous batching, against the same requests run one
    at a time by the plain path: (a) per request nuasm_plan from host
    coordinates, execute with host buffers, destroy; (b) execute with host
    buffers on plans built beforehand (resident), waiting for each."""
    import torch
    from paper_1308_6644_gb300 import workloads as WL
    sets = [WL.serving_point_set(1005, k) for k in range(n_sets)]
    trace = WL.serving_trace(1005, n_requests, len(sets))
    rng = np.random.default_rng(1005)
    host = []
    for st_ in sets:
        nn = st_.n * st_.n
        host.append({"in1": torch.from_numpy(WL.random_phasor(rng, st_.m).astype(np.complex64)).pin_memory(),
                     "in2": torch.from_numpy(WL.random_phasor(rng, nn).astype(np.complex64)).pin_memory(),
                     "out1": [torch.empty(nn, dtype=torch.complex64).pin_memory() for _ in range(2)],
                     "out2": [torch.empty(st_.m, dtype=torch.complex64).pin_memory() for _ in range(2)]})

    def request(i, rec):
        k, t, z, lam, _ = rec
        st_, h = sets[k], host[k]
        params = P.make_params(st_.n, st_.pitch, lam, z, kind="asm", prec="f32")
        inp = h["in1"] if t == 1 else h["in2"]
        out = (h["out1"] if t == 1 else h["out2"])[i % 2]
        return st_, params, t, inp, out

    srv = P.nuasm_server_create(slots=slots)
    # every set binned once (resident from then on)
    warm = []
    for k, st_ in enumerate(sets):
        params = P.make_params(st_.n, st_.pitch, 532e-9, 0.1, kind="asm", prec="f32")
        warm.append(P.nuasm_server_submit(srv, params, 2, st_.x, st_.y, host[k]["in2"], host[k]["out2"][0],
                                          points_id=k + 1))
    for t in warm:
        P.nuasm_server_wait(srv, t)

    def closed_burst(recs):
        t0 = time.perf_counter()
        tk, pts = [], 0
        for i, rec in enumerate(recs):
            st_, params, t, inp, out = request(i, rec)
            tk.append(P.nuasm_server_submit(srv, params, t, st_.x, st_.y, inp, out, points_id=rec[0] + 1))
            pts += st_.m
        for t in tk:
            P.nuasm_server_wait(srv, t)
        return time.perf_counter() - t0, pts

    # warm the pools and staging buffers, then probe the capacity with a closed burst
    closed_burst(trace[: min(len(trace), 4 * slots)])
    burst = trace[: min(len(trace), 16 * slots)]
    el, pts = closed_burst(burst)
    rate = len(burst) / el                               # requests/s the GPU sustains
    capacity = pts / el
    P.nuasm_server_stats(srv, reset=True)
    # Poisson arrivals at the measured capacity (saturating)
    clk_s = ClockSampler(local) if clocks else None
    if clk_s:
        clk_s.start()
    t_start = time.perf_counter()
    arrival = 0.0
    tickets = []
    for i, rec in enumerate(trace):
        arrival += rec[4] / rate
        delay = t_start + arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        st_, params, t, inp, out = request(i, rec)
        tickets.append(P.nuasm_server_submit(srv, params, t, st_.x, st_.y, inp, out, points_id=rec[0] + 1))
    res = [P.nuasm_server_wait(srv, t) for t in tickets]
    clk = clk_s.stop() if clk_s else None
    st = P.nuasm_server_stats(srv)
    srv.destroy()
    failed = sum(1 for r in res if r["status"] != 0)
    served = st["points"] / st["wall_s"]
    # plain path (a): the first requests of the same trace, one at a time, plan per request
    n_plain = min(len(trace), plain_requests)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pts = 0
    for i, rec in enumerate(trace[:n_plain]):
        st_, params, t, inp, out = request(i, rec)
        plan = P.nuasm_plan(params, st_.x, st_.y)
        (P.nuasm1_execute if t == 1 else P.nuasm2_execute)(plan, inp, out)
        plan.destroy()
        pts += st_.m
    plain = pts / (time.perf_counter() - t0)
    # plain path (b): plans of the first requests built beforehand (resident),
    # then one execute at a time with the same host buffers, each waited for
    n_res = min(len(trace), resident_requests)
    stream = torch.cuda.current_stream()
    plans = []
    for i, rec in enumerate(trace[:n_res]):
        st_, params, t, inp, out = request(i, rec)
        plans.append((P.nuasm_plan(params, torch.from_numpy(st_.x).cuda(), torch.from_numpy(st_.y).cuda()),
                      t, inp, out, st_.m))
    for plan, t, inp, out, _ in plans[:2]:
        (P.nuasm1_execute if t == 1 else P.nuasm2_execute)(plan, inp, out, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pts = 0
    for plan, t, inp, out, m in plans:
        (P.nuasm1_execute if t == 1 else P.nuasm2_execute)(plan, inp, out, stream=stream)
        stream.synchronize()
        pts += m
    plain_res = pts / (time.perf_counter() - t0)
    for plan, *_ in plans:
        plan.destroy()
    h2d = d2h = 0
    for rec in trace:
        st_ = sets[rec[0]]
        h2d += 8 * (st_.m if rec[1] == 1 else st_.n * st_.n)
        d2h += 8 * (st_.n * st_.n if rec[1] == 1 else st_.m)
    return {"requests": len(trace), "sets": len(sets), "slots": slots, "warmup_requests": len(burst),
            "failed": failed, "arrival_rate_per_s": rate, "closed_loop_points_per_s": capacity,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "wall_s": st["wall_s"],
            "served_points_per_s": served, "points_served": st["points"],
            "bins_built_during_run": st["bins_built"], "resident_sets": st["resident_sets"],
            "resident_gb": st["resident_bytes"] / 1e9, "peak_budget_gb": st["peak_bytes"] / 1e9,
            "hbm_budget_gb": 150,
            "plain_points_per_s": plain, "plain_requests_timed": n_plain, "served_over_plain": served / plain,
            "plain": "per request: nuasm_plan from host coordinates, execute with host buffers, destroy",
            "plain_resident_points_per_s": plain_res, "plain_resident_requests_timed": n_res,
            "served_over_plain_resident": served / plain_res,
            "plain_resident": "per request: execute with host buffers on a plan built beforehand, waited for",
            "inputs": "pinned host memory, copied in and out by every request",
            "h2d_bytes_per_request": h2d // len(trace), "d2h_bytes_per_request": d2h // len(trace),
            "clocks": clk}


def run_serve(args):
    """The serving loop as its own bench line (see serve_session)."""
    import torch
    ws, rank, local = _dist()
    if ws > 1 and rank != 0:
        return 0          # one server per GPU; replicas add nothing to this line
    torch.cuda.set_device(local)
    from paper_1308_6644_gb300 import _build
    _build.build()
    import paper_1308_6644_gb300 as P
    r = serve_session(P, local, args.requests, args.sets, args.slots, args.plain_requests, args.plain_requests)
    n = r["requests"]
    line = {"metric": METRIC, "value": r["served_points_per_s"], "unit": UNIT, "n_gpus": 1, "steps": n,
            "warmup": r["warmup_requests"], "ms_per_step": 1e3 * r["wall_s"] / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve_poisson_{n}req_{r['sets']}sets_n512-4096",
                       **{k: v for k, v in r.items() if k not in ("clocks", "p50_ms", "p99_ms")}},
            "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"]},
            "e2e": {"value": r["served_points_per_s"], "unit": UNIT,
                    "h2d_bytes_per_step": r["h2d_bytes_per_request"],
                    "d2h_bytes_per_step": r["d2h_bytes_per_request"]},
            "gpu_launches": 4 * n,
            "clocks": r["clocks"]}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=list(SINGLE) + ["batch64", "serve"], default="nuasm2",
                    help="nuasm2: the NU-ASM_2 single-solve benchmark (default); c1: NU-ASM_1 64^2 FP64; "
                         "c3t1/c3t2(f64): NU-FRE types 1/2 at N = 2048, 4M clustered points; batch64: 64 mixed "
                         "planes in one graph; serve: Poisson-arrival serving loop")
    ap.add_argument("--planes", type=int, default=64)
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--sets", type=int, default=12)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--plain-requests", type=int, default=60)
    ap.add_argument("--served-requests", type=int, default=200,
                    help="default workload: requests of the bounded serving trace reported under 'served' (0: skip)")
    ap.add_argument("--served-sets", type=int, default=6)
    ap.add_argument("--kernel", choices=["es", "gaussian"], default="es",
                    help="spreading kernel of the single-solve workloads (gaussian: the paper's Greengard-Lee kernel)")
    ap.add_argument("--tol", type=float, default=0.0,
                    help="NUFFT tolerance of the single-solve workloads (0: the precision's default)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the tile side and split chunks per plane with nuasm_autotune instead of the "
                         "library's rule")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
