"""Benchmark: Levenberg-Marquardt iterations per second on the medium synthetic BA
workload (1,000 cameras, 500,000 points, ~3.0M observations, 1% outliers, Huber
delta 2, PCG <= 100 iterations at 1e-6 relative tolerance), mixed precision.

One step = one LM iteration of the whole hot path: edge linearisation, point and
camera accumulation, camera Schur complement, block-Jacobi PCG on it, point
back-substitution, FP64 retraction, FP64 candidate cost and the FP64 gain-ratio
decision.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp64]
                    [--impl ours|reference]

The line's cpu_baseline is one FP64 CPU oracle LM iteration (exact Schur complement,
dense Cholesky) on the whole workload, timed on the host cores; --impl reference times
the oracle per step on a bounded sub-problem of the same workload (edge-scaled).  Under torchrun every rank solves its own
replica (independent problems: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ba_medium_c1000_p500k_e3M_huber2_outliers1pct"
METRIC = "LM iter/s"


def _cpu_sample_worker(seed: int, ncam: int, iters: int) -> None:
    """Times the oracle (runs in a child process; the BLAS thread count comes from the
    environment).  ncam = 0: the whole workload; ncam < 0: every camera with the first
    2,000 points and their edges; otherwise the closed sub-problem of the first `ncam`
    cameras (their points and the edges among them)."""
    import numpy as np

    from oracle import lm as olm
    from paper_2509_26581_gb300 import synth

    p = synth.ba_medium(seed)
    if ncam == 0:
        ncam = p.n_cams
        prob = olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=p.huber_delta)
        n_edges, n_pts = p.n_edges, p.n_pts
    elif ncam < 0:
        # every camera (the full-size dense camera system) and only the first 2,000
        # points with their edges: the part of an iteration that grows with the cameras
        ncam = p.n_cams
        keep = p.pt_idx < 2000
        prob = olm.ba_problem(p.cams0, p.pts0[:2000], p.cam_idx[keep], p.pt_idx[keep], p.obs[keep],
                              huber_delta=p.huber_delta)
        n_edges, n_pts = int(keep.sum()), 2000
    else:
        keep = np.ones(p.n_pts, bool)
        keep[p.pt_idx[p.cam_idx >= ncam]] = False
        sel = keep[p.pt_idx]
        pts = np.nonzero(keep)[0]
        newid = -np.ones(p.n_pts, np.int64)
        newid[pts] = np.arange(len(pts))
        prob = olm.ba_problem(p.cams0[:ncam], p.pts0[pts], p.cam_idx[sel], newid[p.pt_idx[sel]],
                              p.obs[sel], huber_delta=p.huber_delta)
        n_edges, n_pts = int(sel.sum()), int(len(pts))
    t0 = time.perf_counter()
    olm.levenberg_marquardt(prob, iters)
    dt = time.perf_counter() - t0
    print(json.dumps(dict(seconds=dt, iters=iters, edges=n_edges, points=n_pts, cams=ncam,
                          full_edges=int(p.n_edges))))


def cpu_baseline(seed: int, ncam: int = 0, iters: int = 1, threads: int = 1) -> dict:
    """The FP64 oracle timed on this machine's host cores in a child process: `iters` LM
    iterations (each: cost, linearisation, normal equations, the camera Schur complement
    formed densely, dense Cholesky, back-substitution, candidate cost) on the whole
    workload (ncam = 0) or on the closed sub-problem of the first ncam cameras, whose
    rate is then scaled by edges to the whole workload."""
    t = str(max(1, threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-worker",
                        str(seed), str(ncam), str(iters)], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    value = d["iters"] / d["seconds"] * d["edges"] / d["full_edges"]
    if d["edges"] == d["full_edges"]:
        sample = (f"{d['iters']} FP64 oracle LM iteration(s) on the whole workload ({d['cams']} cameras, "
                  f"{d['points']} points, {d['edges']} edges; exact Schur complement, dense Cholesky of "
                  f"the {9 * d['cams']}-dimensional camera system) in {d['seconds']:.1f} s")
    else:
        sample = (f"{d['iters']} FP64 oracle LM iteration(s) on the closed sub-problem of the first "
                  f"{d['cams']} cameras ({d['points']} points, {d['edges']} edges) in {d['seconds']:.2f} s, "
                  f"scaled by edges to the {d['full_edges']}-edge workload")
    return dict(value=value, unit=METRIC, cores=max(1, threads), kind="oracle", sample=sample,
                nproc=os.cpu_count(), seconds=d["seconds"])


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.window = (0.0, float("inf"))

    def start(self):
        """Start sampling; returns once the first sample has arrived (at most 3 s), so
        that the samples cover the whole timed region that begins on return."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        t0 = time.monotonic()
        while not self.lines and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.window = (time.monotonic(), float("inf"))

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self) -> dict:
        """Stop sampling; the summary covers the samples taken between start() returning
        and this call (all samples if none fell inside)."""
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.window = (self.window[0], time.monotonic())
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lo, hi = self.window
        inside = [ln for t, ln in self.lines if lo <= t <= hi]
        used = inside if inside else [ln for _, ln in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in used:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        return dict(sm_mhz=sm[len(sm) // 2] if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm), samples_in_window=len(inside),
                    interval_ms=self.interval_ms)


# HBM3e nominal bandwidth of the part (8 stacks at 3,996 MHz), reported beside the
# measured copy rate.
NOMINAL_HBM_GBS = 7900.0

# FP64 flops per edge (2 x DFMA + DADD + DMUL thread instructions, counted by ncu) of
# one launch of the BA linearisation and cost kernels on the medium workload, keyed by
# a hash of the kernel sources they were counted from, so changed kernels report null.
FP64_SOURCES = ("schur_common.cuh", "schur_kernels.cuh")
FP64_FLOPS_PER_EDGE = {
    ("k_linearize", "bf16", "d06c2de5842b"): 18.00,
    ("k_linearize", "fp64", "d06c2de5842b"): 588.78,
    # one kernel for every precision (FP64 geometry and cost)
    ("k_cost", "bf16", "d06c2de5842b"): 65.55,
    ("k_cost", "fp32", "d06c2de5842b"): 65.55,
    ("k_cost", "fp64", "d06c2de5842b"): 65.55,
}


def fp64_peak(stream) -> float:
    """Measured FP64 FMA throughput of this GPU (TFLOP/s): gpo_fp64_fma_probe, eight
    CTAs of 256 threads per SM, the median of ten launches timed with CUDA events."""
    import torch

    from paper_2509_26581_gb300 import gpo
    n_ctas = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    iters = 400
    out = torch.empty(n_ctas * 256, dtype=torch.float64, device="cuda")
    for _ in range(3):
        gpo.fp64_fma_probe(stream.cuda_stream, n_ctas, iters, out)
    times = []
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gpo.fp64_fma_probe(stream.cuda_stream, n_ctas, iters, out)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    flops = 2.0 * n_ctas * 256 * iters * 32
    return flops / (ms * 1e-3) / 1e12


def fp64_rooflines(prof: dict, n_edges: int, precision: str, peak_tflops: float) -> dict:
    """FP64-pipe rooflines of the linearisation and cost kernels from their per-launch
    times in a profiled pass and the counted FP64 flops per edge (null when the
    counts are not for the current sources)."""
    h = kernel_source_hash(FP64_SOURCES)
    out = dict(peak_tflops=peak_tflops, peak_source="measured (gpo_fp64_fma_probe)")
    for key, kern in (("linearize", "k_linearize"), ("cost", "k_cost")):
        k = prof.get(key, {})
        ms = k["active_ms"] / k["active"] if k.get("active") else None
        fpe = FP64_FLOPS_PER_EDGE.get((kern, precision, h))
        ach = fpe * n_edges / (ms * 1e-3) / 1e12 if (fpe and ms) else None
        out[key] = dict(kernel=kern, avg_ms=ms, fp64_flops_per_edge=fpe, achieved_tflops=ach,
                        frac=ach / peak_tflops if ach else None)
    return out


def load_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM bytes (read + write) per Schur-product launch on the medium workload, counted by
# ncu, keyed by (precision, kernel, hash of the kernel sources): stale once the sources
# change.
MEASURED_TRAFFIC = {("bf16", "k_spmv_pp", "7fc91d8044b4"): 179.2e6}
SPMV_VARIANTS = {"auto": 0, "staged": 1, "classic": 2, "pipelined": 3, "dynamic": 4, "warpgroup": 5,
                 "warpgroup_staged": 6}
KERNEL_SOURCES = ("schur_common.cuh", "schur_spmv.cuh")


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha1()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2509_26581_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def spmv_kernel(precision: str, knobs: dict, ch_max: int) -> str:
    """The Schur-product kernel the library runs for these knobs (gpo_graph_desc)."""
    v = knobs.get("spmv_variant", 0)
    if v == 6 and ch_max <= 1024 and precision != "fp64":
        return "k_spmv_wgs"
    if v == 5 and ch_max <= 1024 and precision != "fp64":
        return "k_spmv_wg"
    if v == 4 and ch_max <= 512:
        return "k_spmv_dyn"
    if ch_max <= 1024 and (v == 3 or (v == 0 and precision != "fp64")):
        return "k_spmv_pp"
    if ch_max <= 1024 and v == 1:
        return "k_spmv_ws"
    return "k_spmv"


KERNEL_LABEL = {"k_spmv_wgs": "k_spmv_wgs (PCG Schur product, warp groups fed through shared-memory stages)",
                "k_spmv_wg": "k_spmv_wg (PCG Schur product, warp groups)",
                "k_spmv_pp": "k_spmv_pp (PCG Schur product, pipelined persistent)",
                "k_spmv_ws": "k_spmv_ws (PCG Schur product, staged)",
                "k_spmv": "k_spmv (PCG Schur product, classic)",
                "k_spmv_dyn": "k_spmv_dyn (PCG Schur product, dynamic Jacobians; bytes of the stored-row product)",
                "k_full_spmv": "k_full_spmv (PCG product with the full damped system)"}


def spmv_traffic(precision: str, kernel: str):
    return MEASURED_TRAFFIC.get((precision, kernel, kernel_source_hash()))


def spmv_algorithmic_bytes(E: int, P: int, precision: str) -> float:
    """Compulsory HBM bytes of one Schur-product launch: every stored Jacobian value
    (24 per edge) and camera index once, and each point's damped inverse block."""
    sJ = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    sA = 8 if precision == "fp64" else 4
    return E * (24 * sJ + 4) + P * 6 * sA


def knobs(args) -> dict:
    """Schedule knobs given on the command line; none given = the autotuned table's."""
    k = {}
    if args.chunk:
        k["chunk_edges"] = args.chunk
    if args.spmv != "auto":
        k["spmv_variant"] = SPMV_VARIANTS[args.spmv]
    return k


def spmv_algorithmic_bytes_vi(E: int, P: int, precision: str) -> float:
    """Same for the stereo model: 27 stored Jacobian values per edge (3 x 6 pose, 3 x 3
    point; rows padded to 32 are padding, not algorithmic)."""
    sJ = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    sA = 8 if precision == "fp64" else 4
    return E * (27 * sJ + 4) + P * 6 * sA


def full_algorithmic_bytes(E: int, P: int, precision: str) -> float:
    """Compulsory HBM bytes of one full-system product (k_full_spmv): every stored
    Jacobian value and camera index once, and per point its undamped block (6), the
    direction's inputs z and p_old and outputs p and y (3 each) and its edge range."""
    sJ = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    sA = 8 if precision == "fp64" else 4
    return E * (24 * sJ + 4) + P * (6 * sA + 12 * sA + 8)


def extra_full_system(args, p, dev, stream, schur_rate: float, schur_cost: float) -> dict:
    """The paper's own form of the solve on the same workload and precision: block-
    Jacobi PCG on the full damped system (GPO_SOLVER_FULL, same PCG cap and tolerance)
    against the camera Schur complement: LM rate over the same warm-up and timed
    steps, PCG iterations, final cost, the full-system product's time and achieved
    bandwidth (profiled pass), and the device footprint."""
    import torch

    from paper_2509_26581_gb300 import gpo
    prm = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6, solver=gpo.GPO_SOLVER_FULL)
    g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, args.precision,
                             device=dev, stream=stream.cuda_stream, **knobs(args))
    g.optimize(args.warmup, prm)
    cams_w = g.get_state(c0, p.n_cams, 9)
    pts_w = g.get_state(p0, p.n_pts, 3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rep = g.optimize(args.steps, prm)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    its = [h["pcg_iters"] for h in g.history()]
    g.set_initial(c0, cams_w)
    g.set_initial(p0, pts_w)
    g.set_profiling(True)
    g.optimize(args.steps, prm)
    prof = g.profile()
    sp = prof["spmv"]
    spmv_ms = sp["active_ms"] / sp["active"] if sp["active"] else float("nan")
    peak, peak_kind = load_peaks()
    alg = full_algorithmic_bytes(p.n_edges, p.n_pts, args.precision)
    out = dict(solver="full system (cameras and points), block-Jacobi PCG", precision=args.precision,
               lm_iter_per_s=args.steps / (ms / 1e3), schur_lm_iter_per_s=schur_rate,
               pcg_iters_per_step=its, final_cost=rep.final_cost,
               rel_diff_vs_schur=abs(rep.final_cost - schur_cost) / schur_cost,
               product=dict(kernel="k_full_spmv", avg_ms=spmv_ms, algorithmic_bytes=alg,
                            achieved_gbs=alg / (spmv_ms * 1e-3) / 1e9,
                            frac=alg / (spmv_ms * 1e-3) / 1e9 / peak, peak=peak, peak_source=peak_kind),
               kernels_ms={k: round(v["active_ms"], 3) for k, v in prof.items() if v["launches"]},
               footprint_bytes=g.footprint())
    g.close()
    return out


def extra_dynamic(args, p, dev, stream, stored_rate: float, stored_cost: float, stored_footprint: int) -> dict:
    """Dynamic Jacobians (spmv_variant 4: no rows are stored; the Schur preparation, every
    Schur product and the back-substitution evaluate each edge's rows from the state, in
    FP32 for the mixed modes) on the same workload, LM steps and PCG cap: LM rate and
    device footprint against stored rows (Table II's trade of time for memory), final
    cost against the stored-row run, and the product's time per launch (profiled pass)."""
    import torch

    from paper_2509_26581_gb300 import gpo
    prm = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6)
    g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, args.precision,
                             device=dev, stream=stream.cuda_stream, spmv_variant=4, chunk_edges=512)
    g.optimize(args.warmup, prm)
    cams_w = g.get_state(c0, p.n_cams, 9)
    pts_w = g.get_state(p0, p.n_pts, 3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rep = g.optimize(args.steps, prm)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    info = g.info()
    g.set_initial(c0, cams_w)
    g.set_initial(p0, pts_w)
    g.set_profiling(True)
    g.optimize(args.steps, prm)
    prof = g.profile()
    sp = prof["spmv"]
    fp = g.footprint()
    out = dict(kernel="k_spmv_dyn", kernel_dispatched=info["spmv_kernel"], precision=args.precision,
               rows_in="FP32 registers (nothing stored)" if args.precision != "fp64" else "FP64 registers",
               chunk_edges=g.knobs["chunk_edges"], lm_iter_per_s=args.steps / (ms / 1e3),
               stored_rows_lm_iter_per_s=stored_rate, footprint_bytes=fp,
               stored_rows_footprint_bytes=stored_footprint, footprint_vs_stored=fp / stored_footprint,
               j_bytes=info["j_bytes"], final_cost=rep.final_cost,
               rel_diff_vs_stored=abs(rep.final_cost - stored_cost) / stored_cost,
               product_avg_ms=sp["active_ms"] / sp["active"] if sp["active"] else None,
               kernels_ms={k: round(v["active_ms"], 3) for k, v in prof.items() if v["launches"]})
    g.close()
    return out


def extra_autodiff(args, p, dev, stream) -> dict:
    """The forward-mode automatic-differentiation checker on the whole workload: its
    kernel time (every edge's FP64 dual-number residual and rows) against the analytic
    linearisation kernel's, and the largest difference of their rows on 2,000 sampled
    edges (relative to each edge's largest entry; the analytic rows stored in the
    benchmarked precision)."""
    import numpy as np

    from paper_2509_26581_gb300 import gpo
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, args.precision,
                           device=dev, stream=stream.cuda_stream, **knobs(args))
    ids = np.random.default_rng(0).choice(p.n_edges, 2000, replace=False)
    _, J = g.debug_linearize_edges(ids)
    g.set_profiling(True)
    _, Ja = g.debug_autodiff_edges(ids)
    g.optimize(1, gpo.default_params(pcg_max_iters=1))   # one profiled analytic linearisation
    prof = g.profile()
    lin, ad = prof["linearize"], prof["autodiff"]
    scale = np.maximum(np.abs(Ja).reshape(len(ids), -1).max(axis=1), 1e-9)
    rel = (np.abs(J - Ja).reshape(len(ids), -1).max(axis=1) / scale).max()
    g.close()
    return dict(edges=p.n_edges, autodiff_ms=ad["total_ms"] / max(1, ad["timed"]),
                analytic_linearize_ms=lin["active_ms"] / max(1, lin["active"]),
                sampled_edges=len(ids), max_rel_diff_sampled=float(rel), analytic_precision=args.precision)


def _converge(p, prec: str, iters: int, dev, stream, params) -> dict:
    """One solve of `iters` LM iterations from the problem's initial state."""
    import torch

    from paper_2509_26581_gb300 import gpo
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, prec,
                           device=dev, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = g.optimize(iters, params)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h = g.history()
    g.close()
    last = h[-1]["cost"] if h else rep.final_cost
    return dict(final_cost=rep.final_cost, initial_cost=rep.initial_cost, accepted=rep.accepted,
                pcg_iters=rep.pcg_iters_total, pcg_failed=int(sum(r["pcg_failed"] for r in h)),
                pcg_breakdowns=int(sum(r["pcg_breakdown"] for r in h)),
                last_step_rel_decrease=(last - rep.final_cost) / rep.final_cost, seconds=dt)


def extra_convergence(args, p, dev, stream, fp64_peak_tflops: float, iters: int = 50) -> dict:
    """Mixed precision against the FP64 GPU path, each run for the paper's BAL budget of
    50 LM iterations from the same initial state (PCG <= 100 at 1e-6):
    * the benchmark's workload (cameras along a path: long, weakly constrained chains
      whose slow modes need many more iterations; the last step's relative decrease
      says how far each run is from converged);
    * a wide-baseline workload of 300,000 edges (100 cameras on a ring, 50,000 points
      seen by 6 cameras each, 1 % outliers, Huber delta 2) that all three precisions
      solve to convergence within the budget.
    Also the FP64 rate and the FP64-pipe rooflines of the FP64 build's linearisation and
    cost kernels (a profiled pass of two iterations)."""
    from paper_2509_26581_gb300 import gpo, synth
    params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6)
    out = dict(lm_iters=iters, pcg_max_iters=100, pcg_tol=1e-6)
    ring = synth.ba_ring(11, 100, 50000, 6, outlier_frac=0.01, huber_delta=2.0)
    for name, prob in (("workload", p), ("ring_300k", ring)):
        res = {prec: _converge(prob, prec, iters, dev, stream, params) for prec in ("fp64", "fp32", "bf16")}
        f64 = res["fp64"]["final_cost"]
        for prec in ("fp32", "bf16"):
            res[prec]["rel_diff_vs_fp64"] = abs(res[prec]["final_cost"] - f64) / f64
        res["edges"] = prob.n_edges
        res["cameras"] = prob.n_cams
        out[name] = res
    # the FP64 build's rate on the benchmarked schedule and its FP64-pipe rooflines
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp64",
                           device=dev, stream=stream.cuda_stream)
    g.optimize(args.warmup, params)
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.optimize(args.steps, params)
    torch.cuda.synchronize()
    out["fp64_lm_iter_per_s"] = args.steps / (time.perf_counter() - t0)
    g.set_profiling(True)
    g.optimize(2, params)
    out["fp64_build_rooflines"] = fp64_rooflines(g.profile(), p.n_edges, "fp64", fp64_peak_tflops)
    g.close()
    return out


def extra_vi(dev, stream, iters: int = 10) -> dict:
    """Global visual-inertial workload (3,000 stereo keyframes, 200,000 landmarks, ~1.9M
    stereo edges, inertial + bias random-walk edges between consecutive keyframes, bias
    prior): LM iterations per second in FP64, FP32 and BF16 storage, the Schur product's
    achieved bandwidth, and the final-cost difference of each mixed form against FP64.
    PCG <= 100 iterations at 1e-6 relative, rejection-ratio guard off (the inertial
    chain makes the PCG residual rise before it falls)."""
    import torch

    from paper_2509_26581_gb300 import gpo, synth
    p = synth.vi_global()
    params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6, pcg_rejection_ratio=0.0)
    peak, peak_kind = load_peaks()
    out = dict(workload=p.name, keyframes=p.n_kf, landmarks=p.n_pts, stereo_edges=p.n_edges,
               lm_iters=iters)
    costs = {}
    for prec in ("fp64", "fp32", "bf16"):
        g, _, _, _ = gpo.vi_graph(p, precision=prec, device=dev, stream=stream.cuda_stream)
        g.optimize(1, params)                     # finalize + warm
        g.set_initial(0, p.nav0)
        g.set_initial(p.n_kf, p.pts0)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        rep = g.optimize(iters, params)           # production path
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        g.set_initial(0, p.nav0)                  # per-kernel pass, same iterations
        g.set_initial(p.n_kf, p.pts0)
        g.set_profiling(True)
        g.optimize(iters, params)
        prof = g.profile()
        sp = prof["spmv"]
        spmv_ms = sp["active_ms"] / sp["active"] if sp["active"] else float("nan")
        alg = spmv_algorithmic_bytes_vi(p.n_edges, p.n_pts, prec)
        gbs = alg / (spmv_ms * 1e-3) / 1e9 if sp["active"] else 0.0
        costs[prec] = rep.final_cost
        out[prec] = dict(lm_iter_per_s=iters / (ms / 1e3), initial_cost=rep.initial_cost,
                         final_cost=rep.final_cost, accepted=rep.accepted,
                         pcg_iters=rep.pcg_iters_total, footprint_bytes=g.footprint(),
                         spmv=dict(avg_ms=spmv_ms, achieved_gbs=gbs, frac=gbs / peak, peak=peak,
                                   peak_source=peak_kind))
        g.close()
    for prec in ("fp32", "bf16"):
        out[prec]["rel_diff_vs_fp64"] = abs(costs[prec] - costs["fp64"]) / costs["fp64"]
        out[prec]["speedup_vs_fp64"] = out[prec]["lm_iter_per_s"] / out["fp64"]["lm_iter_per_s"]
    return out


def accumulation_bytes(E: int, P: int, NS: int, precision: str) -> float:
    """Compulsory bytes of one linearisation + Schur preparation (the accumulation phase):
    linearisation reads observations, indices, thresholds and point states and writes
    the Jacobian rows, point blocks and camera slot partials; the Schur preparation
    reads the rows and point blocks and writes the point inverses, point records and
    Schur slot partials."""
    sJ = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    sA = 8 if precision == "fp64" else 4
    prb = 64 if precision == "fp64" else 32
    lin = E * (16 + 8 + 8 + 2 + 24 * sJ) + P * (24 + 9 * sA) + NS * 54 * sA
    schur = E * (24 * sJ + 4 + 2) + P * (9 * sA + 6 * sA + prb) + NS * 54 * sA
    return lin + schur


def accumulation_roofline(prof: dict, E: int, P: int, NS: int, precision: str) -> dict:
    """The accumulation phase (a working linearisation plus the Schur preparation) of the
    profiled pass against the HBM roofline: algorithmic bytes of both kernels over the sum
    of their average working-launch times."""
    peak, peak_kind = load_peaks()
    ms = sum(prof[k]["active_ms"] / max(1, prof[k]["active"]) for k in ("linearize", "schur_prepare"))
    alg = accumulation_bytes(E, P, NS, precision)
    ach = alg / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return dict(bound="hbm", kernels="k_linearize + k_schur_prepare", avg_ms=ms, algorithmic_bytes=alg,
                achieved=ach, peak=peak, unit="GB/s", frac=ach / peak, peak_source=peak_kind)


def extra_large(dev, stream, iters: int = 20) -> dict:
    """Large BA workload (13,000 cameras, 4.5M points, ~29M observations, geometric tracks
    of mean 6.5 capped at 200): LM iterations per second over `iters` iterations from the
    initial state (the first ones are rejected: at the initial damping the step is far
    too long for the weakly constrained points), initial and final cost, accepted and
    failed steps, the Schur product's and the accumulation phase's achieved bandwidth
    (a profiled pass of three iterations), and the device footprint, in BF16 and FP32
    storage (mixed precision with the FP64 gain ratio) against the FP64 path."""
    import torch

    from paper_2509_26581_gb300 import gpo, synth
    p = synth.ba_large(2)
    params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6)
    peak, peak_kind = load_peaks()
    out = dict(workload=p.name, cameras=p.n_cams, points=p.n_pts, edges=p.n_edges, lm_iters=iters,
               peak=peak, peak_source=peak_kind)
    for prec in ("bf16", "fp32", "fp64"):
        g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, prec,
                                 device=dev, stream=stream.cuda_stream)
        g.optimize(0, params)                     # finalize: plan and upload
        info = g.info()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        rep = g.optimize(iters, params)           # production path
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        h = g.history()
        g.set_initial(c0, p.cams0)                # per-kernel pass
        g.set_initial(p0, p.pts0)
        g.set_profiling(True)
        g.optimize(3, params)
        prof = g.profile()
        sp = prof["spmv"]
        spmv_ms = sp["active_ms"] / sp["active"] if sp["active"] else float("nan")
        acc_ms = sum(prof[k]["active_ms"] / max(1, prof[k]["active"]) for k in ("linearize", "schur_prepare"))
        alg_s = spmv_algorithmic_bytes(p.n_edges, p.n_pts, prec)
        alg_a = accumulation_bytes(p.n_edges, p.n_pts, info["slots"], prec)
        out[prec] = dict(lm_iter_per_s=iters / (ms / 1e3), initial_cost=rep.initial_cost,
                         final_cost=rep.final_cost, accepted=rep.accepted,
                         first_accepted_iter=next((k for k, r in enumerate(h) if r["accepted"]), None),
                         pcg_failed=int(sum(r["pcg_failed"] for r in h)), pcg_iters=rep.pcg_iters_total,
                         footprint_bytes=g.footprint(), schedule=g.knobs,
                         spmv=dict(kernel=spmv_kernel(prec, g.knobs, info["chunk_edges"]), avg_ms=spmv_ms,
                                   achieved_gbs=alg_s / (spmv_ms * 1e-3) / 1e9,
                                   frac=alg_s / (spmv_ms * 1e-3) / 1e9 / peak),
                         accumulation=dict(avg_ms=acc_ms, achieved_gbs=alg_a / (acc_ms * 1e-3) / 1e9,
                                           frac=alg_a / (acc_ms * 1e-3) / 1e9 / peak))
        g.close()
    for prec in ("bf16", "fp32"):
        out[prec]["footprint_vs_fp64"] = out[prec]["footprint_bytes"] / out["fp64"]["footprint_bytes"]
        out[prec]["speedup_vs_fp64"] = out[prec]["lm_iter_per_s"] / out["fp64"]["lm_iter_per_s"]
        out[prec]["rel_diff_vs_fp64_same_iters"] = (abs(out[prec]["final_cost"] - out["fp64"]["final_cost"])
                                                    / out["fp64"]["final_cost"])
    out["note"] = ("no run is converged after this many iterations (the path's slow modes need "
                   "hundreds), so the final costs differ by trajectory; the convergence comparison "
                   "of the precisions is the 'convergence' record")
    return out


def extra_served(stream, rate: float = 2000.0, duration: float = 10.0, pool: int = 256,
                 sample: int = 32, lm_iters: int = 10) -> dict:
    """Served local-BA windows: Poisson streams of requests over `duration` seconds, each
    request a window of 5-40 keyframes, 300-8,000 landmarks and 2k-50k edges (first
    keyframe fixed) with its own observation noise and initial state, `lm_iters` LM
    iterations in BF16 storage under a 40 GB budget, through the continuous-batching
    server.  Two regimes: the configured 2,000 requests/s (above the service capacity:
    the queue grows and latency is queueing), and 60 % of the capacity measured there
    (steady state: latency is the service time under load).  Against the same requests
    solved one by one with the plain FP64 path; served results against the same
    requests solved alone; and BF16 against FP64 when both run to convergence (50 LM
    iterations, a sample of requests)."""
    import numpy as np

    from paper_2509_26581_gb300 import gpo, serving, synth
    bases = synth.window_pool(7, pool)
    edges = np.array([w.n_edges for w in bases])

    def stream_of(seed, r):
        arr = synth.poisson_arrivals(seed, r, duration)
        pick = synth.Stream(seed, 24).integers(len(arr), 0, pool)
        return arr, (lambda i: synth.fresh_request(bases[int(pick[i])], seed, i))

    out = dict(duration_s=duration, precision="bf16", lm_iters=lm_iters, budget_gb=40, window_pool=pool,
               window_edges=[int(edges.min()), int(edges.max())], mean_window_edges=float(edges.mean()))
    arr, make = stream_of(8, rate)
    r = serving.serve(make, arr, precision="bf16", lm_iters=lm_iters, stream=stream.cuda_stream)
    cap = r["solves_per_s"]

    def summary(r, arr, rate):
        steady = arr >= 0.2 * duration          # after the first fifth of the stream
        lat = r["latency"]
        return dict(rate_per_s=rate, requests=int(len(arr)), solves_per_s=r["solves_per_s"],
                    p50_s=r["p50"], p99_s=r["p99"],
                    p50_steady_s=float(np.percentile(lat[steady], 50)),
                    p99_steady_s=float(np.percentile(lat[steady], 99)),
                    seconds=r["seconds"], steps=r["steps"], max_resident=r["max_resident"],
                    mean_resident=r["mean_resident"], mean_step_ms=1e3 * r["step_seconds"] / max(1, r["steps"]))

    out["configured_rate"] = summary(r, arr, rate)
    arr2, make2 = stream_of(9, 0.6 * cap)
    r2 = serving.serve(make2, arr2, precision="bf16", lm_iters=lm_iters, stream=stream.cuda_stream)
    out["below_capacity"] = summary(r2, arr2, 0.6 * cap)
    # one by one in plain FP64 (baseline rate), and the served results against the same
    # requests solved alone in the same precision (the first `sample` requests)
    ids = np.arange(sample)
    b64 = serving.one_by_one(make, ids, precision="fp64", lm_iters=lm_iters)
    a16 = serving.one_by_one(make, ids, precision="bf16", lm_iters=lm_iters)
    same = np.abs(r["final_cost"][:sample] - a16["final_cost"]) / a16["final_cost"]
    out["one_by_one_fp64_solves_per_s"] = b64["solves_per_s"]
    out["speedup_vs_one_by_one_fp64"] = cap / b64["solves_per_s"]
    out["max_rel_cost_diff_served_vs_alone_same_precision"] = float(same.max())
    # converged: 50 LM iterations, BF16 and FP64, each request alone
    c16 = serving.one_by_one(make, ids, precision="bf16", lm_iters=50)
    c64 = serving.one_by_one(make, ids, precision="fp64", lm_iters=50)
    rel = np.abs(c16["final_cost"] - c64["final_cost"]) / c64["final_cost"]
    out["converged_50_iters"] = dict(requests=sample, max_rel_diff_bf16_vs_fp64=float(rel.max()),
                                     median_rel_diff_bf16_vs_fp64=float(np.median(rel)),
                                     within_1e6=int((rel <= 1e-6).sum()))
    return out


def max_over_ranks(x: float, dist) -> float:
    """The maximum of x over the ranks of the process group (x itself without a group):
    the replicas' timed regions end when the slowest one does."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, steps: int, seconds: float) -> float:
    """Whole-job LM iterations per second: each of the `world` replicas runs `steps`."""
    return world * steps / seconds


def run_vi(args, dev, stream, world: int) -> dict:
    """The global visual-inertial workload as the measured loop (--workload vi_global;
    used for its own launch lists and profiles): K LM iterations after W warm-up ones."""
    import torch

    from paper_2509_26581_gb300 import gpo, synth
    p = synth.vi_global()
    params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6, pcg_rejection_ratio=0.0)
    g, _, _, _ = gpo.vi_graph(p, precision=args.precision, device=dev, stream=stream.cuda_stream,
                              **knobs(args))
    g.optimize(args.warmup, params)
    nav_w = g.get_state(0, p.n_kf, 16)
    pts_w = g.get_state(p.n_kf, p.n_pts, 3)
    torch.cuda.synchronize()
    g.set_profiling(False)
    clocks = ClockSampler(dev)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rep = g.optimize(args.steps, params)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = int(sum(v["launches"] for v in g.profile().values()))
    g.set_initial(0, nav_w)                       # per-kernel pass from the same state
    g.set_initial(p.n_kf, pts_w)
    g.set_profiling(True)
    g.optimize(args.steps, params)
    prof = g.profile()
    sp = prof["spmv"]
    peak, peak_kind = load_peaks()
    alg = spmv_algorithmic_bytes_vi(p.n_edges, p.n_pts, args.precision)
    spmv_ms = sp["active_ms"] / sp["active"] if sp["active"] else float("nan")
    achieved = alg / (spmv_ms * 1e-3) / 1e9 if sp["active"] else 0.0
    return dict(
        metric=METRIC, value=world * args.steps / (ms / 1e3), unit="LM iter/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype={"fp64": "f64", "fp32": "f32", "bf16": "bf16+f32"}[args.precision],
        data="synthetic",
        config=dict(workload=p.name, precision=args.precision, keyframes=p.n_kf, landmarks=p.n_pts,
                    stereo_edges=p.n_edges, pcg_max_iters=100, pcg_tol=1e-6, pcg_rejection_ratio="off",
                    schedule=g.knobs,
                    parallelism=f"replicas x{world}"),
        gpu_launches=launches,
        roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, traffic=None,
                      kernel=KERNEL_LABEL[spmv_kernel(args.precision, g.knobs, g.info()["chunk_edges"])],
                      peak_source=peak_kind, algorithmic_bytes=alg, avg_ms=spmv_ms),
        clocks=clk, final_cost=rep.final_cost,
        kernels_ms={k: round(v["active_ms"], 3) for k, v in prof.items()},
        footprint_bytes=g.footprint())


def run_ours(args, rank: int, world: int, dist) -> dict | None:
    import numpy as np
    import torch

    from paper_2509_26581_gb300 import gpo, synth

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local % max(1, torch.cuda.device_count()))
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    if args.workload == "vi_global":
        return run_vi(args, dev, stream, world)
    p = synth.ba_medium(args.seed)
    solver = gpo.GPO_SOLVER_FULL if args.solver == "full" else gpo.GPO_SOLVER_SCHUR
    params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6, solver=solver)
    g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta,
                             args.precision, device=dev, stream=stream.cuda_stream, **knobs(args))
    g.optimize(args.warmup, params)               # also freezes the topology and plans memory
    cams_w = g.get_state(c0, p.n_cams, 9)         # the state the timed iterations start from
    pts_w = g.get_state(p0, p.n_pts, 3)
    torch.cuda.synchronize()
    g.set_profiling(False)                        # the production path; resets the launch counts
    clocks = ClockSampler(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rep = g.optimize(args.steps, params)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = int(sum(v["launches"] for v in g.profile().values()))
    hist = g.history()
    ms = max_over_ranks(ms, dist)
    # per-kernel times: the same iterations again from the same state (deterministic),
    # every launch bracketed by CUDA events on the stream (direct launches, the camera
    # half and the PCG update timed apart)
    g.set_initial(c0, cams_w)
    g.set_initial(p0, pts_w)
    g.set_profiling(True)
    g.optimize(args.steps, params)
    prof = g.profile()

    # end to end through the public API with host buffers: the timed LM trajectory
    # again (from the same post-warm-up state and initial damping), one call per
    # iteration as a caller stepping the solver makes it: copy the state in from pinned
    # host memory, run one LM iteration (continuing lambda and nu from the previous
    # call's report, so the calls run the timed iterations exactly), read the state back
    # and feed it to the next step
    g.set_profiling(False)
    bufs = [(torch.from_numpy(np.ascontiguousarray(cams_w)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(pts_w)).pin_memory())]
    bufs.append((torch.empty_like(bufs[0][0]).pin_memory(), torch.empty_like(bufs[0][1]).pin_memory()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_e2e = 0 if args.no_e2e else args.steps
    step_params = gpo.default_params(pcg_max_iters=100, pcg_tol=1e-6, solver=solver)
    lam, nu = step_params.initial_damping, 0.0
    e2e_pcg = []
    for k in range(n_e2e):
        cin, pin = bufs[k % 2]
        cout, pout = bufs[(k + 1) % 2]
        g.set_initial(c0, cin.numpy())
        g.set_initial(p0, pin.numpy())
        step_params.initial_damping = lam        # the LM state carried through the ABI
        step_params.initial_nu = nu
        r = g.optimize(1, step_params)
        lam, nu = r.final_lambda, r.final_nu
        e2e_pcg.append(r.pcg_iters_total)
        g.get_state(c0, p.n_cams, 9, out=cout.numpy())
        g.get_state(p0, p.n_pts, 3, out=pout.numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    if rank != 0:
        return None
    sp = prof["spmv"]
    peak, peak_kind = load_peaks()
    kern = spmv_kernel(args.precision, g.knobs, g.info()["chunk_edges"])
    alg = spmv_algorithmic_bytes(p.n_edges, p.n_pts, args.precision)
    if args.solver == "full":   # the full-system product instead of the Schur product
        kern = "k_full_spmv"
        alg = full_algorithmic_bytes(p.n_edges, p.n_pts, args.precision)
    spmv_ms = sp["active_ms"] / sp["active"] if sp["active"] else float("nan")
    achieved = alg / (spmv_ms * 1e-3) / 1e9 if sp["active"] else 0.0
    state_bytes = (p.n_cams * 9 + p.n_pts * 3) * 8
    pcg_iters = [h["pcg_iters"] for h in hist]
    line = dict(
        metric=METRIC, value=replica_rate(world, args.steps, ms / 1e3), unit="LM iter/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype={"fp64": "f64", "fp32": "f32", "bf16": "bf16+f32"}[args.precision],
        data="synthetic",
        config=dict(workload=WORKLOAD, precision=args.precision, cameras=p.n_cams, points=p.n_pts,
                    edges=p.n_edges, pcg_max_iters=100, pcg_tol=1e-6, seed=args.seed,
                    schedule=g.knobs,
                    l2="inputs larger than L2 (Jacobians + observations exceed 129 MB)",
                    parallelism=f"replicas x{world}"),
        e2e=None if args.no_e2e else dict(value=replica_rate(world, args.steps, e2e_s), unit="LM iter/s",
                                          h2d_bytes_per_step=state_bytes, d2h_bytes_per_step=state_bytes,
                                          pcg_iters_per_step=e2e_pcg,
                                          same_trajectory_as_timed=e2e_pcg == [h["pcg_iters"] for h in hist]),
        gpu_launches=launches,
        roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                      traffic=spmv_traffic(args.precision, kern) if args.seed == 1
                      and g.knobs["chunk_edges"] in (0, 512) else None,
                      kernel=KERNEL_LABEL[kern], peak_source=peak_kind,
                      algorithmic_bytes=alg, avg_ms=spmv_ms,
                      peak_nominal=NOMINAL_HBM_GBS, frac_nominal=achieved / NOMINAL_HBM_GBS),
        accumulation=accumulation_roofline(prof, p.n_edges, p.n_pts, g.info()["slots"], args.precision),
        clocks=clk,
        pcg_iters_per_step=pcg_iters,
        accepted_per_step=[int(h["accepted"]) for h in hist],
        final_cost=rep.final_cost,
        kernels_ms={k: round(v["active_ms"], 3) for k, v in prof.items()},
        footprint_bytes=g.footprint(),
        fp64=fp64_rooflines(prof, p.n_edges, args.precision, fp64_peak(stream)),
    )
    if not args.no_extras and world == 1:
        g.close()

        def extra(name, fn, *a):
            try:                  # an extra never takes the headline line down with it
                line[name] = fn(*a)
            except Exception as ex:
                line[name] = dict(error=repr(ex)[:300])

        extra("convergence", extra_convergence, args, p, dev, stream, line["fp64"]["peak_tflops"])
        extra("full_system", extra_full_system, args, p, dev, stream, line["value"], rep.final_cost)
        extra("autodiff", extra_autodiff, args, p, dev, stream)
        extra("dynamic_jacobians", extra_dynamic, args, p, dev, stream, line["value"], rep.final_cost,
              line["footprint_bytes"])
        extra("vi", extra_vi, dev, stream)
        extra("served", extra_served, stream)
        extra("large", extra_large, dev, stream)
    return line


def _oracle_part(seed: int, ncam: int) -> dict:
    """One FP64 oracle LM iteration on a part of the workload (a child process, one BLAS
    thread); returns the worker's record."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-worker", str(seed),
                        str(ncam), "1"], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args, rank: int, world: int) -> dict | None:
    """The oracle on this workload, each step a bounded sample of one LM iteration in two
    measured parts: the closed sub-problem of the first 200 cameras (the work that grows
    with the edges, scaled by edges to the whole workload) and all 1,000 cameras with
    2,000 points (the dense 9,000-dimensional camera system: its forming, Cholesky and
    solves, measured at full size).  The sum comes within about 10 % of the full
    iteration, which is the default run's cpu_baseline (about 40 s)."""
    if rank != 0:
        return None
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps are not needed
    secs = []
    for _ in range(max(1, args.steps)):
        a = _oracle_part(args.seed, 200)
        b = _oracle_part(args.seed, -1)
        secs.append(a["seconds"] * a["full_edges"] / a["edges"] + b["seconds"])
    v = len(secs) / sum(secs)
    sample = (f"per step, one FP64 oracle LM iteration on the closed sub-problem of the first {a['cams']} cameras "
              f"({a['points']} points, {a['edges']} edges, {a['seconds']:.2f} s, scaled by edges to the "
              f"{a['full_edges']}-edge workload) plus one on all {b['cams']} cameras with {b['points']} points "
              f"({b['edges']} edges; the dense {9 * b['cams']}-dimensional camera system at full size, "
              f"{b['seconds']:.2f} s)")
    base = dict(nproc=os.cpu_count(), sample=sample)
    return dict(metric=METRIC, value=v, unit="LM iter/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 / v, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, precision="fp64-oracle", seed=args.seed),
                cpu_baseline=dict(kind="oracle", cores=1, sample=base["sample"], value=v, unit=METRIC,
                                  nproc=base["nproc"]),
                e2e=dict(value=v, unit="LM iter/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--cpu-sample-worker":
        _cpu_sample_worker(int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--chunk", type=int, default=0, help="edges per chunk (0 = library default)")
    ap.add_argument("--spmv", default="auto", choices=sorted(SPMV_VARIANTS),
                    help="Schur-product kernel (a tuning knob; results are bit-identical)")
    ap.add_argument("--solver", default="schur", choices=["schur", "full"],
                    help="linear solver of the LM step: camera Schur complement (default) or the "
                         "full-system PCG")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=1,
                    help="BLAS threads of the oracle's CPU baseline (default 1)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--workload", default="ba_medium", choices=["ba_medium", "vi_global"],
                    help="the measured loop: the 1,000-camera BA workload (default) or the global "
                         "visual-inertial one (for its profiles)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, the visual-inertial and the served-windows measurements")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line:
            print(json.dumps(line))
        return
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "ba_medium":
        base = cpu_baseline(args.seed, threads=args.cpu_threads)   # before any GPU work in this process
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_ours(args, rank, world, dist)
    if line is not None:
        if base is not None:
            line["cpu_baseline"] = base
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
