"""Serving driver over the C ABI's continuous-batching loop (gpo_server_*).

Requests (local bundle-adjustment windows) arrive at given times; the driver builds
and plans every arrived request on worker threads, submits them in arrival order,
advances the server by one step (admit, one LM iteration for every resident window,
retire), and records each request's latency from arrival to retirement.  Every solve
runs in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import gpo


# Schedule of served windows: a server step's launches cover hundreds of windows at once,
# so the chunking and Schur product that suit a large problem serve them best (512-edge
# chunks and the pipelined product gave 12 % more solves/s than the single-window tuning
# of 256-edge chunks on a 2,000 requests/s stream).  The same knobs solve a window alone,
# so served and lone results stay equal.
SERVED_KNOBS = dict(chunk_edges=512, spmv_variant=3)


def window_graph(p, precision: str, fix_first: bool = True, **kw) -> tuple:
    """Graph of a window (first keyframe fixed, as local BA fixes its oldest pose),
    scheduled with SERVED_KNOBS unless knobs are given."""
    kw = kw or dict(SERVED_KNOBS)
    cam_fixed = np.zeros(p.n_cams, bool)
    if fix_first:
        cam_fixed[0] = True
    return gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, precision,
                        cam_fixed=cam_fixed, **kw)


def serve(windows, arrivals: np.ndarray, pick: np.ndarray | None = None, precision: str = "bf16",
          lm_iters: int = 10, params=None, memory_budget: int = 40 << 30,
          max_resident: int = 1024, stream=None, builders: int = 4) -> dict:
    """Runs the request stream; request i arrives at arrivals[i] seconds and is a fresh
    graph of windows[pick[i]] (windows a list), or of the problem windows(i) returns
    (windows a callable, pick unused).  Arrived requests are built and planned on
    `builders` worker threads (problem and graph construction and host planning need no
    GPU and release the interpreter inside the library), submitted in arrival order,
    and the server is stepped on this thread.  Returns latencies (arrival to
    retirement), throughput and final costs."""
    from concurrent.futures import ThreadPoolExecutor

    sv = gpo.Server(precision, stream=stream, memory_budget=memory_budget, max_resident=max_resident)
    n = len(arrivals)
    lat = np.full(n, np.nan)
    cost = np.full(n, np.nan)
    tickets = {}
    graphs = {}
    building = {}
    nxt_build = 0
    nxt = 0
    done = 0
    steps = 0
    max_res = 0
    step_s = 0.0                          # time inside sv.step() (admission + one LM iteration)
    res_sum = 0

    def make(i):
        g, _, _ = window_graph(windows(i) if callable(windows) else windows[pick[i]], precision)
        g.plan()
        return g

    pool = ThreadPoolExecutor(max_workers=max(1, builders))
    t0 = time.perf_counter()
    try:
        while done < n:
            now = time.perf_counter() - t0
            while nxt_build < n and arrivals[nxt_build] <= now:
                building[nxt_build] = pool.submit(make, nxt_build)
                nxt_build += 1
            while nxt < nxt_build and building[nxt].done():
                g = building.pop(nxt).result()
                tickets[sv.submit(g, lm_iters, params)] = nxt
                graphs[nxt] = g
                nxt += 1
            ts = time.perf_counter()
            res, queued, fin = sv.step()
            step_s += time.perf_counter() - ts
            steps += 1
            res_sum += res
            max_res = max(max_res, res)
            if fin:
                tnow = time.perf_counter() - t0
                for t in list(tickets):
                    rep = sv.poll(t)
                    if rep is not None:
                        i = tickets.pop(t)
                        lat[i] = tnow - arrivals[i]
                        cost[i] = rep.final_cost
                        graphs.pop(i).close()
                        done += 1
            if res == 0 and queued == 0:       # idle: wait for a build or the next arrival
                if nxt < nxt_build:
                    building[nxt].result()
                elif nxt_build < n:
                    wait = arrivals[nxt_build] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
    finally:
        pool.shutdown(wait=True)
    total = time.perf_counter() - t0
    sv.close()
    return dict(latency=lat, final_cost=cost, seconds=total, steps=steps, max_resident=max_res,
                mean_resident=res_sum / max(1, steps), step_seconds=step_s,
                solves_per_s=n / total, p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)))


def one_by_one(windows, pick: np.ndarray, precision: str = "fp64", lm_iters: int = 10,
               params=None) -> dict:
    """Baseline: the same requests solved one after another with gpo_optimize (request k
    is windows[pick[k]], or windows(pick[k]) when windows is a callable)."""
    n = len(pick)
    cost = np.empty(n)
    t0 = time.perf_counter()
    for i in range(n):
        g, _, _ = window_graph(windows(pick[i]) if callable(windows) else windows[pick[i]], precision)
        cost[i] = g.optimize(lm_iters, params).final_cost
        g.close()
    total = time.perf_counter() - t0
    return dict(final_cost=cost, seconds=total, solves_per_s=n / total)
