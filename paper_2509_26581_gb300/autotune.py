"""Autotuner of the per-graph schedule knobs.

Two knobs of `gpo_graph_desc` change how the kernels walk a problem, not the method:
  * chunk_edges  -- edges per CTA chunk of the per-edge kernels (256, 512, 1024); the
                    chunking groups the per-camera partial sums, so results agree up to
                    rounding;
  * spmv_variant -- the PCG Schur-product kernel: 2 = classic (one CTA per chunk),
                    1 = staged (persistent CTAs, warp-specialised bulk-copy pipeline),
                    3 = pipelined (persistent CTAs prefetching the next chunk's
                    indices); all give bit-identical results (see the variant tests).
The best choice depends on the problem's size (how many chunks fill the GPU, how many
slots a chunk has) and on the storage precision.  `tune` times every candidate on a
representative problem of a size class -- a few LM iterations after a warm-up, wall
clock around `gpo_optimize` with the device synchronised on both sides -- and keeps the
fastest.  The winners form a table keyed by device name, model, precision and size
class (`tuning.json` beside this file, written by `python -m
paper_2509_26581_gb300.autotune --write` on the target GPU); `choose` looks a graph's
knobs up in it, and `gpo.ba_graph` / `gpo.vi_graph` apply it when no knob is given.
"""
from __future__ import annotations

import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")

# (upper bound on observation edges, class name)
SIZE_CLASSES = [(20_000, "window"), (300_000, "small"), (8_000_000, "medium"), (math.inf, "large")]
CANDIDATES = [dict(chunk_edges=c, spmv_variant=v) for c in (256, 512, 1024) for v in (2, 1, 3)]
DEFAULT = dict(chunk_edges=512, spmv_variant=0)


def size_class(n_edges: int) -> str:
    for bound, name in SIZE_CLASSES:
        if n_edges < bound:
            return name
    return SIZE_CLASSES[-1][1]


_CACHE: dict = {}


def device_name() -> str:
    if "device" not in _CACHE:
        name = "none"
        try:
            import torch
            if torch.cuda.is_available():
                name = torch.cuda.get_device_name(0)
        except Exception:   # no torch or no GPU: the table is not used
            pass
        _CACHE["device"] = name
    return _CACHE["device"]


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def choose(n_edges: int, precision: str, model: str = "ba", table: dict | None = None,
           device: str | None = None) -> dict:
    """Knobs for a graph of n_edges observation edges: the table's entry for this device,
    model, precision and size class, else the library defaults."""
    if table is None:
        if "table" not in _CACHE:
            _CACHE["table"] = load_table()
        table = _CACHE["table"]
    key = f"{device or device_name()}|{model}|{precision}|{size_class(n_edges)}"
    entry = table.get(key)
    return dict(entry["best"]) if entry else dict(DEFAULT)


def tune(build, candidates=CANDIDATES, iters: int = 3, warmup: int = 1, repeats: int = 2) -> dict:
    """Times build(**knobs).optimize(iters) for every candidate (after `warmup` LM
    iterations on the same graph, state reset in between); returns the fastest and all
    timings (seconds per LM iteration, best of `repeats`)."""
    import torch
    timings = []
    for knobs in candidates:
        g, reset = build(**knobs)
        g.optimize(warmup)
        best = math.inf
        for _ in range(repeats):
            reset(g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.optimize(iters)
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) / iters)
        g.close()
        timings.append(dict(knobs=knobs, s_per_iter=best))
    fastest = min(timings, key=lambda t: t["s_per_iter"])
    return dict(best=fastest["knobs"], timings=timings)


def _ba_builder(p, precision):
    from . import gpo

    def build(**knobs):
        g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, precision,
                                 **knobs)

        def reset(graph):
            graph.set_initial(c0, p.cams0)
            graph.set_initial(p0, p.pts0)
        return g, reset
    return build


def _vi_builder(p, precision):
    from . import gpo

    def build(**knobs):
        g, n0, p0, _ = gpo.vi_graph(p, precision=precision, **knobs)

        def reset(graph):
            graph.set_initial(n0, p.nav0)
            graph.set_initial(p0, p.pts0)
        return g, reset
    return build


def representative(model: str, cls: str):
    """A seeded problem of each size class (the large class is left to the medium one's
    choice unless tuned explicitly: generating 29M edges takes minutes)."""
    from . import synth
    if model == "ba":
        return {"window": lambda: synth.ba_window(5, 20, 3000),
                "small": lambda: synth.ba_path(6, 100, 30_000, "pareto"),
                "medium": lambda: synth.ba_medium(1),
                "large": lambda: synth.ba_large(2)}[cls]()
    return {"window": lambda: synth.vi_problem(5, n_kf=20, n_pts=1000),
            "small": lambda: synth.vi_problem(6, n_kf=200, n_pts=10_000),
            "medium": lambda: synth.vi_global(),
            "large": lambda: synth.vi_global()}[cls]()


def tune_all(models=("ba", "vi"), precisions=("fp64", "fp32", "bf16"),
             classes=("window", "small", "medium"), path: str = TABLE) -> dict:
    table = load_table(path)
    dev = device_name()
    for model in models:
        for cls in classes:
            p = representative(model, cls)
            for prec in precisions:
                build = _ba_builder(p, prec) if model == "ba" else _vi_builder(p, prec)
                res = tune(build)
                n_edges = int(p.n_edges)
                table[f"{dev}|{model}|{prec}|{cls}"] = dict(res, edges=n_edges)
                print(model, cls, prec, n_edges, res["best"],
                      {f"{t['knobs']['chunk_edges']}/{t['knobs']['spmv_variant']}": round(t['s_per_iter'] * 1e3, 3)
                       for t in res["timings"]}, flush=True)
                with open(path, "w") as f:      # after every entry: a partial run keeps its results
                    json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    import sys
    if "--write" in sys.argv:
        tune_all()
    else:
        print(__doc__)
