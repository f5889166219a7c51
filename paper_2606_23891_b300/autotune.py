"""Autotuner of the batched offload pipeline.

Times one batched step (density -> ghost -> gradient -> force) of the caller's
particle set for every candidate (CTA size, target cells per bundle) and
keeps the fastest.  Every candidate runs the same kernels on the same data, so
the choice changes speed only, never results beyond rounding order.
"""
from __future__ import annotations

import torch

from . import sph


def candidates(ncells: int):
    """CTA sizes x bundle sizes (all targets, and two splits into smaller
    bundles whose dedup buffers stay closer to L2 size)."""
    bundles = [0]
    for div in (8, 64):
        if ncells // div >= 64:
            bundles.append(ncells // div)
    return [(t, b) for t in (64, 128, 256) for b in bundles]


def time_batched_step(off, reps: int = 2, step: str = "batched") -> float:
    """ms per batched step on the offload's stream (after one warm step);
    ``step`` "list" times the neighbour-list variant."""
    fn = off.list_step if step == "list" else off.batch_step
    fn()
    torch.cuda.synchronize(off.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize(off.device)
    return e0.elapsed_time(e1) / reps


def tune(off, reps: int = 2, configs=None, step: str = "batched") -> dict:
    """Try every candidate on `off` (an Offload), leave the best plan built on
    it, and return {"threads", "max_target_cells", "ms", "table"}."""
    ncells = off.info["nonempty_cells"]
    table = []
    for threads, mtc in (configs or candidates(ncells)):
        off.batch(max_target_cells=mtc, threads=threads)
        ms = time_batched_step(off, reps, step)
        table.append({"threads": threads, "max_target_cells": mtc, "ms": ms,
                      "bundles": off.binfo["nbundles"]})
    best = min(table, key=lambda r: r["ms"])
    off.batch(max_target_cells=best["max_target_cells"], threads=best["threads"])
    return {"threads": best["threads"], "max_target_cells": best["max_target_cells"],
            "ms": best["ms"], "table": table}


def tune_tree(off, leaf_maxes=(64, 128, 256), threads=(64, 128, 256), reps: int = 1,
              step: str = "batched") -> dict:
    """Tree plan: pick the leaf size at 128 threads, then the CTA size at that
    leaf size; leave the best plan built on `off` and return the table."""
    table = []

    def trial(lm, t):
        off.batch(threads=t, leaf_max=lm)
        ms = time_batched_step(off, reps, step)
        table.append({"leaf_max": lm, "threads": t, "ms": ms, "leaves": off.binfo["cells"],
                      "nbrs": off.binfo["nbrs"]})
        return ms

    best_lm = min(leaf_maxes, key=lambda lm: trial(lm, 128))
    for t in threads:
        if t != 128:
            trial(best_lm, t)
    best = min(table, key=lambda r: r["ms"])
    off.batch(threads=best["threads"], leaf_max=best["leaf_max"])
    return {"threads": best["threads"], "leaf_max": best["leaf_max"], "ms": best["ms"],
            "table": table}


class GraphStep:
    """The batched step recorded once into a CUDA graph and replayed.  All
    calls of the step are asynchronous library launches on the capture
    stream; one eager step runs first so that one-time set-up (occupancy
    queries) happens outside the capture."""

    def __init__(self, off, step=None):
        self.off = off
        step = step or off.batch_step
        step()
        torch.cuda.synchronize(off.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            step()
        torch.cuda.synchronize(off.device)

    def replay(self) -> None:
        self.graph.replay()
