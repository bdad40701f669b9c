"""Autotuner of batched factorizations: the tile size b of every matrix and
the batch's dense threshold, picked by timing candidate configurations on
this GPU.

For each distinct shape (m, n) of the batch, one representative problem is
compressed and factored with every candidate tile size b (b must divide m
and n) and dense threshold; the fastest b is kept per shape, and the dense
threshold that minimises the batch's summed time (shapes weighted by how
often they occur) is kept for the batch.  Results can be cached in a JSON
file keyed by GPU, kernel, tolerance, precision and shape.

This module only chooses options and times library calls: the work runs in
the library.  The scheduler width stays at one CTA per SM and the rank
capacity of a tile is fixed by b (b/2), so there is no separate width or
rank-bucket knob to tune.
"""
from __future__ import annotations

import collections
import json
import os

from . import blr
from . import workloads as W

CANDIDATE_B = (256, 512)
CANDIDATE_DENSE = (16, 32, 64)


def _time_one(kernel, m, n, b, sx, sy, tol, precision, dense_rank) -> float:
    pr = W.kernel_problem(kernel, m, n, b, sx, sy)
    opts = blr.blr_opts_default(b=b, tol=tol, precision=precision, dense_rank=dense_rank)
    a = blr.blr_compress_kernel(pr.x, pr.y, kernel, opts)
    f = blr.blr_qr(a, opts)
    sec = blr.blr_stats(f)["seconds"]
    f.destroy()
    return sec


def tune(problems, kernel: str, tol: float, precision: int, cache_path: str | None = None,
         candidates_b=CANDIDATE_B, candidates_dense=CANDIDATE_DENSE) -> dict:
    """problems: (m, n, seed_x, seed_y) tuples.  Returns {"b": [b per
    problem], "dense_rank": int, "table": {shape: {config: seconds}}}."""
    import torch
    gpu = torch.cuda.get_device_name(0)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    shapes = collections.OrderedDict()
    for (m, n, sx, sy) in problems:
        shapes.setdefault((m, n), (sx, sy))
    weight = collections.Counter((m, n) for (m, n, _, _) in problems)
    # warm the library up (module load, first launch) on a tiny problem
    _time_one(kernel, 1024, 512, 256, 1, 2, tol, precision, 16)
    table = {}
    for (m, n), (sx, sy) in shapes.items():
        row = {}
        for b in candidates_b:
            if m % b or n % b:
                continue
            for dr in candidates_dense:
                key = f"{gpu}|{kernel}|{tol:g}|{precision}|{m}x{n}|b{b}|d{dr}"
                if key not in cache:
                    cache[key] = _time_one(kernel, m, n, b, sx, sy, tol, precision, dr)
                row[(b, dr)] = cache[key]
        table[(m, n)] = row
    best_b = {shape: min({b for b, _ in row}, key=lambda b: min(t for (bb, _), t in row.items() if bb == b))
              for shape, row in table.items()}
    best_dense = min(candidates_dense,
                     key=lambda dr: sum(weight[s] * table[s][(best_b[s], dr)] for s in table))
    if cache_path:
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=0)
    return {"b": [best_b[(m, n)] for (m, n, _, _) in problems], "dense_rank": best_dense,
            "table": {f"{m}x{n}": {f"b{b}/d{dr}": t for (b, dr), t in row.items()} for (m, n), row in table.items()}}
