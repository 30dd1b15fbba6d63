"""Autotuner for the batched SVD (one captured graph of many uneven problems).

For each size class of the batch (m and n binned by powers of two) it times the
candidate launch parameters of ``rr_batch_svd_tuned`` on a sample batch of that
class, on the GPU it runs on, and keeps the fastest: the number of concurrent
graph branches, the cap on each tensor-core product's K splits (a product that
would fill the GPU alone shares it with the other branches) and the launch
order.  The table persists as JSON keyed by "m-class,n-class,dtype".
``batch_svd`` then runs each class of a batch with its tuned parameters.
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

from . import api

DEFAULT = {"branches": 16, "max_splits": 0, "order": 0}
CANDIDATES = [{"branches": b, "max_splits": c, "order": o}
              for b in (8, 16, 32) for c in (0, 1, 4) for o in (0, 1)]


def size_class(m: int, n: int, dtype: str = "bf16") -> str:
    """Power-of-two bins of m and n: "9,7,bf16" holds 512 <= m < 1024, 128 <= n < 256."""
    return f"{int(math.log2(max(m, 1)))},{int(math.log2(max(n, 1)))},{dtype}"


def _time(ops, params, seed, tuning, reps):
    """Median wall time of `reps` batch launches (graph capture and instantiation
    included, as a caller pays them) after one warm-up, and the pairs converged."""
    api.rr_batch_svd(ops, params, seed, tuning=tuning)
    times = []
    conv = 0
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, infos = api.rr_batch_svd(ops, params, seed, tuning=tuning)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        conv = sum(i["n_converged"] for i in infos)
    times.sort()
    return times[len(times) // 2], conv


def tune(samples, params, dtype="bf16", candidates=None, reps=3, seed=1, log=None):
    """samples: {class key: list of rr_operator} (each list a representative batch of
    that class).  Returns the table {class key: {branches, max_splits, order, ms,
    default_ms}}.  A candidate must converge at least as many pairs as the defaults
    (the sweep count is fixed in batch mode, so launch parameters should not change
    it; the check guards against any that would)."""
    table = {}
    for key, ops in samples.items():
        t_def, c_def = _time(ops, params, seed, DEFAULT, reps)
        best = (t_def, DEFAULT)
        for cand in candidates or CANDIDATES:
            t, c = _time(ops, params, seed, cand, reps)
            if log:
                log(f"{key} {cand} {1e3 * t:.2f} ms, {c} pairs")
            if c >= c_def and t < best[0]:
                best = (t, cand)
        chosen = dict(best[1])
        chosen["ms"] = 1e3 * best[0]
        chosen["default_ms"] = 1e3 * t_def
        table[key] = chosen
    return table


def save(table, path):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path=None):
    """A saved table; without a path, the table tuned on a GB300 that ships with
    the package (``tuning_gb300.json``, written by ``bench.py --stage batch --table``)."""
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
    with open(path) as f:
        return json.load(f)


def batch_svd(ops, params, seed, table=None, dtype="bf16"):
    """The batch split by size class, each class in one graph launch with its tuned
    parameters (the defaults for classes the table lacks).  Returns the outputs,
    statuses and infos in the order of ``ops``."""
    groups = {}
    for i, op in enumerate(ops):
        groups.setdefault(size_class(op.m, op.n, dtype), []).append(i)
    outs, st, infos = [None] * len(ops), [None] * len(ops), [None] * len(ops)
    for key, idx in groups.items():
        tuning = (table or {}).get(key)
        tuning = {k: tuning[k] for k in ("branches", "max_splits", "order")} if tuning else DEFAULT
        o, s, inf = api.rr_batch_svd([ops[i] for i in idx], params, seed + idx[0], tuning=tuning)
        for j, i in enumerate(idx):
            outs[i], st[i], infos[i] = o[j], s[j], inf[j]
    return outs, st, infos
