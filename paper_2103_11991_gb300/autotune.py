"""Autotuner of the accumulator geometry: hash-table load factors (table
sizes), the team width rule (vector walk for long B rows, flattened walk for
short ones) and the tier thresholds, searched per matrix family on training
matrices (seeded families disjoint from the evaluation inputs) and persisted
per device as JSON.

The search times the plain two-phase path (or the batched form for the
``batch`` family) through the C ABI with CUDA events and keeps the fastest
option set.  ``tuned_options(family)`` returns the stored choice (or {}).
"""
from __future__ import annotations

import itertools
import json
import os

from . import inputs as I
from . import spgemm as K

PKG = os.path.dirname(os.path.abspath(__file__))
TUNED = os.path.join(PKG, "tuned")

SPACE = {
    "team_vec_min_len": [8, 12, 20],
    "sym_load_pct": [50, 75],
    "num_load_pct": [25, 50],
    "use_window": [0, 1],
}


def training_problems(family: str):
    """Training products of a family (sizes and seeds other than the evaluation ones)."""
    if family == "stencil3d":
        return [(A, A) for A in (I.stencil_3d(36, 36, 36, 27, 26.0, -1.0),
                                 I.stencil_3d(48, 48, 48, 7, 6.0, -1.0))]
    if family == "stencil2d":
        return [(A, A) for A in (I.stencil_2d(192, 192, 5), I.stencil_2d(160, 160, 9, 8.0))]
    if family == "rmat":
        return [(A, A) for A in (I.rmat(14, 16, seed=1500),)]
    if family == "amg":
        d = I.config_inputs("amg_galerkin_128", scale=48)
        return [(d["A"], d["P"])]
    if family == "batch":
        return [("batch", I.batch_pairs(60, seed0=9000, rows_lo=100, rows_hi=20000))]
    raise KeyError(family)


def _device_name():
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def _time_plain(dA, dB, opts, reps=3):
    import torch
    with K.SpGEMM(**opts) as op:
        rp, nnz = op.symbolic(dA, dB)
        ci, va = op.numeric(dA, dB, rp, nnz)
        op.sync()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            rp, nnz = op.symbolic(dA, dB)
            op.numeric(dA, dB, rp, nnz, ci, va)
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps


def _time_batched(dAs, dBs, opts, reps=3):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with K.BatchedSpGEMM(stream=stream, **opts) as op:
            rp, off, total = op.symbolic(dAs, dBs)
            ci, va = op.numeric(dAs, dBs, rp, total)
            op.sync()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            for _ in range(reps):
                rp, off, total = op.symbolic(dAs, dBs)
                op.numeric(dAs, dBs, rp, total, ci, va)
            e.record(stream)
            torch.cuda.synchronize()
            return s.elapsed_time(e) / reps


def tune_family(family: str, space=None, reps: int = 3):
    """Returns (best options, {str(options): ms})."""
    space = space or SPACE
    keys = list(space)
    combos = [dict(zip(keys, vals)) for vals in itertools.product(*(space[k] for k in keys))]
    probs = training_problems(family)
    results = {}
    if family == "batch":
        pairs = probs[0][1]
        dAs = [K.DeviceCSR.from_host(A) for A, _ in pairs]
        dBs = [K.DeviceCSR.from_host(B) for _, B in pairs]
        for c in combos:
            results[json.dumps(c, sort_keys=True)] = _time_batched(dAs, dBs, c, reps)
    else:
        dev = [(K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)) for A, B in probs]
        for c in combos:
            results[json.dumps(c, sort_keys=True)] = sum(_time_plain(a, b, c, reps) for a, b in dev)
    best = min(results, key=results.get)
    return json.loads(best), results


def tune_all(families=("stencil3d", "stencil2d", "rmat", "amg", "batch"), path=None):
    out = {}
    for f in families:
        best, res = tune_family(f)
        out[f] = {"options": best, "ms": res[json.dumps(best, sort_keys=True)],
                  "candidates": len(res)}
    os.makedirs(TUNED, exist_ok=True)
    path = path or os.path.join(TUNED, f"autotune_{_device_name()}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    return out, path


def tuned_options(family: str, path=None) -> dict:
    try:
        path = path or os.path.join(TUNED, f"autotune_{_device_name()}.json")
        with open(path) as fh:
            return dict(json.load(fh)[family]["options"])
    except Exception:
        return {}
