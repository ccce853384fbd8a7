"""Autotuner of the accumulator geometry: hash-table load factors (table
sizes), the team width rule (vector walk for long B rows, flattened walk for
short ones), the window tier, and the bin thresholds that send rows to the
team, CTA and dense tiers (symbolic: by flop bound; numeric: by nnz(C(i,:))),
searched per matrix family on training matrices (seeded families disjoint from
the evaluation inputs) and persisted per device as JSON.

The search times the plain two-phase path (or the batched form for the
``batch`` family) through the C ABI with CUDA events.  The space is the
product of the axes below, too large to time whole, so it is searched by
coordinate descent: from the library's defaults, each axis in turn is set to
its fastest value with the others held, for a few rounds or until no axis
changes.  ``tuned_options(family)`` returns the stored choice (or {}).
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
    "sym_team_max_flop": [1536, 3072, 6144],
    "sym_cta_max_flop": [12288, 24576, 49152],
    "num_team_max_nnz": [512, 1024, 2048],
    "num_cta_max_nnz": [2048, 4096, 8192],
}
# the library's defaults (kk_spgemm_options_default), the descent's start
DEFAULTS = {"team_vec_min_len": 12, "sym_load_pct": 75, "num_load_pct": 50, "use_window": 1,
            "sym_team_max_flop": 3072, "sym_cta_max_flop": 24576, "num_team_max_nnz": 1024,
            "num_cta_max_nnz": 4096}


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


def _valid(c: dict) -> bool:
    """Threshold orders the library requires (team below CTA)."""
    return (c.get("sym_team_max_flop", 0) < c.get("sym_cta_max_flop", 1 << 30) and
            c.get("num_team_max_nnz", 0) < c.get("num_cta_max_nnz", 1 << 30))


def tune_family(family: str, space=None, reps: int = 3, rounds: int = 2, start=None):
    """Coordinate descent over ``space`` from ``start`` (the defaults restricted
    to the space's axes).  Returns (best options, {str(options): ms}) with every
    timed candidate."""
    space = space or SPACE
    keys = list(space)
    cur = {k: (start or DEFAULTS).get(k, space[k][0]) for k in keys}
    for k in keys:
        if cur[k] not in space[k]:
            cur[k] = space[k][0]
    probs = training_problems(family)
    results = {}
    if family == "batch":
        pairs = probs[0][1]
        dAs = [K.DeviceCSR.from_host(A) for A, _ in pairs]
        dBs = [K.DeviceCSR.from_host(B) for _, B in pairs]

        def cost(c):
            return _time_batched(dAs, dBs, c, reps)
    else:
        dev = [(K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)) for A, B in probs]

        def cost(c):
            return sum(_time_plain(a, b, c, reps) for a, b in dev)

    def timed(c):
        key = json.dumps(c, sort_keys=True)
        if key not in results:
            results[key] = cost(c)
        return results[key]

    best_ms = timed(cur)
    for _ in range(rounds):
        changed = False
        for k in keys:
            for v in space[k]:
                cand = dict(cur, **{k: v})
                if cand == cur or not _valid(cand):
                    continue
                ms = timed(cand)
                if ms < best_ms:
                    best_ms, cur, changed = ms, cand, True
        if not changed:
            break
    return cur, results


def tune_all(families=("stencil3d", "stencil2d", "rmat", "amg", "batch"), path=None):
    out = {}
    for f in families:
        best, res = tune_family(f)
        out[f] = {"options": best, "ms": res[json.dumps(best, sort_keys=True)],
                  "default_ms": res.get(json.dumps({k: DEFAULTS[k] for k in SPACE}, sort_keys=True)),
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
