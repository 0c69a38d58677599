"""Launch-shape autotuner for the local update (an addition: the paper has no counterpart).

For each (form, chi, d) bucket it times one Trotter layer of a seeded synthetic saturated
state for every candidate launch shape and keeps the fastest:
  * "max_slots": local updates in flight per batch (how many triples share each grouped
    launch and each cooperative reduction), and
  * "panel_blocks": blocks per SM of the tridiagonal reduction's cooperative grid.
Neither changes the arithmetic or its order (results are bitwise the same for every
choice), only how the work is cut into launches.  The table is written as JSON and read
back by `tuned_options` (or `TEBD(..., tuning=...)` through `apply_tuning`).

    python -m paper_2401_05301_gb300.autotune --out tuning.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

SLOTS = (4, 8, 16, 24)
PANEL_BLOCKS = (1, 2, 3)
BUCKETS = (("dense", 64, 4), ("dense", 128, 4), ("dense", 256, 4), ("dense", 256, 5),
           ("u1", 256, 5), ("u1", 512, 5), ("u1", 1024, 5))


def _state(form: str, L: int, d: int, chi: int, seed: int):
    # seeded synthetic inputs live in the repository's input module (no part of the method)
    import workloads
    if form == "u1":
        return workloads.synthetic_state_u1(L, d, chi, L // 2, seed=seed)
    B, lam, _ = workloads.synthetic_state(L, d, chi, seed=seed)
    return B, lam, None


def _time_layer(form, L, d, chi, state, slots, pblocks, reps=2):
    import torch
    from .binding import TEBD
    B, lam, q = state
    g = TEBD(L, d - 1, chi, 3.0, 1.0, 0.1, 0.003, (L + 1) / 2, 0.005, precision=1, u1=(form == "u1"))
    g.set_option("max_slots", slots)
    g.set_option("panel_blocks", pblocks)
    g.set_state(B, lam)
    if q is not None:
        g.set_charges(q)
    g.layer(0, False)  # warm-up: workspace and arenas
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        g.set_state(B, lam)
        if q is not None:
            g.set_charges(q)
        torch.cuda.synchronize()
        t = time.perf_counter()
        g.layer(0, False)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
    g.close()
    return best


def tune(buckets=BUCKETS, L: int = 16, seed: int = 240105301):
    import torch
    out = {"device": torch.cuda.get_device_name(0), "layer": f"layer A of an L={L} synthetic saturated state, "
           "precision 1", "buckets": []}
    for form, chi, d in buckets:
        state = _state(form, L, d, chi, seed)
        trials = []
        for slots in SLOTS:
            for pb in PANEL_BLOCKS:
                trials.append((_time_layer(form, L, d, chi, state, slots, pb), slots, pb))
        t, slots, pb = min(trials)
        default = next(x for x in trials if x[1] == 24 and x[2] == 3)[0]
        out["buckets"].append({"form": form, "chi": chi, "d": d, "max_slots": slots, "panel_blocks": pb,
                               "layer_ms": 1e3 * t, "default_layer_ms": 1e3 * default,
                               "trials_ms": {f"{s}x{p}": 1e3 * x for x, s, p in trials}})
    return out


def tuned_options(table: dict, form: str, chi: int, d: int) -> dict:
    """The options of the bucket nearest to (form, chi, d): same form, the same d if any,
    then the nearest chi on a log scale.  Empty if the table has no bucket of that form."""
    cand = [b for b in table.get("buckets", []) if b["form"] == form]
    if not cand:
        return {}
    same_d = [b for b in cand if b["d"] == d]
    cand = same_d or cand
    b = min(cand, key=lambda x: abs(np.log(x["chi"]) - np.log(max(chi, 1))))
    return {"max_slots": b["max_slots"], "panel_blocks": b["panel_blocks"]}


def apply_tuning(sim, table: dict, form: str, chi: int, d: int):
    """Set the tuned launch options on a fresh handle (before its first step)."""
    for k, v in tuned_options(table, form, chi, d).items():
        sim.set_option(k, v)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="tuning.json")
    ap.add_argument("--L", type=int, default=16)
    args = ap.parse_args()
    table = tune(L=args.L)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    for b in table["buckets"]:
        print(f"{b['form']:5s} chi={b['chi']:5d} d={b['d']}: max_slots={b['max_slots']:2d} "
              f"panel_blocks={b['panel_blocks']}  {b['layer_ms']:.1f} ms (default {b['default_layer_ms']:.1f} ms)")


if __name__ == "__main__":
    main()
