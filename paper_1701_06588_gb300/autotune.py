"""Autotuner for the launch shape of two-center plans.

Candidates: schedule (one launch per class, or one persistent launch with
tiles in decreasing estimated cost), threads per CTA (1, 2 or 4 warps, each
warp owning a class-pure tile of up to 32 pairs), persistent CTAs per SM and,
for the double-float fused pass, the compiled kernel variant (register count
left to the compiler, or capped for one more resident CTA per SM).
Each candidate runs the requested operators a few times (CUDA events, after a
warm-up); the fastest is cached in a JSON file keyed by GPU name, precision,
operators and a signature of the workload's (la, lb, Ka*Kb) histogram.
The cache path is $SHG_AUTOTUNE_CACHE, else ~/.cache/shg_gb300/autotune.json.
"""
import hashlib
import json
import os

import numpy as np
import torch

from . import api

CANDIDATES = ([("per_class", t, 0) for t in (32, 64, 128)] +
              [("persistent", t, c) for t in (32, 64, 128) for c in (0, 1, 2, 4, 8)])
VARIANTS = {"mixed_fused": (0, 1, 2), "fp64_fused": (0, 1, 2)}


def cache_path():
    return os.environ.get("SHG_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "shg_gb300",
                                                                 "autotune.json")


def workload_signature(basis, pair_a, pair_b):
    l = basis.l.astype(np.int64)
    k = basis.nprim.astype(np.int64)
    key = (l[pair_a] * 7 + l[pair_b]) * 1024 + np.minimum(k[pair_a] * k[pair_b], 1023)
    hist = np.bincount(key, minlength=49 * 1024)
    return hashlib.sha256(hist.astype(np.int64).tobytes()).hexdigest()[:16]


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(db):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def tune_2c(basis, pair_a, pair_b, ops, omegas, out_offsets, outs, precision="fp64", reps=3, force=False):
    """Best (schedule, threads_per_cta, ctas_per_sm) for this workload; times in ms per pass over `ops`.
    precision "fp64_fused" / "mixed_fused" tunes the fused multi-operator pass (one exec_fused per pass)."""
    fused = precision.endswith("_fused")

    def one_pass(plan):
        if fused:
            plan.exec_fused(ops, out_offsets, outs, omegas=omegas, precision=precision[:-len("_fused")])
        else:
            for op, om, o in zip(ops, omegas, outs):
                plan.exec(op, out_offsets, o, omega=om, precision=precision)

    key = "|".join(["v3", torch.cuda.get_device_name(), precision, ",".join(map(str, ops)),
                    workload_signature(basis, pair_a, pair_b)])
    db = _load()
    if not force and key in db:
        return db[key]
    results = []
    plans = {}
    for sched, threads, ctas in CANDIDATES:
        if sched not in plans:
            plans[sched] = api.Plan2c(basis, pair_a, pair_b, schedule=sched)
        plan = plans[sched]
        for variant in VARIANTS.get(precision, (0,)):
            api.set_launch(plan, threads, ctas, variant)
            one_pass(plan)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                one_pass(plan)
            e1.record()
            torch.cuda.synchronize()
            results.append((e0.elapsed_time(e1) / reps, sched, threads, ctas, variant))
    for p in plans.values():
        p.close()
    results.sort()
    ms, sched, threads, ctas, variant = results[0]
    best = {"schedule": sched, "threads_per_cta": threads, "ctas_per_sm": ctas, "variant": variant, "ms": ms,
            "candidates": [{"ms": r[0], "schedule": r[1], "threads_per_cta": r[2], "ctas_per_sm": r[3],
                            "variant": r[4]} for r in results]}
    db[key] = best
    _save(db)
    return best


def tuned_plan(basis, pair_a, pair_b, config):
    plan = api.Plan2c(basis, pair_a, pair_b, schedule=config["schedule"])
    api.set_launch(plan, config["threads_per_cta"], config["ctas_per_sm"], config.get("variant", 1))
    return plan
