"""Cache of measured per-class-pair schedules (fock_autotune).

A schedule is measured once per workload shape and GPU and kept in a JSON
file: the key is the GPU name, the precision options, the threshold and the
shell composition of every molecule (counts of shells by angular momentum and
contraction degree, and the basis size), so that other geometries of the same
molecules reuse it.  The measurement itself runs in the library.
"""
from __future__ import annotations

import hashlib
import json
import os
from collections import Counter

from . import fock


def workload_key(bases, schwarz_thresh: float, opts: fock.fock_opts | None, device_name: str) -> str:
    o = opts if opts is not None else fock.make_opts()
    comp = []
    for b in bases:
        c = Counter((int(l), int(k)) for l, k in zip(b["l"], b["nprim"]))
        nbf = sum((int(l) + 1) * (int(l) + 2) // 2 for l in b["l"])
        comp.append([nbf, sorted([list(k), v] for k, v in c.items())])
    desc = {"gpu": device_name, "precision": int(o.precision), "fp32_cutoff": float(o.fp32_cutoff),
            "prune_eps": float(o.prune_eps), "warp_scratch": int(o.warp_scratch), "reg_max_L": int(o.reg_max_L),
            "tau": float(schwarz_thresh), "molecules": comp}
    return hashlib.sha1(json.dumps(desc, sort_keys=True).encode()).hexdigest()


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_opts(bases, Ds, schwarz_thresh: float, opts: fock.fock_opts | None = None, cache: str | None = None,
               reps: int = 3, stream=None, device_name: str | None = None):
    """Options with a measured schedule for this workload: from `cache` when
    it holds the key, else measured by fock_autotune (and stored there).
    Returns (opts, record) with record = {"ms_base", "ms_tuned", "schedule",
    "cached"}.  device_name: the key's GPU name (default: the current
    device's)."""
    base = opts if opts is not None else fock.make_opts()
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    key = workload_key(bases, schwarz_thresh, base, device_name)
    db = _load(cache) if cache else {}
    if key in db:
        rec = db[key]
        out = fock.fock_opts.from_buffer_copy(base)
        out.tune_isolate = 0
        for i in range(fock.NCLASS * fock.NCLASS):
            out.schedule[i] = 0
        for k, v in rec["schedule"].items():
            c1, c2 = (int(x) for x in k.split(","))
            out.schedule[c1 * fock.NCLASS + c2] = int(v)
        return out, dict(rec, cached=True)
    out, ms, pair = fock.fock_autotune(bases, Ds, schwarz_thresh, base, reps, stream)
    rec = {"ms_base": ms[0], "ms_tuned": ms[1],
           "schedule": {f"{a},{b}": v for (a, b), v in fock.schedule_of(out).items()},
           "pair_ms_base": {f"{a},{b}": v for (a, b), v in pair.items()}}
    if cache:
        db = _load(cache)
        db[key] = rec
        d = os.path.dirname(os.path.abspath(cache))
        os.makedirs(d, exist_ok=True)
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return out, dict(rec, cached=False)
