"""Autotuner of the launch configuration of grp_step.

Candidates: the flat per-step kernel sequence; the split form (grid-wide flux
kernel + a per-domain-group kernel for update, repair and bookkeeping) with
threads per block x cells per block; and the fused persistent kernel with
threads x cells per block (the tile of whole domains a block owns) x steps per
launch (the temporal depth of one launch).  Each
candidate advances a copy of the caller's initial data for a few steps and is
timed on the device (stream-synchronised wall clock around the steps; the
kernels are FP64-bound and run for milliseconds, so the host clock suffices).
The winner is cached in a JSON file keyed by the GPU name and a signature of
the problem (system, degree, number of domains, cell-count histogram).  The
configuration never changes results, only speed.
"""
import hashlib
import json
import os
import time

import numpy as np

from . import grprec

CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "grprec_autotune.json")


def signature(prob):
    n = np.asarray(prob["n_cells"])
    hist = np.histogram(np.log2(np.maximum(n, 1)), bins=12, range=(0, 24))[0]
    key = "sys%d-M%d-D%d-cells%d-h%s-bc%d" % (prob["system"], prob["M"], len(n), int(n.sum()),
                                           hashlib.sha1(hist.tobytes()).hexdigest()[:8],
                                           int(np.asarray(prob["bc"]).sum()))
    return key


def gpu_name(device=0):
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return "cuda%d" % device


def candidates(prob):
    out = [(grprec.GRP_LAUNCH_FLAT, 256, 2048, 1)]
    if int(np.max(prob["n_cells"])) <= 1 << 16:
        for threads in (128, 256):
            for cells in (512, 2048, 8192):
                out.append((grprec.GRP_LAUNCH_SPLIT, threads, cells, 1))
        for threads in (128, 256):
            for cells in (1024, 4096):
                for k in (1, 16):
                    out.append((grprec.GRP_LAUNCH_FUSED, threads, cells, k))
    return out


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _time(s, avg, lim_minus, lim_plus, cfg, warm, steps):
    s.set_launch(*cfg)
    s.set_initial(avg, lim_minus, lim_plus)
    s.step(warm)                               # warm-up (graph capture, first-launch set-up)
    s.get_stats()
    t0 = time.perf_counter()
    s.step(steps)
    s.get_stats()                              # synchronises
    return (time.perf_counter() - t0) / steps


def tune(prob, avg, lim_minus, lim_plus, device=0, warm=16, steps=32, finalists=3, use_cache=True,
         verbose=False, solver=None):
    """Best (mode, threads, cells_per_block, steps_per_launch) for this problem.
    Every candidate runs `warm` steps, then `steps` timed steps, from the
    initial data; the `finalists` fastest run again for 2 x `steps` and the
    fastest of that round wins.  ``solver``: tune on this Solver (its guess
    model and settings) instead of a new one; its launch configuration is left
    at the winner and its state must be set again by the caller."""
    key = gpu_name(device) + "|" + signature(prob) + ("|guess%d" % int(prob.get("guess", 0)))
    cache = _load() if use_cache else {}
    if key in cache:
        best = tuple(cache[key]["config"])
        if solver is not None:
            solver.set_launch(*best)
        return best
    s = solver or grprec.Solver(prob, device=device)
    results = []
    for cfg in candidates(prob):
        dt = _time(s, avg, lim_minus, lim_plus, cfg, warm, steps)
        results.append((dt, cfg))
        if verbose:
            print("autotune %-28s %8.3f ms/step" % (cfg, 1e3 * dt))
    results.sort()
    final = []
    for dt0, cfg in results[:finalists]:
        dt = _time(s, avg, lim_minus, lim_plus, cfg, warm, 2 * steps)
        final.append((dt, cfg))
        if verbose:
            print("autotune final %-22s %8.3f ms/step" % (cfg, 1e3 * dt))
    best_dt, best = min(final)
    if solver is None:
        s.close()
    else:
        solver.set_launch(*best)
    if use_cache:
        cache = _load()
        cache[key] = {"config": list(best), "ms_per_step": 1e3 * best_dt}
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            with open(CACHE + ".tmp", "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(CACHE + ".tmp", CACHE)
        except OSError:
            pass
    return best
