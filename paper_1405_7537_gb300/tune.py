"""Autotuner for the launch shape of the solve kernels (lanes per eigenvalue, warps per
block, blocks per SM).

The best shape depends on the problem sizes: small problems want narrow lane groups
(few terms per lane, short reductions), large ones want whole warps.  ``tune`` times
every candidate shape with CUDA events on a sample batch drawn from the caller's size
distribution and caches the winner in ``_lib/tune_cache.json`` under a key made of the
size histogram (log2 buckets) and the GPU name, so later calls with a similar size mix
reuse it.
"""
import json
import os
import time

import numpy as np
import torch

from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")
CANDIDATES = [(l, w, b) for l in (8, 16, 32) for w in (4, 8) for b in ((1, 2, 4) if w == 8 else (1, 2, 4, 8))]


def size_key(sizes, zero_finder=0):
    sizes = np.asarray(sizes, dtype=np.int64)
    sizes = sizes[sizes > 0]
    if sizes.size == 0:
        return "empty"
    h = np.bincount(np.minimum(np.log2(sizes).astype(int), 20), minlength=21)
    frac = np.round(h / h.sum(), 1)
    return "%s|zf%d|%s" % (torch.cuda.get_device_name(), zero_finder, ",".join("%g" % f for f in frac))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)


def _sample_batch(sizes, max_total, rng):
    sizes = np.asarray(sizes, dtype=np.int64)
    if sizes.sum() <= max_total:
        pick = sizes
    else:
        pick = []
        tot = 0
        for s in rng.permutation(sizes):
            if tot + s > max_total:
                break
            pick.append(s)
            tot += s
        pick = np.array(pick if pick else [min(int(sizes.max()), max_total)], dtype=np.int64)
    ds, zs = [], []
    for n in pick:
        d = np.sort(rng.uniform(-1, 1, int(n)))[::-1]
        while np.any(np.diff(d) >= 0):
            d = np.sort(rng.uniform(-1, 1, int(n)))[::-1]
        ds.append(d)
        zs.append(rng.uniform(-1, 1, int(n)))
    return pick, np.concatenate(ds), np.concatenate(zs), rng.uniform(0.1, 10, pick.size)


def tune(sizes, device="cuda", max_total=200_000, reps=2, force=False, verbose=False, zero_finder=0):
    """Returns (lanes, warps_per_block, blocks_per_sm) for this size distribution and zero finder
    (the accelerated solve does a few evaluations per eigenvalue and prefers other shapes)."""
    key = size_key(sizes, zero_finder)
    cache = _load()
    if not force and key in cache:
        return tuple(cache[key]["shape"])
    rng = np.random.default_rng(12345)
    pick, d, z, rho = _sample_batch(sizes, max_total, rng)
    bt = B.Batch(pick, device=device, want_vectors=False)
    dt = torch.tensor(d, device=device)
    zt = torch.tensor(z, device=device)
    rt = torch.tensor(rho, device=device)
    best, best_ms, results = None, float("inf"), {}
    for shape in CANDIDATES:
        o = B.default_options(lanes=shape[0], warps_per_block=shape[1], blocks_per_sm=shape[2],
                              zero_finder=zero_finder)
        bt.solve(dt, zt, rt, options=o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            bt.solve(dt, zt, rt, options=o)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        results["%d/%d/%d" % shape] = ms
        if verbose:
            print("shape lanes=%d warps=%d blocks/SM=%d: %.3f ms" % (shape + (ms,)))
        if ms < best_ms:
            best, best_ms = shape, ms
    cache[key] = {"shape": list(best), "ms": best_ms, "sample_eigenpairs": int(pick.sum()), "all_ms": results,
                  "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    _store(cache)
    return best


def options_for(sizes, device="cuda", zero_finder=0, **kw):
    """dpr1_options with the tuned launch shape for this size distribution and zero finder."""
    l, w, b = tune(sizes, device=device, zero_finder=zero_finder, **kw)
    return B.default_options(lanes=l, warps_per_block=w, blocks_per_sm=b, zero_finder=zero_finder)
