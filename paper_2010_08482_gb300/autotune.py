"""Launch-configuration autotuner for the trace kernels.

The kernels expose a few launch choices through ``ctq_eval_opts`` (see
``include/ctq.h``): threads per CTA and resident CTAs per SM of the FP64
kernel, resident CTAs per SM of the small-block tensor-core kernel, and the
pipeline depth and tile order of the large-block kernel.  ``tune()`` times
every candidate on the caller's own batch with CUDA events on the launching
stream and keeps the fastest; results are cached in a JSON file keyed by the
GPU, the impurity's sector structure, the precision and the batch shape, so a
workload is tuned once per machine.

The timing loop and cache are host logic; every candidate runs the same
library kernels (there is no alternative code path), so a tuned
configuration changes speed only -- results agree to the rounding of the
changed reduction order.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Iterable, List, Optional

from . import ctq

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ctq_autotune.json")


def engine(imp: "ctq.Impurity", precision: int) -> str:
    """Which trace kernel a (impurity, precision) pair runs on (the
    library's own choice when the impurity has a device copy)."""
    try:
        k = ctq.trace_kernel(imp, precision)
        return {ctq.KERNEL_FP64_SHARED: "fp64", ctq.KERNEL_FP64_LARGE: "fp64big",
                ctq.KERNEL_TC_SMALL: "tc", ctq.KERNEL_TC_LARGE: "big"}[k]
    except ctq.CtqError:  # host-only impurity: the same rule from the sector sizes
        if precision == ctq.FP64:
            return "fp64"
        return "big" if (imp.is_complex or imp.max_dim > 112) else "tc"


def candidates(imp: "ctq.Impurity", precision: int) -> List[Dict[str, int]]:
    """Launch configurations worth timing for this kernel (the first is the
    library default)."""
    eng = engine(imp, precision)
    out: List[Dict[str, int]] = [{}]
    if eng == "fp64":
        for threads in (32, 64, 128, 256, 512):
            if threads < 32 * ((imp.max_dim + 31) // 32):
                continue  # fewer threads than rows of the largest block
            for cap in (0, 8, 4):
                if threads * max(cap, 1) > 2048:
                    continue
                out.append({"threads_per_cta": threads, "ctas_per_sm": cap})
    elif eng == "fp64big":
        for order in (2, 3):  # row-major, groups of 8 column tiles (the default is column-major)
            out.append({"tile_order": order})
    elif eng == "tc":
        if precision != ctq.TF32X3:  # 3xTF32 holds all tensor memory: one CTA per SM
            out.append({"ctas_per_sm": 1})
    else:
        stages = (2, 3) if precision != ctq.TF32 else (2, 3, 4)  # deeper pipelines are refused if they do not fit
        for st in stages:
            for order in (0, 1, 3):  # default (row-major), column-major, groups of 8 column tiles
                out.append({"stages": st, "tile_order": order})
    # drop duplicates of the default, keep order
    seen, uniq = set(), []
    for c in out:
        key = tuple(sorted((k, v) for k, v in c.items() if v))
        if key in seen:
            continue
        seen.add(key)
        uniq.append({k: v for k, v in c.items() if v})
    return uniq


def cache_key(imp: "ctq.Impurity", precision: int, n_chains: int, max_ops: int, segment: int, lazy: bool,
              device_name: str) -> str:
    """Stable key: GPU, sector structure of the impurity, precision and the
    batch shape (chain count and longest chain rounded up to powers of two)."""
    dims, _, _, s = imp.sectors()
    h = hashlib.sha256()
    h.update(repr((list(map(int, dims)), [int(x) for x in s.ravel()], bool(imp.is_complex))).encode())
    shape = (1 << max(0, int(n_chains - 1).bit_length()), 1 << max(0, int(max_ops - 1).bit_length()))
    return f"{device_name}|{h.hexdigest()[:16]}|p{precision}|c{shape[0]}|o{shape[1]}|S{segment}|L{int(lazy)}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(imp: "ctq.Impurity", db: "ctq.DeviceBatch", precision: int, segment: int = 8, lazy: bool = False,
         reps: int = 3, cache_path: Optional[str] = DEFAULT_CACHE, cands: Optional[Iterable[dict]] = None,
         verbose: bool = False) -> Dict[str, int]:
    """Fastest launch configuration for evaluating `db` on `imp`.  Each
    candidate runs once untimed, then `reps` times between CUDA events on the
    current stream; the minimum counts.  With a cache path, a previous
    result for the same key is returned without timing."""
    import torch
    key = cache_key(imp, precision, db.n_chains, db.max_ops, segment, lazy, torch.cuda.get_device_name())
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache and "best" in cache[key]:
        return dict(cache[key]["best"])
    stream = torch.cuda.current_stream()
    timings = []
    for cand in (list(cands) if cands is not None else candidates(imp, precision)):
        ev = ctq.TraceEvaluator(imp, db.n_chains, max(1, db.max_ops), precision=precision, segment=segment,
                                tune=cand)
        try:
            ev(db, lazy=lazy)
        except RuntimeError:
            continue  # a configuration this launch cannot take (CTQ_ERR_UNSUPPORTED)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ev(db, lazy=lazy)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        timings.append((best, cand))
        if verbose:
            print(f"autotune {engine(imp, precision)} {cand}: {best:.3f} ms")
    if not timings:
        raise RuntimeError("no launch configuration ran")
    timings.sort(key=lambda x: x[0])
    best_ms, best = timings[0]
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"best": best, "ms": best_ms,
                      "timings": [{"ms": t, "tune": c} for t, c in timings]}
        save_cache(cache_path, cache)
    return dict(best)
