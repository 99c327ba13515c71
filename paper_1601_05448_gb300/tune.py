"""Autotuner for the solver's work decomposition.

For a grid size and precision it times a fixed number of Krylov iterations of a real solve
(the caller's density and right-hand side) for a set of candidate layouts -- the stencil sweep
variant (direct register march or TMA-staged pipeline), threads per unit (which fixes the row
tile), number of work units (z chunks), pipeline stages, and launch pairs per host check -- and
keeps the fastest.  Results are cached in a JSON file keyed by device name, grid and precision
($VDP_TUNE_CACHE, default ~/.cache/paper_1601_05448_gb300/tune.json).

The chosen options change only how the work is split, not what is computed; but the split fixes
the order of the partial sums, so results are bitwise reproducible for a fixed tuned layout
(the batch engine relies on each member keeping its own layout).
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import PRECISIONS, Solver, VdpError

_lock = threading.Lock()
TUNABLE = ("stencil", "threads", "units", "stages", "tile_y", "steps_per_sync")


def cache_path() -> str:
    return os.environ.get("VDP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_1601_05448_gb300", "tune.json"))


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def _key(nx, ny, nz, precision, batchable=False) -> str:
    return f"{_device_name()}|{nx}x{ny}x{nz}|{precision}" + ("|batch" if batchable else "")


def _load_cache() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(key: str, entry: dict) -> None:
    with _lock:
        data = _load_cache()
        data[key] = entry
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def cached_options(nx: int, ny: int, nz: int, precision: str, batchable: bool = False):
    """Tuned options for this grid and precision (batchable: for batch members), or None."""
    e = _load_cache().get(_key(nx, ny, nz, precision, batchable))
    return dict(e["options"]) if e else None


def _direct_threads(nx: int, precision: str):
    v = 2 if precision == "fp64" else 4
    tpr = nx // v
    unit = tpr // math.gcd(tpr, 32) * 32
    out = []
    for t in (256, 192, 128, 96, 64):
        if t % unit == 0 and t >= unit and t not in out:
            out.append(t)
    return out[:2]


def candidates(nx: int, ny: int, nz: int, precision: str, batchable: bool = False):
    """Candidate option sets (zero = the library's automatic choice).  Batch members run the
    direct stencil sweep and the batch's own launch schedule, so `batchable` keeps only the
    direct-sweep splits."""
    cands = []
    for t in _direct_threads(nx, precision):
        for units in (0, 608, 1216, 2432):
            cands.append({"stencil": 0, "threads": t, "units": units})
    if batchable:
        return cands
    for stages in (4, 6):
        cands.append({"stencil": 1, "stages": stages})
    for sps in (8, 32):
        cands.append({"stencil": 0, "steps_per_sync": sps})
    return cands


def time_options(nx, ny, nz, L, rho, f, precision, options, iters=40, reps=2) -> float:
    """Milliseconds per Krylov iteration with `options` (inf if the layout cannot run)."""
    import torch
    try:
        with Solver(nx, ny, nz, L, precision=precision, max_iter=iters, **options) as s:
            s.set_density(rho)
            p = torch.empty_like(f)
            best = float("inf")
            for _ in range(reps + 1):
                st = s.solve(f, p, 1e-30, check=False)
                if st.iters > 0:
                    best = min(best, st.ms / st.iters)
            return best
    except VdpError:
        return float("inf")


def tune(nx: int, ny: int, nz: int, L: float, rho, f, precision: str = "mixed", iters: int = 40,
         use_cache: bool = True, verbose: bool = False, batchable: bool = False) -> dict:
    """Pick the fastest layout for this grid/precision; returns the options (cached).
    batchable: only layouts a batch member can use (vdp_batch_add accepts them)."""
    assert precision in PRECISIONS
    key = _key(nx, ny, nz, precision, batchable)
    if use_cache:
        e = _load_cache().get(key)
        if e:
            return dict(e["options"])
    results = []
    for opt in candidates(nx, ny, nz, precision, batchable):
        ms = time_options(nx, ny, nz, L, rho, f, precision, opt, iters=iters)
        results.append((ms, opt))
        if verbose:
            print(f"tune {key} {opt}: {ms * 1e3:.1f} us/iter")
    results.sort(key=lambda t: t[0])
    best_ms, best = results[0]
    _store(key, {"options": best, "us_per_iter": best_ms * 1e3,
                 "tried": [{"options": o, "us_per_iter": (m * 1e3 if math.isfinite(m) else None)} for m, o in results]})
    return dict(best)
