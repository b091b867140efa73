"""Tile-shape autotuner for the 2D stage kernel.

The tile of a warp is 28 output columns by H rows; a thread block holds W warps. Both change only
the schedule, never the result. For a configuration (degree, equation, precision, mesh size) the
tuner times a few SSP-RK3 steps of a scratch solver for each candidate (H, W) with CUDA events and
keeps the fastest; results are cached in a JSON file keyed by device and configuration.
"""
from __future__ import annotations

import json
import os

from . import _native as N
from . import inputs as I

CACHE = os.environ.get("DGJF_TILE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "paper_2407_19169_gb300", "tiles.json"))
H_CANDIDATES = (8, 16, 32, 64, 128)
W_CANDIDATES = (2, 4, 8)


def _key(device_name, k, eq, precision, nx, ny):
    return "%s|k%d|eq%d|prec%d|%dx%d" % (device_name, k, eq, precision, nx, ny)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_2d(nx, ny, k=2, eq=N.EQ_EULER, precision=N.PREC_FP32_MIXED, steps=3, use_cache=True):
    """Best (tile_rows, tile_warps) for a 2D mesh; times `steps` steps per candidate."""
    import torch

    dev = torch.cuda.get_device_name()
    key = _key(dev, k, eq, precision, nx, ny)
    db = _load() if use_cache else {}
    if key in db:
        return tuple(db[key]["best"])
    stream = torch.cuda.Stream()
    results = {}
    for H in H_CANDIDATES:
        if H > ny:
            continue
        for W in W_CANDIDATES:
            s = N.Solver(dim=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(N.BC_OUTFLOW,) * 4, k=k,
                         eq=eq, precision=precision, stream=stream.cuda_stream, tile_rows=H, tile_warps=W)
            if eq == N.EQ_EULER:
                s.set_initial(N.IC_QUADRANT2D, I.quadrant_params(1))
            else:
                s.set_initial(N.IC_SINE, [0.5, 1.0, 6.283185307179586, 0.0])
            s.advance_steps(1)
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.advance_steps(steps)
            e1.record(stream)
            stream.synchronize()
            st = s.sync()[0]
            s.close()
            if st == 0:
                results["%d,%d" % (H, W)] = e0.elapsed_time(e1) / steps
    best = min(results, key=results.get)
    H, W = (int(x) for x in best.split(","))
    if use_cache:
        db = _load()
        db[key] = {"best": [H, W], "ms_per_step": results}
        _store(db)
    return H, W
