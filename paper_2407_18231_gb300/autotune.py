"""Launch-configuration autotuner.

Sweeps threads per block, resident blocks per SM (the size of the persistent grids) and
the LS work split (how many neighbour MDs a warp stages in shared memory; 1 = one warp per
MD everywhere) on a sample batch, times each point as the chain really runs (the captured
graph, with its second stream; median wall time of whole batches, so any overlap between
the streams counts), checks that every point returns bit-identical track candidates (the
configuration must never change results), and keeps the fastest.  The choice is cached
per device name in a JSON file.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import Session, lst_config  # noqa: F401

SPACE = {"block_size": [128, 256, 512], "blocks_per_sm": [2, 4, 8, 12], "ls_list_cap": [1, 128, 512, 1024]}
DEFAULT = {"block_size": 256, "blocks_per_sm": 4, "ls_list_cap": 512}


def _device_name(device: int) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:  # noqa: BLE001
        return "unknown"


def measure(sess: Session, events, reps: int = 3) -> tuple[float, bytes]:
    """Median wall time (ms) of the chain on `events` (graph replay) and the candidates' bytes."""
    ids = sess.run_batch(events)  # sizes the buffers and captures the graph
    ref = b"".join(sess.candidates(i).tobytes() for i in ids)
    for i in ids:
        sess.release(i)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ids = sess.run_batch(events)
        times.append((time.perf_counter() - t0) * 1e3)
        for i in ids:
            sess.release(i)
    return float(np.median(times)), ref


def tune(modules, events, *, device: int = 0, space=None, reps: int = 3, cache: str | None = None,
         log=None) -> dict:
    """Run the sweep; returns {"best": config, "table": [...], "device": name}."""
    space = space or SPACE
    sess = Session(modules, device=device)
    table = []
    ref = None
    for bs, bps, cap in itertools.product(space["block_size"], space["blocks_per_sm"], space["ls_list_cap"]):
        sess.set_tuning(bs, bps, cap)
        ms, out = measure(sess, events, reps)
        if ref is None:
            ref = out
        if out != ref:
            raise RuntimeError(f"configuration {bs}/{bps}/{cap} changed the track candidates")
        table.append({"block_size": bs, "blocks_per_sm": bps, "ls_list_cap": cap, "ms": ms})
        if log:
            log(f"block {bs:4d} blocks/SM {bps:2d} ls list {cap:4d}: {ms:.3f} ms")
    sess.close()
    best = min(table, key=lambda r: r["ms"])
    result = {"device": _device_name(device), "events": len(events),
              "best": {k: best[k] for k in ("block_size", "blocks_per_sm", "ls_list_cap")}, "table": table}
    if cache:
        db = json.load(open(cache)) if os.path.exists(cache) else {}
        db[result["device"]] = result
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return result


def cached(cache: str, device: int = 0) -> dict | None:
    """The cached best configuration for this device, if any."""
    if not os.path.exists(cache):
        return None
    rec = json.load(open(cache)).get(_device_name(device))
    return rec["best"] if rec else None
