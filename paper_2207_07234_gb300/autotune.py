"""Autotuner of the persistent batch launch (pdhg_batch_set_launch).

For a batch of 1D instances it times batch iterations on the GPU and chooses, by
coordinate descent, the resident blocks per multiprocessor of the persistent launch
the queue order and, for every size class present, the row items per queue entry (the
class of an instance is log2 of its row transform length - 8: the Bluestein length for
nx not a power of two, nx/2 otherwise), and compares the best persistent launch with
the four per-stage launches.  The choice is written to batch_tiles.json beside this
file; Batch (binding.py) applies it to every batch it creates.  Run on the GPU:

    python -m paper_2207_07234_gb300.autotune        # the 256-instance workload, float32
"""
from __future__ import annotations

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TILES_FILE = os.path.join(HERE, "batch_tiles.json")


def size_class(p) -> int:
    """The size class of one 1D instance (the rule of pdhg_batch_set_launch)."""
    nx = p.nx
    pow2 = nx > 0 and (nx & (nx - 1)) == 0
    if p.nmodes == 1 and not pow2:
        lg = math.ceil(math.log2(2 * nx - 1))              # Bluestein length
    else:
        lg = max(0, math.ceil(math.log2(max(nx // 2, 1))))
    return min(7, max(0, lg - 8))


def time_iterations(bt, iters, stream):
    import torch
    bt.iterate(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    bt.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def search(measure, present, candidates=(1, 2, 4, 8), blocks=(0, 1, 2, 3), orders=(0, 1), unsupported=()):
    """Coordinate descent over the launch choices, given measure(persistent,
    blocks_per_sm, order, tiles) -> ms per batch iteration: the per-stage launches
    once, then every (order, blocks per multiprocessor) of the persistent launch with
    untiled queue entries (a choice whose measure raises one of `unsupported` is
    skipped), then, at the best of those, each present size class's tile in turn,
    kept where it is faster.  Returns the choice dict without the timings."""
    tiles = [1] * 8
    per_stage = measure(False, 0, 0, tiles)
    best, best_bps, best_order = None, 0, 0
    for order in orders:
        for bps in blocks:
            try:
                ms = measure(True, bps, order, tiles)
            except unsupported:
                continue
            if best is None or ms < best:
                best, best_bps, best_order = ms, bps, order
    if best is None:                                       # no persistent form fits
        return {"persistent": False, "blocks_per_sm": 0, "order": 0, "tiles": tiles,
                "persistent_ms": None, "per_stage_ms": per_stage, "classes_present": list(present)}
    for c in present:
        for g in candidates:
            if g == tiles[c]:
                continue
            trial = list(tiles)
            trial[c] = g
            ms = measure(True, best_bps, best_order, trial)
            if ms < best:
                best, tiles = ms, trial
    return {"persistent": bool(best < per_stage), "blocks_per_sm": best_bps, "order": best_order, "tiles": tiles,
            "persistent_ms": best, "per_stage_ms": per_stage, "classes_present": list(present)}


def tune(problems, precision="fp32", iters=3, candidates=(1, 2, 4, 8), blocks=(0, 1, 2, 3), orders=(0, 1)):
    """Returns the chosen launch (the persistent one with its best blocks per
    multiprocessor, queue order and tiles, or the per-stage launches when those are
    faster) and every timing taken (ms per batch iteration)."""
    import torch
    from . import binding
    present = sorted({size_class(p) for p in problems})
    stream = torch.cuda.Stream()
    log = []
    with binding.Batch(problems, precision=precision, stream=stream) as bt:
        def run(persistent, bps, order, tiles):
            bt.set_launch(persistent=persistent, blocks_per_sm=bps, order=order, tiles=tiles)
            ms = time_iterations(bt, iters, stream)
            log.append({"persistent": persistent, "blocks_per_sm": bps, "order": order, "tiles": list(tiles),
                        "ms": ms})
            return ms
        res = search(run, present, candidates, blocks, orders, unsupported=(binding.PdhgError,))
    res["timings"] = log
    return res


def main(argv=None):
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TILES_FILE, help="where to write the choice (default: beside this file)")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    import pdhg_workloads as W
    from . import binding
    binding.load()
    if os.path.exists(TILES_FILE):
        os.environ["PDHG_BATCH_TILES"] = "none"          # tune from the untuned launch
    probs = W.batch_instances()
    res = tune(probs)
    res["workload"] = f"{len(probs)} mixed 1D instances (pdhg_workloads.batch_instances), float32"
    res["device"] = torch.cuda.get_device_name(0)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({k: v for k, v in res.items() if k != "timings"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
