"""Launch-shape autotuner: times each candidate configuration of a system on
the device with CUDA events and keeps the fastest, caching the choice in a
JSON file keyed by GPU name and workload signature.

The knobs are launch shapes only (results do not depend on them): the
particles per cell tile (tile width in cells along x, `tile_target`), the
number of blocks of the persistent tile sweeps (`sweep_blocks`: 0 = as
many as fit at once, -1 = one block per tile, k > 0 = k blocks) and, for the
batched replicas, the one-launch step (its register bound) or the separate
calls with the force sweep's threads per block (`sweep_threads`: 128, 256,
512).  Tile width and block size together set the cells a warp covers
(reported as `cells_per_warp`).

Cache file: $FPM_AUTOTUNE_CACHE, else ~/.cache/fpm/autotune.json.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

import torch


def cache_path() -> str:
    p = os.environ.get("FPM_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "fpm", "autotune.json")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: tuning still works, it is just not remembered


def signature(obj) -> str:
    """A short stable hash of a JSON-able workload description."""
    return hashlib.sha1(json.dumps(obj, sort_keys=True).encode()).hexdigest()[:16]


def time_steps(step, steps: int, warmup: int) -> float:
    """Mean device milliseconds of step() over `steps` calls, after `warmup`."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(key: str, space: dict, apply, measure, use_cache: bool = True) -> dict:
    """Grid search over `space` (knob -> candidate values).  apply(config)
    puts a configuration in place; measure() returns its cost (lower is
    better).  Returns {"config", "ms", "trials", "cached", "seconds"} and
    leaves the best configuration applied."""
    path = cache_path()
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    full = f"{dev}|{key}|{signature(space)}"
    if use_cache:
        hit = _load(path).get(full)
        if hit is not None:
            apply(hit["config"])
            return {**hit, "cached": True, "seconds": 0.0}
    t0 = time.time()
    names = list(space)
    trials = []
    best = None
    for values in itertools.product(*(space[k] for k in names)):
        cfg = dict(zip(names, values))
        apply(cfg)
        ms = float(measure())
        trials.append({"config": cfg, "ms": ms})
        if best is None or ms < best["ms"]:
            best = {"config": cfg, "ms": ms}
    apply(best["config"])
    out = {"config": best["config"], "ms": best["ms"], "trials": trials}
    if use_cache:
        data = _load(path)
        data[full] = out
        _store(path, data)
    return {**out, "cached": False, "seconds": time.time() - t0}


def tune_batch(system, steps: int = 20, warmup: int = 5, tile_targets=(128, 170, 230, 300, 420),
               sweep_blocks=None, sweep_threads=(128, 256, 512), step_blocks=(0,), step_minb=(2, 3, 4),
               use_cache: bool = True) -> dict:
    """Tunes an LJBatch: tile_target (re-plans and rebuilds) x the launch
    shape, one of
      ["step", blocks, minb]     the one-launch step (fpm_batch_step) on
                                 `blocks` blocks (0: all that fit at once),
                                 its registers bounded for minb blocks per SM;
      ["split", blocks, threads] the four separate calls, the force sweep on
                                 `blocks` blocks of `threads` threads (a tile
                                 larger than the block takes more than one
                                 particle per thread; one much smaller leaves
                                 lanes idle)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if sweep_blocks is None:
        sweep_blocks = (0, -1, 2 * sms, 4 * sms)
    shapes = [["step", int(b), int(m)] for b in step_blocks for m in step_minb]
    shapes += [["split", int(b), int(t)] for b in sweep_blocks for t in sweep_threads]
    space = {"tile_target": list(tile_targets), "shape": shapes}
    key = "lj_batch:" + signature({"counts": list(system.counts), "L": [round(float(L[0]), 6) for L in system.L],
                                   "r_list": system.r_list, "cap": system.cap})

    def apply(cfg):
        mode, blocks, third = cfg["shape"]
        if cfg["tile_target"] != system.tile_target:
            system.plan(cfg["tile_target"], blocks)
        system.fused = mode == "step"
        system.set_sweep_blocks(blocks)
        system.set_sweep_threads(0 if mode == "step" else third)
        system.set_step_blocks_per_sm(third if mode == "step" else 0)

    def measure():
        return time_steps(system._step, steps, warmup)

    out = tune(key, space, apply, measure, use_cache)
    # cells of the tile per warp of the chosen block: the tiles' mean width
    # in cells over the warps of a block
    widths = [int(system.reps[r].grid.nc[0]) / max(1, int(system.reps[r].grid.tiles_x)) for r in range(system.R)]
    threads = (out["config"]["shape"][2] or 256) if out["config"]["shape"][0] == "split" else 256
    out["cells_per_warp"] = (sum(widths) / len(widths)) / (threads / 32)
    return out


def tune_system(system, steps: int = 20, warmup: int = 5, cells_per_tile=(6, 8, 10, 13), sweep_blocks=(0, -1),
                use_cache: bool = True) -> dict:
    """Tunes an LJSystem: cells per tile along x (re-tiles and rebuilds) x
    sweep blocks, timing whole steps."""
    nc0 = int(system.grid.nc[0])
    tiles = sorted({max(1, -(-nc0 // int(w))) for w in cells_per_tile})
    space = {"tiles_x": tiles, "sweep_blocks": list(sweep_blocks)}
    key = "lj_system:" + signature({"n": system.n, "L": [float(x) for x in system.L], "r_list": system.r_list,
                                    "prec": system.prec})

    def apply(cfg):
        if cfg["tiles_x"] != system.grid.tiles_x:
            system.retile(cfg["tiles_x"], cfg["sweep_blocks"])
        system.grid.sweep_blocks = int(cfg["sweep_blocks"])
        system._graph = None

    def measure():
        return time_steps(system._step, steps, warmup)

    return tune(key, space, apply, measure, use_cache)


def tune_sph(system, steps: int = 6, warmup: int = 2, tile_targets=(60, 90, 130, 170), sweep_blocks=(0, -1),
             use_cache: bool = True) -> dict:
    """Tunes an SPHSystem: particles per tile (re-tiles and rebuilds) x sweep
    blocks, timing whole steps."""
    space = {"tile_target": list(tile_targets), "sweep_blocks": list(sweep_blocks)}
    key = "sph:" + signature({"n": system.n, "L": [float(x) for x in system.L], "r_list": system.r_list})

    def apply(cfg):
        if cfg["tile_target"] != system.tile_target:
            system.retile(cfg["tile_target"], cfg["sweep_blocks"])
        system.grid.sweep_blocks = int(cfg["sweep_blocks"])
        system._graph = None

    def measure():
        return time_steps(system._step, steps, warmup)

    return tune(key, space, apply, measure, use_cache)
