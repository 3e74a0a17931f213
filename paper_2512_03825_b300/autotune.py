"""Autotuner for the batched kernel's launch shape.

Knobs: the batched strategy (lock-step tiles dealt by the host or handed out by a device
queue, the same tiles in one dataflow launch, or one persistent cluster kernel); for the tile strategies the words per warp tile (the words
each lane updates per tile: tile_words / 32) and, for the lock-step ones, the number of
streams the batch is split over (parts of equal work whose launches overlap); for the cluster kernel the CTAs per
thread-block cluster and the lattice size from which a problem is spread over a whole
cluster instead of one CTA. They change only how work is
distributed, never a result: `tune` checks that every candidate leaves every problem in the
same state (spins, temperature map, swap counters) before it compares times.

Choices are cached per device name in ``autotune_cache.json`` next to this module.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import time
from typing import Dict, List, Optional, Sequence, Tuple

from ._lib import check, lib

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")
FLAT, CLUSTER, FLOW, QUEUE = 0, 1, 2, 3
DEFAULT = {"strategy": FLAT, "cluster": 4, "joint_min_L": 128, "tile_words": 512, "streams": 1}
# (strategy, cluster, joint_min_L, tile_words, streams)
CANDIDATES: Tuple[Tuple[int, int, int, int, int], ...] = (
    (FLAT, 1, 128, 256, 1), (FLAT, 1, 128, 512, 1), (FLAT, 1, 128, 1024, 1),
    (QUEUE, 1, 128, 256, 1), (QUEUE, 1, 128, 512, 1), (QUEUE, 1, 128, 1024, 1),
    (FLAT, 1, 128, 512, 2), (FLAT, 1, 128, 512, 3), (FLAT, 1, 128, 512, 4),
    (FLAT, 1, 128, 256, 4), (FLAT, 1, 128, 1024, 4),
    (QUEUE, 1, 128, 512, 2), (QUEUE, 1, 128, 512, 4), (QUEUE, 1, 128, 1024, 4),
    (FLOW, 1, 128, 256, 1), (FLOW, 1, 128, 512, 1),
    (CLUSTER, 1, 1 << 20, 512, 1), (CLUSTER, 2, 128, 512, 1), (CLUSTER, 3, 128, 512, 1),
    (CLUSTER, 4, 256, 512, 1), (CLUSTER, 4, 128, 512, 1), (CLUSTER, 4, 96, 512, 1),
    (CLUSTER, 6, 128, 512, 1), (CLUSTER, 8, 128, 512, 1))


def set_tuning(strategy: int, cluster: int, joint_min_L: int, tile_words: int = 512,
               streams: int = 1) -> None:
    check(lib.pt_set_batch_tuning(int(strategy), int(cluster), int(joint_min_L)),
          "pt_set_batch_tuning")
    check(lib.pt_set_batch_tile_words(int(tile_words)), "pt_set_batch_tile_words")
    check(lib.pt_set_batch_streams(int(streams)), "pt_set_batch_streams")


def get_tuning() -> Dict[str, int]:
    s, c, j, w, n = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    check(lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(j)), "pt_get_batch_tuning")
    check(lib.pt_get_batch_tile_words(C.byref(w)), "pt_get_batch_tile_words")
    check(lib.pt_get_batch_streams(C.byref(n)), "pt_get_batch_streams")
    return {"strategy": s.value, "cluster": c.value, "joint_min_L": j.value,
            "tile_words": w.value, "streams": n.value}


def _device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/sm%d%d/%dSM" % (p.name, p.major, p.minor, p.multi_processor_count)


def _load_cache() -> dict:
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def apply_cached_or_default(workload: str = "batched") -> Dict[str, int]:
    """Apply the cached choice for this device (or the default) and return it."""
    entry = _load_cache().get(_device_key(), {}).get(workload, DEFAULT)
    set_tuning(entry.get("strategy", FLAT), entry["cluster"], entry["joint_min_L"],
               entry.get("tile_words", DEFAULT["tile_words"]), entry.get("streams", 1))
    return get_tuning()


def _snapshot(handles):
    out = []
    for h in handles:
        att, acc = h.swap_stats()
        out.append((h.spins().tobytes(), h.chain_map().tobytes(), att.tobytes(), acc.tobytes()))
    return out


def tune(problems: Sequence, sweeps: int = 200, every: int = 1,
         candidates: Sequence[Tuple[int, ...]] = CANDIDATES, workload: str = "batched",
         repeats: int = 2, save: bool = True, log=None) -> Dict[str, object]:
    """Time every candidate launch shape on `problems` (workload Problems); keep the fastest.
    Raises if two candidates disagree on any problem's final state."""
    import torch

    from .api import PTProblem, sweep_batch

    results: List[Tuple[float, Tuple[int, ...]]] = []
    reference = None
    for cand in candidates:
        set_tuning(*cand)
        best = float("inf")
        for rep in range(repeats):
            hs = [PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in problems]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sweep_batch(hs, sweeps, every)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
            if rep == 0:
                snap = _snapshot(hs)
                if reference is None:
                    reference = snap
                elif snap != reference:
                    raise RuntimeError("launch shape %r changed a result" % (cand,))
            for h in hs:
                h.close()
        results.append((best, cand))
        if log:
            full = tuple(cand) + (1,) * (5 - len(cand))
            log("strategy=%d cluster=%d joint_min_L=%d tile_words=%d streams=%d: %.4f s"
                % (full + (best,)))
    results.sort(key=lambda r: r[0])
    best_t, cand = results[0]
    st, cl, jm, tw, ns = tuple(cand) + (1,) * (5 - len(cand))
    choice = {"strategy": st, "cluster": cl, "joint_min_L": jm, "tile_words": tw, "streams": ns}
    set_tuning(st, cl, jm, tw, ns)
    if save:
        cache = _load_cache()
        cache.setdefault(_device_key(), {})[workload] = dict(choice, seconds=best_t,
                                                             when=time.strftime("%Y-%m-%d"))
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return {"choice": choice, "timings": [(c, t) for t, c in results]}
