"""Autotuners for the launch shapes of the batched path and of the plain (one problem) path.

Knobs: the batched strategy (lock-step tiles dealt by the host or handed out by a device
queue, the same tiles in one dataflow launch, or one persistent cluster kernel); for the tile strategies the words per warp tile (the words
each lane updates per tile: tile_words / 32) and, for the lock-step ones, the number of
streams the batch is split over (parts of equal work whose launches overlap); for the cluster kernel the CTAs per
thread-block cluster and the lattice size from which a problem is spread over a whole
cluster instead of one CTA. They change only how work is
distributed, never a result: `tune` checks that every candidate leaves every problem in the
same state (spins, temperature map, swap counters) before it compares times.

For the plain path (`tune_single`) the knobs are the halo scheme of the persistent sweep
(each CTA owning strided words of a plane, with a grid barrier between the colours, or a
band of whole rows in shared memory whose halo rows it recomputes, with one grid barrier a
sweep), the words of each colour a thread owns, and one launch per half sweep instead of a
persistent launch; the choice is kept per problem shape (L, R, J, h).

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
DEFAULT = {"strategy": FLAT, "cluster": 4, "joint_min_L": 128, "tile_words": 512, "streams": 1,
           "graphs": 0}
# (strategy, cluster, joint_min_L, tile_words, streams[, graphs])
CANDIDATES: Tuple[Tuple[int, int, int, int, int], ...] = (
    (FLAT, 1, 128, 256, 1), (FLAT, 1, 128, 512, 1), (FLAT, 1, 128, 1024, 1),
    (QUEUE, 1, 128, 256, 1), (QUEUE, 1, 128, 512, 1), (QUEUE, 1, 128, 1024, 1),
    (FLAT, 1, 128, 512, 2), (FLAT, 1, 128, 512, 3), (FLAT, 1, 128, 512, 4),
    (FLAT, 1, 128, 256, 4), (FLAT, 1, 128, 1024, 4),
    (QUEUE, 1, 128, 512, 2), (QUEUE, 1, 128, 512, 4), (QUEUE, 1, 128, 1024, 4),
    (FLOW, 1, 128, 256, 1), (FLOW, 1, 128, 512, 1),
    (CLUSTER, 1, 1 << 20, 512, 1), (CLUSTER, 2, 128, 512, 1), (CLUSTER, 3, 128, 512, 1),
    (CLUSTER, 4, 256, 512, 1), (CLUSTER, 4, 128, 512, 1), (CLUSTER, 4, 96, 512, 1),
    (CLUSTER, 6, 128, 512, 1), (CLUSTER, 8, 128, 512, 1),
    # graph replay of the lock-step shapes (worth it where a batch's shape repeats)
    (FLAT, 1, 128, 512, 1, 1), (FLAT, 1, 128, 512, 2, 1), (FLAT, 1, 128, 512, 4, 1),
    (FLAT, 1, 128, 256, 4, 1), (FLAT, 1, 128, 1024, 4, 1), (QUEUE, 1, 128, 512, 4, 1),
    (QUEUE, 1, 128, 1024, 4, 1))


def set_tuning(strategy: int, cluster: int, joint_min_L: int, tile_words: int = 512,
               streams: int = 1, graphs: int = 0) -> None:
    check(lib.pt_set_batch_tuning(int(strategy), int(cluster), int(joint_min_L)),
          "pt_set_batch_tuning")
    check(lib.pt_set_batch_tile_words(int(tile_words)), "pt_set_batch_tile_words")
    check(lib.pt_set_batch_streams(int(streams)), "pt_set_batch_streams")
    check(lib.pt_set_batch_graphs(int(graphs)), "pt_set_batch_graphs")


def get_tuning() -> Dict[str, int]:
    s, c, j, w, n, g = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    check(lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(j)), "pt_get_batch_tuning")
    check(lib.pt_get_batch_tile_words(C.byref(w)), "pt_get_batch_tile_words")
    check(lib.pt_get_batch_streams(C.byref(n)), "pt_get_batch_streams")
    check(lib.pt_get_batch_graphs(C.byref(g)), "pt_get_batch_graphs")
    return {"strategy": s.value, "cluster": c.value, "joint_min_L": j.value,
            "tile_words": w.value, "streams": n.value, "graphs": g.value}


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
               entry.get("tile_words", DEFAULT["tile_words"]), entry.get("streams", 1),
               entry.get("graphs", 0))
    return get_tuning()


def _snapshot(handles):
    out = []
    for h in handles:
        att, acc = h.swap_stats()
        out.append((h.spins().tobytes(), h.chain_map().tobytes(), att.tobytes(), acc.tobytes()))
    return out


def _full(cand) -> Tuple[int, int, int, int, int, int]:
    """A candidate with the knobs it leaves out at their defaults (512-word tiles, one
    stream, no graph replay)."""
    return tuple(cand) + (512, 1, 0)[len(cand) - 3:] if len(cand) < 6 else tuple(cand)


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
            log("strategy=%d cluster=%d joint_min_L=%d tile_words=%d streams=%d graphs=%d: "
                "%.4f s" % (_full(cand) + (best,)))
    results.sort(key=lambda r: r[0])
    best_t, cand = results[0]
    # within half a percent of the fastest, prefer graph replay: the same device time with
    # the host free (a 2000-sweep call issues in 0.2 ms instead of 183 ms)
    for t, c in results:
        if t <= 1.005 * results[0][0] and _full(c)[5] == 1:
            best_t, cand = t, c
            break
    st, cl, jm, tw, ns, gr = _full(cand)
    choice = {"strategy": st, "cluster": cl, "joint_min_L": jm, "tile_words": tw, "streams": ns,
              "graphs": gr}
    set_tuning(st, cl, jm, tw, ns, gr)
    if save:
        cache = _load_cache()
        cache.setdefault(_device_key(), {})[workload] = dict(choice, seconds=best_t,
                                                             when=time.strftime("%Y-%m-%d"))
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return {"choice": choice, "timings": [(c, t) for t, c in results]}


# ---------------------------------------------------------------------------------------
# plain path: one problem per pt_sweep call
# ---------------------------------------------------------------------------------------
SWEEP_AUTO, SWEEP_LAUNCHES, SWEEP_PERSISTENT, SWEEP_BANDS = 0, 1, 2, 3
# (strategy, words_per_thread)
SINGLE_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (SWEEP_PERSISTENT, 1), (SWEEP_PERSISTENT, 2), (SWEEP_PERSISTENT, 4), (SWEEP_PERSISTENT, 8),
    (SWEEP_BANDS, 1), (SWEEP_BANDS, 2), (SWEEP_BANDS, 4), (SWEEP_LAUNCHES, 1))


def shape_key(L: int, R: int, J: float, h: float) -> str:
    return "L%d_R%d_J%g_h%g" % (L, R, J, h)


def _single_snapshot(h):
    att, acc = h.swap_stats()
    return (h.spins().tobytes(), h.chain_map().tobytes(), att.tobytes(), acc.tobytes(),
            h.energies_int().tobytes())


def tune_single(problem, sweeps: int = 200, every: int = 1,
                candidates: Sequence[Tuple[int, int]] = SINGLE_CANDIDATES, repeats: int = 2,
                save: bool = True, log=None) -> Dict[str, object]:
    """Time every plain-path shape on `problem` (a workload Problem), each on a fresh copy
    from the same seed, with CUDA events on the copy's stream; keep the fastest. A shape the
    problem does not fit (pt_sweep answers PT_EINVAL) is skipped. Raises if two shapes
    disagree on the final state (spins, energies, temperature map, swap counters)."""
    import torch

    from ._lib import PTError
    from .api import PTProblem

    stream = torch.cuda.Stream()
    results: List[Tuple[float, Tuple[int, int]]] = []
    reference = None
    for cand in candidates:
        best = float("inf")
        try:
            for rep in range(repeats):
                h = PTProblem(problem.L, problem.betas, J=problem.J, h=problem.h,
                              seed=problem.seed, stream=stream)
                try:
                    h.set_sweep_tuning(*cand)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    h.sweep(sweeps, every)
                    b.record(stream)
                    h.synchronize()
                    best = min(best, a.elapsed_time(b) / 1e3)
                    if rep == 0:
                        snap = _single_snapshot(h)
                        if reference is None:
                            reference = snap
                        elif snap != reference:
                            raise RuntimeError("sweep shape %r changed a result" % (cand,))
                finally:
                    h.close()
        except PTError as e:
            if log:
                log("strategy=%d words_per_thread=%d: does not fit (%s)" % (cand + (e,)))
            continue
        results.append((best, tuple(cand)))
        if log:
            log("strategy=%d words_per_thread=%d: %.6f s" % (tuple(cand) + (best,)))
    if not results:
        raise RuntimeError("no plain-path shape fits this problem")
    results.sort(key=lambda r: r[0])
    best_t, (st, wpt) = results[0]
    choice = {"strategy": st, "words_per_thread": wpt}
    if save:
        cache = _load_cache()
        key = shape_key(problem.L, len(problem.betas), problem.J, problem.h)
        cache.setdefault(_device_key(), {}).setdefault("single", {})[key] = dict(
            choice, seconds=best_t, sweeps=sweeps, every=every, when=time.strftime("%Y-%m-%d"))
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return {"choice": choice, "timings": [(c, t) for t, c in results]}


def apply_single(handle, L: int, R: int, J: float, h: float) -> Optional[Dict[str, int]]:
    """Give `handle` (an api.PTProblem) the cached plain-path shape of its problem shape on
    this device; None (and the library's default, PT_SWEEP_AUTO) when there is none."""
    entry = _load_cache().get(_device_key(), {}).get("single", {}).get(shape_key(L, R, J, h))
    if entry is None:
        return None
    handle.set_sweep_tuning(entry["strategy"], entry["words_per_thread"])
    return {"strategy": entry["strategy"], "words_per_thread": entry["words_per_thread"]}


def main(argv=None) -> int:
    """python -m paper_2512_03825_b300.autotune {batched,serve,single} [--out PATH]: tune on
    this device's GPU and update the cache (and copy it to PATH)."""
    import argparse
    import shutil

    import torch

    from . import workloads as W

    ap = argparse.ArgumentParser(prog="python -m paper_2512_03825_b300.autotune")
    ap.add_argument("workload", choices=["batched", "serve", "single"])
    ap.add_argument("--out", default=None, help="also copy the updated cache here")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)

    def log(s):
        print(s, flush=True)

    tiles = [c for c in CANDIDATES if c[0] in (FLAT, FLOW, QUEUE)]
    if args.workload == "batched":
        r = tune(W.batched_problems(), sweeps=200, every=1, candidates=tiles,
                 workload="batched", repeats=3, log=log)
        log("batched: %r" % (r["choice"],))
    elif args.workload == "serve":
        # no graph replay for the server: its batch changes shape whenever a request
        # arrives or leaves, so nearly every call would pay a capture (the tuner's repeats of
        # one fixed sample would hide that)
        reqs = W.serving_requests(n=96, rate_per_s=1.0, draw_seed=4242)
        r = tune([q.problem for q in reqs], sweeps=100, every=1,
                 candidates=[c for c in tiles if _full(c)[5] == 0],
                 workload="serve", repeats=3, log=log)
        log("serve: %r" % (r["choice"],))
    else:
        for name, p in list(W.SINGLE.items()) + [("paper", W.paper_problem())]:
            sweeps = 2000 if p.L <= 128 else 200
            r = tune_single(p, sweeps=sweeps, every=p.every, log=log)
            log("single %s: %r" % (name, r["choice"]))
    if args.out:
        shutil.copy(CACHE, args.out)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
