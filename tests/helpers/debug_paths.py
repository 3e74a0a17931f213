"""Run every sweep path of the debug build of the library on small cases (test support).

Run as a separate process with PT_LIBRARY=debug, so that the package loads libpt_debug.so,
whose kernels check every spin-word, count and trace index before the access and tag every
store with its half sweep (pt_debug_report). For each case the problems must end with no
failed check, with every word stored by its own half sweep of the last sweep, and equal to
the oracle. Two planted mistakes (pt_debug_inject) must be caught. Prints one JSON object.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_03825_b300 import _lib, api, autotune  # noqa: E402
from paper_2512_03825_b300 import workloads as W  # noqa: E402

LAUNCHES, PERSISTENT, BANDS = 1, 2, 3
FLAT, CLUSTER, FLOW, QUEUE = 0, 1, 2, 3


def report(g):
    v, k, i, u = C.c_uint64(), C.c_int32(), C.c_uint64(), C.c_uint64()
    rc = _lib.lib.pt_debug_report(g.handle, C.byref(v), C.byref(k), C.byref(i), C.byref(u))
    assert rc == 0, _lib.lib.pt_last_error().decode()
    return {"violations": v.value, "first_kind": k.value, "first_index": i.value,
            "unwritten": u.value}


def oracle_run(p, calls):
    o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
    for kind, n, m in calls:
        if kind == "sweep":
            o.sweep(n, m)
        else:
            o.flip(n, m)
    return o


def same(g, o):
    return (np.array_equal(g.spins(), o.spins()) and np.array_equal(g.energies_int(), o.energies_int())
            and np.array_equal(g.magnetisations(), o.magnetisations())
            and np.array_equal(g.chain_map(), o.chain_map())
            and all(np.array_equal(a, b) for a, b in zip(g.swap_stats(), o.swap_stats())))


def check(results, name, g, p, calls):
    rep = report(g)
    ok = rep["violations"] == 0 and rep["unwritten"] == 0
    equal = same(g, oracle_run(p, calls))
    results.append({"case": name, "L": p.L, "R": p.R, "h": p.h, "report": rep,
                    "oracle_equal": bool(equal), "ok": bool(ok and equal)})


def main():
    assert _lib.lib.pt_debug_build() == 1, "not the debug build: " + _lib.LIB_PATH
    oracle.set_threads(os.cpu_count() or 1)
    res = []
    P = W.Problem
    # plain path: persistent (cooperative grid, cluster grid, one CTA with its plane in shared
    # memory), one launch per half sweep, generic mode, traced
    plain = [("persistent cooperative L128 R32", P(L=128, betas=W.linear_ladder(0.3, 0.55, 32), seed=11), PERSISTENT),
             ("persistent cluster L32 R40", P(L=32, betas=W.linear_ladder(0.2, 0.7, 40), seed=12), PERSISTENT),
             ("persistent shared-memory plane L16 R8", P(L=16, betas=W.geometric_ladder(0.2, 0.6, 8), seed=13), PERSISTENT),
             ("persistent generic L20 R6", P(L=20, betas=W.linear_ladder(0.3, 0.6, 6), h=0.1, seed=14), PERSISTENT),
             ("launches generic L24 R37", P(L=24, betas=W.linear_ladder(0.2, 0.7, 37), h=0.1, seed=15), LAUNCHES),
             ("launches ferro L16 R8", P(L=16, betas=W.geometric_ladder(0.2, 0.6, 8), seed=16), LAUNCHES),
             ("launches antiferro L12 R3", P(L=12, betas=W.linear_ladder(0.3, 0.5, 3), J=-1.0, h=0.25, seed=17), LAUNCHES),
             ("bands L128 R32", P(L=128, betas=W.linear_ladder(0.3, 0.55, 32), seed=22), BANDS),
             ("bands generic uneven L90 R40", P(L=90, betas=W.linear_ladder(0.3, 0.6, 40), h=0.1, seed=23), BANDS)]
    for name, p, strategy in plain:
        g = api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        g.set_sweep_tuning(strategy)
        g.sweep(7, 2)
        g.sweep(6, 3)
        check(res, name, g, p, [("sweep", 7, 2), ("sweep", 6, 3)])
    # traced plain run (every sweep counted, trace rows written)
    p = P(L=24, betas=W.linear_ladder(0.3, 0.6, 9), seed=18)
    for strategy in (LAUNCHES, PERSISTENT, BANDS):
        g = api.PTProblem(p.L, p.betas, seed=p.seed)
        g.set_sweep_tuning(strategy)
        g.trace_start(5)
        g.sweep(9, 2)
        check(res, "traced %s" % {LAUNCHES: "launches", PERSISTENT: "persistent",
                                  BANDS: "bands"}[strategy], g, p, [("sweep", 9, 2)])
    # batches: every strategy, ferro and generic problems mixed, uneven n and m
    rng = np.random.Generator(np.random.PCG64(5150))
    probs = []
    for j in range(10):
        L = int(rng.choice([8, 16, 24, 32, 48]))
        R = int(rng.integers(1, 70))
        J, h = [(1.0, 0.0), (1.0, 0.1), (-1.0, 0.25), (1.0, -0.1)][j % 4]
        probs.append(P(L=L, betas=W.linear_ladder(0.2, 0.8, R), J=J, h=h, seed=2000 + j))
    ns = [int(x) for x in rng.integers(1, 9, size=len(probs))]
    ms = [int(x) for x in rng.integers(0, 3, size=len(probs))]
    before = autotune.get_tuning()
    for strategy, name in ((FLAT, "batch dealt"), (QUEUE, "batch queued"), (FLOW, "batch dataflow"),
                           (CLUSTER, "batch cluster")):
        autotune.set_tuning(strategy=strategy, cluster=2, joint_min_L=24, tile_words=64)
        gs = [api.PTProblem(q.L, q.betas, J=q.J, h=q.h, seed=q.seed) for q in probs]
        api.sweep_batch(gs, ns, ms)
        api.sweep_batch(gs, [3] * len(gs), ms)
        for q, g, n, m in zip(probs, gs, ns, ms):
            check(res, name, g, q, [("sweep", n, m), ("sweep", 3, m)])
    # graph replay (needs a stream of its own): one capture, then replays of the same shape
    import torch
    st = torch.cuda.Stream()
    for strategy, name in ((FLAT, "batch dealt, graph replay"), (QUEUE, "batch queued, graph replay")):
        autotune.set_tuning(strategy=strategy, cluster=2, joint_min_L=24, tile_words=64,
                            streams=2, graphs=1)
        gs = [api.PTProblem(q.L, q.betas, J=q.J, h=q.h, seed=q.seed, stream=st) for q in probs]
        for _ in range(3):
            api.sweep_batch(gs, [3] * len(gs), ms)
        for q, g, m in zip(probs, gs, ms):
            check(res, name, g, q, [("sweep", 3, m)] * 3)
    autotune.set_tuning(strategy=QUEUE, cluster=2, joint_min_L=24, tile_words=64)
    gs = [api.PTProblem(q.L, q.betas, J=q.J, h=q.h, seed=q.seed) for q in probs]
    api.sweep_batch_static(gs, ns, ms)
    for q, g, n, m in zip(probs, gs, ns, ms):
        check(res, "batch static", g, q, [("sweep", n, m)])
    # a traced problem in a batch, and the batched read (one count launch over all problems)
    gs = [api.PTProblem(q.L, q.betas, J=q.J, h=q.h, seed=q.seed) for q in probs[:4]]
    gs[1].trace_start(4)
    api.sweep_batch(gs, [5] * 4, [1] * 4)
    api.read_batch(gs)
    for q, g in zip(probs[:4], gs):
        check(res, "batch traced + batched read", g, q, [("sweep", 5, 1)])
    autotune.set_tuning(**before)
    # single-spin flips (replicas in shared memory, and the global-word kernel), then sweeps
    p = P(L=20, betas=W.linear_ladder(0.3, 0.6, 40), seed=19)
    for shared in (True, False):
        g = api.PTProblem(p.L, p.betas, seed=p.seed)
        g.set_flip_tuning(shared)
        g.flip(300, 50)
        g.sweep(4, 1)
        check(res, "flip %s + sweeps" % ("shared" if shared else "global"), g, p,
              [("flip", 300, 50), ("sweep", 4, 1)])
    # a checkpoint round trip, then sweeps on the loaded problem
    p = P(L=16, betas=W.linear_ladder(0.3, 0.6, 12), h=0.1, seed=20)
    g = api.PTProblem(p.L, p.betas, h=p.h, seed=p.seed)
    g.sweep(5, 1)
    g2 = api.PTProblem.load(g.save())
    g2.sweep(4, 1)
    check(res, "checkpoint load + sweeps", g2, p, [("sweep", 9, 1)])
    # planted mistakes must be caught (and poison only their own problem)
    caught = {}
    for kind in (1, 2):
        p = P(L=16, betas=W.geometric_ladder(0.2, 0.6, 8), seed=21)
        g = api.PTProblem(p.L, p.betas, seed=p.seed)
        g.set_sweep_tuning(LAUNCHES)
        assert _lib.lib.pt_debug_inject(g.handle, kind) == 0
        g.sweep(2, 1)
        rep = report(g)
        rc = _lib.lib.pt_synchronize(g.handle)
        caught[kind] = {"report": rep, "synchronize_rc": rc,
                        "message": _lib.lib.pt_last_error().decode()}
    out = {"cases": res, "all_ok": all(r["ok"] for r in res), "planted": caught}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
