"""The continuous-batching server on the GPU: requests that arrive while others run are
admitted as memory frees up, advance together in shared batches, and every result equals the
same request run alone (and the oracle's, on a sample) -- exactly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    from paper_2512_03825_b300 import build as B
    B.build()
    import torch
    from paper_2512_03825_b300 import serve
    torch.cuda.set_device(0)
    return serve.LibEngine()


def small_stream(n=24, seed=31, gap=0.01):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n):
        L = int(rng.choice([32, 64, 96]))
        R = int(rng.integers(8, 40))
        out.append(W.Request(rid=j, arrival=j * gap, problem=W.Problem(
            L=L, betas=W.linear_ladder(0.3, 0.6, R), J=1.0, h=float(rng.choice([0.0, 0.1])),
            seed=0x5EED3000 + j, sweeps=int(rng.integers(20, 200)), every=int(rng.integers(1, 4)))))
    return out


def alone(engine, p):
    h = engine.create(p)
    h.sweep(p.sweeps, p.every)
    data = engine.read(h)
    engine.destroy(h)
    return data


def test_served_results_equal_alone(engine):
    from paper_2512_03825_b300 import serve
    reqs = small_stream()
    srv = serve.Server(engine, budget_bytes=10 ** 10, slice_sweeps=25)
    res = srv.run(reqs, realtime=True, timeout_s=120)
    assert sorted(res) == [r.rid for r in reqs]
    assert srv.ticks > 1 and max(srv.peak_used, 0) > 0
    for r in reqs:
        ref = alone(engine, r.problem)
        got = res[r.rid]
        for key in ("E_int", "M", "slot_of_temp", "attempted", "accepted"):
            np.testing.assert_array_equal(getattr(got, key), ref[key], err_msg="%d %s" % (r.rid, key))
    s = srv.summary()
    assert s["requests"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0
    # a sample against the oracle
    oracle.set_threads(8)
    for r in reqs[:4]:
        p = r.problem
        o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        o.sweep(p.sweeps, p.every)
        np.testing.assert_array_equal(res[r.rid].E_int, o.energies_int())
        np.testing.assert_array_equal(res[r.rid].slot_of_temp, o.chain_map())


def test_tight_budget_queues_and_still_serves_everything(engine):
    from paper_2512_03825_b300 import serve
    reqs = small_stream(n=10, seed=32, gap=0.0)
    need = max(engine.estimate_bytes(r.problem) for r in reqs)
    srv = serve.Server(engine, budget_bytes=2 * need, slice_sweeps=50)
    res = srv.run(reqs, realtime=False, timeout_s=120)
    assert sorted(res) == [r.rid for r in reqs]
    assert srv.peak_used <= 2 * need
    assert srv.used == 0
