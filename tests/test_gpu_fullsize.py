"""Parity at the full workload sizes, in the launch configurations bench.py times.

The oracle cannot run thousands of sweeps of an L = 1024 lattice, so each full run is checked
on outputs the oracle can compute one by one: the GPU runs every sweep but the last, its exact
state (spins of every slot, temperature map, counters, swap statistics) is handed to the
oracle, both take the last sweep (and its swap iteration), and every spin, energy, map entry and
counter must agree. Properties that hold at any size are checked on every problem: the oracle's
energies of the GPU's final configurations equal the GPU's, attempt counts follow the closed
form, and each temperature map is a permutation."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(16)
    return A


def handoff(g, prob):
    """An oracle problem holding exactly the GPU problem's current state."""
    o = oracle.OracleProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    so = g.chain_map()
    sp = np.empty((prob.R, prob.L, prob.L), np.int8)
    for k in range(prob.R):
        sp[so[k]] = g.spins(k)
    att, acc = g.swap_stats()
    o.load_state(sp, so, *g.counters(), att, acc)
    return o


def assert_same(g, o, where):
    np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where)
    for k in range(o.R):
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg="%s spins %d" % (where, k))
    np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where)
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where)
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y, err_msg=where)
    assert g.counters() == o.counters(), where


def closed_form_attempts(R, n, m):
    n_ex = n // m if m else 0
    return np.array([sum(1 for e in range(n_ex) if e % 2 == k % 2) for k in range(R - 1)],
                    dtype=np.uint64)


def check_properties(g, prob, n):
    so = g.chain_map()
    assert sorted(so.tolist()) == list(range(prob.R))
    att, acc = g.swap_stats()
    np.testing.assert_array_equal(att, closed_form_attempts(prob.R, n, prob.every))
    assert (acc <= att).all()
    o = handoff(g, prob)  # oracle energies of the GPU's configurations
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations())


def test_L1024_R64_full_run_plain_path(api):
    prob = W.SINGLE["L1024_R64"]
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    g.sweep(prob.sweeps - 1, prob.every)
    o = handoff(g, prob)
    g.sweep(1, prob.every)            # sweep 1000, then swap iteration 199
    o.sweep(1, prob.every)
    assert_same(g, o, "L1024 R64 last sweep")
    check_properties(g, prob, prob.sweeps)


def test_L128_R32_full_run_batched_and_plain(api):
    prob = W.SINGLE["L128_R32"]
    b = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    api.sweep_batch([b], prob.sweeps - 1, prob.every)
    o = handoff(b, prob)
    api.sweep_batch([b], 1, prob.every)
    o.sweep(1, prob.every)
    assert_same(b, o, "L128 R32 last sweep (batched)")
    check_properties(b, prob, prob.sweeps)
    p = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    p.sweep(prob.sweeps, prob.every)
    for x, y in zip(b.spins(), p.spins()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(b.chain_map(), p.chain_map())


@pytest.fixture
def bench_tuning(api):
    """The batch launch shape bench.py times (the autotuner's cached choice for this GPU),
    restored to the previous one afterwards."""
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    chosen = autotune.apply_cached_or_default("batched")
    yield chosen
    autotune.set_tuning(**before)


def test_batched_256_full_run(api, bench_tuning):
    import torch
    probs = W.batched_problems()
    n = probs[0].sweeps
    st = torch.cuda.Stream()  # as bench.py: problems created on a side stream, no host wait
    gs = [api.PTProblem(p.L, p.betas, seed=p.seed, stream=st) for p in probs]
    api.sweep_batch(gs, n - 1, 1)
    order = sorted(range(len(probs)), key=lambda j: probs[j].L ** 2 * probs[j].R)
    sample = [order[0], order[len(order) // 2], order[-1]]
    handed = {j: handoff(gs[j], probs[j]) for j in sample}
    api.sweep_batch(gs, 1, 1)
    for j in sample:
        handed[j].sweep(1, 1)
        assert_same(gs[j], handed[j], "batched problem %d last sweep" % j)
    for j, (g, p) in enumerate(zip(gs, probs)):
        so = g.chain_map()
        assert sorted(so.tolist()) == list(range(p.R)), j
        att, acc = g.swap_stats()
        np.testing.assert_array_equal(att, closed_form_attempts(p.R, n, 1), err_msg=str(j))
        assert g.counters() == (n, n)
    for j in order[::32]:
        check_properties(gs[j], probs[j], n)


def test_4096_problem_batch_sample(api, bench_tuning):
    """The bench's beyond-L2 leg: 4096 problems of the default mix (about 360 MB of spin
    words, more than the L2) in the tuned launch shape, 12 sweeps with an exchange after each.
    Every 512th problem, from creation, equals the oracle in every output; every problem keeps
    a permutation for its map and the closed-form attempt counts."""
    import torch
    probs = W.batched_problems(n=4096, sweeps=12)
    st = torch.cuda.Stream()
    gs = [api.PTProblem(p.L, p.betas, seed=p.seed, stream=st) for p in probs]
    api.sweep_batch(gs, 12, 1)
    torch.cuda.synchronize()
    oracle.set_threads(os.cpu_count() or 1)
    for j in range(0, len(probs), 512):
        p = probs[j]
        o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
        o.sweep(12, 1)
        assert_same(gs[j], o, "problem %d of 4096" % j)
    for j in range(0, len(probs), 97):
        g, p = gs[j], probs[j]
        assert sorted(g.chain_map().tolist()) == list(range(p.R)), j
        np.testing.assert_array_equal(g.swap_stats()[0], closed_form_attempts(p.R, 12, 1),
                                      err_msg=str(j))
    for g in gs:
        g.close()
