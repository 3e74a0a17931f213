"""Problem creation on a caller's stream from the page-locked creation images, against the
oracle. Problems created on a side stream start without a host wait, share one image when
their ladder, couplings and (where it shapes a table) lattice reach agree, and start and
continue exactly as the oracle's. An image above the page-locked limit (the paper's
1500-temperature ladder on L = 300, about 311 MiB of tables) takes the pageable copy and gives
the same problem as a creation without a stream."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(8)
    return A


def assert_same(g, o, where):
    np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where)
    np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where)
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where)
    for k in range(o.R):
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg="%s spins %d" % (where, k))
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y, err_msg=where)
    assert g.counters() == o.counters(), where


LADDER = W.linear_ladder(0.3, 0.6, 40)
PROBLEMS = [
    # L = 8 reaches |n| <= 256, inside every pair's saturation range: reach-shaped tables
    W.Problem(L=8, betas=LADDER, seed=31),
    W.Problem(L=8, betas=LADDER, seed=32),
    # L = 64 and 96 reach beyond it: whole tables, one image for both lattices
    W.Problem(L=64, betas=LADDER, seed=33),
    W.Problem(L=96, betas=LADDER, seed=34),
    # a field: the generic thresholds and a table stride of 2 (gcd(4 J_int, 2 h_int) = 2)
    W.Problem(L=16, betas=LADDER, h=0.1, seed=35),
    W.Problem(L=12, betas=W.linear_ladder(0.2, 0.5, 9), J=-1.0, h=0.25, seed=36),
]


def test_stream_creation_matches_oracle(api):
    import torch
    st = torch.cuda.Stream()
    for r in range(2):  # the second round takes every image from the cache
        gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=st)
              for p in PROBLEMS]
        os_ = [oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in PROBLEMS]
        for j, (g, o) in enumerate(zip(gs, os_)):
            assert_same(g, o, "round %d problem %d initial" % (r, j))
        api.sweep_batch(gs, 5, 1)
        for o in os_:
            o.sweep(5, 1)
        for j, (g, o) in enumerate(zip(gs, os_)):
            assert_same(g, o, "round %d problem %d after 5 sweeps" % (r, j))
        for g in gs:
            g.close()


def test_metropolis_rule_gets_its_own_image(api):
    """Same ladder, both swap rules, created back to back on one stream: each problem runs
    with its own rule's tables."""
    import torch
    st = torch.cuda.Stream()
    p = W.Problem(L=10, betas=W.linear_ladder(0.25, 0.55, 12), seed=41)
    for rule in (0, 1, 0):
        g = api.PTProblem(p.L, p.betas, seed=p.seed, stream=st, swap_rule=rule)
        o = oracle.OracleProblem(p.L, p.betas, seed=p.seed, swap_rule=rule)
        g.sweep(30, 1)
        o.sweep(30, 1)
        assert_same(g, o, "rule %d" % rule)
        g.close()


def test_large_image_takes_the_pageable_copy(api):
    import torch
    prob = W.paper_problem()
    assert api.estimate_device_bytes(prob.L, prob.betas) > 2 ** 28
    st = torch.cuda.Stream()
    a = api.PTProblem(prob.L, prob.betas, seed=prob.seed, stream=st)
    b = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    for g in (a, b):
        g.set_sweep_tuning(2)
        g.sweep(2, 1)
    np.testing.assert_array_equal(a.chain_map(), b.chain_map())
    np.testing.assert_array_equal(a.energies_int(), b.energies_int())
    for x, y in zip(a.swap_stats(), b.swap_stats()):
        np.testing.assert_array_equal(x, y)
    for k in (0, 31, 32, 1499):
        np.testing.assert_array_equal(a.spins(k), b.spins(k))
    a.close()
    b.close()


def test_small_cache_limit_evicts_without_freeing_live_images(api):
    """A 96 KiB cache limit: the images (5-25 KiB) are page-locked and the cache is emptied
    again and again while the problems created from them are alive and still running. With
    a limit of 0 every image goes through pageable memory. Every problem matches the
    oracle."""
    import torch
    st = torch.cuda.Stream()
    limit = 96 << 10
    api.set_image_cache_limit(limit)
    try:
        probs = [W.Problem(L=8 + 2 * (k % 3), betas=W.linear_ladder(0.2 + 0.01 * k, 0.6, 6 + 3 * k),
                           seed=50 + k) for k in range(10)]
        gs = []
        for p in probs:
            gs.append(api.PTProblem(p.L, p.betas, seed=p.seed, stream=st))
            gs[-1].sweep(3, 1)
            assert api.image_cache_bytes() <= limit
        api.sweep_batch(gs, 4, 2)
        for j, (p, g) in enumerate(zip(probs, gs)):
            o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
            o.sweep(3, 1)
            o.sweep(4, 2)
            assert_same(g, o, "problem %d" % j)
        for g in gs:
            g.close()
        api.set_image_cache_limit(0)
        assert api.image_cache_bytes() == 0
        g = api.PTProblem(probs[0].L, probs[0].betas, seed=probs[0].seed, stream=st)
        assert api.image_cache_bytes() == 0
        o = oracle.OracleProblem(probs[0].L, probs[0].betas, seed=probs[0].seed)
        g.sweep(5, 1)
        o.sweep(5, 1)
        assert_same(g, o, "no cache")
        g.close()
    finally:
        api.set_image_cache_limit(1 << 30)
