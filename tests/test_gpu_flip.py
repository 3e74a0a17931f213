"""The single-spin-flip variant on the GPU (one thread per replica, one random site per
iteration) against the oracle bit for bit: alone and interleaved with sweeps (they share the
swap index), at the paper's full workload through a hand-off of the GPU state, across a
checkpoint, and with its bounded barrier wait made to run out on purpose."""
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


def assert_same(g, o, where=""):
    np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where)
    np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=where)
    np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where)
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where)
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y, err_msg=where)
    assert g.counters() == o.counters(), where
    assert g.iterations == o.iterations, where


CASES = [
    W.Problem(L=8, betas=W.linear_ladder(0.2, 0.7, 8), seed=201),
    W.Problem(L=16, betas=W.linear_ladder(0.25, 0.65, 70), seed=202),             # 3 planes
    W.Problem(L=12, betas=W.linear_ladder(0.3, 0.6, 6), J=1.0, h=0.1, seed=203),  # field
    W.Problem(L=10, betas=(0.44,), J=-1.0, seed=204),                             # one slot
    W.Problem(L=12, betas=(0.0, 0.0, 0.3, 10.0), seed=205),       # beta 0 and frozen: saturated
    W.Problem(L=12, betas=(0.0, 0.3, 10.0), h=0.2, seed=206),     # the same with a field
    W.Problem(L=10, betas=W.linear_ladder(0.1, 0.8, 12), J=0.0, h=0.5, seed=207),  # no coupling
    W.Problem(L=6, betas=W.linear_ladder(0.05, 0.3, 10), J=3.0, h=1.0, seed=208),  # L / 2 odd
]


@pytest.mark.parametrize("shared", [True, False])
@pytest.mark.parametrize("m", [0, 1, 7])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_flip_matches_oracle(api, k, m, shared):
    """Both kernels: replicas in shared memory (the default) and in the global spin words."""
    pr = CASES[k]
    g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    g.set_flip_tuning(shared)
    o = oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    for n in (1, 60, 139):          # several calls: counters and energies carry over
        g.flip(n, m)
        o.flip(n, m)
    assert_same(g, o, "case %d m %d shared %d" % (k, m, shared))


def test_flips_and_sweeps_share_the_swap_index(api):
    pr = CASES[1]
    g = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    o = oracle.OracleProblem(pr.L, pr.betas, seed=pr.seed)
    for step in (("flip", 33, 5), ("sweep", 3, 2), ("flip", 20, 4), ("sweep", 1, 1)):
        getattr(g, step[0])(step[1], step[2])
        getattr(o, step[0])(step[1], step[2])
    assert_same(g, o, "interleaved")


def test_paper_workload_single_flip_handoff(api):
    """The paper's run read literally (L = 300, 1500 replicas, swaps every 100 iterations):
    the GPU runs 1000 iterations, the oracle takes over the GPU's exact state, and both run
    the next 150 iterations (one more swap iteration) identically."""
    prob = W.paper_problem()
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    g.flip(1000, 100)
    so = g.chain_map()
    sp = np.empty((prob.R, prob.L, prob.L), np.int8)
    for k in range(prob.R):
        sp[so[k]] = g.spins(k)
    att, acc = g.swap_stats()
    o = oracle.OracleProblem(prob.L, prob.betas, seed=prob.seed)
    o.load_state(sp, so, *g.counters(), att, acc)
    o.set_iterations(g.iterations)
    g.flip(150, 100)
    o.flip(150, 100)
    np.testing.assert_array_equal(g.chain_map(), o.chain_map())
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations())
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y)
    for k in (0, 31, 32, 777, 1499):
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg=str(k))


def test_checkpoint_carries_iterations(api):
    pr = CASES[2]
    ref = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    ref.flip(90, 7)
    ref.sweep(4, 2)
    a = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    a.flip(50, 7)
    b = api.PTProblem.load(a.save())
    assert b.iterations == 50
    b.flip(40, 7)
    b.sweep(4, 2)
    for x, y in zip((b.spins(), b.chain_map(), b.energies_int(), *b.swap_stats()),
                    (ref.spins(), ref.chain_map(), ref.energies_int(), *ref.swap_stats())):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("shared", [True, False])
def test_flip_wait_runs_out(api, shared):
    from paper_2512_03825_b300 import _lib
    pr = CASES[1]
    g = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    g.set_flip_tuning(shared)
    g.set_wait_limit(0.05)
    g.debug_stall_barrier(1)
    g.flip(20, 5)
    with pytest.raises(_lib.PTError) as ei:
        g.synchronize()
    assert ei.value.code == _lib.PT_ETIMEOUT
