"""Bit-exact parity of the CUDA path with the CPU oracle on the same seeded inputs: every spin
of every replica, every energy and magnetisation, the temperature map and every swap
counter. Integer work, so the bar is equality."""
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
    return A


def assert_same(gpu, ref, where=""):
    np.testing.assert_array_equal(gpu.chain_map(), ref.chain_map(), err_msg=where + " chain map")
    np.testing.assert_array_equal(gpu.energies_int(), ref.energies_int(), err_msg=where + " E")
    np.testing.assert_array_equal(gpu.magnetisations(), ref.magnetisations(),
                                  err_msg=where + " M")
    for k in range(ref.R):
        np.testing.assert_array_equal(gpu.spins(k), ref.spins(k), err_msg=where + " spins %d" % k)
    for a, b in zip(gpu.swap_stats(), ref.swap_stats()):
        np.testing.assert_array_equal(a, b, err_msg=where + " swap stats")
    assert gpu.counters() == ref.counters()


def pair(api, prob, threads=8):
    g = api.PTProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    o = oracle.OracleProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    oracle.set_threads(threads)
    return g, o


def test_initial_state(api):
    for prob in [W.SINGLE["L16_R8"], W.Problem(L=6, betas=(0.1, 0.2, 0.3), seed=3),
                 W.Problem(L=48, betas=W.linear_ladder(0.3, 0.6, 37), seed=11)]:
        g, o = pair(api, prob)
        assert_same(g, o, "init")


def test_first_sweep_and_first_exchange(api):
    prob = W.SINGLE["L128_R32"]
    g, o = pair(api, prob)
    g.sweep(1, 0)
    o.sweep(1, 0)
    assert_same(g, o, "after one sweep")
    g.sweep(1, 2)
    o.sweep(1, 2)
    assert_same(g, o, "after the first exchange")


def test_config_L16_R8_full(api):
    prob = W.SINGLE["L16_R8"]
    g, o = pair(api, prob)
    g.sweep(prob.sweeps, prob.every)
    o.sweep(prob.sweeps, prob.every)
    assert_same(g, o, "L16 R8 1000 sweeps")


def test_config_L128_R32_prefix(api):
    prob = W.SINGLE["L128_R32"]
    g, o = pair(api, prob)
    for n in (1, 9, 40):
        g.sweep(n, prob.every)
        o.sweep(n, prob.every)
        assert_same(g, o, "L128 R32 after %d more" % n)


def test_config_L1024_R64_prefix(api):
    prob = W.SINGLE["L1024_R64"]
    g, o = pair(api, prob)
    g.sweep(5, prob.every)
    o.sweep(5, prob.every)
    assert_same(g, o, "L1024 R64 5 sweeps")


@pytest.mark.parametrize("prob", [
    W.Problem(L=4, betas=(0.2, 0.44, 0.6), seed=1),
    W.Problem(L=6, betas=W.linear_ladder(0.2, 0.7, 5), seed=2),
    W.Problem(L=10, betas=W.linear_ladder(0.1, 0.9, 33), seed=3),        # second plane, 1 slot
    W.Problem(L=30, betas=W.linear_ladder(0.3, 0.6, 63), seed=4),
    W.Problem(L=8, betas=(0.4,), seed=5),                                # single replica
    W.Problem(L=12, betas=(0.0, 0.0, 0.3, 10.0), seed=6),                # beta 0 and frozen
    W.Problem(L=16, betas=W.linear_ladder(0.2, 0.7, 7), h=0.1, seed=7),  # field: generic path
    W.Problem(L=14, betas=W.linear_ladder(0.2, 0.7, 9), J=-1.0, h=0.25, seed=8),  # antiferro
    W.Problem(L=20, betas=W.linear_ladder(0.3, 0.5, 40), J=0.5, h=-0.3, seed=9),
    W.Problem(L=96, betas=W.linear_ladder(0.3, 0.6, 48), seed=10),
    # exchange tables strided by 2^k in n (k = 1, 3, 1): no coupling, J_int = 2, and
    # gcd(4 J_int, 2 h_int) = 2
    W.Problem(L=10, betas=W.linear_ladder(0.1, 0.8, 12), J=0.0, h=0.5, seed=13),
    W.Problem(L=12, betas=W.linear_ladder(0.1, 0.4, 12), J=2.0, seed=14),
    W.Problem(L=8, betas=W.linear_ladder(0.05, 0.3, 10), J=3.0, h=1.0, seed=15),
], ids=lambda p: "L%d_R%d_J%g_h%g" % (p.L, p.R, p.J, p.h))
@pytest.mark.parametrize("every", [0, 1, 3])
def test_edge_cases(api, prob, every):
    g, o = pair(api, prob)
    g.sweep(7, every)
    o.sweep(7, every)
    assert_same(g, o)
    g.sweep(6, every)
    o.sweep(6, every)
    assert_same(g, o)


def test_set_spins_roundtrip_and_parity(api):
    prob = W.Problem(L=24, betas=W.linear_ladder(0.3, 0.6, 10), seed=12)
    g, o = pair(api, prob)
    for k in range(prob.R):
        s = W.random_spins(prob.L, 100 + k)
        g.set_spins(k, s)
        o.set_spins(k, s)
        np.testing.assert_array_equal(g.spins(k), s)
    g.sweep(10, 2)
    o.sweep(10, 2)
    assert_same(g, o)


def test_splitting_invariance(api):
    prob = W.Problem(L=32, betas=W.linear_ladder(0.3, 0.6, 20), seed=13)
    a = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    b = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    a.sweep(17, 3)
    for n in (5, 0, 1, 11):
        b.sweep(n, 3)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.chain_map(), b.chain_map())
    assert a.counters() == b.counters() == (17, 5)


def test_bad_calls(api):
    from paper_2512_03825_b300 import _lib
    g = api.PTProblem(8, [0.3, 0.4], seed=1)
    with pytest.raises(_lib.PTError):
        g.sweep(-1, 0)
    with pytest.raises(_lib.PTError):
        g.sweep(1, -2)
    with pytest.raises(_lib.PTError):
        g.spins(2)
    with pytest.raises(_lib.PTError):
        g.set_spins(0, np.zeros((8, 8), np.int8))
    g.sweep(3, 1)
    g.synchronize()
