"""The ways pt_sweep runs one problem -- one launch per half sweep, or one persistent
cooperative launch whose CTAs meet at grid barriers, in its strided form or with a band of
rows per CTA (one grid barrier per sweep) -- against the CPU oracle, bit for bit, on grids of
one CTA, several CTAs per plane, several planes with a ragged last plane, ragged word shares
and uneven bands; switching between them (and the batched path) mid-run; more sweeps than
one persistent launch takes; and the bounded barrier wait, made to run out on purpose by
waiting for CTAs that do not exist."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu

AUTO, LAUNCHES, PERSISTENT, BANDS = 0, 1, 2, 3


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(8)
    return A


def assert_same(g, o, where=""):
    np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where + " chain map")
    np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where + " E")
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where + " M")
    for k in range(o.R):
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg=where + " spins %d" % k)
    for a, b in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(a, b, err_msg=where + " swap stats")
    assert g.counters() == o.counters(), where


def make(api, prob, strategy, wpt=0):
    g = api.PTProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    g.set_sweep_tuning(strategy, wpt)
    o = oracle.OracleProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    return g, o


CASES = [
    # (L, R, J, h, words per thread, sweeps, exchange_every)
    (4, 1, 1.0, 0.0, 0, 25, 1),        # smallest lattice, one replica, one CTA
    (6, 3, 1.0, 0.0, 1, 30, 1),        # L/2 odd
    (16, 8, 1.0, 0.0, 1, 40, 3),
    (30, 5, -1.0, 0.25, 2, 30, 2),     # generic mode (antiferromagnet in a field)
    (64, 33, 1.0, 0.0, 1, 24, 1),      # two planes, the second with one slot
    (64, 70, 1.0, 0.1, 3, 20, 4),      # three planes, generic, ragged shares
    (130, 40, 0.5, 0.0, 7, 12, 5),     # s = 2, ragged shares
    (128, 32, 1.0, 0.0, 0, 15, 0),     # no exchanges
    # one CTA per plane, the plane in shared memory: two planes (the swap iterations meet
    # at the grid barrier), 8 words per thread; and the largest such plane (L = 128: 64 KB)
    # in the generic mode
    (64, 40, 1.0, 0.0, 8, 20, 1),
    (128, 33, 1.0, 0.1, 32, 6, 2),
]


@pytest.mark.parametrize("strategy", [LAUNCHES, PERSISTENT])
@pytest.mark.parametrize("L,R,J,h,wpt,n,m", CASES)
def test_strategy_matches_oracle(api, strategy, L, R, J, h, wpt, n, m):
    prob = W.Problem(L=L, betas=W.linear_ladder(0.2, 0.7, R), J=J, h=h,
                     seed=0x9E00 + 7 * L + R)
    g, o = make(api, prob, strategy, wpt)
    s, w, grid = g.sweep_tuning()
    assert s == strategy
    if strategy == PERSISTENT:
        W_planes = (R + 31) // 32
        assert grid > 0 and grid % W_planes == 0
        if wpt * 256 >= L * L // 2:  # one CTA per plane
            assert grid == W_planes
    for k in (1, n - 1):                # two calls: the state carries over between launches
        g.sweep(k, m)
        o.sweep(k, m)
    assert_same(g, o, "L%d R%d strategy %d" % (L, R, strategy))


BAND_CASES = [
    # (L, R, J, h, words per thread, sweeps, exchange_every); the band height is the largest
    # whose colour-0 rows (band + 2 halo rows) a CTA of 256 threads updates in one pass
    (24, 8, 1.0, 0.0, 1, 30, 1),       # 2 bands of 12 rows: the halo rows are the other band's
    (30, 5, -1.0, 0.25, 1, 30, 2),     # generic, L/2 odd, 2 bands of 15 rows
    (32, 40, 1.0, 0.0, 1, 24, 1),      # two planes, 3 uneven bands each, one cluster
    (64, 33, 1.0, 0.0, 1, 20, 3),      # 11 uneven bands per plane, the second plane one slot
    (90, 9, 1.0, 0.1, 1, 16, 1),       # 30 bands of 3 rows, generic
    (128, 32, 1.0, 0.0, 1, 20, 1),     # 64 bands of 2 rows, cooperative grid
    (128, 70, 1.0, 0.1, 1, 10, 2),     # three planes, 192 CTAs, generic
    (130, 40, 0.5, 0.0, 1, 12, 5),     # s = 2, bands of one row, two planes
    (256, 32, 1.0, 0.0, 1, 10, 0),     # 256 bands of one row, no exchanges
    (512, 40, 1.0, 0.0, 1, 6, 1),      # taller bands so that the grid stays resident
    (128, 32, 1.0, 0.0, 2, 12, 1),     # 16 bands of 8 rows: one cluster
]


@pytest.mark.parametrize("L,R,J,h,wpt,n,m", BAND_CASES)
def test_bands_match_oracle(api, L, R, J, h, wpt, n, m):
    prob = W.Problem(L=L, betas=W.linear_ladder(0.2, 0.7, R), J=J, h=h,
                     seed=0xBA00 + 7 * L + R)
    g, o = make(api, prob, BANDS, wpt)
    s, w, grid = g.sweep_tuning()
    assert s == BANDS and grid >= 2 * ((R + 31) // 32)
    for k in (1, n - 1):                # two launches: the bands are reloaded by the second
        g.sweep(k, m)
        o.sweep(k, m)
    assert_same(g, o, "bands L%d R%d" % (L, R))


def test_bands_traced_and_switched(api):
    """The band form with a trace (every sweep counted), then the strided form and the band
    form again on the same problem: every trace row and the final state equal the oracle."""
    prob = W.Problem(L=48, betas=W.linear_ladder(0.3, 0.6, 12), J=1.0, h=0.1, seed=0xBA77)
    g, o = make(api, prob, BANDS, 1)
    g.trace_start(20)
    g.sweep(8, 3)
    g.set_sweep_tuning(PERSISTENT, 1)
    g.sweep(5, 3)
    g.set_sweep_tuning(BANDS, 1)
    g.sweep(7, 3)
    E, M = o.trace(20, 3)
    first, Eg, Mg = g.trace()
    assert first == 1
    np.testing.assert_array_equal(Eg, E)
    np.testing.assert_array_equal(Mg, M)
    assert_same(g, o, "bands traced")


def test_bands_refused_where_they_do_not_fit(api):
    from paper_2512_03825_b300 import _lib
    # L = 4096: a band of every resident CTA's share of rows (14 rows and 2 halo rows of 2048
    # words each) does not fit the 48 KB of shared copies
    g = api.PTProblem(4096, [0.3])
    g.set_sweep_tuning(BANDS)
    assert g.sweep_tuning()[2] == 0
    with pytest.raises(_lib.PTError) as ei:
        g.sweep(1, 1)
    assert ei.value.code == _lib.PT_EINVAL
    g.set_sweep_tuning(AUTO)
    g.sweep(1, 1)
    g.synchronize()


def test_grid_follows_words_per_thread(api):
    prob = W.Problem(L=256, betas=W.linear_ladder(0.3, 0.6, 64), seed=5)
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    grids = []
    for wpt in (1, 4, 16, 64, 255):
        g.set_sweep_tuning(PERSISTENT, wpt)
        grids.append(g.sweep_tuning()[2])
    words = 256 * 128
    assert all(x % 2 == 0 for x in grids)
    assert grids == sorted(grids, reverse=True)
    assert grids[-1] == 2 and grids[3] == 2 * words // (64 * 256)


def test_switching_strategies_mid_run(api):
    """Launches, persistent, batched and persistent again, one after the other on one
    problem, equal the oracle: each path leaves the maps, thresholds and counts as the next
    one expects."""
    prob = W.Problem(L=96, betas=W.linear_ladder(0.25, 0.65, 48), J=1.0, h=0.0, seed=77)
    g, o = make(api, prob, LAUNCHES)
    g.sweep(7, 2)
    o.sweep(7, 2)
    g.set_sweep_tuning(PERSISTENT, 1)
    g.sweep(9, 2)
    o.sweep(9, 2)
    assert_same(g, o, "launches then persistent")
    api.sweep_batch([g], 5, 2)
    o.sweep(5, 2)
    g.sweep(6, 3)
    o.sweep(6, 3)
    assert_same(g, o, "then batched, then persistent")
    g.set_sweep_tuning(LAUNCHES)
    g.sweep(4, 3)
    o.sweep(4, 3)
    assert_same(g, o, "then launches again")


def test_more_sweeps_than_one_launch(api):
    """70000 sweeps is two persistent launches (65536 + 4464)."""
    prob = W.Problem(L=4, betas=(0.3, 0.45, 0.6), seed=123)
    g, o = make(api, prob, PERSISTENT)
    g.sweep(70000, 7)
    o.sweep(70000, 7)
    assert_same(g, o, "70000 sweeps")


def test_persistent_equals_launches_at_L512(api):
    prob = W.Problem(L=512, betas=W.linear_ladder(0.35, 0.5, 64), seed=0x5EED0042)
    a = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    b = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    a.set_sweep_tuning(LAUNCHES)
    b.set_sweep_tuning(PERSISTENT)
    a.sweep(40, 5)
    b.sweep(40, 5)
    np.testing.assert_array_equal(a.chain_map(), b.chain_map())
    np.testing.assert_array_equal(a.energies_int(), b.energies_int())
    for x, y in zip(a.swap_stats(), b.swap_stats()):
        np.testing.assert_array_equal(x, y)
    for k in range(0, 64, 9):
        np.testing.assert_array_equal(a.spins(k), b.spins(k))


def test_tuning_arguments_checked(api):
    from paper_2512_03825_b300 import _lib
    g = api.PTProblem(8, [0.3])
    for call in (lambda: g.set_sweep_tuning(4), lambda: g.set_sweep_tuning(PERSISTENT, 256),
                 lambda: g.set_sweep_tuning(PERSISTENT, -1), lambda: g.set_wait_limit(0.0),
                 lambda: g.set_wait_limit(61.0), lambda: g.debug_stall_barrier(-1)):
        with pytest.raises(_lib.PTError) as ei:
            call()
        assert ei.value.code == _lib.PT_EINVAL
    g.sweep(3, 1)                       # nothing above changed the problem
    g.synchronize()


@pytest.mark.parametrize("strategy", [PERSISTENT, BANDS])
def test_barrier_wait_runs_out_and_context_survives(api, strategy):
    """The first grid barrier waits for one CTA more than the launch has: every wait gives
    up after the 50 ms limit, the problem reports PT_ETIMEOUT and stays poisoned, and a new
    problem on the same context still matches the oracle."""
    from paper_2512_03825_b300 import _lib
    prob = W.Problem(L=64, betas=W.linear_ladder(0.3, 0.5, 40), seed=9)
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    g.set_sweep_tuning(strategy, 1)
    g.set_wait_limit(0.05)
    g.debug_stall_barrier(1)
    g.sweep(3, 1)
    with pytest.raises(_lib.PTError) as ei:
        g.synchronize()
    assert ei.value.code == _lib.PT_ETIMEOUT
    with pytest.raises(_lib.PTError) as ei:
        g.sweep(1, 1)
    assert ei.value.code in (_lib.PT_ETIMEOUT, _lib.PT_ESTATE)
    g.close()
    h, o = make(api, prob, strategy, 1)
    h.sweep(12, 1)
    o.sweep(12, 1)
    assert_same(h, o, "after a timed-out launch")


def test_kernel_smem_limits_survive_smaller_problems(api):
    """A kernel's dynamic shared-memory limit is process-wide: planning a small problem must
    not lower it under a larger problem that was planned before (persistent sweep and the
    shared-memory single-flip kernel)."""
    big = W.Problem(L=64, betas=W.linear_ladder(0.3, 0.6, 2048), seed=61)
    small = W.Problem(L=16, betas=W.linear_ladder(0.3, 0.6, 4), seed=62)
    a = api.PTProblem(big.L, big.betas, seed=big.seed)
    b = api.PTProblem(small.L, small.betas, seed=small.seed)
    a.set_sweep_tuning(2)
    b.set_sweep_tuning(2)
    a.sweep(2, 1)       # plans the large problem
    b.sweep(2, 1)       # plans the small one
    a.sweep(2, 1)       # the large problem's launch still fits the kernel's limit
    a.flip(40, 10)
    b.flip(40, 10)
    a.flip(40, 10)
    o = oracle.OracleProblem(big.L, big.betas, seed=big.seed)
    oracle.set_threads(8)
    o.sweep(4, 1)
    o.flip(80, 10)
    np.testing.assert_array_equal(a.energies_int(), o.energies_int())
    np.testing.assert_array_equal(a.chain_map(), o.chain_map())


def test_plain_path_tuner_compares_equal_results(api, tmp_path, monkeypatch):
    """The plain-path autotuner times the halo schemes (strided words, bands of rows) and
    words-per-thread settings on fresh copies of one problem, skips the shapes the problem
    does not fit, checks that all of them end in the same state (the oracle's), and the
    choice it caches is the one apply_single gives a new handle."""
    from paper_2512_03825_b300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    p = W.Problem(L=64, betas=W.linear_ladder(0.3, 0.6, 40), seed=515, every=2)
    r = autotune.tune_single(p, sweeps=30, every=2, save=True)
    shapes = [c for c, _ in r["timings"]]
    assert (PERSISTENT, 1) in shapes and (LAUNCHES, 1) in shapes and (BANDS, 1) in shapes
    assert tuple(r["choice"].values()) in shapes
    g = api.PTProblem(p.L, p.betas, seed=p.seed)
    got = autotune.apply_single(g, p.L, p.R, p.J, p.h)
    assert got == r["choice"]
    assert g.sweep_tuning()[:2] == (got["strategy"], got["words_per_thread"])
    g.sweep(30, 2)
    o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
    o.sweep(30, 2)
    assert_same(g, o, "tuned shape")
    assert autotune.apply_single(g, 48, p.R, p.J, p.h) is None


@pytest.mark.parametrize("L,R,m", [(128, 32, 3), (128, 32, 0), (64, 33, 3), (96, 40, 2)])
def test_bands_launch_ends_and_count_buffers(api, L, R, m):
    """Band-form launches of many lengths, ending on even and odd sweep indices, with and
    without a swap iteration on their last sweep: a band copies its last colour 1 back into
    the spin array only after every band is done reading it, and the three count buffers
    take turns without one being counted into before it is cleared."""
    prob = W.Problem(L=L, betas=W.linear_ladder(0.2, 0.7, R), seed=0xBE00 + L + R)
    g, o = make(api, prob, BANDS, 1)
    for k in (1, 19, 2, 4, 7, 6, 3, 10):
        g.sweep(k, m)
        o.sweep(k, m)
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg="after %d more" % k)
    assert_same(g, o, "bands L%d R%d m%d" % (L, R, m))
