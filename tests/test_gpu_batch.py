"""The batched paths (lock-step launches, cluster kernel, dataflow launch): each problem
advanced inside a batch is bit-identical to the same problem advanced alone (plain path) and
to the CPU oracle, for every launch shape the autotuner may pick, and batches compose with
plain sweeps and with each other. The dataflow launch's bounded waits are made to run out
once, on purpose, by a wait for tiles that do not exist."""
from __future__ import annotations

import ctypes as C

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


@pytest.fixture
def tuning(api):
    from paper_2512_03825_b300._lib import lib
    import ctypes as C
    s, c, j = C.c_int(), C.c_int(), C.c_int()
    lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(j))

    def setter(cl, jm, strategy=1):
        assert lib.pt_set_batch_tuning(strategy, cl, jm) == 0
    yield setter
    lib.pt_set_batch_tuning(s.value, c.value, j.value)


def state(g):
    return (g.spins(), g.energies_int(), g.magnetisations(), g.chain_map(),
            *g.swap_stats(), g.counters())


def assert_state_equal(a, b, where=""):
    for x, y in zip(state(a) if not isinstance(a, tuple) else a,
                    state(b) if not isinstance(b, tuple) else b):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y), err_msg=where)


def mixed_problems(n=24, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n):
        L = int(rng.choice([4, 6, 8, 12, 16, 24, 32, 48, 64]))
        R = int(rng.integers(1, 70))
        J, h = [(1.0, 0.0), (1.0, 0.1), (-1.0, 0.25), (1.0, 0.0)][j % 4]
        out.append(W.Problem(L=L, betas=W.linear_ladder(0.2, 0.8, R), J=J, h=h,
                             seed=1000 + j, sweeps=int(rng.integers(0, 30)),
                             every=int(rng.integers(0, 4))))
    return out


def test_batch_equals_plain_and_oracle(api, tuning):
    probs = mixed_problems()
    plain = []
    for pr in probs:
        g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
        g.sweep(pr.sweeps, pr.every)
        plain.append(state(g))
    for st, cl, jm in [(0, 1, 4), (3, 1, 4), (2, 1, 4), (1, 4, 16), (1, 1, 4), (1, 2, 8),
                       (1, 8, 16), (1, 3, 8), (1, 6, 12), (1, 4, 1 << 20)]:
        tuning(cl, jm, st)
        batch = [api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed) for pr in probs]
        api.sweep_batch(batch, [pr.sweeps for pr in probs], [pr.every for pr in probs])
        for j, (b, ref) in enumerate(zip(batch, plain)):
            assert_state_equal(state(b), ref,
                               "strategy %d cluster %d joint>=%d problem %d" % (st, cl, jm, j))
    oracle.set_threads(8)
    for pr in probs[:6]:
        o = oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
        o.sweep(pr.sweeps, pr.every)
        g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
        api.sweep_batch([g], [pr.sweeps], [pr.every])
        np.testing.assert_array_equal(g.spins(), o.spins())
        np.testing.assert_array_equal(g.chain_map(), o.chain_map())
        np.testing.assert_array_equal(g.energies_int(), o.energies_int())


@pytest.mark.parametrize("strategy", [0, 1, 2, 3])
def test_batch_composes_with_plain(api, tuning, strategy):
    tuning(4, 16, strategy)
    pr = W.Problem(L=64, betas=W.linear_ladder(0.3, 0.6, 40), seed=77)
    a = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    b = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    a.sweep(23, 3)
    api.sweep_batch([b], [5], [3])
    b.sweep(7, 3)
    api.sweep_batch([b], [11], [3])
    assert_state_equal(a, b)


@pytest.mark.parametrize("strategy", [0, 1, 2, 3])
def test_batched_workload_sample_vs_oracle(api, tuning, strategy):
    """A sample of the 256-problem batched workload, short runs, against the oracle."""
    tuning(4, 128, strategy)
    probs = W.batched_problems()[:12]
    gs = [api.PTProblem(p.L, p.betas, seed=p.seed) for p in probs]
    api.sweep_batch(gs, 6, 1)
    oracle.set_threads(8)
    for p, g in zip(probs, gs):
        o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
        o.sweep(6, 1)
        np.testing.assert_array_equal(g.spins(), o.spins())
        np.testing.assert_array_equal(g.chain_map(), o.chain_map())
        for x, y in zip(g.swap_stats(), o.swap_stats()):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("tile_words", [64, 160, 1024])
def test_tile_size_never_changes_a_result(api, tuning, tile_words):
    """Lock-step, dataflow and allocation-free batches at several tile sizes equal the plain
    path (the mixed problem set: ragged L, R from 1 to 69, every mode)."""
    import ctypes as C
    from paper_2512_03825_b300._lib import lib
    probs = mixed_problems(n=16, seed=11)
    plain = []
    for pr in probs:
        g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
        g.sweep(pr.sweeps, pr.every)
        plain.append(state(g))
    old = C.c_int()
    lib.pt_get_batch_tile_words(C.byref(old))
    try:
        assert lib.pt_set_batch_tile_words(tile_words) == 0
        for st in (0, 3, 2, "static-dealt", "static-queued"):
            if isinstance(st, int):
                tuning(1, 4, st)
            else:  # the allocation-free entry hands tiles out as the strategy set says
                tuning(1, 4, 3 if st == "static-queued" else 0)
            batch = [api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed) for pr in probs]
            run = api.sweep_batch_static if isinstance(st, str) else api.sweep_batch
            run(batch, [pr.sweeps for pr in probs], [pr.every for pr in probs])
            for j, (b, ref) in enumerate(zip(batch, plain)):
                assert_state_equal(state(b), ref, "tile %d strategy %s problem %d"
                                   % (tile_words, st, j))
    finally:
        lib.pt_set_batch_tile_words(old.value)


def test_batch_rejects_bad_input(api):
    from paper_2512_03825_b300._lib import PTError
    g = api.PTProblem(8, [0.3, 0.4], seed=1)
    with pytest.raises(PTError):
        api.sweep_batch([g, g], 1, 1)
    with pytest.raises(PTError):
        api.sweep_batch([g], -1, 1)
    api.sweep_batch([g], 0, 0)
    assert g.counters() == (0, 0)


def test_flow_uneven_lengths_and_long_runs(api, tuning):
    """Dataflow launch: problems with different sweep counts and exchange periods, many
    tiles per problem (L = 256) next to one-tile problems, equal to the lock-step path."""
    probs = [W.Problem(L=256, betas=W.linear_ladder(0.3, 0.6, 40), seed=11, sweeps=37, every=1),
             W.Problem(L=8, betas=W.linear_ladder(0.3, 0.6, 5), seed=12, sweeps=120, every=3),
             W.Problem(L=96, betas=W.linear_ladder(0.3, 0.6, 33), J=1.0, h=0.1, seed=13,
                       sweeps=64, every=2),
             W.Problem(L=32, betas=(0.4,), seed=14, sweeps=90, every=1)]
    out = {}
    for st in (0, 2):
        tuning(1, 4, st)
        gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
        api.sweep_batch(gs, [p.sweeps for p in probs], [p.every for p in probs])
        api.sweep_batch(gs, [5, 0, 9, 1], [1, 3, 2, 1])
        out[st] = [state(g) for g in gs]
    for j in range(len(probs)):
        assert_state_equal(out[0][j], out[2][j], "problem %d" % j)


def test_flow_wait_runs_out_and_context_survives(api, tuning):
    """One problem's first colour-1 wait expects one tile more than exists: the wait gives
    up after its 50 ms limit, every problem of the call reports PT_ETIMEOUT, and a new
    batch on the same context still equals the oracle."""
    from paper_2512_03825_b300 import _lib
    tuning(1, 4, 2)
    probs = [W.Problem(L=64, betas=W.linear_ladder(0.3, 0.5, 20), seed=21),
             W.Problem(L=32, betas=W.linear_ladder(0.3, 0.5, 9), seed=22)]
    gs = [api.PTProblem(p.L, p.betas, seed=p.seed) for p in probs]
    for g in gs:
        g.set_wait_limit(0.05)
    gs[1].debug_stall_barrier(1)
    api.sweep_batch(gs, 4, 1)
    for g in gs:
        with pytest.raises(_lib.PTError) as ei:
            g.synchronize()
        assert ei.value.code == _lib.PT_ETIMEOUT
        g.close()
    hs = [api.PTProblem(p.L, p.betas, seed=p.seed) for p in probs]
    api.sweep_batch(hs, 6, 1)
    oracle.set_threads(8)
    for p, h in zip(probs, hs):
        o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
        o.sweep(6, 1)
        np.testing.assert_array_equal(h.spins(), o.spins())
        np.testing.assert_array_equal(h.chain_map(), o.chain_map())


@pytest.mark.parametrize("strategy", [0, 3])
@pytest.mark.parametrize("streams", [2, 3, 4])
def test_batch_over_several_streams(api, strategy, streams):
    """The lock-step batch split into parts on their own streams: every problem ends exactly
    as when advanced alone, and the problems' stream is ordered after every part -- a plain
    sweep queued right after the batch, on the same stream, sees the batch's result (checked
    against the oracle)."""
    import torch
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    probs = mixed_problems(n=20, seed=23 + streams)
    try:
        autotune.set_tuning(strategy, 1, 128, 128, streams)
        st = torch.cuda.Stream()
        batch = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=st)
                 for p in probs]
        api.sweep_batch(batch, [p.sweeps for p in probs], [p.every for p in probs])
        for b in batch[:5]:
            b.sweep(3, 2)   # on the problems' stream, right behind the batch's parts
        api.sweep_batch(batch[5:], 2, 1)
    finally:
        autotune.set_tuning(**before)
    oracle.set_threads(8)
    for j, (pr, b) in enumerate(zip(probs, batch)):
        o = oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
        o.sweep(pr.sweeps, pr.every)
        o.sweep(3, 2) if j < 5 else o.sweep(2, 1)
        np.testing.assert_array_equal(b.spins(), o.spins(), err_msg="problem %d" % j)
        np.testing.assert_array_equal(b.energies_int(), o.energies_int(), err_msg=str(j))
        np.testing.assert_array_equal(b.chain_map(), o.chain_map(), err_msg=str(j))
        for x, y in zip(b.swap_stats(), o.swap_stats()):
            np.testing.assert_array_equal(x, y, err_msg=str(j))


@pytest.mark.parametrize("strategy", [0, 3])
def test_field_signs_and_class_sets_match_oracle(api, strategy):
    """Batched problems whose trials compare with five class thresholds (J > 0, 0 < |h| < 2J,
    either sign of the field: the class sets the kernel knows at compile time) and with other
    class counts (|h| >= 2J, J < 0) all equal the oracle."""
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    cases = [(1.0, 0.1), (1.0, -0.1), (1.0, 0.7), (1.0, -1.3), (1.0, 2.5), (-1.0, 0.25),
             (0.5, -0.2), (2.0, 0.0)]
    probs = [W.Problem(L=24 + 8 * (j % 3), betas=W.linear_ladder(0.2, 0.7, 5 + 9 * j), J=J,
                       h=h, seed=7700 + j) for j, (J, h) in enumerate(cases)]
    try:
        autotune.set_tuning(strategy, 1, 128, 128, 1)
        gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
        api.sweep_batch(gs, 9, 2)
    finally:
        autotune.set_tuning(**before)
    oracle.set_threads(8)
    for p, g in zip(probs, gs):
        o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        o.sweep(9, 2)
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg="J %g h %g" % (p.J, p.h))
        np.testing.assert_array_equal(g.energies_int(), o.energies_int())
        np.testing.assert_array_equal(g.chain_map(), o.chain_map())


def test_autotuner_compares_equal_results(api, tuning):
    """The autotuner times a few candidates (tile sizes, strategies), checks that they all
    leave the problems in the same state, and applies the fastest without saving it."""
    from paper_2512_03825_b300 import autotune
    probs = W.batched_problems(n=10)
    cands = [(0, 1, 128, 128, 1, 0), (3, 1, 128, 1024, 1, 0), (2, 1, 128, 256, 1, 0),
             (1, 2, 64, 512, 1, 0), (0, 1, 128, 512, 3, 0), (3, 1, 128, 512, 2, 0),
             (0, 1, 128, 512, 2, 1), (3, 1, 128, 256, 1, 1)]
    out = autotune.tune(probs, sweeps=4, every=1, candidates=cands, repeats=2, save=False)
    assert tuple(out["choice"].values()) in cands
    assert len(out["timings"]) == len(cands)
    assert autotune.get_tuning() == out["choice"]
    autotune.set_tuning(**autotune.DEFAULT)


def test_read_batch_equals_single_getters(api):
    """pt_read_batch returns, for every problem of a mixed set (one slot, several planes,
    the generic mode), exactly what the single getters return."""
    probs = mixed_problems(n=12, seed=17) + [W.Problem(L=8, betas=(0.4,), seed=5)]
    gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
    api.sweep_batch(gs, [max(p.sweeps, 1) for p in probs], [p.every for p in probs])
    api.sweep_batch(gs, 3, 2)  # ends between swap iterations: the counts are recomputed
    listed = gs + [gs[3], gs[0], gs[3]]  # a problem listed again is read once
    got = api.read_batch(listed)
    assert len(got) == len(listed)
    for j, (g, r) in enumerate(zip(listed, got)):
        np.testing.assert_array_equal(r["E_int"], g.energies_int(), err_msg=str(j))
        np.testing.assert_array_equal(r["M"], g.magnetisations(), err_msg=str(j))
        np.testing.assert_array_equal(r["chain_map"], g.chain_map(), err_msg=str(j))
        tm = np.empty(g.R, np.int32)
        from paper_2512_03825_b300._lib import lib
        assert lib.pt_temperature_map(g.handle, tm.ctypes.data_as(C.POINTER(C.c_int32))) == 0
        np.testing.assert_array_equal(tm, r["chain_map"], err_msg=str(j))
        att, acc = g.swap_stats()
        np.testing.assert_array_equal(r["attempted"], att, err_msg=str(j))
        np.testing.assert_array_equal(r["accepted"], acc, err_msg=str(j))
    assert api.read_batch([]) == []


# the plain path's edge cases (test_gpu_parity), here in one batch: beta = 0 and frozen
# temperatures (every threshold saturated either way), one replica, a plane with one slot,
# L / 2 odd, the field and antiferromagnetic modes, no coupling, and exchange tables strided
# by 2^k in n
EDGE_BATCH = [
    W.Problem(L=4, betas=(0.2, 0.44, 0.6), seed=1),
    W.Problem(L=6, betas=W.linear_ladder(0.2, 0.7, 5), seed=2),
    W.Problem(L=10, betas=W.linear_ladder(0.1, 0.9, 33), seed=3),
    W.Problem(L=30, betas=W.linear_ladder(0.3, 0.6, 63), seed=4),
    W.Problem(L=8, betas=(0.4,), seed=5),
    W.Problem(L=12, betas=(0.0, 0.0, 0.3, 10.0), seed=6),
    W.Problem(L=12, betas=(0.0, 0.0, 0.3, 10.0), h=0.1, seed=16),
    W.Problem(L=16, betas=W.linear_ladder(0.2, 0.7, 7), h=0.1, seed=7),
    W.Problem(L=14, betas=W.linear_ladder(0.2, 0.7, 9), J=-1.0, h=0.25, seed=8),
    W.Problem(L=20, betas=W.linear_ladder(0.3, 0.5, 40), J=0.5, h=-0.3, seed=9),
    W.Problem(L=10, betas=W.linear_ladder(0.1, 0.8, 12), J=0.0, h=0.5, seed=13),
    W.Problem(L=12, betas=W.linear_ladder(0.1, 0.4, 12), J=2.0, seed=14),
    W.Problem(L=8, betas=W.linear_ladder(0.05, 0.3, 10), J=3.0, h=1.0, seed=15),
]


@pytest.mark.parametrize("strategy,streams", [(0, 1), (0, 4), (3, 3), (2, 1), (1, 1)])
def test_edge_cases_in_one_batch(api, strategy, streams):
    """Every edge case of the plain path, advanced together by one batch call under each
    batch strategy (dealt and queued tiles on one or several streams, dataflow, cluster),
    with exchange intervals 0, 1 and 3 mixed: each problem equals the oracle."""
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    every = [(0, 1, 3)[j % 3] for j in range(len(EDGE_BATCH))]
    try:
        autotune.set_tuning(strategy, 2, 16, 64, streams)
        gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in EDGE_BATCH]
        api.sweep_batch(gs, 7, every)
        api.sweep_batch(gs, 6, every)
    finally:
        autotune.set_tuning(**before)
    oracle.set_threads(8)
    for j, (p, g) in enumerate(zip(EDGE_BATCH, gs)):
        o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        o.sweep(13, every[j])
        where = "L%d R%d J%g h%g every %d" % (p.L, p.R, p.J, p.h, every[j])
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=where)
        np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where)
        np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where)
        np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where)
        for x, y in zip(g.swap_stats(), o.swap_stats()):
            np.testing.assert_array_equal(x, y, err_msg=where)



@pytest.mark.parametrize("strategy,streams", [(0, 1), (0, 3), (3, 2)])
def test_graph_replay_matches_oracle(api, strategy, streams):
    """Batches replayed from captured graphs (pt_set_batch_graphs): a mixed batch (both
    modes, uneven sweeps, exchange intervals and schedule phases, a traced problem) runs
    three calls of one shape -- the first captures, the next two replay with the problems'
    advanced counters -- then calls of other shapes until the least recently used graph is
    dropped, then the first shape again (captured anew). Every problem equals the oracle, the
    trace rows included, and results equal those of launches without replay."""
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    probs = mixed_problems(n=18, seed=71 + streams)
    ns = [p.sweeps for p in probs]
    ms = [p.every for p in probs]
    plan = [(ns, ms), (ns, ms), (ns, ms)]
    plan += [([k + 1] * len(probs), ms) for k in range(5)]   # five more shapes: evictions
    plan += [(ns, ms)]
    import torch
    st = torch.cuda.Stream()  # replay needs a stream other than the legacy default one
    try:
        autotune.set_tuning(strategy, 1, 128, 128, streams, 1)
        gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=st) for p in probs]
        gs[2].trace_start(64)
        for n, m in plan:
            api.sweep_batch(gs, n, m)
        autotune.set_tuning(strategy, 1, 128, 128, streams, 0)
        hs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs[:6]]
        for n, m in plan:
            api.sweep_batch(hs, n[:6], m[:6])
    finally:
        autotune.set_tuning(**before)
    oracle.set_threads(8)
    for j, (p, g) in enumerate(zip(probs, gs)):
        o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
        for n, m in plan:
            o.sweep(n[j], m[j])
        where = "problem %d" % j
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=where)
        np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where)
        np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where)
        for x, y in zip(g.swap_stats(), o.swap_stats()):
            np.testing.assert_array_equal(x, y, err_msg=where)
        if j < 6:
            np.testing.assert_array_equal(g.spins(), hs[j].spins(), err_msg=where)
    # the traced problem's rows, sweep by sweep across all calls (the ring keeps the last 64)
    first, Eg, Mg = gs[2].trace()
    o = oracle.OracleProblem(probs[2].L, probs[2].betas, J=probs[2].J, h=probs[2].h,
                             seed=probs[2].seed)
    rows = [o.trace(n[2], m[2]) for n, m in plan]
    E = np.concatenate([r[0] for r in rows])
    M = np.concatenate([r[1] for r in rows])
    assert first >= 1 and len(Eg) == min(64, len(E))
    np.testing.assert_array_equal(Eg, E[first - 1:first - 1 + len(Eg)])
    np.testing.assert_array_equal(Mg, M[first - 1:first - 1 + len(Mg)])


def test_graph_replay_with_new_problems_and_streams(api):
    """A replayed graph serves any problems of its shape: each call here creates fresh
    problems (new device arrays, the same shapes), alternating between two streams, and the
    problems of every call equal the oracle -- the descriptors, not the graph, carry the
    problems."""
    import torch
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    probs = mixed_problems(n=10, seed=404)
    ns = [max(1, p.sweeps) for p in probs]
    ms = [p.every for p in probs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    finals = []
    try:
        autotune.set_tuning(0, 1, 128, 128, 2, 1)
        for k in range(4):
            st = streams[k % 2]
            gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed + 100 * k, stream=st)
                  for p in probs]
            api.sweep_batch(gs, ns, ms)
            finals.append([(g.spins(), g.energies_int(), g.chain_map()) for g in gs])
            for g in gs:
                g.close()
    finally:
        autotune.set_tuning(**before)
    oracle.set_threads(8)
    for k in range(4):
        for j, p in enumerate(probs):
            o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed + 100 * k)
            o.sweep(ns[j], ms[j])
            s, e, c = finals[k][j]
            where = "call %d problem %d" % (k, j)
            np.testing.assert_array_equal(s, o.spins(), err_msg=where)
            np.testing.assert_array_equal(e, o.energies_int(), err_msg=where)
            np.testing.assert_array_equal(c, o.chain_map(), err_msg=where)
