"""Observable traces: the device ring of per-sweep (E_int, M) rows by temperature index equals
the oracle's trace (recorded after each sweep and its swap iteration) bit for bit, through
every sweep strategy and the batched path, across calls, after the ring wraps, and when the
trace starts in mid-run."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu

LAUNCHES, PERSISTENT = 1, 2


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(8)
    return A


PROBS = [
    W.Problem(L=16, betas=W.geometric_ladder(0.2, 0.6, 8), seed=0x5EED0001),       # config 1
    W.Problem(L=24, betas=W.linear_ladder(0.2, 0.7, 37), seed=41),                   # two planes
    W.Problem(L=20, betas=W.linear_ladder(0.3, 0.6, 6), J=1.0, h=0.1, seed=42),      # generic
    W.Problem(L=12, betas=(0.44,), J=-1.0, h=0.0, seed=43),                          # one slot
]


def oracle_of(pr):
    return oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)


def gpu_of(api, pr, strategy):
    g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    g.set_sweep_tuning(strategy)
    return g


@pytest.mark.parametrize("strategy", [LAUNCHES, PERSISTENT])
@pytest.mark.parametrize("k", range(len(PROBS)))
def test_trace_equals_oracle(api, strategy, k):
    pr = PROBS[k]
    for m in (0, 1, 3):
        g, o = gpu_of(api, pr, strategy), oracle_of(pr)
        g.trace_start(64)
        g.sweep(17, m)
        g.sweep(5, m)  # a second call continues the ring
        first, E, M = g.trace()
        Eo, Mo = o.trace(22, m)
        assert first == 1 and E.shape == (22, pr.R)
        np.testing.assert_array_equal(E, Eo, err_msg="E, m=%d" % m)
        np.testing.assert_array_equal(M, Mo, err_msg="M, m=%d" % m)
        np.testing.assert_array_equal(E[-1], g.energies_int())
        np.testing.assert_array_equal(M[-1], g.magnetisations())


@pytest.mark.parametrize("strategy", [LAUNCHES, PERSISTENT])
def test_ring_wraps_and_late_start(api, strategy):
    pr = PROBS[1]
    g, o = gpu_of(api, pr, strategy), oracle_of(pr)
    g.sweep(9, 2)          # untraced
    o.sweep(9, 2)
    g.trace_start(7)
    g.sweep(30, 2)
    first, E, M = g.trace()
    Eo, Mo = o.trace(30, 2)
    assert first == 9 + 24 and E.shape[0] == 7      # sweeps 33..39 done
    np.testing.assert_array_equal(E, Eo[-7:])
    np.testing.assert_array_equal(M, Mo[-7:])
    first3, E3, _ = g.trace(3)                       # the newest three only
    assert first3 == 37
    np.testing.assert_array_equal(E3, Eo[-3:])
    bytes_on = g.device_bytes
    g.trace_stop()
    assert g.device_bytes == bytes_on - 7 * pr.R * 16
    from paper_2512_03825_b300 import _lib
    with pytest.raises(_lib.PTError) as ei:
        g.trace()
    assert ei.value.code == _lib.PT_ESTATE
    g.sweep(3, 2)          # untraced again, still equal to the oracle
    o.sweep(3, 2)
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())


@pytest.mark.parametrize("strategy", [0, 1, 3])
def test_batch_with_traced_and_untraced_problems(api, strategy):
    """The batch runs a lock-step path when a problem is traced (the queued one when it is
    set, else the dealt one); the traced problems' rows equal the oracle's and the untraced
    ones are unaffected."""
    import ctypes as C
    from paper_2512_03825_b300._lib import lib
    s, c, jm = C.c_int(), C.c_int(), C.c_int()
    lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(jm))
    assert lib.pt_set_batch_tuning(strategy, 4, 128) == 0
    try:
        _traced_batch(api)
    finally:
        lib.pt_set_batch_tuning(s.value, c.value, jm.value)


def _traced_batch(api):
    probs = PROBS + [W.Problem(L=32, betas=W.linear_ladder(0.3, 0.6, 20), seed=44)]
    gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
    for g in gs[::2]:
        g.trace_start(100)
    ns = [12, 7, 20, 3, 15]
    ms = [1, 2, 0, 1, 5]
    api.sweep_batch(gs, ns, ms)
    for j, (g, p) in enumerate(zip(gs, probs)):
        o = oracle_of(p)
        Eo, Mo = o.trace(ns[j], ms[j])
        np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=str(j))
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=str(j))
        if j % 2 == 0:
            first, E, M = g.trace()
            assert first == 1
            np.testing.assert_array_equal(E, Eo, err_msg=str(j))
            np.testing.assert_array_equal(M, Mo, err_msg=str(j))


def test_trace_arguments(api):
    from paper_2512_03825_b300 import _lib
    g = api.PTProblem(8, [0.3, 0.4])
    for cap in (0, -5):
        with pytest.raises(_lib.PTError) as ei:
            g.trace_start(cap)
        assert ei.value.code == _lib.PT_EINVAL
    g.trace_stop()         # no trace: a no-op
    g.trace_start(4)
    first, E, M = g.trace()
    assert E.shape == (0, 2)
