"""The documented size limits on the GPU against the oracle, bit for bit: the largest
replica count (PT_MAX_R = 2048 temperatures, 64 planes, 2047 swap pairs) through every sweep
path, the batched strategies and the single-flip kernels, and the largest lattice
(PT_MAX_L = 16384: 2^28 sites, a 1 GiB plane)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_R = 2048
MAX_L = 16384


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
    np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=where)
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y, err_msg=where)
    assert g.counters() == o.counters(), where


MAX_R_PROBLEMS = [
    W.Problem(L=8, betas=W.linear_ladder(0.05, 1.0, MAX_R), seed=0x11AA),
    W.Problem(L=6, betas=W.linear_ladder(0.1, 0.9, MAX_R), J=1.0, h=0.2, seed=0x11AB),
]


@pytest.mark.parametrize("path", ["persistent", "launches", "batch-dealt", "batch-queued",
                                  "batch-flow", "static"])
@pytest.mark.parametrize("k", range(len(MAX_R_PROBLEMS)))
def test_max_replicas_sweeps(api, path, k):
    from paper_2512_03825_b300._lib import lib
    pr = MAX_R_PROBLEMS[k]
    assert pr.R == MAX_R
    g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    o = oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed)
    s, c, jm = C.c_int(), C.c_int(), C.c_int()
    lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(jm))
    try:
        strategy = {"batch-dealt": 0, "batch-queued": 3, "batch-flow": 2, "static": 0}
        if path in strategy:
            assert lib.pt_set_batch_tuning(strategy[path], 1, 128) == 0
        for n, m in ((3, 1), (4, 2)):
            if path in ("persistent", "launches"):
                g.set_sweep_tuning(2 if path == "persistent" else 1)
                g.sweep(n, m)
            elif path == "static":
                api.sweep_batch_static([g], n, m)
            else:
                api.sweep_batch([g], n, m)
            o.sweep(n, m)
        assert_same(g, o, "R=2048 %s problem %d" % (path, k))
    finally:
        lib.pt_set_batch_tuning(s.value, c.value, jm.value)


@pytest.mark.parametrize("shared", [True, False])
def test_max_replicas_single_flips(api, shared):
    pr = MAX_R_PROBLEMS[0]
    g = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    g.set_flip_tuning(shared)
    o = oracle.OracleProblem(pr.L, pr.betas, seed=pr.seed)
    g.flip(130, 20)
    o.flip(130, 20)
    assert_same(g, o, "R=2048 flips shared=%d" % shared)


def test_max_lattice_one_sweep(api):
    """L = 16384 with two temperatures: one sweep with its swap iteration, every spin
    compared."""
    pr = W.Problem(L=MAX_L, betas=(0.3, 0.5), seed=0x11AC)
    g = api.PTProblem(pr.L, pr.betas, seed=pr.seed)
    o = oracle.OracleProblem(pr.L, pr.betas, seed=pr.seed)
    g.sweep(1, 1)
    o.sweep(1, 1)
    np.testing.assert_array_equal(g.chain_map(), o.chain_map())
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations())
    for k in range(pr.R):
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg="temperature %d" % k)
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y)
