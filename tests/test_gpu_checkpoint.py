"""Checkpoint / resume and the Metropolis swap option on the GPU. A problem restored from a
checkpoint continues exactly as the saved one would have (against an uninterrupted run and,
through an independent decoder of the documented byte layout, against the oracle); the
Metropolis swap rule equals the oracle's bit for bit on every path."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W
from tests.helpers import checkpoint as ck

pytestmark = pytest.mark.gpu

BARKER, METROPOLIS = 0, 1


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(8)
    return A


def state(g):
    return (g.spins(), g.energies_int(), g.magnetisations(), g.chain_map(), *g.swap_stats(),
            np.array(g.counters()))


def assert_same(a, b, where=""):
    for x, y in zip(state(a), state(b)):
        np.testing.assert_array_equal(x, y, err_msg=where)


CASES = [
    W.Problem(L=16, betas=W.linear_ladder(0.2, 0.7, 8), seed=101),
    W.Problem(L=24, betas=W.linear_ladder(0.25, 0.65, 41), seed=102),              # two planes
    W.Problem(L=20, betas=W.linear_ladder(0.3, 0.6, 6), J=1.0, h=0.1, seed=103),   # generic
]


@pytest.mark.parametrize("rule", [BARKER, METROPOLIS])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_resume_equals_uninterrupted_run(api, rule, k):
    pr = CASES[k]
    ref = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed, swap_rule=rule)
    ref.sweep(23, 3)
    a = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed, swap_rule=rule)
    a.sweep(13, 3)
    data = a.save()
    a.close()
    b = api.PTProblem.load(data)
    assert b.L == pr.L and b.R == pr.R and b.swap_rule == rule
    assert b.save() == data                     # save -> load -> save is the identity
    b.sweep(10, 3)
    assert_same(b, ref, "rule %d case %d" % (rule, k))


def test_checkpoint_decoded_into_the_oracle(api):
    """The documented byte layout, decoded by the test's own reader, is the state the oracle
    continues from: both then take the same sweeps."""
    pr = CASES[1]
    g = api.PTProblem(pr.L, pr.betas, seed=pr.seed, swap_rule=METROPOLIS)
    g.sweep(9, 2)
    c = ck.parse(g.save())
    assert (c["L"], c["R"], c["t"], c["e"], c["rule"]) == (pr.L, pr.R, 9, 4, METROPOLIS)
    spins = ck.words_to_spins(c["words"], pr.R)
    o = oracle.OracleProblem(pr.L, pr.betas, seed=pr.seed, swap_rule=oracle.SWAP_METROPOLIS)
    o.load_state(spins, c["slot_of_temp"], c["t"], c["e"], c["attempted"], c["accepted"])
    g.sweep(7, 2)
    o.sweep(7, 2)
    np.testing.assert_array_equal(g.chain_map(), o.chain_map())
    np.testing.assert_array_equal(g.spins(), o.spins())
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("path", ["persistent", "launches", "batch"])
def test_metropolis_rule_matches_oracle(api, path):
    for pr in CASES:
        g = api.PTProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed, swap_rule=METROPOLIS)
        o = oracle.OracleProblem(pr.L, pr.betas, J=pr.J, h=pr.h, seed=pr.seed,
                                 swap_rule=oracle.SWAP_METROPOLIS)
        if path == "batch":
            api.sweep_batch([g], 30, 1)
        else:
            g.set_sweep_tuning(2 if path == "persistent" else 1)
            g.sweep(30, 1)
        o.sweep(30, 1)
        np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=path)
        np.testing.assert_array_equal(g.spins(), o.spins(), err_msg=path)
        for x, y in zip(g.swap_stats(), o.swap_stats()):
            np.testing.assert_array_equal(x, y, err_msg=path)
    # the two rules differ: at equal temperatures Metropolis accepts every swap
    g = api.PTProblem(12, [0.4] * 5, seed=9, swap_rule=METROPOLIS)
    g.sweep(40, 1)
    att, acc = g.swap_stats()
    assert (att == acc).all() and att.sum() > 0
