"""The paper's own workload (Sec. 4: 300 x 300 lattice, J = 1, B = 0, temperatures
T_i = 1 + 3i/|R| for 1500 replicas, 47 replica words per site) on the GPU: it runs on the
persistent plain path, its last sweep equals the oracle's continuation of the GPU's state bit
for bit, and its magnetisation-versus-temperature curve (the paper's Fig. 3a) follows
Onsager's exact spontaneous magnetisation away from the critical temperature."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W
from tests.stats import BETA_C, onsager_magnetisation

pytestmark = pytest.mark.gpu

PERSISTENT = 2


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(16)
    return A


def test_paper_workload_runs_persistent_and_matches_oracle(api):
    prob = W.paper_problem()
    assert prob.L == 300 and prob.R == 1500
    assert abs(1.0 / prob.betas[0] - 1.0) < 1e-12 and abs(1.0 / prob.betas[-1] - 3.998) < 1e-12
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    g.set_sweep_tuning(PERSISTENT)
    _, _, grid = g.sweep_tuning()
    assert grid > 0 and grid % 47 == 0
    g.sweep(3, 2)                                  # one swap iteration (after sweep 2)
    # the oracle continues from the GPU's exact state
    so = g.chain_map()
    sp = np.empty((prob.R, prob.L, prob.L), np.int8)
    for k in range(prob.R):
        sp[so[k]] = g.spins(k)
    att, acc = g.swap_stats()
    o = oracle.OracleProblem(prob.L, prob.betas, seed=prob.seed)
    o.load_state(sp, so, *g.counters(), att, acc)
    g.sweep(1, 2)                                  # sweep 4 and swap iteration 1 (odd pairs)
    o.sweep(1, 2)
    np.testing.assert_array_equal(g.chain_map(), o.chain_map())
    np.testing.assert_array_equal(g.energies_int(), o.energies_int())
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations())
    for x, y in zip(g.swap_stats(), o.swap_stats()):
        np.testing.assert_array_equal(x, y)
    for k in (0, 1, 31, 32, 750, 1468, 1499):      # first, plane edges, middle, last plane
        np.testing.assert_array_equal(g.spins(k), o.spins(k), err_msg="temperature %d" % k)


def test_paper_magnetisation_curve(api):
    """Fig. 3a: |M| / L^2 against T. All replicas start fully ordered (the paper gives every
    replica the same +1 / -1 ratio); 1500 sweeps with a swap iteration every 10 settle them,
    and the mean over the next 1500 sweeps (from the device trace) is compared with Onsager's
    m(T) = (1 - sinh^-4(2/T))^(1/8) below T_c and with zero above it, away from T_c where
    the finite lattice and critical slowing down blur the curve."""
    prob = W.paper_problem()
    g = api.PTProblem(prob.L, prob.betas, seed=prob.seed)
    up = np.ones((prob.L, prob.L), np.int8)
    for k in range(prob.R):
        g.set_spins(k, up)
    g.sweep(1500, 10)
    g.trace_start(1500)
    g.sweep(1500, 10)
    _, _, M = g.trace()
    m = np.abs(M).mean(axis=0) / (prob.L * prob.L)
    T = 1.0 / np.asarray(prob.betas)
    Tc = 1.0 / BETA_C
    low = T < 1.9
    exact = np.array([onsager_magnetisation(b) for b in prob.betas])
    assert np.max(np.abs(m[low] - exact[low])) < 0.01
    assert np.all(m[T > 2.8] < 0.06)
    # the phase transition: the curve falls from > 0.9 to < 0.3 across T_c
    assert m[(T > 2.0) & (T < 2.1)].mean() > 0.85 and m[(T > 2.45) & (T < 2.55)].mean() < 0.3
    assert 2.1 < Tc < 2.4
