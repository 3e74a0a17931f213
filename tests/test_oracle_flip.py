"""Pins of the oracle's single-spin-flip variant (the paper's "iteration", Sec. 2.1, read as
one Metropolis trial at one uniformly chosen site): closed forms at infinite temperature, the
exact stationary moments of a 4 x 4 lattice, the swap schedule counted in iterations, and
its independence of the thread count."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import stats


def test_infinite_temperature_decay_pins_uniform_sites():
    """beta = 0: every trial flips. From the all-up state, spin i after n iterations is
    (-1)^{k_i} with k_i ~ Binomial(n, p_i); uniform sites (p_i = 1/N) give
    E[M] = N (1 - 2/N)^n. Averaged over 2048 independent replicas."""
    L, R = 8, 2048
    N = L * L
    o = oracle.OracleProblem(L, [0.0] * R, seed=77)
    up = np.ones((L, L), np.int8)
    for k in range(R):
        o.set_spins(k, up)
    oracle.set_threads(8)
    for n_total in (16, 64):
        o.flip(n_total - (16 if n_total == 64 else 0), 0)
        M = o.magnetisations().astype(np.float64)
        expect = N * (1 - 2 / N) ** n_total
        var = N * (1 - (1 - 4 / N) ** n_total) - 0  # upper bound of Var M for uniform sites
        se = math.sqrt(max(var, 1.0) / R)
        assert abs(M.mean() - expect) < 4 * se, (n_total, M.mean(), expect, se)
        # half of the sites alone would leave E[M] = N/2 + N/2 (1 - 4/N)^n: far away
        assert abs(N / 2 + N / 2 * (1 - 4 / N) ** n_total - expect) > 10 * se
    oracle.set_threads(1)


@pytest.mark.parametrize("h", [0.0, 0.1])
def test_4x4_single_flip_moments_match_exact_enumeration(h):
    """The single-flip chain at a fixed temperature samples the Boltzmann distribution of
    Eq. 2 (exact 4 x 4 enumeration): E and M means within 3 standard errors."""
    L, J = 4, 1.0
    betas = np.array([0.25, 0.45])
    En, Mn = stats.enumerate_lattice(L, J, h)
    o = oracle.OracleProblem(L, betas, J=J, h=h, seed=0xF11F)
    o.flip(2000, 0)
    Es, Ms = [], []
    for _ in range(4000):
        o.flip(16, 0)      # one lattice's worth of iterations between samples
        Es.append(o.energies_int() / o.scale)
        Ms.append(o.magnetisations())
    Es, Ms = np.array(Es, np.float64), np.array(Ms, np.float64)
    for k, beta in enumerate(betas):
        ex = stats.exact_moments(En, Mn, beta)
        mE, seE = stats.blocked_mean_se(Es[:, k])
        mM, seM = stats.blocked_mean_se(Ms[:, k])
        assert abs(mE - ex["E"]) < 3 * seE, (beta, mE, ex["E"], seE)
        assert abs(mM - ex["M"]) < 3 * seM, (beta, mM, ex["M"], seM)


def test_swap_schedule_in_iterations_and_shared_swap_index():
    """Swap iterations follow the iteration count (after every m-th) and share the swap index
    with sweeps: pairs alternate even / odd across both kinds of step."""
    o = oracle.OracleProblem(6, np.linspace(0.3, 0.6, 6), seed=5)
    o.flip(7, 2)                 # iterations 2, 4, 6: swap iterations 0, 1, 2
    assert o.counters() == (0, 3) and o.iterations == 7
    assert o.swap_stats()[0].tolist() == [2, 1, 2, 1, 2]
    o.sweep(1, 1)                # swap iteration 3 (odd pairs)
    assert o.counters() == (1, 4)
    assert o.swap_stats()[0].tolist() == [2, 2, 2, 2, 2]
    o.flip(1, 2)                 # iteration count 8: swap iteration 4 (even pairs)
    assert o.swap_stats()[0].tolist() == [3, 2, 3, 2, 3]


def test_flip_is_independent_of_threads_and_splitting():
    a = oracle.OracleProblem(10, np.linspace(0.2, 0.7, 9), J=1.0, h=0.1, seed=8)
    b = oracle.OracleProblem(10, np.linspace(0.2, 0.7, 9), J=1.0, h=0.1, seed=8)
    oracle.set_threads(1)
    a.flip(500, 7)
    oracle.set_threads(8)
    b.flip(123, 7)
    b.flip(377, 7)
    oracle.set_threads(1)
    np.testing.assert_array_equal(a.spins(), b.spins())
    np.testing.assert_array_equal(a.chain_map(), b.chain_map())
    assert a.iterations == b.iterations == 500
