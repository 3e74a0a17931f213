"""Statistical pins of the oracle's Markov chain (Sec. 2.1 Eq. 1 with the Boltzmann target of
Eq. 2 on the Ising energy of Eq. 3; Sec. 3 replica exchange):

* 4x4 lattice, all 2^16 states enumerated: run averages of E, |M| (and M with a field) at
  each temperature agree with the exact Boltzmann averages within 3 standard errors, with
  and without replica exchange. A wrong sign or a wrong factor in either acceptance rule
  moves the stationary distribution and fails these.
* The exchange acceptance rate of each adjacent pair agrees with its exact expectation over
  the product of the two exact energy distributions.
* L = 256 against Onsager's exact internal energy and spontaneous magnetisation.
* The magnetisation collapses across the critical temperature (the qualitative claim of
  Sec. 4.1, Fig. 3a).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import stats


def _run_trace(L, betas, J, h, seed, burn, n, m, threads=4, start=None,
               swap_rule=oracle.SWAP_BARKER):
    p = oracle.OracleProblem(L, betas, J=J, h=h, seed=seed, swap_rule=swap_rule)
    if start is not None:
        for k in range(len(betas)):
            p.set_spins(k, start)
    oracle.set_threads(threads)
    try:
        p.sweep(burn, m)
        E, M = p.trace(n, m)
    finally:
        oracle.set_threads(1)
    return p, E.astype(np.float64) / p.scale, M.astype(np.float64)


@pytest.mark.parametrize("m", [0, 1])
def test_4x4_exact_enumeration_h0(m):
    L, J, h = 4, 1.0, 0.0
    betas = np.array([0.2, 0.3, 0.44, 0.6])
    En, Mn = stats.enumerate_lattice(L, J, h)
    _, E, M = _run_trace(L, betas, J, h, seed=0x4A4A + m, burn=2000, n=200_000, m=m,
                         threads=1)
    for k, beta in enumerate(betas):
        ex = stats.exact_moments(En, Mn, beta)
        mE, seE = stats.blocked_mean_se(E[:, k])
        mA, seA = stats.blocked_mean_se(np.abs(M[:, k]))
        assert abs(mE - ex["E"]) < 3 * seE, (beta, mE, ex["E"], seE)
        assert abs(mA - ex["absM"]) < 3 * seA, (beta, mA, ex["absM"], seA)


def test_4x4_exact_enumeration_field():
    # E = +h sum(sigma) (Eq. 3 sign): h > 0 favours negative magnetisation
    L, J, h = 4, 1.0, 0.1
    betas = np.array([0.15, 0.25, 0.35, 0.45])
    En, Mn = stats.enumerate_lattice(L, J, h)
    _, E, M = _run_trace(L, betas, J, h, seed=0x4A4B, burn=2000, n=200_000, m=1, threads=1)
    for k, beta in enumerate(betas):
        ex = stats.exact_moments(En, Mn, beta)
        assert ex["M"] < 0
        mE, seE = stats.blocked_mean_se(E[:, k])
        mM, seM = stats.blocked_mean_se(M[:, k])
        assert abs(mE - ex["E"]) < 3 * seE, (beta, mE, ex["E"], seE)
        assert abs(mM - ex["M"]) < 3 * seM, (beta, mM, ex["M"], seM)


@pytest.mark.parametrize("rule", [oracle.SWAP_BARKER, oracle.SWAP_METROPOLIS])
def test_4x4_swap_acceptance_matches_exact_expectation(rule):
    """Acceptance of each adjacent pair vs E_{pi_k x pi_k+1}[S(y)] / 2^32 with the exact
    energy distributions, for both swap rules: this also checks the sign convention of y (a
    reversed sign gives a different, larger rate whenever the two distributions differ)."""
    L, J, h = 4, 1.0, 0.0
    betas = np.array([0.2, 0.3, 0.4, 0.5, 0.6])
    En, _ = stats.enumerate_lattice(L, J, h)
    levels, inv = np.unique(En, return_inverse=True)
    n_sweeps = 200_000
    p, _, _ = _run_trace(L, betas, J, h, seed=0x5A5A, burn=1000, n=10, m=1, threads=1,
                         swap_rule=rule)
    att0, acc0 = p.swap_stats()
    p.sweep(n_sweeps, 1)
    att, acc = p.swap_stats()
    att = att - att0
    acc = acc - acc0
    s = p.scale
    for k in range(len(betas) - 1):
        pk = np.bincount(inv, weights=stats.boltzmann_weights(En, betas[k]), minlength=levels.size)
        pk1 = np.bincount(inv, weights=stats.boltzmann_weights(En, betas[k + 1]),
                          minlength=levels.size)
        expect = 0.0
        wrong_sign = 0.0
        for a, Ea in enumerate(levels):
            for b, Eb in enumerate(levels):
                w = pk[a] * pk1[b]
                if w < 1e-14:
                    continue
                n = int(round((Ea - Eb) * s))
                expect += w * oracle.swap_threshold(betas[k], betas[k + 1], n, s, rule) / 2.0 ** 32
                wrong_sign += w * oracle.swap_threshold(betas[k], betas[k + 1], -n, s,
                                                        rule) / 2.0 ** 32
        rate = acc[k] / att[k]
        # successive attempts are correlated through the chain: allow 3 SE of a binomial with
        # an effective sample size reduced tenfold
        se = math.sqrt(expect * (1 - expect) / (att[k] / 10.0))
        assert abs(rate - expect) < 3 * se, (k, rate, expect, se)
        assert abs(wrong_sign - expect) > 6 * se


def test_swap_rate_equal_betas_is_one_half():
    p = oracle.OracleProblem(6, [0.4] * 6, seed=31)
    p.sweep(4000, 1)
    att, acc = p.swap_stats()
    rate = acc.sum() / att.sum()
    assert abs(rate - 0.5) < 4 * math.sqrt(0.25 / att.sum())


@pytest.mark.parametrize("beta,ordered", [(0.30, False), (0.35, False), (0.50, True),
                                          (0.55, True)])
def test_onsager_L256(beta, ordered):
    """Energy per spin within 3 SE plus a 1e-3 finite-size allowance of Onsager's u(beta);
    |M| per spin likewise against the spontaneous magnetisation in the ordered phase.
    Ordered-phase chains start from the all-up state (equilibrating from a random start
    means coarsening domains over ~L^2 sweeps)."""
    L = 256
    start = np.ones((L, L), np.int8) if ordered else None
    _, E, M = _run_trace(L, [beta], 1.0, 0.0, seed=0x0A5A + int(beta * 100), burn=300, n=700,
                         m=0, threads=8, start=start)
    u, se = stats.blocked_mean_se(E[:, 0] / (L * L), min_blocks=16)
    assert abs(u - stats.onsager_energy_per_spin(beta)) < 3 * se + 1e-3, (u, se)
    if ordered:
        mabs, se_m = stats.blocked_mean_se(np.abs(M[:, 0]) / (L * L), min_blocks=16)
        assert abs(mabs - stats.onsager_magnetisation(beta)) < 3 * se_m + 2e-3, (mabs, se_m)


def test_onsager_helpers_against_library():
    import scipy.special
    for k in (0.1, 0.5, 0.9, 0.999):
        assert abs(stats.ellipk(k) - scipy.special.ellipk(k * k)) < 1e-12
    # u(beta_c) = -sqrt(2) J (the elliptic term vanishes at the critical point)
    assert abs(stats.onsager_energy_per_spin(stats.BETA_C + 1e-5) + math.sqrt(2.0)) < 2e-3
    assert abs(stats.onsager_energy_per_spin(stats.BETA_C - 1e-5) + math.sqrt(2.0)) < 2e-3
    assert stats.onsager_magnetisation(0.3) == 0.0


def test_magnetisation_collapses_across_critical_temperature():
    """Sec. 4.1 / Fig. 3a: ordered (large |M|) well below T_c, disordered well above."""
    L = 48
    betas = np.array([0.25, 0.33, 0.55, 0.7])
    start = np.ones((L, L), np.int8)
    _, _, M = _run_trace(L, betas, 1.0, 0.0, seed=77, burn=500, n=500, m=1, threads=4,
                         start=start)
    pct = 100.0 * np.abs(M).mean(axis=0) / (L * L)
    assert pct[0] < 15 and pct[1] < 25
    assert pct[2] > 85 and pct[3] > 95
