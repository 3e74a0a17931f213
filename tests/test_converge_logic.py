"""The convergence criterion of the Fig. 3b benchmark (Sec. 4.1) on the host: first crossing
of the random-start energy below the ordered-start energy, per temperature, on hand-made
traces whose answers are known, and on oracle traces of a small lattice."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import converge as CV
from paper_2512_03825_b300 import workloads as W


def test_first_crossing_known_rows():
    # temperature 0 crosses at row 2 (sweep 3), temperature 1 at row 0 (ties count),
    # temperature 2 never
    hot = np.array([[10, 5, 9], [8, 4, 9], [6, 3, 9], [7, 2, 9]])
    cold = np.array([[4, 5, 1], [5, 6, 1], [6, 7, 1], [8, 8, 1]])
    got = CV.first_crossing(hot, cold, first_sweep=1)
    np.testing.assert_array_equal(got, [3, 1, CV.NOT_YET])
    assert CV.converged_at(got) == CV.NOT_YET
    np.testing.assert_array_equal(CV.first_crossing(hot, cold, first_sweep=101), [103, 101, -1])
    assert CV.converged_at(np.array([3, 1, 7])) == 7


def test_first_crossing_rejects_mismatched_traces():
    with pytest.raises(ValueError):
        CV.first_crossing(np.zeros((3, 2)), np.zeros((3, 3)))


def test_fit_exponent_recovers_power_laws():
    Ls = [16, 32, 64, 128]
    assert CV.fit_exponent(Ls, [3.0 * L ** 2 for L in Ls]) == pytest.approx(2.0, abs=1e-12)
    assert CV.fit_exponent(Ls, [0.5 * L ** 2.17 for L in Ls]) == pytest.approx(2.17, abs=1e-12)


def test_summarise_counts_censored_runs_at_their_cap():
    res = {16: [10, 20, 30, CV.NOT_YET], 32: [40, 80, 120, 160]}
    s = CV.summarise(res, {16: 1000, 32: 4000})
    assert s["per_L"]["16"]["censored"] == 1
    assert s["per_L"]["16"]["median_sweeps"] == pytest.approx(25.0)
    assert s["per_L"]["32"]["median_sweeps"] == pytest.approx(100.0)
    assert s["exponent_sweeps"] == pytest.approx(np.log2(100.0 / 25.0))
    assert s["exponent_iterations"] == pytest.approx(s["exponent_sweeps"] + 2.0)


def oracle_pair(L, R, seed, n, every=1):
    p = CV.paper_ladder_problem(L, R, seed, every)
    hot = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
    cold = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
    CV.cold_start(cold, L, R)
    Eh, _ = hot.trace(n, every)
    Ec, _ = cold.trace(n, every)
    return Eh, Ec


def test_ordered_start_is_the_ground_state_and_random_start_is_not():
    L, R = 8, 4
    p = CV.paper_ladder_problem(L, R, 5, 1)
    cold = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
    CV.cold_start(cold, L, R)
    np.testing.assert_array_equal(cold.energies_int(), np.full(R, -2 * L * L))
    hot = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
    assert (hot.energies_int() > -2 * L * L).all()


def test_oracle_runs_converge_on_a_small_lattice():
    # at L = 8 on the paper's ladder every temperature converges well within 2000 sweeps, and
    # the hottest one (T close to 4) within a few sweeps
    oracle.set_threads(4)
    Eh, Ec = oracle_pair(8, 8, 0x5EED4000, 2000)
    per_k = CV.first_crossing(Eh, Ec)
    assert (per_k != CV.NOT_YET).all()
    assert per_k[-1] <= 20
    assert CV.converged_at(per_k) == per_k.max()


def test_slowest_temperature_counts():
    det = {(16, 1): [3, 9, 4], (16, 2): [8, 2, 1], (32, 1): [5, 6, CV.NOT_YET]}
    assert CV.slowest_temperatures(det) == {"16": {"1": 1, "0": 1}}
