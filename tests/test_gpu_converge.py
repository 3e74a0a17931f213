"""The Fig. 3b convergence benchmark on the GPU (Sec. 4.1): the per-sweep traces of the
random-start and ordered-start runs equal the oracle's over the whole measured window, row for
row, so the convergence sweep computed from either is the same; the batched, chunked driver
(converge.measure) finds the same sweeps."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import converge as CV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(8)
    return A


CASES = [(16, 8, 0x5EED4000, 1500), (16, 8, 0x5EED4001, 1500), (32, 12, 0x5EED4002, 3000)]


@pytest.mark.parametrize("L,R,seed,n", CASES)
def test_traces_and_convergence_sweep_equal_the_oracle(api, L, R, seed, n):
    p = CV.paper_ladder_problem(L, R, seed, 1)
    hot = api.PTProblem(p.L, p.betas, seed=p.seed)
    cold = api.PTProblem(p.L, p.betas, seed=p.seed)
    CV.cold_start(cold, L, R)
    for g in (hot, cold):
        g.trace_start(n)
        g.sweep(n, 1)
    f_h, Eg_h, Mg_h = hot.trace(n)
    f_c, Eg_c, Mg_c = cold.trace(n)
    assert f_h == f_c == 1
    Eo_h, Eo_c = [], []
    for start in ("hot", "cold"):
        o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
        if start == "cold":
            CV.cold_start(o, L, R)
        E, M = o.trace(n, 1)
        (Eo_h if start == "hot" else Eo_c).append((E, M))
    np.testing.assert_array_equal(Eg_h, Eo_h[0][0])
    np.testing.assert_array_equal(Mg_h, Eo_h[0][1])
    np.testing.assert_array_equal(Eg_c, Eo_c[0][0])
    np.testing.assert_array_equal(Mg_c, Eo_c[0][1])
    t_gpu = CV.converged_at(CV.first_crossing(Eg_h, Eg_c))
    t_orc = CV.converged_at(CV.first_crossing(Eo_h[0][0], Eo_c[0][0]))
    assert t_gpu == t_orc != CV.NOT_YET


def test_chunked_batched_driver_finds_the_same_sweeps(api):
    seeds = [0x5EED4000, 0x5EED4001]
    got = CV.measure(api, [16], seeds, R=8, every=1, cap_min=1500, cap_factor=0.0,
                     chunk_min=64, chunk_factor=0.0)
    for s, t in zip(seeds, got[16]):
        p = CV.paper_ladder_problem(16, 8, s, 1)
        E = []
        for start in ("hot", "cold"):
            o = oracle.OracleProblem(p.L, p.betas, seed=p.seed)
            if start == "cold":
                CV.cold_start(o, 16, 8)
            E.append(o.trace(1500, 1)[0])
        assert t == CV.converged_at(CV.first_crossing(E[0], E[1]))
