"""Full-length parity from creation: the GPU and the oracle each start from pt_create's seed
and run the whole workload (every sweep and swap iteration the workload asks for), then every
spin of every temperature, the exact energies and magnetisations, the temperature map, the
swap statistics and the counters must agree bit for bit. Nothing is handed from one side to
the other, so a divergence at any sweep of the run (a rare race, a wrong counter on sweep
500) shows in the final state.

Covered at their stated sizes:
  * L = 128, R = 32, 10^4 sweeps, a swap iteration after every sweep (plain path);
  * L = 1024, R = 64, 1000 sweeps, a swap iteration every 5 (plain path, its default
    persistent kernel);
  * the batched workload: all 256 problems advanced together for 2000 sweeps in the launch
    shape the benchmark times; every 16th problem is checked in full against the oracle;
  * the served workload: the 2000-request Poisson stream served at about 80% load with an
    80 GB budget; every 50th request with at most 2e9 spin-flip attempts is checked in full
    against the oracle (28 requests, 12 of them with a field).

The oracle runs take several minutes on a 16-core host in all (about 6.5e10, 5e9, 2.5e10 and
1.7e10 attempts at 2.3-2.5e8 attempts/s)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2512_03825_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def api():
    from paper_2512_03825_b300 import build as B
    B.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2512_03825_b300 import api as A
    oracle.set_threads(os.cpu_count() or 1)
    return A


def run_oracle(p, sweeps=None, every=None):
    o = oracle.OracleProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed)
    o.sweep(p.sweeps if sweeps is None else sweeps, p.every if every is None else every)
    return o


def assert_same_state(g, o, where):
    """Every output of the GPU problem g equals the oracle problem o's."""
    np.testing.assert_array_equal(g.chain_map(), o.chain_map(), err_msg=where + ": map")
    np.testing.assert_array_equal(g.energies_int(), o.energies_int(), err_msg=where + ": E")
    np.testing.assert_array_equal(g.magnetisations(), o.magnetisations(), err_msg=where + ": M")
    for x, y, name in zip(g.swap_stats(), o.swap_stats(), ("attempted", "accepted")):
        np.testing.assert_array_equal(x, y, err_msg=where + ": " + name)
    assert g.counters() == o.counters(), where
    for k in range(o.R):
        np.testing.assert_array_equal(g.spins(k), o.spins(k),
                                      err_msg="%s: spins at temperature %d" % (where, k))


def test_L128_R32_all_10000_sweeps_from_creation(api):
    p = W.SINGLE["L128_R32"]
    assert (p.sweeps, p.every) == (10_000, 1)
    g = api.PTProblem(p.L, p.betas, seed=p.seed)
    g.sweep(p.sweeps, p.every)
    o = run_oracle(p)
    assert_same_state(g, o, "L128 R32 after 10^4 sweeps")
    assert g.counters() == (10_000, 10_000)


def test_L1024_R64_all_1000_sweeps_from_creation(api):
    p = W.SINGLE["L1024_R64"]
    assert (p.sweeps, p.every) == (1000, 5)
    g = api.PTProblem(p.L, p.betas, seed=p.seed)
    assert g.sweep_tuning()[2] > 0  # the default strategy runs the persistent kernel here
    g.sweep(p.sweeps, p.every)
    o = run_oracle(p)
    assert_same_state(g, o, "L1024 R64 after 1000 sweeps")
    assert g.counters() == (1000, 200)


@pytest.fixture
def bench_tuning(api):
    """The batch launch shape bench.py times (the autotuner's cached choice for this GPU),
    restored afterwards."""
    from paper_2512_03825_b300 import autotune
    before = autotune.get_tuning()
    chosen = autotune.apply_cached_or_default("batched")
    yield chosen
    autotune.set_tuning(**before)


def test_batched_256_all_2000_sweeps_from_creation(api, bench_tuning):
    import torch
    probs = W.batched_problems()
    n = probs[0].sweeps
    assert n == 2000 and len(probs) == 256
    st = torch.cuda.Stream()  # as bench.py: created on a side stream, no host wait
    gs = [api.PTProblem(p.L, p.betas, seed=p.seed, stream=st) for p in probs]
    api.sweep_batch(gs, n, 1)  # one call, the whole run, as one benchmark step
    torch.cuda.synchronize()
    for j in range(0, len(probs), 16):
        assert_same_state(gs[j], run_oracle(probs[j]), "batched problem %d" % j)


class _KeepSpins:
    """A serving engine that also keeps the final spins of chosen requests (by seed)."""

    def __init__(self, base, seeds):
        self.base, self.seeds, self.spins, self.counters = base, set(seeds), {}, {}

    def __getattr__(self, name):
        return getattr(self.base, name)

    def _keep(self, h):
        if h.seed in self.seeds:
            self.spins[h.seed] = h.spins()
            self.counters[h.seed] = h.counters()

    def read(self, h):
        data = self.base.read(h)
        self._keep(h)
        return data

    def read_many(self, hs):
        datas = self.base.read_many(hs)
        for h in hs:
            self._keep(h)
        return datas


def test_served_stream_2000_requests_sample_from_creation(api):
    import time

    import torch
    from paper_2512_03825_b300 import autotune, serve
    before = autotune.get_tuning()
    autotune.apply_cached_or_default("serve")
    try:
        st = torch.cuda.Stream()
        base = serve.LibEngine(stream=st)
        # the arrival rate the benchmark uses: 80% of the batched rate on a probe of the mix
        probe = W.serving_requests(n=64, rate_per_s=1.0, draw_seed=4242)
        hs = [base.create(r.problem) for r in probe]
        torch.cuda.synchronize()
        k = [min(200, r.problem.sweeps) for r in probe]
        t0 = time.perf_counter()
        base.advance(hs, k, [1] * len(hs))
        torch.cuda.synchronize()
        peak = sum(r.problem.L ** 2 * r.problem.R * m for r, m in zip(probe, k))
        peak /= time.perf_counter() - t0
        for h in hs:
            base.destroy(h)
        unit = W.serving_requests(n=2000, rate_per_s=1.0)
        rate = 0.8 * peak / serve.mean_attempts(unit)
        reqs = W.serving_requests(n=2000, rate_per_s=rate)
        sample = [r for r in reqs[::50] if r.problem.attempts <= 2 * 10 ** 9]
        assert len(sample) == 28 and sum(r.problem.h > 0 for r in sample) == 12
        eng = _KeepSpins(base, [r.problem.seed for r in sample])
        srv = serve.Server(eng, budget_bytes=80 * 10 ** 9, slice_sweeps=100)
        res = srv.run(reqs, realtime=True, timeout_s=600)
        assert sorted(res) == list(range(2000)) and not srv.rejected
    finally:
        autotune.set_tuning(**before)
    for r in sample:
        p, got = r.problem, res[r.rid]
        o = run_oracle(p)
        where = "request %d (L %d, R %d, %d sweeps, h %g)" % (r.rid, p.L, p.R, p.sweeps, p.h)
        np.testing.assert_array_equal(got.E_int, o.energies_int(), err_msg=where + ": E")
        np.testing.assert_array_equal(got.M, o.magnetisations(), err_msg=where + ": M")
        np.testing.assert_array_equal(got.slot_of_temp, o.chain_map(), err_msg=where + ": map")
        att, acc = o.swap_stats()
        np.testing.assert_array_equal(got.attempted, att, err_msg=where + ": attempted")
        np.testing.assert_array_equal(got.accepted, acc, err_msg=where + ": accepted")
        assert eng.counters[p.seed] == o.counters(), where
        np.testing.assert_array_equal(eng.spins[p.seed], o.spins(), err_msg=where + ": spins")
