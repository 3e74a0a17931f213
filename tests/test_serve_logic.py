"""Scheduling logic of the continuous-batching server, without a GPU: a fake engine that
does the bookkeeping stands in for libpt. Failures are made on the host (an allocation that
fails, a cancelled request, a budget too small), never on a device."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2512_03825_b300 import serve
from paper_2512_03825_b300 import workloads as W


class FakeEngine(serve.Engine):
    def __init__(self, bytes_per_site=4, fail_on=()):
        self.bytes_per_site = bytes_per_site
        self.fail_on = set(fail_on)
        self.live = {}
        self.calls = []
        self.next = 0

    def estimate_bytes(self, p):
        return p.L * p.L * self.bytes_per_site

    def create(self, p):
        if p.seed in self.fail_on:
            raise MemoryError("injected allocation failure")
        self.next += 1
        self.live[self.next] = dict(p=p, t=0, e=0)
        return self.next

    def advance(self, handles, n, every):
        assert len(handles) == len(n) == len(every)
        self.calls.append(list(zip(handles, n)))
        for h, k, m in zip(handles, n, every):
            st = self.live[h]
            if m:
                st["e"] += (st["t"] + k) // m - st["t"] // m
            st["t"] += k

    def read(self, h):
        st = self.live[h]
        R = st["p"].R
        return dict(E_int=np.full(R, st["t"], np.int64), M=np.zeros(R, np.int64), scale=1,
                    slot_of_temp=np.arange(R, dtype=np.int32),
                    attempted=np.full(max(R - 1, 0), st["e"], np.uint64),
                    accepted=np.zeros(max(R - 1, 0), np.uint64))

    def destroy(self, h):
        del self.live[h]


def reqs(n, L=32, sweeps=250, every=1, gap=0.0):
    return [W.Request(rid=j, arrival=j * gap,
                      problem=W.Problem(L=L, betas=(0.3, 0.4, 0.5), seed=j, sweeps=sweeps,
                                        every=every)) for j in range(n)]


def test_slices_and_completion():
    eng = FakeEngine()
    srv = serve.Server(eng, budget_bytes=10 ** 9, slice_sweeps=100)
    out = srv.run(reqs(5, sweeps=250), realtime=False)
    assert sorted(out) == list(range(5))
    for r in out.values():
        assert r.E_int[0] == 250                 # every sweep was run
        assert r.attempted[0] == 250             # exchange counts follow the global sweep count
    assert [sorted(k for _, k in c) for c in eng.calls] == [[100] * 5, [100] * 5, [50] * 5]
    assert not eng.live and srv.used == 0


def test_budget_limits_residency_and_frees_memory():
    eng = FakeEngine()
    one = 32 * 32 * 4
    srv = serve.Server(eng, budget_bytes=3 * one, slice_sweeps=50)
    srv.run(reqs(10, sweeps=100), realtime=False)
    assert len(srv.results) == 10
    assert srv.peak_used <= 3 * one
    assert max(len(c) for c in eng.calls) == 3   # never more than three resident
    assert srv.used == 0 and not eng.live


def test_continuous_batching_mixes_requests():
    eng = FakeEngine()
    srv = serve.Server(eng, budget_bytes=10 ** 9, slice_sweeps=10)
    srv.t0 = 0.0
    srv.clock = lambda: 0.0
    srv.realtime = True
    a = reqs(3, sweeps=30)
    srv.submit(a[0])
    srv.step()                      # request 0 alone
    srv.submit(a[1])
    srv.submit(a[2])
    srv.step()                      # requests 1 and 2 join while 0 is running
    assert [len(c) for c in eng.calls] == [1, 3]
    while not srv.idle():
        srv.step()
    assert sorted(srv.results) == [0, 1, 2]


def test_rejections_and_failures():
    eng = FakeEngine(fail_on={3})
    srv = serve.Server(eng, budget_bytes=40 * 40 * 4, slice_sweeps=100)
    stream = reqs(5, L=32) + [W.Request(rid=99, arrival=0.0,
                                        problem=W.Problem(L=64, betas=(0.3,), seed=99,
                                                          sweeps=10))]
    srv.run(stream, realtime=False)
    assert 99 in srv.rejected and "budget" in srv.rejected[99]
    assert 3 in srv.rejected and "injected" in srv.rejected[3]
    assert sorted(srv.results) == [0, 1, 2, 4]
    assert srv.used == 0 and not eng.live


def test_cancel_running_request_returns_memory():
    eng = FakeEngine()
    srv = serve.Server(eng, budget_bytes=10 ** 9, slice_sweeps=10)
    srv.t0 = 0.0
    srv.clock = lambda: 0.0
    for r in reqs(2, sweeps=100):
        srv.submit(r)
    srv.step()
    assert srv.used > 0
    assert srv.cancel(0)
    assert 0 in srv.rejected and len(eng.live) == 1
    while not srv.idle():
        srv.step()
    assert sorted(srv.results) == [1] and srv.used == 0


def test_bad_server_arguments():
    with pytest.raises(ValueError):
        serve.Server(FakeEngine(), budget_bytes=0)
    with pytest.raises(ValueError):
        serve.Server(FakeEngine(), slice_sweeps=0)


def test_serving_workload_shape():
    rs = W.serving_requests(n=2000, rate_per_s=10.0)
    L = np.array([r.problem.L for r in rs])
    R = np.array([r.problem.R for r in rs])
    sw = np.array([r.problem.sweeps for r in rs])
    h = np.array([r.problem.h for r in rs])
    assert (L % 32 == 0).all() and L.min() >= 32 and L.max() <= 512
    assert R.min() >= 8 and R.max() <= 64
    assert sw.min() >= 100 and sw.max() <= 10000
    assert set(np.unique(h).tolist()) == {0.0, 0.1}
    gaps = np.diff([r.arrival for r in rs])
    assert abs(gaps.mean() - 0.1) < 0.01     # Poisson at 10 per second
