"""pt_sweep_batch_static, the batch entry point that allocates nothing, against
pt_sweep_batch (lock-step strategy): two calls in a row through the C ABI must leave every
problem in exactly the same state (spins, energies, temperature map, swap counters).

The static variant is for callers that cannot allocate device memory while they run (a
fixed memory budget, memory owned by an allocator the library cannot see, or code that must
not let an allocation synchronise the device); its work lists live in one fixed device array
of the library. This file is collected last so that a failure here cannot hide another
test's."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_2512_03825_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import _lib
    return _lib


def _problems():
    rng = np.random.Generator(np.random.PCG64(909))
    out = []
    for j in range(20):
        L = int(rng.choice([4, 8, 16, 32, 48, 64]))
        R = int(rng.integers(1, 70))
        J, h = [(1.0, 0.0), (1.0, 0.1), (-1.0, 0.25)][j % 3]
        out.append(W.Problem(L=L, betas=W.linear_ladder(0.2, 0.8, R), J=J, h=h, seed=4000 + j))
    return out


def _state(g):
    att, acc = g.swap_stats()
    return [g.spins(), g.energies_int(), g.magnetisations(), g.chain_map(), att, acc,
            np.array(g.counters())]


def _batch(lib, fn, handles, n, m):
    k = len(handles)
    hs = (C.c_void_p * k)(*[h.handle.value for h in handles])
    ns = np.ascontiguousarray(n, dtype=np.int64)
    ms = np.ascontiguousarray(m, dtype=np.int32)
    return fn(hs, k, ns.ctypes.data_as(C.POINTER(C.c_int64)),
              ms.ctypes.data_as(C.POINTER(C.c_int32)))


def test_static_batch_matches_allocating_batch(lib):
    from paper_2512_03825_b300 import api
    s, c, j = C.c_int(), C.c_int(), C.c_int()
    lib.lib.pt_get_batch_tuning(C.byref(s), C.byref(c), C.byref(j))
    assert lib.lib.pt_set_batch_tuning(lib.PT_BATCH_FLAT, c.value, j.value) == 0
    try:
        probs = _problems()
        a = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
        b = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed) for p in probs]
        rng = np.random.Generator(np.random.PCG64(910))
        for call in range(2):  # two calls in a row: the shared array is reused
            n = rng.integers(0, 12, size=len(probs))
            m = rng.integers(0, 4, size=len(probs))
            assert _batch(lib, lib.lib.pt_sweep_batch, a, n, m) == 0
            rc = _batch(lib, lib.lib.pt_sweep_batch_static, b, n, m)
            assert rc == 0, lib.lib.pt_last_error().decode()
            for k, (ga, gb) in enumerate(zip(a, b)):
                for x, y in zip(_state(ga), _state(gb)):
                    np.testing.assert_array_equal(x, y, err_msg="call %d problem %d" % (call, k))
    finally:
        lib.lib.pt_set_batch_tuning(s.value, c.value, j.value)


def test_static_batch_rejects_oversize(lib):
    from paper_2512_03825_b300 import api
    big = api.PTProblem(8192, [0.4], seed=1)  # 65536 tiles of 512 words: over 1 MiB of lists
    rc = _batch(lib, lib.lib.pt_sweep_batch_static, [big], [1], [0])
    assert rc == lib.PT_EINVAL
    assert "static work area" in lib.lib.pt_last_error().decode()
    assert big.counters() == (0, 0)
    big.sweep(1, 0)  # the problem is still usable
    big.synchronize()


def test_static_batch_refuses_stream_capture(lib):
    """Under stream capture the call must refuse cleanly: its copies read host arrays that the
    next call overwrites, so it cannot be recorded. The refusal comes before anything is
    queued, and the problems stay usable and exact."""
    import torch
    from paper_2512_03825_b300 import api
    st = torch.cuda.Stream()
    probs = _problems()[:3]
    gs = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=st) for p in probs]
    ref = [api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=st) for p in probs]
    assert _batch(lib, lib.lib.pt_sweep_batch_static, gs, [2, 2, 2], [1, 1, 1]) == 0
    assert _batch(lib, lib.lib.pt_sweep_batch, ref, [2, 2, 2], [1, 1, 1]) == 0
    torch.cuda.synchronize()
    x = torch.zeros(16, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        x.add_(1.0)  # something to capture besides the refused call
        rc = _batch(lib, lib.lib.pt_sweep_batch_static, gs, [3, 3, 3], [1, 1, 1])
        msg = lib.lib.pt_last_error().decode()
    assert rc == lib.PT_EINVAL, (rc, msg)
    assert "captured" in msg
    graph.replay()
    torch.cuda.synchronize()
    for g in gs:
        assert g.counters() == (2, 2)  # nothing was queued
    # the problems go on exactly as the allocating path's twins
    assert _batch(lib, lib.lib.pt_sweep_batch_static, gs, [3, 3, 3], [1, 1, 1]) == 0
    assert _batch(lib, lib.lib.pt_sweep_batch, ref, [3, 3, 3], [1, 1, 1]) == 0
    for k, (ga, gb) in enumerate(zip(gs, ref)):
        for a, b in zip(_state(ga), _state(gb)):
            np.testing.assert_array_equal(a, b, err_msg="problem %d" % k)
