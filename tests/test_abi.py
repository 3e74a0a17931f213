"""The C-ABI library without a GPU: it loads, exports every function include/pt.h declares,
its host-built tables equal the oracle's value for value, and device calls fail loudly
(PT_ENODEV) instead of falling back to the CPU."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from tests.conftest import ROOT

TWO32 = 1 << 32


@pytest.fixture(scope="module")
def pt():
    from paper_2512_03825_b300 import build as B
    B.build()
    from paper_2512_03825_b300 import _lib
    return _lib


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_exports_every_declared_function(pt):
    declared = _declared_functions()
    assert len(declared) >= 20
    raw = C.CDLL(pt.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name
    bound = {n for n, _, _ in pt.SIGNATURES}
    assert set(declared) == bound


def test_only_pt_symbols_exported(pt):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", pt.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = [line.split()[-1] for line in out.splitlines() if " T " in line]
    assert syms and all(s.startswith("pt_") for s in syms), syms


def test_quantise_matches_oracle(pt):
    from paper_2512_03825_b300 import api
    for J, h in [(1, 0), (1, 0.1), (0.5, 0), (1 / 3, 0), (-1, 0.25), (2, -0.3), (0, 1)]:
        assert api.quantise(J, h) == oracle.quantise(J, h)
    with pytest.raises(Exception):
        api.quantise(np.pi, 0)


def test_spin_thresholds_equal_oracle(pt):
    from paper_2512_03825_b300 import api
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(20000):
        beta = float(rng.uniform(0, 2.0)) if rng.random() > 0.05 else 0.0
        dE = int(rng.integers(-100, 100))
        s = int(rng.choice([1, 2, 10, 1000]))
        assert api.spin_threshold(beta, dE, s) == oracle.spin_threshold(beta, dE, s)


@pytest.mark.parametrize("blo,bhi,s", [
    (0.30, 0.30 + 0.25 / 31, 1), (0.35, 0.35 + 0.15 / 63, 1), (0.3, 0.3 + 0.3 / 63, 10),
    (0.5, 0.4, 1), (0.4, 0.4, 1), (0.2, 0.6, 1), (0.0, 1e-3, 2), (1.0, 0.2, 10)])
def test_swap_table_equals_oracle(pt, blo, bhi, s):
    """Every n where the table or its saturated ends decide: equal to the oracle's direct
    evaluation of the rule (checked on the whole interior, its edges and far outside)."""
    from paper_2512_03825_b300 import api
    d = bhi - blo
    if d == 0:
        ns = list(range(-50, 51)) + [10 ** 9, -10 ** 9]
    else:
        N = int(np.ceil(46.0 * s / abs(d)))
        ns = list(range(-N, N + 1, max(1, N // 20000))) + [N + 5, -N - 5, 10 ** 12, -10 ** 12]
        # dense around both saturation edges
        lo_edge = int(np.floor(-36.8 * s / d)) if d > 0 else int(np.floor(36.8 * s / -d))
        hi_edge = int(np.floor(22.2 * s / d)) if d > 0 else int(np.floor(-22.2 * s / -d))
        for e in (lo_edge, hi_edge):
            ns += list(range(e - 300, e + 300))
    for n in ns:
        assert api.swap_threshold(blo, bhi, n, s) == oracle.swap_threshold(blo, bhi, n, s), n


def test_no_gpu_fails_loudly(pt):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2512_03825_b300 import api
    with pytest.raises(pt.PTError) as ei:
        api.PTProblem(16, [0.3, 0.4])
    assert ei.value.code == pt.PT_ENODEV


def test_bad_arguments_rejected_before_device(pt):
    from paper_2512_03825_b300 import api
    for L, betas, J, h in [(5, [0.1], 1, 0), (2, [0.1], 1, 0), (8, [], 1, 0), (8, [-0.1], 1, 0),
                           (8, [float("nan")], 1, 0), (8, [0.1], np.pi, 0),
                           (32768, [0.1], 1, 0)]:
        with pytest.raises(pt.PTError) as ei:
            api.PTProblem(L, betas, J=J, h=h)
        assert ei.value.code == pt.PT_EINVAL
    assert api.estimate_device_bytes(5, [0.1]) == 0
    assert api.estimate_device_bytes(1024, np.linspace(0.35, 0.5, 64)) > 8 * 2 ** 20


def test_allocator_hooks_are_kept_alive(pt):
    """Re-enabling the torch allocator must not free the callbacks that existing problems
    will call when they are destroyed."""
    from paper_2512_03825_b300 import api
    api.use_torch_allocator(True)
    first = api._torch_hooks
    api.use_torch_allocator(True)
    assert api._torch_hooks is first
    api.use_torch_allocator(False)
    api.use_torch_allocator(True)
    assert first in api._all_hooks
    api.use_torch_allocator(False)


@pytest.mark.parametrize("blo,bhi,s", [(0.30, 0.30 + 0.25 / 31, 1), (0.5, 0.4, 1), (0.4, 0.4, 1),
                                       (0.2, 0.6, 1), (1.0, 0.2, 10)])
def test_metropolis_swap_table_equals_oracle(pt, blo, bhi, s):
    """The host tables of the Metropolis swap option give the oracle's threshold for every n
    around and far outside the range where they are tabulated."""
    from paper_2512_03825_b300 import api
    d = bhi - blo
    N = int(np.ceil(46.0 * s / abs(d))) if d else 50
    ns = list(range(-N, N + 1, max(1, N // 20000))) + [10 ** 9, -10 ** 9, 0, 1, -1]
    for n in ns:
        assert api.swap_threshold_rule(blo, bhi, n, s, 1) == \
            oracle.swap_threshold(blo, bhi, n, s, oracle.SWAP_METROPOLIS), n
        assert api.swap_threshold_rule(blo, bhi, n, s, 0) == oracle.swap_threshold(blo, bhi, n, s)
    assert api.swap_threshold_rule(0.3, 0.4, 5, 1, 2) == (1 << 64) - 1


def test_create_ex_rejects_bad_options(pt):
    import ctypes as C
    from paper_2512_03825_b300 import api
    for rule in (2, -1):
        with pytest.raises(pt.PTError) as ei:
            api.PTProblem(8, [0.3, 0.4], swap_rule=rule)
        assert ei.value.code == pt.PT_EINVAL
    b = np.array([0.3, 0.4])
    h = C.c_void_p()
    opt = pt.PTOptions(2, 0)  # size too small
    rc = pt.lib.pt_create_ex(8, b.ctypes.data_as(C.POINTER(C.c_double)), 2, 1.0, 0.0, 1,
                             C.byref(opt), C.byref(h))
    assert rc == pt.PT_EINVAL


def _load_rc(pt, data):
    import ctypes as C
    buf = C.create_string_buffer(bytes(data), len(data))
    h = C.c_void_p()
    return pt.lib.pt_load(buf, len(data), C.byref(h))


def test_load_validates_before_the_device(pt):
    """pt_load checks the whole checkpoint on the host: a well-formed one gets past every
    check to the device (PT_ENODEV here, no GPU); every kind of damage is PT_EINVAL."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from tests.helpers import checkpoint as ck
    L, R = 6, 35
    rng = np.random.Generator(np.random.PCG64(3))
    betas = np.linspace(0.2, 0.6, R)
    spins = np.where(rng.random((R, L, L)) < 0.5, 1, -1).astype(np.int8)
    words = ck.spins_to_words(spins)
    np.testing.assert_array_equal(ck.words_to_spins(words, R), spins)
    sot = rng.permutation(R).astype(np.int32)
    att = rng.integers(0, 100, R - 1).astype(np.uint64)
    acc = (att // 2).astype(np.uint64)
    good = ck.build(L, betas, 1.0, 0.0, 7, 40, 13, 1, sot, att, acc, words)
    assert ck.parse(good)["t"] == 40
    assert _load_rc(pt, good) == pt.PT_ENODEV
    bad = []
    bad.append(b"XTCKPT01" + good[8:])                                       # magic
    bad.append(good[:-1])                                                    # size
    b = bytearray(good); b[100] ^= 1; bad.append(bytes(b))                   # checksum
    bad.append(ck.build(L, betas, 1.0, 0.0, 7, 40, 13, 1, np.zeros(R, np.int32), att, acc,
                        words))                                              # not a permutation
    bad.append(ck.build(L, betas, 1.0, 0.0, 7, 40, 13, 1, sot, att, att + 1, words))  # acc > att
    w2 = words.copy(); w2[1, 0, 0, 0] |= 1 << 31
    bad.append(ck.build(L, betas, 1.0, 0.0, 7, 40, 13, 1, sot, att, acc, w2))  # unused slot bit
    bad.append(ck.build(L, betas, 1.0, 0.0, 7, 40, 13, 5, sot, att, acc, words))  # swap rule
    bad.append(ck.build(5, betas, 1.0, 0.0, 7, 40, 13, 1, sot, att, acc, words))  # odd L
    for k, data in enumerate(bad):
        assert _load_rc(pt, data) == pt.PT_EINVAL, k


def test_batch_tile_words_validated(pt):
    """The tile size knob: multiples of 32 in [64, 1024] only; host state, no device."""
    old = C.c_int()
    assert pt.lib.pt_get_batch_tile_words(C.byref(old)) == 0
    assert old.value % 32 == 0 and 64 <= old.value <= 1024
    try:
        for bad in (0, 32, 63, 100, 1056, 4096, -64):
            assert pt.lib.pt_set_batch_tile_words(bad) == pt.PT_EINVAL, bad
        for good in (64, 256, 1024):
            assert pt.lib.pt_set_batch_tile_words(good) == 0
            got = C.c_int()
            assert pt.lib.pt_get_batch_tile_words(C.byref(got)) == 0 and got.value == good
        assert pt.lib.pt_get_batch_tile_words(None) == pt.PT_EINVAL
    finally:
        pt.lib.pt_set_batch_tile_words(old.value)


def test_exchange_tables_limited_to_reachable_energies(pt):
    """A problem's exchange tables cover only the energy differences its lattice can reach
    (|n| <= 2 (2 L^2 |J_int| + L^2 |h_int|)): a long, dense ladder on a small lattice needs a
    few MiB, not the GiB that the whole non-saturated range of every pair would take."""
    from paper_2512_03825_b300 import api
    from paper_2512_03825_b300 import workloads as W
    small = api.estimate_device_bytes(8, W.linear_ladder(0.05, 1.0, 2048))
    assert 0 < small < 64 * 2 ** 20
    # a lattice that reaches the whole range keeps every entry it can look up: L = 300 with
    # the paper's ladder T_i = 1 + 3 i / 1500 holds more than 256 MiB of tables (every n
    # would take 1.2 GiB; only multiples of 4 occur, and only those are kept)
    paper = api.estimate_device_bytes(300, [1.0 / (1.0 + 3.0 * i / 1500) for i in range(1500)])
    assert 2 ** 28 < paper < 2 ** 30


def test_image_cache_limit_without_a_device(pt):
    """The cache limit is a host setting: it can be set and read with no GPU, and nothing
    is cached when no problem could be created."""
    assert pt.lib.pt_set_image_cache_limit(1 << 20) == 0
    assert pt.lib.pt_image_cache_bytes() == 0
    assert pt.lib.pt_set_image_cache_limit(1 << 30) == 0


def test_getters_reject_a_null_problem(pt):
    """Every per-problem getter answers PT_EINVAL for a NULL handle, before touching a
    device."""
    import ctypes as C
    out32 = (C.c_int32 * 4)()
    out64 = (C.c_int64 * 4)()
    outd = (C.c_double * 4)()
    assert pt.lib.pt_chain_map(None, out32) == pt.PT_EINVAL
    assert pt.lib.pt_temperature_map(None, out32) == pt.PT_EINVAL
    assert pt.lib.pt_energies(None, outd) == pt.PT_EINVAL
    assert pt.lib.pt_energies_int(None, out64, None, None) == pt.PT_EINVAL


def test_release_library_has_no_debug_checks(pt):
    # the release library compiles none of the debug build's checks, and its debug entry points
    # refuse (a NULL problem is refused before anything else)
    assert pt.lib.pt_debug_build() == 0
    assert pt.lib.pt_debug_report(None, None, None, None, None) == pt.PT_EINVAL
    assert pt.lib.pt_debug_inject(None, 1) != 0


def test_batch_streams_validated(pt):
    import ctypes as C
    n = C.c_int()
    assert pt.lib.pt_get_batch_streams(C.byref(n)) == 0
    before = n.value
    for bad in (0, -1, 5):
        assert pt.lib.pt_set_batch_streams(bad) == pt.PT_EINVAL
    assert pt.lib.pt_set_batch_streams(3) == 0
    assert pt.lib.pt_get_batch_streams(C.byref(n)) == 0 and n.value == 3
    assert pt.lib.pt_get_batch_streams(None) == pt.PT_EINVAL
    assert pt.lib.pt_set_batch_streams(before) == 0


def test_empty_batches_are_no_ops(pt):
    """A batch of no problems is a no-op that succeeds before any device is touched (so it
    does here, without a GPU); a negative count, or a positive one without its arrays, is
    PT_EINVAL."""
    lib = pt.lib
    for fn in (lib.pt_sweep_batch, lib.pt_sweep_batch_static):
        assert fn(None, 0, None, None) == 0
        assert fn(None, -1, None, None) == pt.PT_EINVAL
        assert fn(None, 2, None, None) == pt.PT_EINVAL
    assert lib.pt_read_batch(None, 0, None, None, None, None, None) == 0
    assert lib.pt_read_batch(None, -1, None, None, None, None, None) == pt.PT_EINVAL
    assert lib.pt_read_batch(None, 3, None, None, None, None, None) == pt.PT_EINVAL


def test_batch_graphs_validated(pt):
    import ctypes as C
    g = C.c_int()
    assert pt.lib.pt_get_batch_graphs(C.byref(g)) == 0
    before = g.value
    for bad in (-1, 2, 7):
        assert pt.lib.pt_set_batch_graphs(bad) == pt.PT_EINVAL
    assert pt.lib.pt_set_batch_graphs(1) == 0
    assert pt.lib.pt_get_batch_graphs(C.byref(g)) == 0 and g.value == 1
    assert pt.lib.pt_get_batch_graphs(None) == pt.PT_EINVAL
    assert pt.lib.pt_set_batch_graphs(before) == 0
