"""Pins of the CPU oracle against things other than itself: an independent Philox4x32-10
(PyTorch's header-only engine), closed-form energies and symmetries of Eq. 3, exact
special cases of the Metropolis rule (beta = 0, zero temperature), high-precision values of
both threshold formulas, and closed forms of the swap schedule. The statistical pins (exact
enumeration, Onsager, swap detailed balance) are in test_oracle_statistics.py."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.conftest import ROOT

TWO32 = 1 << 32


def test_swap_threshold_metropolis_values():
    """The Metropolis-form option min(1, e^{-y}): exact values (40-digit arithmetic), the
    detailed-balance ratio p(y) / p(-y) = e^{-y} that every valid swap rule has -- checked
    against the Barker form's own ratio, so each formula pins the other -- and p >= Barker
    pointwise."""
    import mpmath
    mpmath.mp.dps = 40
    M = oracle.SWAP_METROPOLIS
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(2000):
        b0 = float(rng.uniform(0.0, 1.0))
        b1 = b0 + float(rng.uniform(-0.1, 0.1))
        s = int(rng.choice([1, 10]))
        n = int(rng.integers(-3000, 3000))
        y = mpmath.mpf(b1 - b0) * n / s
        S = oracle.swap_threshold(b0, b1, n, s, M)
        if y <= 0:
            assert S == TWO32
        elif y > 44:
            assert S == 0
        else:
            exact = mpmath.mpf(TWO32) * mpmath.exp(-y)
            assert S == int(mpmath.floor(exact)) or abs(exact - mpmath.nint(exact)) < 1e-5
        assert S >= oracle.swap_threshold(b0, b1, n, s) - 1
        if 0 < abs(y) < 8:  # thresholds above 1.4e6: the floor moves a ratio by < 1e-6
            Sm = oracle.swap_threshold(b0, b1, -n, s, M)
            Bp, Bm = oracle.swap_threshold(b0, b1, n, s), oracle.swap_threshold(b0, b1, -n, s)
            ratio_m, ratio_b = S / Sm, Bp / Bm
            assert abs(ratio_m / float(mpmath.exp(-y)) - 1) < 3e-6
            assert abs(ratio_m / ratio_b - 1) < 3e-6
    assert oracle.swap_threshold(0.4, 0.4, 12345, 1, M) == TWO32   # equal temperatures
    assert oracle.swap_threshold(0.0, 1.0, 45, 1, M) == 0
    assert oracle.swap_threshold(0.0, 1.0, -45, 1, M) == TWO32


def test_swap_rule_selects_the_formula():
    """A problem created with the Metropolis rule takes exactly the Metropolis decisions: at
    equal temperatures every swap is accepted (y = 0), under Barker half of them."""
    a = oracle.OracleProblem(6, [0.4] * 6, seed=31, swap_rule=oracle.SWAP_METROPOLIS)
    a.sweep(200, 1)
    att, acc = a.swap_stats()
    assert (acc == att).all() and att.sum() > 0
    b = oracle.OracleProblem(6, [0.4] * 6, seed=31)
    b.sweep(200, 1)
    assert b.swap_stats()[1].sum() < att.sum()
    with pytest.raises(ValueError):
        oracle.OracleProblem(6, [0.4] * 6, seed=31, swap_rule=2)


# --------------------------------------------------------------------------------------
# Philox4x32-10 vs PyTorch's own engine (ATen/core/PhiloxRNGEngine.h), built on the CPU
# --------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def torch_philox():
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    src = os.path.join(ROOT, "tests", "helpers", "torch_philox.cpp")
    out_dir = os.path.join(ROOT, "tests", "helpers", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libtorch_philox.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + inc, "-o", so,
                        src], check=True)
    lib = C.CDLL(so)
    lib.torch_philox_blocks.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    lib.torch_philox_blocks.restype = None

    def run(ctr, key):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
        key = np.ascontiguousarray(key, dtype=np.uint32)
        out = np.zeros((ctr.shape[0], 4), dtype=np.uint32)
        lib.torch_philox_blocks(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0])
        return out
    return run


def test_philox_matches_torch_engine(torch_philox):
    rng = np.random.Generator(np.random.PCG64(11))
    n = 4096
    ctr = rng.integers(0, TWO32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, TWO32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge words: all zeros, all ones, and the counter layouts the method uses
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    ctr[2] = [5, 17, 3, 0]
    ctr[3] = [1023, 0, 15, 2]
    ctr[4] = [7, 42, 0, 1 | (3 << 8)]
    ref = torch_philox(ctr, key)
    mine = np.stack([oracle.philox4x32_10(ctr[i], key[i]) for i in range(n)])
    np.testing.assert_array_equal(mine, ref)


# --------------------------------------------------------------------------------------
# Quantisation of J and h
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("J,h,expect", [
    (1.0, 0.0, (1, 1, 0)),
    (1.0, 0.1, (10, 10, 1)),
    (0.5, 0.0, (2, 1, 0)),
    (1.0 / 3.0, 0.0, (3, 1, 0)),
    (-1.0, 0.25, (4, -4, 1)),
    (2.0, -0.3, (10, 20, -3)),
    (0.0, 1.0, (1, 0, 1)),
])
def test_quantise(J, h, expect):
    assert oracle.quantise(J, h) == expect


@pytest.mark.parametrize("J,h", [(np.pi, 0.0), (1.0, np.sqrt(2.0)), (float("nan"), 0.0),
                                 (1.0, float("inf")), (1e7, 0.0)])
def test_quantise_rejects(J, h):
    with pytest.raises(ValueError):
        oracle.quantise(J, h)


# --------------------------------------------------------------------------------------
# Eq. 3 energies: closed forms and symmetries
# --------------------------------------------------------------------------------------

def _with_state(L, sigma, J=1.0, h=0.0):
    p = oracle.OracleProblem(L, [0.3], J=J, h=h, seed=1)
    p.set_spins(0, sigma)
    return p


@pytest.mark.parametrize("L", [4, 6, 16])
@pytest.mark.parametrize("J,h", [(1.0, 0.0), (1.0, 0.1), (-0.5, 0.25)])
def test_energy_closed_forms(L, J, h):
    s, Ji, hi = oracle.quantise(J, h)
    n = L * L
    up = np.ones((L, L), np.int8)
    # all up: every one of the 2 L^2 bonds satisfied, M = L^2
    p = _with_state(L, up, J, h)
    assert p.energies_int()[0] == -Ji * 2 * n + hi * n
    assert p.magnetisations()[0] == n
    # all down: same bonds, field term flips sign
    p = _with_state(L, -up, J, h)
    assert p.energies_int()[0] == -Ji * 2 * n - hi * n
    # Neel state: every bond unsatisfied, M = 0
    yy, xx = np.mgrid[0:L, 0:L]
    neel = np.where((xx + yy) % 2 == 0, 1, -1).astype(np.int8)
    p = _with_state(L, neel, J, h)
    assert p.energies_int()[0] == Ji * 2 * n
    assert p.magnetisations()[0] == 0
    # stripes along x (rows alternate): horizontal bonds satisfied, vertical unsatisfied
    stripes = np.where(yy % 2 == 0, 1, -1).astype(np.int8)
    p = _with_state(L, stripes, J, h)
    assert p.energies_int()[0] == 0
    # one flipped spin in the all-up state, at a corner (periodic wrap) and in the bulk:
    # four bonds turn unsatisfied, M drops by 2
    for (y, x) in [(0, 0), (L - 1, L - 1), (L // 2, 1)]:
        st = up.copy()
        st[y, x] = -1
        p = _with_state(L, st, J, h)
        assert p.energies_int()[0] == -Ji * (2 * n - 8) + hi * (n - 2)


def test_energy_symmetries():
    rng = np.random.Generator(np.random.PCG64(3))
    for L in (4, 8, 10):
        for (J, h) in [(1.0, 0.0), (1.0, 0.1), (-1.0, 0.3)]:
            sig = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
            e0 = _with_state(L, sig, J, h).energies_int()[0]
            # translation, transposition and mirror invariance of the periodic lattice
            for t in (np.roll(sig, 3, axis=0), np.roll(sig, -1, axis=1), sig.T.copy(),
                      sig[:, ::-1].copy(), sig[::-1, :].copy()):
                assert _with_state(L, t, J, h).energies_int()[0] == e0
            # global flip: bond term unchanged, field term negated
            s, Ji, hi = oracle.quantise(J, h)
            m = int(sig.sum())
            e1 = _with_state(L, -sig, J, h).energies_int()[0]
            assert e0 - e1 == 2 * hi * m


@pytest.mark.parametrize("J,h", [(1.0, 0.0), (1.0, 0.1), (-1.0, 0.25), (0.0, 0.5), (2.0, 0.0),
                                 (3.0, 1.0)])
def test_energy_differences_lie_on_a_lattice(J, h):
    """Two spin states' E_int differ by a multiple of g = gcd(4 J_int, 2 h_int), and random
    states reach differences whose gcd is g itself: the number of unsatisfied bonds is even
    (one flip changes it by 4 - 2k), so the bond sum moves in steps of 4, and M in steps of
    2. The exchange tables hold the threshold only at multiples of the power of two in g."""
    import math
    rng = np.random.Generator(np.random.PCG64(11))
    s, Ji, hi = oracle.quantise(J, h)
    g = math.gcd(4 * abs(Ji), 2 * abs(hi))
    for L in (4, 6, 10):
        es = [_with_state(L, rng.choice(np.array([-1, 1], np.int8), size=(L, L)), J, h)
              .energies_int()[0] for _ in range(24)]
        diffs = [int(e - es[0]) for e in es[1:]]
        assert all(d % g == 0 for d in diffs), (L, diffs)
        assert math.gcd(*diffs) == g, (L, diffs)


# --------------------------------------------------------------------------------------
# Threshold formulas vs high-precision arithmetic
# --------------------------------------------------------------------------------------

def test_spin_threshold_values():
    import mpmath
    mpmath.mp.dps = 40
    assert oracle.spin_threshold(0.4, 0, 1) == TWO32
    assert oracle.spin_threshold(0.4, -8, 1) == TWO32
    assert oracle.spin_threshold(0.0, 8, 1) == TWO32          # beta = 0 accepts everything
    assert oracle.spin_threshold(1000.0, 1, 10) == 0          # zero temperature rejects
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(2000):
        beta = float(rng.uniform(0.0, 3.0))
        s = int(rng.choice([1, 2, 10, 100]))
        dE = int(rng.integers(1, 100))
        exact = mpmath.mpf(TWO32) * mpmath.exp(-mpmath.mpf(beta) * dE / s)
        T = oracle.spin_threshold(beta, dE, s)
        # the floor of the exact value, unless that value sits within rounding error of an
        # integer (FP64 exp carries ~1e-16 relative error, i.e. ~1e-6 absolute here)
        assert T == int(mpmath.floor(exact)) or abs(exact - mpmath.nint(exact)) < 1e-5
    # monotone: decreasing in dE and in beta
    for beta in (0.1, 0.44, 0.9):
        seq = [oracle.spin_threshold(beta, d, 1) for d in range(1, 30)]
        assert all(a >= b for a, b in zip(seq, seq[1:]))
    seq = [oracle.spin_threshold(b, 4, 1) for b in np.linspace(0, 2, 50)]
    assert all(a >= b for a, b in zip(seq, seq[1:]))


def test_swap_threshold_values():
    import mpmath
    mpmath.mp.dps = 40
    rng = np.random.Generator(np.random.PCG64(6))
    for _ in range(2000):
        b0 = float(rng.uniform(0.0, 1.0))
        b1 = b0 + float(rng.uniform(-0.1, 0.1))
        s = int(rng.choice([1, 10]))
        n = int(rng.integers(-3000, 3000))
        y = mpmath.mpf(b1 - b0) * n / s
        S = oracle.swap_threshold(b0, b1, n, s)
        if y > 44:
            assert S == 0
        elif y < -44:
            assert S == TWO32
        else:
            exact = mpmath.mpf(TWO32) / (1 + mpmath.exp(y))
            assert S == int(mpmath.floor(exact)) or abs(exact - mpmath.nint(exact)) < 1e-5
        # Barker form: p(y) + p(-y) = 1
        S2 = oracle.swap_threshold(b0, b1, -n, s)
        assert abs(S + S2 - TWO32) <= 2
    # equal temperatures: exactly one half
    assert oracle.swap_threshold(0.4, 0.4, 12345, 1) == 1 << 31
    # the cut-off at 44 in both directions
    assert oracle.swap_threshold(0.0, 1.0, 45, 1) == 0
    assert oracle.swap_threshold(0.0, 1.0, -45, 1) == TWO32
    # Lower energy at the colder temperature (n < 0 with beta_hi > beta_lo) is the favoured
    # order, so swapping it away is unlikely: y = (b_hi - b_lo) n / s < 0 gives S > 2^31 only
    # when the hotter replica holds the lower energy.
    assert oracle.swap_threshold(0.3, 0.5, 100, 1) < (1 << 31)
    assert oracle.swap_threshold(0.3, 0.5, -100, 1) > (1 << 31)


# --------------------------------------------------------------------------------------
# Exact special cases of the Metropolis sweep
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("h", [0.0, 0.1])
def test_beta_zero_flips_every_spin(h):
    L, R = 8, 5
    p = oracle.OracleProblem(L, np.zeros(R), J=1.0, h=h, seed=77)
    s0 = p.spins()
    for n in range(1, 6):
        p.sweep(1)
        np.testing.assert_array_equal(p.spins(), s0 * (-1) ** n)


def _zero_temperature_quench(sig, sweeps):
    """Zero-temperature checkerboard dynamics written from the textbook rule: a spin turns
    over exactly when at least half of its four neighbours point the other way."""
    sig = sig.astype(np.int64).copy()
    L = sig.shape[0]
    yy, xx = np.mgrid[0:L, 0:L]
    for _ in range(sweeps):
        for colour in (0, 1):
            mask = ((xx + yy) % 2) == colour
            nb = [np.roll(sig, 1, 0), np.roll(sig, -1, 0), np.roll(sig, 1, 1), np.roll(sig, -1, 1)]
            against = sum((n != sig).astype(np.int64) for n in nb)
            turn = mask & (against >= 2)
            sig[turn] = -sig[turn]
    return sig.astype(np.int8)


def test_zero_temperature_quench():
    L = 12
    p = oracle.OracleProblem(L, [1000.0, 1000.0, 1000.0], J=1.0, h=0.0, seed=123)
    s0 = p.spins()
    p.sweep(7)
    for k in range(3):
        np.testing.assert_array_equal(p.spins(k), _zero_temperature_quench(s0[k], 7))


def test_global_flip_symmetry_h0():
    L, betas = 8, [0.25, 0.4, 0.5, 0.7]
    a = oracle.OracleProblem(L, betas, seed=9)
    b = oracle.OracleProblem(L, betas, seed=9)
    for k in range(len(betas)):
        b.set_spins(k, -a.spins(k))
    a.sweep(60, 3)
    b.sweep(60, 3)
    np.testing.assert_array_equal(b.spins(), -a.spins())
    np.testing.assert_array_equal(a.energies_int(), b.energies_int())
    for x, y in zip(a.swap_stats(), b.swap_stats()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.chain_map(), b.chain_map())


def test_splitting_and_threading_invariance():
    L, betas = 10, np.linspace(0.3, 0.6, 6)
    a = oracle.OracleProblem(L, betas, seed=21)
    a.sweep(13, 4)
    a.sweep(0, 4)
    a.sweep(20, 4)
    b = oracle.OracleProblem(L, betas, seed=21)
    oracle.set_threads(4)
    try:
        b.sweep(33, 4)
    finally:
        oracle.set_threads(1)
    np.testing.assert_array_equal(a.spins(), b.spins())
    for x, y in zip(a.swap_stats(), b.swap_stats()):
        np.testing.assert_array_equal(x, y)
    assert a.counters() == b.counters() == (33, 8)


@pytest.mark.parametrize("R,n,m", [(8, 1000, 10), (5, 37, 3), (2, 10, 1), (1, 10, 1), (7, 9, 0),
                                   (5, 37, 4), (3, 7, 1), (2, 1, 1), (6, 15, 5)])
def test_attempt_counts_closed_form(R, n, m):
    p = oracle.OracleProblem(4, np.linspace(0.2, 0.6, R), seed=5)
    p.sweep(n, m)
    att, acc = p.swap_stats()
    n_exch = n // m if m else 0
    for k in range(R - 1):
        assert att[k] == sum(1 for e in range(n_exch) if e % 2 == k % 2)
        assert acc[k] <= att[k]
    assert p.counters() == (n, n_exch)
    # the chain map is a permutation
    assert sorted(p.chain_map().tolist()) == list(range(R))


def test_first_exchange_pairs_even_neighbours():
    """Sec. 3: the first swap iteration pairs (0,1), (2,3), ...; the second (1,2), (3,4), ..."""
    p = oracle.OracleProblem(4, np.linspace(0.2, 0.6, 6), seed=8)
    p.sweep(1, 1)
    assert p.swap_stats()[0].tolist() == [1, 0, 1, 0, 1]
    p.sweep(1, 1)
    assert p.swap_stats()[0].tolist() == [1, 1, 1, 1, 1]


def test_replica_streams_are_independent():
    """Every slot draws its own random numbers: slots started from one configuration at one
    temperature part ways, and so does a rerun with another seed."""
    L, R = 16, 12
    p = oracle.OracleProblem(L, np.full(R, 0.42), seed=4)
    q = oracle.OracleProblem(L, np.full(R, 0.42), seed=5)
    start = np.ones((L, L), np.int8)
    start[::3, ::5] = -1
    for k in range(R):
        p.set_spins(k, start)
        q.set_spins(k, start)
    p.sweep(6)
    q.sweep(6)
    s = p.spins().reshape(R, -1)
    for a in range(R):
        assert (s[a] != q.spins(a).reshape(-1)).mean() > 0.02
        for b in range(a + 1, R):
            assert (s[a] != s[b]).mean() > 0.02, (a, b)


def test_initial_state_uniform():
    L, R = 128, 8
    p = oracle.OracleProblem(L, np.full(R, 0.4), seed=0x5EED0002)
    s = p.spins()
    assert set(np.unique(s).tolist()) == {-1, 1}
    n = s.size
    frac = (s == 1).mean()
    assert abs(frac - 0.5) < 4 * 0.5 / np.sqrt(n)
    # different temperature indices and different seeds draw different lattices
    assert (s[0] != s[1]).mean() > 0.45
    q = oracle.OracleProblem(L, np.full(R, 0.4), seed=0x5EED0003)
    assert (q.spins(0) != s[0]).mean() > 0.45


def test_create_rejects_bad_arguments():
    for L, betas, J, h in [(5, [0.1], 1, 0), (2, [0.1], 1, 0), (8, [], 1, 0), (8, [-0.1], 1, 0),
                           (8, [float("nan")], 1, 0), (8, [0.1], np.pi, 0)]:
        with pytest.raises(ValueError):
            oracle.OracleProblem(L, betas, J=J, h=h)
