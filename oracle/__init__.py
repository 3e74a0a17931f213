"""ctypes binding of the CPU oracle (``pt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the plain, slow reference for Metropolis-Hastings with Parallel
Tempering on the periodic 2D Ising model (arXiv 2512.03825, Secs. 2.1, 2.2 and 3). Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it. It imports
nothing from the CUDA package and the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
        L.oracle_philox4x32_10.restype = None
        L.oracle_quantise.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.oracle_quantise.restype = C.c_int
        L.oracle_spin_threshold.argtypes = [C.c_double, C.c_int64, C.c_int64]
        L.oracle_spin_threshold.restype = C.c_uint64
        L.oracle_swap_threshold.argtypes = [C.c_double, C.c_double, C.c_int64, C.c_int64]
        L.oracle_swap_threshold.restype = C.c_uint64
        L.oracle_create.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double,
                                    C.c_double, C.c_uint64, C.POINTER(P)]
        L.oracle_create.restype = C.c_int
        L.oracle_create_ex.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double,
                                       C.c_double, C.c_uint64, C.c_int, C.POINTER(P)]
        L.oracle_create_ex.restype = C.c_int
        L.oracle_swap_threshold_metropolis.argtypes = [C.c_double, C.c_double, C.c_int64,
                                                       C.c_int64]
        L.oracle_swap_threshold_metropolis.restype = C.c_uint64
        L.oracle_destroy.argtypes = [P]
        L.oracle_destroy.restype = None
        L.oracle_sweep.argtypes = [P, C.c_int64, C.c_int]
        L.oracle_sweep.restype = C.c_int
        L.oracle_trace.argtypes = [P, C.c_int64, C.c_int, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]
        L.oracle_trace.restype = C.c_int
        L.oracle_energy_int.argtypes = [P, C.c_int]
        L.oracle_energy_int.restype = C.c_int64
        L.oracle_magnetisation.argtypes = [P, C.c_int]
        L.oracle_magnetisation.restype = C.c_int64
        L.oracle_flip.argtypes = [P, C.c_int64, C.c_int]
        L.oracle_flip.restype = C.c_int
        L.oracle_iterations.argtypes = [P]
        L.oracle_iterations.restype = C.c_uint64
        L.oracle_set_iterations.argtypes = [P, C.c_uint64]
        L.oracle_set_iterations.restype = None
        L.oracle_scale.argtypes = [P]
        L.oracle_scale.restype = C.c_int64
        L.oracle_get_spins.argtypes = [P, C.c_int, C.POINTER(C.c_int8)]
        L.oracle_get_spins.restype = C.c_int
        L.oracle_set_spins.argtypes = [P, C.c_int, C.POINTER(C.c_int8)]
        L.oracle_set_spins.restype = C.c_int
        L.oracle_chain_map.argtypes = [P, C.POINTER(C.c_int32)]
        L.oracle_chain_map.restype = None
        L.oracle_swap_stats.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.oracle_swap_stats.restype = None
        L.oracle_counters.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.oracle_counters.restype = None
        L.oracle_load_state.argtypes = [P, C.POINTER(C.c_int8), C.POINTER(C.c_int32),
                                        C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64),
                                        C.POINTER(C.c_uint64)]
        L.oracle_load_state.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_set_threads.restype = None
        L.oracle_get_threads.argtypes = []
        L.oracle_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 uint32, key = 2 uint32 -> 4 uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def quantise(J, h):
    """(s, J_int, h_int) with s*J = J_int and s*h = h_int exactly, or ValueError."""
    s, ji, hi = C.c_int64(), C.c_int64(), C.c_int64()
    rc = lib().oracle_quantise(float(J), float(h), C.byref(s), C.byref(ji), C.byref(hi))
    if rc != 0:
        raise ValueError("J=%r, h=%r cannot be quantised" % (J, h))
    return s.value, ji.value, hi.value


def spin_threshold(beta, dE_int, s):
    """Metropolis threshold T in [0, 2^32] (accept iff u < T)."""
    return int(lib().oracle_spin_threshold(float(beta), int(dE_int), int(s)))


SWAP_BARKER, SWAP_METROPOLIS = 0, 1


def swap_threshold(beta_lo, beta_hi, n, s, rule=SWAP_BARKER):
    """Replica-exchange threshold S in [0, 2^32] (accept iff u < S), Barker or Metropolis."""
    f = lib().oracle_swap_threshold_metropolis if rule == SWAP_METROPOLIS \
        else lib().oracle_swap_threshold
    return int(f(float(beta_lo), float(beta_hi), int(n), int(s)))


def set_threads(n):
    lib().oracle_set_threads(int(n))


def get_threads():
    return int(lib().oracle_get_threads())


class OracleProblem:
    """One PT problem held by the oracle: int8 spins [R][L][L], temperature-indexed."""

    def __init__(self, L, betas, J=1.0, h=0.0, seed=0, swap_rule=SWAP_BARKER):
        b = np.ascontiguousarray(betas, dtype=np.float64)
        h_ = C.c_void_p()
        rc = lib().oracle_create_ex(int(L), _ptr(b, C.c_double), int(b.size), float(J),
                                    float(h), int(seed) & 0xFFFFFFFFFFFFFFFF, int(swap_rule),
                                    C.byref(h_))
        if rc != 0:
            raise ValueError("oracle_create failed (%d) for L=%r R=%r J=%r h=%r rule=%r"
                             % (rc, L, b.size, J, h, swap_rule))
        self._h = h_
        self.L, self.R = int(L), int(b.size)
        self.betas = b.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().oracle_destroy(h)
            self._h = None

    def sweep(self, n, exchange_every=0):
        rc = lib().oracle_sweep(self._h, int(n), int(exchange_every))
        if rc != 0:
            raise ValueError("oracle_sweep failed (%d)" % rc)

    def flip(self, n, exchange_every=0):
        """n single-spin-flip iterations of every replica (one random site each), a swap
        iteration after every iteration count that is a multiple of exchange_every."""
        rc = lib().oracle_flip(self._h, int(n), int(exchange_every))
        if rc != 0:
            raise ValueError("oracle_flip failed (%d)" % rc)

    @property
    def iterations(self):
        return int(lib().oracle_iterations(self._h))

    def set_iterations(self, it):
        lib().oracle_set_iterations(self._h, int(it))

    def trace(self, n, exchange_every=0):
        """Run n sweeps; return (E_int[n][R], M[n][R]) recorded after each sweep."""
        E = np.zeros((int(n), self.R), dtype=np.int64)
        M = np.zeros((int(n), self.R), dtype=np.int64)
        rc = lib().oracle_trace(self._h, int(n), int(exchange_every), _ptr(E, C.c_int64),
                                _ptr(M, C.c_int64))
        if rc != 0:
            raise ValueError("oracle_trace failed (%d)" % rc)
        return E, M

    @property
    def scale(self):
        return int(lib().oracle_scale(self._h))

    def energies_int(self):
        return np.array([lib().oracle_energy_int(self._h, k) for k in range(self.R)],
                        dtype=np.int64)

    def magnetisations(self):
        return np.array([lib().oracle_magnetisation(self._h, k) for k in range(self.R)],
                        dtype=np.int64)

    def energies(self):
        return self.energies_int().astype(np.float64) / self.scale

    def spins(self, k=None):
        """int8 spins of temperature k ([L][L]) or of all temperatures ([R][L][L])."""
        if k is None:
            return np.stack([self.spins(j) for j in range(self.R)])
        out = np.zeros((self.L, self.L), dtype=np.int8)
        rc = lib().oracle_get_spins(self._h, int(k), _ptr(out, C.c_int8))
        if rc != 0:
            raise ValueError("bad temperature index %r" % k)
        return out

    def set_spins(self, k, arr):
        a = np.ascontiguousarray(arr, dtype=np.int8).reshape(self.L, self.L)
        rc = lib().oracle_set_spins(self._h, int(k), _ptr(a, C.c_int8))
        if rc != 0:
            raise ValueError("oracle_set_spins failed")

    def chain_map(self):
        out = np.zeros(self.R, dtype=np.int32)
        lib().oracle_chain_map(self._h, _ptr(out, C.c_int32))
        return out

    def swap_stats(self):
        n = max(self.R - 1, 0)
        att = np.zeros(max(n, 1), dtype=np.uint64)
        acc = np.zeros(max(n, 1), dtype=np.uint64)
        lib().oracle_swap_stats(self._h, _ptr(att, C.c_uint64), _ptr(acc, C.c_uint64))
        return att[:n], acc[:n]

    def counters(self):
        t, e = C.c_uint64(), C.c_uint64()
        lib().oracle_counters(self._h, C.byref(t), C.byref(e))
        return t.value, e.value

    def load_state(self, spins_by_slot, slot_of_temp, t, e, attempted, accepted):
        """Continue the chain from a given state: spins [R][L][L] by slot, the temperature
        map, the counters and the swap statistics."""
        sp = np.ascontiguousarray(spins_by_slot, dtype=np.int8).reshape(self.R, self.L, self.L)
        so = np.ascontiguousarray(slot_of_temp, dtype=np.int32)
        att = np.ascontiguousarray(attempted, dtype=np.uint64)
        acc = np.ascontiguousarray(accepted, dtype=np.uint64)
        if att.size == 0:
            att = np.zeros(1, np.uint64)
            acc = np.zeros(1, np.uint64)
        rc = lib().oracle_load_state(self._h, _ptr(sp, C.c_int8), _ptr(so, C.c_int32), int(t),
                                     int(e), _ptr(att, C.c_uint64), _ptr(acc, C.c_uint64))
        if rc != 0:
            raise ValueError("oracle_load_state failed (%d)" % rc)
