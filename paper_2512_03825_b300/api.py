"""Python face of libpt: one PT problem per `PTProblem`, `sweep_batch` for many at once.

PyTorch provides the device memory (through `use_torch_allocator`) and the streams; all
sampling work is done by the library's kernels.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from ._lib import ALLOC_FN, FREE_FN, PTOptions, check, lib


def _dptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class PTProblem:
    """Metropolis-Hastings with parallel tempering on an L x L periodic Ising lattice with R
    temperatures (inverse temperatures `betas`), coupling J and field h."""

    def __init__(self, L: int, betas: Sequence[float], J: float = 1.0, h: float = 0.0,
                 seed: int = 0, stream=None, swap_rule: int = 0, _handle=None):
        b = np.ascontiguousarray(betas, dtype=np.float64)
        if _handle is None:
            h_ = C.c_void_p()
            raw = int(getattr(stream, "cuda_stream", stream) or 0)
            opt = PTOptions(C.sizeof(PTOptions), int(swap_rule), C.c_void_p(raw))
            check(lib.pt_create_ex(int(L), _dptr(b, C.c_double), int(b.size), float(J),
                                   float(h), int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(opt),
                                   C.byref(h_)), "pt_create_ex")
        else:
            h_ = _handle
        self._h = h_
        self.L, self.R = int(L), int(b.size)
        self.betas = b.copy()
        self.J, self.h, self.seed = float(J), float(h), int(seed)
        self.swap_rule = int(swap_rule)
        if stream is not None and _handle is not None:
            self.set_stream(stream)

    # -- checkpoints ---------------------------------------------------------------------
    def save(self) -> bytes:
        """The problem's whole sampler state as a checkpoint (format in include/pt.h)."""
        n = int(lib.pt_checkpoint_bytes(self._h))
        buf = C.create_string_buffer(n)
        check(lib.pt_save(self._h, buf, n), "pt_save")
        return buf.raw

    @classmethod
    def load(cls, data: bytes, stream=None) -> "PTProblem":
        """A new problem that continues exactly from a checkpoint made by `save`."""
        import struct
        buf = C.create_string_buffer(bytes(data), len(data))
        h_ = C.c_void_p()
        check(lib.pt_load(buf, len(data), C.byref(h_)), "pt_load")
        L, R = struct.unpack_from("<II", data, 8)
        J, h = struct.unpack_from("<dd", data, 16)
        seed, = struct.unpack_from("<Q", data, 32)
        rule, = struct.unpack_from("<i", data, 56)
        betas = np.frombuffer(data, np.float64, R, 72)
        return cls(L, betas, J=J, h=h, seed=seed, stream=stream, swap_rule=rule, _handle=h_)

    # -- lifetime ------------------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.pt_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (default)."""
        raw = getattr(stream, "cuda_stream", stream)
        check(lib.pt_set_stream(self._h, C.c_void_p(int(raw or 0))), "pt_set_stream")

    # -- work ----------------------------------------------------------------------------
    def sweep(self, n: int, exchange_every: int = 0):
        check(lib.pt_sweep(self._h, int(n), int(exchange_every)), "pt_sweep")

    def synchronize(self):
        check(lib.pt_synchronize(self._h), "pt_synchronize")

    def flip(self, n: int, exchange_every: int = 0):
        """n single-spin-flip iterations of every replica (one random site each)."""
        check(lib.pt_flip(self._h, int(n), int(exchange_every)), "pt_flip")

    def set_flip_tuning(self, shared_memory: bool = True):
        check(lib.pt_set_flip_tuning(self._h, int(bool(shared_memory))), "pt_set_flip_tuning")

    @property
    def iterations(self) -> int:
        it = C.c_uint64()
        check(lib.pt_iterations(self._h, C.byref(it)), "pt_iterations")
        return it.value

    def trace_start(self, capacity: int):
        """Record (E_int, M) of every temperature after each later sweep, in a device ring of
        `capacity` rows."""
        check(lib.pt_trace_start(self._h, int(capacity)), "pt_trace_start")

    def trace_stop(self):
        check(lib.pt_trace_stop(self._h), "pt_trace_stop")

    def trace(self, max_rows: Optional[int] = None):
        """(first_sweep, E_int[rows][R], M[rows][R]) of the newest trace rows, oldest first;
        first_sweep = sweeps done when the first row was taken."""
        if max_rows is None:
            max_rows = self.counters()[0]
        max_rows = int(max_rows)
        E = np.zeros((max(max_rows, 1), self.R), np.int64)
        M = np.zeros((max(max_rows, 1), self.R), np.int64)
        first, rows = C.c_uint64(), C.c_int64()
        check(lib.pt_trace_read(self._h, max_rows, _dptr(E, C.c_int64), _dptr(M, C.c_int64),
                                C.byref(first), C.byref(rows)), "pt_trace_read")
        n = rows.value
        return first.value, E[:n].copy(), M[:n].copy()

    def set_sweep_tuning(self, strategy: int = 0, words_per_thread: int = 0):
        """strategy: PT_SWEEP_AUTO (0), PT_SWEEP_LAUNCHES (1) or PT_SWEEP_PERSISTENT (2)."""
        check(lib.pt_set_sweep_tuning(self._h, int(strategy), int(words_per_thread)),
              "pt_set_sweep_tuning")

    def sweep_tuning(self):
        """(strategy, words_per_thread, persistent grid or 0)."""
        s, w, g = C.c_int(), C.c_int(), C.c_int()
        check(lib.pt_get_sweep_tuning(self._h, C.byref(s), C.byref(w), C.byref(g)),
              "pt_get_sweep_tuning")
        return s.value, w.value, g.value

    def set_wait_limit(self, seconds: float):
        check(lib.pt_set_wait_limit(self._h, float(seconds)), "pt_set_wait_limit")

    def debug_stall_barrier(self, arrivals: int):
        check(lib.pt_debug_stall_barrier(self._h, int(arrivals)), "pt_debug_stall_barrier")

    # -- observables ---------------------------------------------------------------------
    def energies_int(self):
        E = np.zeros(self.R, np.int64)
        check(lib.pt_energies_int(self._h, _dptr(E, C.c_int64), None, None), "pt_energies_int")
        return E

    def magnetisations(self):
        M = np.zeros(self.R, np.int64)
        check(lib.pt_energies_int(self._h, None, _dptr(M, C.c_int64), None), "pt_energies_int")
        return M

    @property
    def scale(self):
        s = C.c_int64()
        check(lib.pt_energies_int(self._h, None, None, C.byref(s)), "pt_energies_int")
        return s.value

    def energies(self):
        out = np.zeros(self.R, np.float64)
        check(lib.pt_energies(self._h, _dptr(out, C.c_double)), "pt_energies")
        return out

    def magnetisations_f(self):
        out = np.zeros(self.R, np.float64)
        check(lib.pt_magnetisations(self._h, _dptr(out, C.c_double)), "pt_magnetisations")
        return out

    def swap_stats(self):
        n = max(self.R - 1, 0)
        att = np.zeros(max(n, 1), np.uint64)
        acc = np.zeros(max(n, 1), np.uint64)
        check(lib.pt_swap_stats(self._h, _dptr(att, C.c_uint64), _dptr(acc, C.c_uint64)),
              "pt_swap_stats")
        return att[:n], acc[:n]

    def chain_map(self):
        out = np.zeros(self.R, np.int32)
        check(lib.pt_chain_map(self._h, _dptr(out, C.c_int32)), "pt_chain_map")
        return out

    def counters(self):
        t, e = C.c_uint64(), C.c_uint64()
        check(lib.pt_counters(self._h, C.byref(t), C.byref(e)), "pt_counters")
        return t.value, e.value

    def spins(self, k: Optional[int] = None):
        if k is None:
            return np.stack([self.spins(j) for j in range(self.R)])
        out = np.zeros((self.L, self.L), np.int8)
        check(lib.pt_get_spins(self._h, int(k), _dptr(out, C.c_int8)), "pt_get_spins")
        return out

    def set_spins(self, k: int, arr):
        a = np.ascontiguousarray(arr, dtype=np.int8).reshape(self.L, self.L)
        check(lib.pt_set_spins(self._h, int(k), _dptr(a, C.c_int8)), "pt_set_spins")

    @property
    def device_bytes(self):
        return int(lib.pt_device_bytes(self._h))


def _batch_call(fn, name, problems, n, exchange_every):
    k = len(problems)
    if k == 0:
        return
    ns = np.ascontiguousarray(np.broadcast_to(np.asarray(n, np.int64), (k,)))
    ms = np.ascontiguousarray(np.broadcast_to(np.asarray(exchange_every, np.int32), (k,)))
    hs = (C.c_void_p * k)(*[p.handle.value for p in problems])
    check(fn(hs, k, _dptr(ns, C.c_int64), _dptr(ms, C.c_int32)), name)


def sweep_batch(problems: Sequence[PTProblem], n, exchange_every):
    """Advance all problems together with the batched strategy (n, exchange_every: an int
    or one value per problem)."""
    _batch_call(lib.pt_sweep_batch, "pt_sweep_batch", problems, n, exchange_every)


def sweep_batch_static(problems: Sequence[PTProblem], n, exchange_every):
    """The same batch through pt_sweep_batch_static: the lock-step strategy with its work
    lists in the library's fixed device array (no device allocation; returns after the
    lists are uploaded, the sweeps still queued on the problems' stream)."""
    _batch_call(lib.pt_sweep_batch_static, "pt_sweep_batch_static", problems, n,
                exchange_every)


def read_batch(problems: Sequence[PTProblem]):
    """Energies (E_int), magnetisations, temperature maps and swap counters of many problems
    in one transfer (pt_read_batch): a list of dicts with keys E_int, M, chain_map,
    attempted, accepted (numpy arrays by temperature index / pair)."""
    k = len(problems)
    if k == 0:
        return []
    out = []
    for p in problems:
        npairs = max(p.R - 1, 0)
        out.append({"E_int": np.empty(p.R, np.int64), "M": np.empty(p.R, np.int64),
                    "chain_map": np.empty(p.R, np.int32),
                    "attempted": np.empty(npairs, np.uint64),
                    "accepted": np.empty(npairs, np.uint64)})

    def ptrs(key, ctype):
        arr = (C.POINTER(ctype) * k)()
        for j, o in enumerate(out):
            arr[j] = o[key].ctypes.data_as(C.POINTER(ctype))
        return arr
    hs = (C.c_void_p * k)(*[p.handle.value for p in problems])
    check(lib.pt_read_batch(hs, k, ptrs("E_int", C.c_int64), ptrs("M", C.c_int64),
                            ptrs("chain_map", C.c_int32), ptrs("attempted", C.c_uint64),
                            ptrs("accepted", C.c_uint64)), "pt_read_batch")
    return out


def set_batch_tile_words(tile_words: int) -> None:
    """Words per warp tile of the tile strategies (a multiple of 32 in [64, 1024])."""
    check(lib.pt_set_batch_tile_words(int(tile_words)), "pt_set_batch_tile_words")


def batch_tile_words() -> int:
    w = C.c_int()
    check(lib.pt_get_batch_tile_words(C.byref(w)), "pt_get_batch_tile_words")
    return w.value


def estimate_device_bytes(L, betas, J=1.0, h=0.0):
    b = np.ascontiguousarray(betas, dtype=np.float64)
    return int(lib.pt_estimate_device_bytes(int(L), _dptr(b, C.c_double), int(b.size),
                                            float(J), float(h)))


def set_image_cache_limit(nbytes: int) -> None:
    """Page-locked host bytes the creation-image cache may hold (default 1 GiB)."""
    check(lib.pt_set_image_cache_limit(int(nbytes)), "pt_set_image_cache_limit")


def image_cache_bytes() -> int:
    """Page-locked host bytes the creation-image cache holds now."""
    return int(lib.pt_image_cache_bytes())


def quantise(J, h):
    s, ji, hi = C.c_int64(), C.c_int64(), C.c_int64()
    check(lib.pt_quantise(float(J), float(h), C.byref(s), C.byref(ji), C.byref(hi)),
          "pt_quantise")
    return s.value, ji.value, hi.value


def spin_threshold(beta, dE_int, s):
    return int(lib.pt_spin_threshold(float(beta), int(dE_int), int(s)))


def swap_threshold_rule(beta_lo, beta_hi, n, s, rule):
    """The device's exchange threshold for either swap rule (0 Barker, 1 Metropolis)."""
    return int(lib.pt_swap_threshold_ex(float(beta_lo), float(beta_hi), int(n), int(s),
                                        int(rule)))


def swap_threshold(beta_lo, beta_hi, n, s):
    return int(lib.pt_swap_threshold(float(beta_lo), float(beta_hi), int(n), int(s)))


# -- PyTorch as the device-memory provider -------------------------------------------------
# Every problem remembers the free function it was allocated with, so the ctypes callbacks
# handed to the library must outlive every problem: they are kept for the whole process and
# installed at most once.
_torch_hooks = None
_all_hooks = []


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator (idempotent).
    With enable=False, later problems go back to cudaMalloc; problems created through torch
    keep releasing their memory through it."""
    global _torch_hooks
    if not enable:
        check(lib.pt_set_allocator(ALLOC_FN(), FREE_FN(), None), "pt_set_allocator")
        _torch_hooks = None
        return
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or None))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        if ptr:
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:  # interpreter shutdown
                pass

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _all_hooks.append(hooks)
    check(lib.pt_set_allocator(hooks[0], hooks[1], None), "pt_set_allocator")
    _torch_hooks = hooks
