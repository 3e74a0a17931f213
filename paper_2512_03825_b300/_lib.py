"""ctypes binding of libpt.so (declarations in include/pt.h). Argument marshalling only:
every step of the sampler runs in the library's CUDA kernels.

The library is loaded from this package's directory. If it is missing the import of this
module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# PT_LIBRARY=debug selects the debug build (libpt_debug.so: bounds and write-set checks in
# every kernel); the default is the release library.
LIB_PATH = os.path.join(HERE, "libpt_debug.so" if os.environ.get("PT_LIBRARY") == "debug"
                        else "libpt.so")

PT_OK = 0
PT_EINVAL = -1
PT_ENOMEM = -2
PT_ECUDA = -3
PT_ETIMEOUT = -4
PT_ESTATE = -5
PT_ENODEV = -6
PT_EINTERNAL = -7
PT_BATCH_FLAT = 0
PT_BATCH_CLUSTER = 1
PT_BATCH_FLOW = 2
PT_SWEEP_AUTO = 0
PT_SWEEP_LAUNCHES = 1
PT_SWEEP_PERSISTENT = 2
PT_MAX_L = 16384
PT_MAX_R = 2048

PT_SWAP_BARKER = 0
PT_SWAP_METROPOLIS = 1


class PTOptions(C.Structure):
    """struct pt_options of include/pt.h."""
    _fields_ = [("size", C.c_uint32), ("swap_rule", C.c_int32), ("stream", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every function include/pt.h declares
P = C.c_void_p
SIGNATURES = [
    ("pt_create", C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_double,
                            C.c_uint64, C.POINTER(P)]),
    ("pt_create_ex", C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double,
                               C.c_double, C.c_uint64, C.POINTER(PTOptions), C.POINTER(P)]),
    ("pt_destroy", None, [P]),
    ("pt_set_stream", C.c_int, [P, P]),
    ("pt_sweep", C.c_int, [P, C.c_int64, C.c_int]),
    ("pt_flip", C.c_int, [P, C.c_int64, C.c_int]),
    ("pt_iterations", C.c_int, [P, C.POINTER(C.c_uint64)]),
    ("pt_set_flip_tuning", C.c_int, [P, C.c_int]),
    ("pt_set_sweep_tuning", C.c_int, [P, C.c_int, C.c_int]),
    ("pt_get_sweep_tuning", C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
    ("pt_set_wait_limit", C.c_int, [P, C.c_double]),
    ("pt_debug_build", C.c_int, []),
    ("pt_debug_report", C.c_int, [P, C.POINTER(C.c_uint64), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("pt_debug_inject", C.c_int, [P, C.c_int]),
    ("pt_debug_stall_barrier", C.c_int, [P, C.c_int]),
    ("pt_sweep_batch", C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int)]),
    ("pt_sweep_batch_static", C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int)]),
    ("pt_set_batch_tuning", C.c_int, [C.c_int, C.c_int, C.c_int]),
    ("pt_get_batch_tuning", C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
    ("pt_set_batch_tile_words", C.c_int, [C.c_int]),
    ("pt_set_batch_streams", C.c_int, [C.c_int]),
    ("pt_get_batch_streams", C.c_int, [C.POINTER(C.c_int)]),
    ("pt_set_batch_graphs", C.c_int, [C.c_int]),
    ("pt_get_batch_graphs", C.c_int, [C.POINTER(C.c_int)]),
    ("pt_read_batch", C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.POINTER(C.c_int64)),
                                C.POINTER(C.POINTER(C.c_int64)), C.POINTER(C.POINTER(C.c_int32)),
                                C.POINTER(C.POINTER(C.c_uint64)),
                                C.POINTER(C.POINTER(C.c_uint64))]),
    ("pt_get_batch_tile_words", C.c_int, [C.POINTER(C.c_int)]),
    ("pt_energies", C.c_int, [P, C.POINTER(C.c_double)]),
    ("pt_magnetisations", C.c_int, [P, C.POINTER(C.c_double)]),
    ("pt_swap_stats", C.c_int, [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("pt_energies_int", C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
    ("pt_get_spins", C.c_int, [P, C.c_int, C.POINTER(C.c_int8)]),
    ("pt_set_spins", C.c_int, [P, C.c_int, C.POINTER(C.c_int8)]),
    ("pt_chain_map", C.c_int, [P, C.POINTER(C.c_int32)]),
    ("pt_temperature_map", C.c_int, [P, C.POINTER(C.c_int32)]),
    ("pt_counters", C.c_int, [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("pt_checkpoint_bytes", C.c_size_t, [P]),
    ("pt_save", C.c_int, [P, C.c_void_p, C.c_size_t]),
    ("pt_load", C.c_int, [C.c_void_p, C.c_size_t, C.POINTER(P)]),
    ("pt_trace_start", C.c_int, [P, C.c_int64]),
    ("pt_trace_stop", C.c_int, [P]),
    ("pt_trace_read", C.c_int, [P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_uint64), C.POINTER(C.c_int64)]),
    ("pt_synchronize", C.c_int, [P]),
    ("pt_device_bytes", C.c_size_t, [P]),
    ("pt_estimate_device_bytes", C.c_size_t, [C.c_int, C.POINTER(C.c_double), C.c_int,
                                              C.c_double, C.c_double]),
    ("pt_set_image_cache_limit", C.c_int, [C.c_size_t]),
    ("pt_image_cache_bytes", C.c_size_t, []),
    ("pt_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, P]),
    ("pt_strerror", C.c_char_p, [C.c_int]),
    ("pt_last_error", C.c_char_p, []),
    ("pt_quantise", C.c_int, [C.c_double, C.c_double, C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("pt_spin_threshold", C.c_uint64, [C.c_double, C.c_int64, C.c_int64]),
    ("pt_swap_threshold", C.c_uint64, [C.c_double, C.c_double, C.c_int64, C.c_int64]),
    ("pt_swap_threshold_ex", C.c_uint64, [C.c_double, C.c_double, C.c_int64, C.c_int64,
                                          C.c_int]),
    ("pt_version", C.c_char_p, []),
]


class PTError(RuntimeError):
    """A libpt call returned a PT_E* code."""

    def __init__(self, code, where, detail):
        self.code = code
        super().__init__("%s failed: %s (%d): %s" % (where, _strerror(code), code, detail))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built; run `python -m paper_2512_03825_b300.build` or "
                          "__graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _strerror(code):
    return lib.pt_strerror(int(code)).decode()


def check(rc, where):
    if rc != PT_OK:
        raise PTError(rc, where, lib.pt_last_error().decode())
    return rc
