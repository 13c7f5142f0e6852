"""Integer-pipe peak of the GPU, measured by libselscan_peak.so
(include/selscan_peak.h): the denominators of the scan kernels' integer
roofline.  Each entry is one operation in independent chains over 64
resident warps per SM, timed with CUDA events."""
from __future__ import annotations

import ctypes
import os
from typing import Dict

_PKG = os.path.dirname(os.path.abspath(__file__))
PEAK_LIB_PATH = os.path.join(_PKG, "libselscan_peak.so")
OPS = ("LOP3", "PRMT", "IMNMX", "VIMNMX2", "POPC", "SHF", "IADD3")
EXPORTS = ("selscan_peak_int", "selscan_peak_scratch_bytes")


class selscan_peak_result(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_double), ("ms", ctypes.c_double), ("ops_per_s", ctypes.c_double),
                ("cycles", ctypes.c_double), ("ops_per_sm_per_cycle", ctypes.c_double),
                ("clock_mhz_attr", ctypes.c_double), ("clock_mhz_implied", ctypes.c_double),
                ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def load_library():
    global _lib
    if _lib is None:
        if not os.path.exists(PEAK_LIB_PATH):
            raise RuntimeError(f"{PEAK_LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(PEAK_LIB_PATH)
        lib.selscan_peak_scratch_bytes.restype = ctypes.c_size_t
        lib.selscan_peak_scratch_bytes.argtypes = []
        lib.selscan_peak_int.restype = ctypes.c_int
        lib.selscan_peak_int.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.POINTER(selscan_peak_result)]
        _lib = lib
    return _lib


def measure(iters: int = 2048) -> Dict[str, Dict[str, float]]:
    """Per operation: ops/s, ops per SM per cycle, and the clock implied by the
    in-kernel cycle count (MHz)."""
    import torch
    lib = load_library()
    n = int(lib.selscan_peak_scratch_bytes())
    scratch = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    out = {}
    for i, name in enumerate(OPS):
        r = selscan_peak_result()
        rc = lib.selscan_peak_int(i, iters, ctypes.c_void_p(scratch.data_ptr()), n, ctypes.byref(r))
        if rc != 0:
            raise RuntimeError(f"selscan_peak_int({name}) failed: {rc}")
        out[name] = {"ops_per_s": r.ops_per_s, "ops_per_sm_per_cycle": r.ops_per_sm_per_cycle,
                     "clock_mhz": r.clock_mhz_implied, "ms": r.ms}
    return out
