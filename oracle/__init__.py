"""CPU oracle for EHH / iHS / XPEHH (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``selscan_oracle.c``, a
literal string-enumeration implementation of the paper's Eq. 1, 3, 4 and 5
and of the truncation / gap / MAF rules of Sections 1.2-1.3, and shares no
code with the CUDA library.

Every public function takes packed marker-major rows (uint64 [m, ld]; bit
h % 64 of word h // 64 is haplotype h) plus positions (int64 bp) and a
genetic map (float64), and returns plain numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "selscan_oracle.c")
_LIB = os.path.join(_HERE, "libselscan_oracle.so")
_lib = None

# per-locus status codes (Section 1.2 rules; readings c6, c7, c11)
OK, MAF_FILTERED, UNDEFINED, ABORT_EDGE, ABORT_GAP = 0, 1, 2, 3, 4


class Params(ctypes.Structure):
    _fields_ = [("ehh_cut_num", ctypes.c_uint32), ("ehh_cut_den", ctypes.c_uint32),
                ("maf_num", ctypes.c_uint32), ("maf_den", ctypes.c_uint32),
                ("gap_scale_bp", ctypes.c_int64), ("max_gap_bp", ctypes.c_int64),
                ("include_crossing_term", ctypes.c_int32),
                ("xpehh_maf_filter", ctypes.c_int32),
                ("use_physical_map", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def params(ehh_cut=(1, 20), maf=(1, 20), gap_scale_bp=20_000, max_gap_bp=200_000,
           include_crossing_term=0, xpehh_maf_filter=0, use_physical_map=0) -> Params:
    """Section 1.2 defaults: EHH cutoff 0.05, MAF 0.05, 20 kbp scale, 200 kbp abort;
    use_physical_map=1 integrates over physical distance (the Section 2 option)."""
    return Params(ehh_cut[0], ehh_cut[1], maf[0], maf[1], gap_scale_bp, max_gap_bp,
                  include_crossing_term, xpehh_maf_filter, use_physical_map, 0)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", "-std=gnu11", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_ihs.restype = ctypes.c_int
        lib.oracle_ihs.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, P, P,
                                   ctypes.POINTER(Params), P, ctypes.c_int64, ctypes.c_int,
                                   P, P, P, P, P, P, P]
        lib.oracle_xpehh.restype = ctypes.c_int
        lib.oracle_xpehh.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, P, P, ctypes.POINTER(Params), P,
                                     ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P]
        lib.oracle_ehh.restype = ctypes.c_int
        lib.oracle_ehh.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, P, P,
                                   ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int64,
                                   P, P, P, P, P, P]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _cores(cores, m):
    if cores is None:
        return None, m
    c = _c(cores, np.int64)
    if c.size and (c.min() < 0 or c.max() >= m):
        raise ValueError("core index out of range")
    return c, c.size


def ihs(rows, n: int, pos, gmap, p: Optional[Params] = None,
        cores: Optional[Sequence[int]] = None, threads: int = 0) -> dict:
    """Unstandardised iHS at each core (all markers if cores is None)."""
    lib = _load()
    rows = _c(rows, np.uint64)
    pos, gmap = _c(pos, np.int64), _c(gmap, np.float64)
    m = rows.shape[0]
    c, k = _cores(cores, m)
    out = dict(status=np.zeros(k, np.int8), n1=np.zeros(k, np.int32),
               ihh1=np.zeros(k), ihh0=np.zeros(k), lnratio=np.zeros(k),
               stop=np.zeros((k, 4), np.int32), digest=np.zeros((k, 4), np.uint64))
    p = p or params()
    rc = lib.oracle_ihs(rows.ctypes.data, rows.shape[1], n, m, pos.ctypes.data, gmap.ctypes.data,
                        ctypes.byref(p), None if c is None else c.ctypes.data, k, threads,
                        *(out[f].ctypes.data for f in
                          ("status", "n1", "ihh1", "ihh0", "lnratio", "stop", "digest")))
    if rc != 0:
        raise ValueError("oracle_ihs: invalid arguments")
    return out


def xpehh(rows, nA: int, nB: int, pos, gmap, p: Optional[Params] = None,
          cores: Optional[Sequence[int]] = None, threads: int = 0) -> dict:
    """Unstandardised XPEHH at each core; rows hold W_A words of A then W_B of B."""
    lib = _load()
    rows = _c(rows, np.uint64)
    pos, gmap = _c(pos, np.int64), _c(gmap, np.float64)
    m = rows.shape[0]
    c, k = _cores(cores, m)
    out = dict(status=np.zeros(k, np.int8), n1=np.zeros(k, np.int32),
               ihhA=np.zeros(k), ihhB=np.zeros(k), lnratio=np.zeros(k),
               stop=np.zeros((k, 2), np.int32), digest=np.zeros((k, 6), np.uint64))
    p = p or params()
    rc = lib.oracle_xpehh(rows.ctypes.data, rows.shape[1], nA, nB, m, pos.ctypes.data,
                          gmap.ctypes.data, ctypes.byref(p),
                          None if c is None else c.ctypes.data, k, threads,
                          *(out[f].ctypes.data for f in
                            ("status", "n1", "ihhA", "ihhB", "lnratio", "stop", "digest")))
    if rc != 0:
        raise ValueError("oracle_xpehh: invalid arguments")
    return out


def ehh(rows, n: int, pos, gmap, locus: int, capacity: int,
        p: Optional[Params] = None) -> dict:
    """Per-step S(i) around one locus: walks [allele 1, allele 0, whole] x [down, up]."""
    lib = _load()
    rows = _c(rows, np.uint64)
    pos, gmap = _c(pos, np.int64), _c(gmap, np.float64)
    m = rows.shape[0]
    out = dict(S=np.zeros((3, 2, capacity), np.uint64), len=np.zeros((3, 2), np.int64),
               stop=np.zeros((3, 2), np.int32), status=np.zeros((3, 2), np.int8),
               ihh=np.zeros((3, 2)), denom=np.zeros(3, np.uint64))
    p = p or params()
    rc = lib.oracle_ehh(rows.ctypes.data, rows.shape[1], n, m, pos.ctypes.data, gmap.ctypes.data,
                        ctypes.byref(p), locus, capacity,
                        *(out[f].ctypes.data for f in ("S", "len", "stop", "status", "ihh",
                                                       "denom")))
    if rc != 0:
        raise ValueError("oracle_ehh: invalid arguments")
    return out


def normalize(score, status, n1, n: int, nbins: int) -> dict:
    """Standardised scores: Eq. 7 (iHS, nbins equal bins of the core's derived
    allele frequency n1 / n) and Eq. 11 (XPEHH, nbins = 1, genome-wide).  Only
    markers of status OK enter a bin; a bin's E and SD are its mean and sample
    standard deviation (count - 1); scores of bins with fewer than two values
    or SD 0, and markers that are not OK, are NaN."""
    score = np.asarray(score, dtype=np.float64)
    status = np.asarray(status)
    n1 = np.asarray(n1, dtype=np.int64)
    if nbins == 1:
        bins = np.zeros(score.size, dtype=np.int64)
    else:
        bins = np.minimum(nbins - 1, (n1 * nbins) // n)
    ok = status == OK
    out = np.full(score.size, np.nan)
    count = np.zeros(nbins, dtype=np.int64)
    mean = np.full(nbins, np.nan)
    sd = np.full(nbins, np.nan)
    for b in range(nbins):
        sel = ok & (bins == b)
        vals = score[sel]
        count[b] = vals.size
        if vals.size >= 1:
            mean[b] = vals.mean()
        if vals.size >= 2:
            sd[b] = vals.std(ddof=1)
            if sd[b] > 0:
                out[sel] = (vals - mean[b]) / sd[b]
    return dict(score=out, count=count, mean=mean, sd=sd)
