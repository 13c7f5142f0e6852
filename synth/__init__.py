"""Seeded synthetic inputs for the EHH / iHS / XPEHH scans.

This module only makes input data (packed haplotype rows, physical positions
and a genetic map); it holds none of the statistic's arithmetic.  Both the CPU
oracle tests and the GPU path draw their inputs from here.  The heavy lifting
is ``synth.c`` (a Li-Stephens mosaic generator with counter-based SplitMix64
draws), compiled on first use into ``libsynth.so`` next to this file.

Layout of the packed matrix (shared by every consumer): marker-major rows of
``ld`` uint64 words; haplotype h of a population whose words start at
``word_off`` is bit ``h % 64`` of word ``word_off + h // 64``; pad bits above
n in the last word are 0.  Allele 1 is derived, 0 ancestral (Section 1.1).

Named workloads (the shapes of the paper's data sets, Section 2):

* ``plain``  - 100 haplotypes x 2,000 SNPs on 2 Mb, 10 founders, 1 cM/Mb.
* ``chr22``  - 204 x 22,147 SNPs on 35 Mb (the CEU22 shape), 30 founders,
  1.2 cM/Mb +-50 % per 1 Mb segment, one planted 400 kb sweep at 17.5 Mb
  carried by 60 %, and eight planted gaps (20,000 / 20,001 / 45,000 /
  120,000 / 200,000 / 200,001 / 350,000 / 3,000,000 bp) that exercise the gap
  scaling and gap abort rules of Section 1.2.
* ``xpehh``  - pop A = the chr22 population, pop B = 210 haplotypes from 60
  independent founders without the sweep, same positions and map (the
  CEUYRI22 shape).
* ``ihs1m``  - 5,000 x 1,000,000 SNPs on 250 Mb, 200 founders, 20 planted
  sweeps (widths U(50, 500) kb, carrier frequency U(0.3, 0.9)).
* ``served_request(i)`` - one request of the served mix (70 % iHS / 30 %
  XPEHH, haplotypes and SNP counts log-uniform), seed 1000 + i.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

SWITCH_PER_CM = 5.0
FLIP_PROB = 1e-3


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Pop(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("founders", ctypes.c_int32),
                ("switch_per_cM", ctypes.c_double), ("flip_prob", ctypes.c_double),
                ("n_sweeps", ctypes.c_int32),
                ("sweep_center_bp", ctypes.POINTER(ctypes.c_double)),
                ("sweep_width_bp", ctypes.POINTER(ctypes.c_double)),
                ("sweep_freq", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_uniform.restype = ctypes.c_double
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_positions_map.restype = ctypes.c_int
        lib.synth_positions_map.argtypes = [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_haplotypes.restype = ctypes.c_int
        lib.synth_haplotypes.argtypes = [
            ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(_Pop), ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int64]
        _lib = lib
    return _lib


def uniform(seed: int, stream: int, index: int) -> float:
    """One counter-based uniform draw in [0, 1)."""
    return _load().synth_uniform(seed, stream, index)


def words(n: int) -> int:
    return (n + 63) // 64


@dataclass
class PopSpec:
    n: int
    founders: int
    sweeps: List[Tuple[float, float, float]] = field(default_factory=list)  # (centre bp, width bp, freq)
    switch_per_cM: float = SWITCH_PER_CM
    flip_prob: float = FLIP_PROB


@dataclass
class ScanSpec:
    """Everything needed to regenerate one scan's inputs bit for bit."""
    name: str
    mode: str                      # "ihs" or "xpehh"
    m: int
    len_bp: int
    seed: int
    pops: List[PopSpec]
    map_rate: float = 1.0          # cM / Mb
    map_spread: float = 0.0        # +- fraction per 1 Mb segment
    gaps: List[Tuple[int, int]] = field(default_factory=list)  # (marker index, exact step bp)

    @property
    def n(self) -> int:
        return self.pops[0].n

    @property
    def W(self) -> int:
        return sum(words(p.n) for p in self.pops)


@dataclass
class ScanData:
    spec: ScanSpec
    rows: np.ndarray               # uint64 [m, ld]
    pos: np.ndarray                # int64 [m]
    gmap: np.ndarray               # float64 [m]

    @property
    def ld(self) -> int:
        return self.rows.shape[1]


def positions_map(seed: int, m: int, len_bp: int, gaps=(), map_rate=1.0, map_spread=0.0):
    lib = _load()
    pos = np.empty(m, dtype=np.int64)
    gmap = np.empty(m, dtype=np.float64)
    gi = np.array([g[0] for g in gaps] or [0], dtype=np.int64)
    gb = np.array([g[1] for g in gaps] or [0], dtype=np.int64)
    rc = lib.synth_positions_map(seed, m, len_bp, len(gaps), gi.ctypes.data, gb.ctypes.data,
                                 float(map_rate), float(map_spread), pos.ctypes.data,
                                 gmap.ctypes.data)
    if rc != 0:
        raise ValueError("synth_positions_map: bad arguments")
    return pos, gmap


def generate(spec: ScanSpec, ld: Optional[int] = None) -> ScanData:
    """Generate packed rows (populations side by side, each word aligned)."""
    lib = _load()
    pos, gmap = positions_map(spec.seed, spec.m, spec.len_bp, spec.gaps, spec.map_rate,
                              spec.map_spread)
    W = spec.W
    ld = W if ld is None else ld
    if ld < W:
        raise ValueError("ld < W")
    rows = np.zeros((spec.m, ld), dtype=np.uint64)
    off = 0
    for k, p in enumerate(spec.pops):
        c = np.array([s[0] for s in p.sweeps] or [0.0], dtype=np.float64)
        w = np.array([s[1] for s in p.sweeps] or [0.0], dtype=np.float64)
        f = np.array([s[2] for s in p.sweeps] or [0.0], dtype=np.float64)
        pop = _Pop(p.n, p.founders, p.switch_per_cM, p.flip_prob, len(p.sweeps),
                   c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                   w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                   f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        rc = lib.synth_haplotypes(spec.seed, k, ctypes.byref(pop), spec.m, pos.ctypes.data,
                                  gmap.ctypes.data, rows.ctypes.data, ld, off)
        if rc != 0:
            raise ValueError("synth_haplotypes: bad arguments")
        off += words(p.n)
    return ScanData(spec, rows, pos, gmap)


def sweep_cores(data: "ScanData", pop: int = 0) -> np.ndarray:
    """Core marker of each planted sweep of population `pop`: the marker
    nearest to the sweep's centre (the first of two equally near), the rule
    synth.c plants the sweep's derived allele at."""
    pos = data.pos
    out = []
    for c, _, _ in data.spec.pops[pop].sweeps:
        k = int(np.searchsorted(pos, c, side="left"))
        k = min(k, pos.size - 1)
        if k > 0 and (c - pos[k - 1]) <= (pos[k] - c):
            k -= 1
        out.append(k)
    return np.array(out, dtype=np.int64)


# ---------------------------------------------------------------- workloads
CHR22_GAP_FRACTIONS = (0.05, 0.15, 0.30, 0.45, 0.60, 0.70, 0.80, 0.90)
CHR22_GAP_BP = (20_000, 20_001, 45_000, 120_000, 200_000, 200_001, 350_000, 3_000_000)


def _chr22_gaps(m: int):
    return [(int(f * m), b) for f, b in zip(CHR22_GAP_FRACTIONS, CHR22_GAP_BP)]


def spec(name: str, seed: int = 0) -> ScanSpec:
    if name == "plain":
        return ScanSpec("plain", "ihs", 2000, 2_000_000, seed, [PopSpec(100, 10)])
    if name == "chr22":
        m = 22147
        return ScanSpec("chr22", "ihs", m, 35_000_000, seed,
                        [PopSpec(204, 30, [(17_500_000.0, 400_000.0, 0.6)])],
                        map_rate=1.2, map_spread=0.5, gaps=_chr22_gaps(m))
    if name == "xpehh":
        m = 22147
        return ScanSpec("xpehh", "xpehh", m, 35_000_000, seed,
                        [PopSpec(204, 30, [(17_500_000.0, 400_000.0, 0.6)]), PopSpec(210, 60)],
                        map_rate=1.2, map_spread=0.5, gaps=_chr22_gaps(m))
    if name == "ihs200k":
        # a smaller analogue of ihs1m whose sweep centres the oracle checks in
        # full: 1,000 haplotypes x 200,000 SNPs on 50 Mb, 4 planted sweeps
        m, L, ns = 200_000, 50_000_000, 4
        sweeps = []
        for k in range(ns):
            width = 50_000.0 + 450_000.0 * uniform(seed, 1, k)
            freq = 0.3 + 0.6 * uniform(seed, 2, k)
            sweeps.append(((k + 0.5) / ns * L, width, freq))
        return ScanSpec(name, "ihs", m, L, seed, [PopSpec(1000, 200, sweeps)],
                        map_rate=1.2, map_spread=0.5)
    if name in ("ihs1m", "ihs250k"):
        # ihs250k: the same recipe on a quarter of the chromosome (5 sweeps), a
        # profiling-sized case whose matrix (158 MB) still exceeds L2
        m, L, ns = (1_000_000, 250_000_000, 20) if name == "ihs1m" else (250_000, 62_500_000, 5)
        sweeps = []
        for k in range(ns):
            width = 50_000.0 + 450_000.0 * uniform(seed, 1, k)
            freq = 0.3 + 0.6 * uniform(seed, 2, k)
            sweeps.append(((k + 0.5) / ns * L, width, freq))
        return ScanSpec(name, "ihs", m, L, seed, [PopSpec(5000, 200, sweeps)],
                        map_rate=1.2, map_spread=0.5)
    if name in ("xpehh1m", "xpehh200k"):
        # XPEHH at scale: A carries the 1M recipe's sweeps, B (other founders)
        # none; 2,500 + 2,500 haplotypes on 1M SNPs, or 1,000 + 1,000 on 200k
        m, L, ns, nA = ((1_000_000, 250_000_000, 20, 2500) if name == "xpehh1m"
                        else (200_000, 50_000_000, 4, 1000))
        sweeps = []
        for k in range(ns):
            width = 50_000.0 + 450_000.0 * uniform(seed, 1, k)
            freq = 0.3 + 0.6 * uniform(seed, 2, k)
            sweeps.append(((k + 0.5) / ns * L, width, freq))
        return ScanSpec(name, "xpehh", m, L, seed, [PopSpec(nA, 200, sweeps), PopSpec(nA, 150)],
                        map_rate=1.2, map_spread=0.5)
    if name in TABLE_SHAPES:
        # stand-ins for the paper's runtime-table data sets: its sample sizes and
        # SNP counts on a 4 Mbp neutral region (no sweep), 1 cM/Mb map
        mode, nA, nB, m = TABLE_SHAPES[name]
        pops = [PopSpec(nA, 100)] + ([PopSpec(nB, 100)] if mode == "xpehh" else [])
        return ScanSpec(name, mode, m, 4_000_000, seed, pops)
    raise KeyError(name)


def complexity_spec(n: int, snps_per_mb: int, len_bp: int = 20_000_000, seed: int = 0) -> ScanSpec:
    """Neutral iHS region for the complexity sweeps over sample size and SNP
    density: a 100-founder mosaic on ``len_bp`` with a 1 cM/Mb map.  The
    per-marker allele noise is scaled by 5,000 / density so that the noise per
    Mb, and with it the physical length of a walk, does not depend on the
    density (a walk then spans a number of markers proportional to it)."""
    m = int(round(snps_per_mb * len_bp / 1e6))
    pop = PopSpec(n, 100, flip_prob=FLIP_PROB * 5000.0 / snps_per_mb)
    return ScanSpec(f"cplx_n{n}_d{snps_per_mb}", "ihs", m, len_bp, seed, [pop])


# name: (mode, n or n_A, n_B, SNPs) of the data sets of the paper's runtime tables
TABLE_SHAPES = {
    "IHS250": ("ihs", 250, 0, 9_625), "IHS500": ("ihs", 500, 0, 10_646),
    "IHS1000": ("ihs", 1000, 0, 11_655), "IHS2000": ("ihs", 2000, 0, 12_724),
    "XP250": ("xpehh", 125, 125, 12_920), "XP500": ("xpehh", 250, 250, 14_989),
    "XP1000": ("xpehh", 500, 500, 17_142), "XP2000": ("xpehh", 1000, 1000, 19_567),
}


def _log_uniform(u: float, lo: float, hi: float) -> float:
    return math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def served_request(i: int, n_range=(100, 5000), m_range=(10_000, 500_000)) -> ScanSpec:
    """Request i of the served mix: 70 % iHS / 30 % XPEHH, seed 1000 + i."""
    seed = 1000 + i
    is_ihs = uniform(seed, 10, 0) < 0.7
    m = int(round(_log_uniform(uniform(seed, 11, 0), *m_range)))

    def pop(stream):
        n = int(round(_log_uniform(uniform(seed, stream, 0), *n_range)))
        return PopSpec(n, int(min(200, max(10, round(n / 25)))))

    pops = [pop(12)] if is_ihs else [pop(12), pop(13)]
    return ScanSpec(f"req{i}", "ihs" if is_ihs else "xpehh", m, 250 * m, seed, pops)


def tiny_random(n: int, m: int, seed: int, p1: float = 0.5, len_bp: Optional[int] = None,
                ld: Optional[int] = None):
    """Unstructured tiny case: iid alleles, positions 1 kb apart (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hap = (rng.random((m, n)) < p1).astype(np.uint8)
    pos = np.arange(1, m + 1, dtype=np.int64) * 1000
    gmap = pos.astype(np.float64) * 1e-6
    return hap, pos, gmap


def pack(hap01: np.ndarray, ld: Optional[int] = None) -> np.ndarray:
    """uint8 [m, n] (marker-major 0/1) -> packed uint64 [m, ld] (LSB first)."""
    m, n = hap01.shape
    W = words(n)
    ld = W if ld is None else ld
    padded = np.zeros((m, W * 64), dtype=np.uint8)
    padded[:, :n] = hap01 & 1
    bits = np.packbits(padded.reshape(m, W, 64), axis=2, bitorder="little")  # [m, W, 8]
    out = np.zeros((m, ld), dtype=np.uint64)
    out[:, :W] = bits.view(np.uint64).reshape(m, W)
    return out


def unpack(rows: np.ndarray, n: int, word_off: int = 0) -> np.ndarray:
    """packed uint64 [m, ld] -> uint8 [m, n]."""
    m = rows.shape[0]
    W = words(n)
    block = np.ascontiguousarray(rows[:, word_off:word_off + W])
    bits = np.unpackbits(block.view(np.uint8).reshape(m, W * 8), axis=1, bitorder="little")
    return bits[:, :n].astype(np.uint8)


def tiny_mosaic(n: int, m: int, seed: int, founders: int = 3, switch: float = 0.1,
                flip: float = 0.02, spacing_bp: int = 1000, dyadic_map: bool = True):
    """Small structured case (numpy PCG64): n haplotypes copying `founders`
    random founder sequences, jumping with probability `switch` between
    markers, alleles flipped with probability `flip`.  Long shared stretches
    make the walks run many steps.  With dyadic_map the map steps are
    integer multiples of 2^-12 cM, so every map difference is exact."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fnd = (rng.random((m, founders)) < 0.5).astype(np.uint8)
    cur = rng.integers(0, founders, size=n)
    hap = np.zeros((m, n), dtype=np.uint8)
    for k in range(m):
        jump = rng.random(n) < switch
        cur = np.where(jump, rng.integers(0, founders, size=n), cur)
        hap[k] = fnd[k, cur]
    hap ^= (rng.random((m, n)) < flip).astype(np.uint8)
    pos = np.cumsum(rng.integers(spacing_bp // 2, spacing_bp * 3 // 2 + 1, size=m)).astype(np.int64)
    if dyadic_map:
        gmap = np.cumsum(rng.integers(1, 64, size=m)).astype(np.float64) / 4096.0
    else:
        gmap = pos.astype(np.float64) * 1e-6
    return hap, pos, gmap
