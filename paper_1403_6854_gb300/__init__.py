"""GB300-native EHH / iHS / XPEHH scans (selscan, arXiv:1403.6854).

Thin ctypes binding of ``libselscan_gb300.so`` (C ABI in include/selscan.h).
Every function here only marshals arguments: buffers are torch CUDA tensors
(PyTorch is the device allocator and supplies the stream), all arithmetic runs
in the library's sm_103a kernels.  There is no CPU fallback: if the library is
missing, importing the binding's functions raises.

Names follow the C ABI: ``selscan_ihs``, ``selscan_xpehh``, ``selscan_ehh``,
``selscan_pack``, ``selscan_workspace_bytes``, ``selscan_default_params``,
``selscan_strerror``.  The tensor-level helpers allocate outputs (and a
workspace, unless one is passed) and return them in a dict; calls are
asynchronous on the current (or given) stream; ``check(out)`` synchronises
and raises on a device-side error.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libselscan_gb300.so")

# return codes and per-locus status codes (include/selscan.h)
OK = 0
ERR_INVALID_ARG, ERR_UNSORTED, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
ERR_INTERNAL = -7
LOCUS_OK, LOCUS_MAF_FILTERED, LOCUS_UNDEFINED, LOCUS_ABORT_EDGE, LOCUS_ABORT_GAP = 0, 1, 2, 3, 4
MODE_IHS, MODE_XPEHH, MODE_EHH = 0, 1, 2
SCHED_DEFAULT, SCHED_LONGEST_FIRST, SCHED_IN_ORDER, SCHED_PLAIN, SCHED_SWEEP = -1, 0, 1, 2, 3

_P = ctypes.c_void_p


class selscan_params(ctypes.Structure):
    _fields_ = [("ehh_cut_num", ctypes.c_uint32), ("ehh_cut_den", ctypes.c_uint32),
                ("maf_num", ctypes.c_uint32), ("maf_den", ctypes.c_uint32),
                ("gap_scale_bp", ctypes.c_int64), ("max_gap_bp", ctypes.c_int64),
                ("include_crossing_term", ctypes.c_int32), ("xpehh_maf_filter", ctypes.c_int32),
                ("use_physical_map", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class selscan_launch(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("smem_entries", ctypes.c_int32),
                ("probe_steps", ctypes.c_int32), ("window_rows", ctypes.c_int32),
                ("cores_per_fetch", ctypes.c_int32), ("min_ctas_per_sm", ctypes.c_int32),
                ("walk_begin_event", ctypes.c_void_p), ("walk_end_event", ctypes.c_void_p),
                ("big_group_entries", ctypes.c_int32), ("sweep_warmup", ctypes.c_int32),
                ("sweep_stage_cores", ctypes.c_int32), ("sweep_threads", ctypes.c_int32),
                ("sweep_split_tile", ctypes.c_int32), ("sweep_ctas_per_sm", ctypes.c_int32),
                ("sweep_done_event", ctypes.c_void_p)]


class selscan_ihs_out(ctypes.Structure):
    _fields_ = [(f, _P) for f in ("status", "n1", "ihh1", "ihh0", "lnratio", "stop", "digest",
                                  "error")]


class selscan_xpehh_out(ctypes.Structure):
    _fields_ = [(f, _P) for f in ("status", "n1", "ihhA", "ihhB", "lnratio", "stop", "digest",
                                  "error")]


class selscan_ehh_out(ctypes.Structure):
    _fields_ = [(f, _P) for f in ("S", "len", "stop", "status", "ihh", "denom", "error")]


class selscan_scan(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("nA", ctypes.c_int32), ("nB", ctypes.c_int32),
                ("m", ctypes.c_int64), ("ld", ctypes.c_int64), ("hap", _P), ("pos_bp", _P),
                ("gmap", _P), ("params", selscan_params), ("status", _P), ("n1", _P),
                ("ihh_a", _P), ("ihh_b", _P), ("lnratio", _P), ("stop", _P), ("digest", _P),
                ("error", _P), ("items", _P)]


EXPORTS = ("selscan_default_params", "selscan_workspace_bytes", "selscan_ihs", "selscan_xpehh",
           "selscan_ihs_range", "selscan_xpehh_range", "selscan_normalize_bin_sums",
           "selscan_normalize_finish", "selscan_normalize_apply",
           "selscan_ehh", "selscan_ehh_noalloc", "selscan_pack", "selscan_strerror",
           "selscan_batch_item_bytes", "selscan_batch_workspace_bytes", "selscan_batch_prepare",
           "selscan_batch_run", "selscan_batch_finalize", "selscan_launch_count",
           "selscan_default_schedule", "selscan_sweep_work",
           "selscan_normalize", "selscan_normalize_workspace_bytes", "selscan_read_tped")
EHH_NOALLOC_MAX_N = 8192

_lib = None


def load_library():
    """Load the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    lib.selscan_default_params.restype = None
    lib.selscan_default_params.argtypes = [ctypes.POINTER(selscan_params)]
    lib.selscan_workspace_bytes.restype = ctypes.c_size_t
    lib.selscan_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.POINTER(selscan_launch)]
    lib.selscan_ihs.restype = ctypes.c_int
    lib.selscan_ihs.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                ctypes.POINTER(selscan_params), ctypes.POINTER(selscan_ihs_out),
                                _P, ctypes.c_size_t, ctypes.POINTER(selscan_launch), _P]
    lib.selscan_xpehh.restype = ctypes.c_int
    lib.selscan_xpehh.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int64, _P, _P, ctypes.POINTER(selscan_params),
                                  ctypes.POINTER(selscan_xpehh_out), _P, ctypes.c_size_t,
                                  ctypes.POINTER(selscan_launch), _P]
    lib.selscan_ihs_range.restype = ctypes.c_int
    lib.selscan_ihs_range.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int64, _P, _P,
                                      ctypes.POINTER(selscan_params),
                                      ctypes.POINTER(selscan_ihs_out), _P, ctypes.c_size_t,
                                      ctypes.POINTER(selscan_launch), _P]
    lib.selscan_xpehh_range.restype = ctypes.c_int
    lib.selscan_xpehh_range.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                        ctypes.POINTER(selscan_params),
                                        ctypes.POINTER(selscan_xpehh_out), _P, ctypes.c_size_t,
                                        ctypes.POINTER(selscan_launch), _P]
    lib.selscan_normalize_bin_sums.restype = ctypes.c_int
    lib.selscan_normalize_bin_sums.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                               ctypes.c_size_t, _P]
    lib.selscan_normalize_finish.restype = ctypes.c_int
    lib.selscan_normalize_finish.argtypes = [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P]
    lib.selscan_normalize_apply.restype = ctypes.c_int
    lib.selscan_normalize_apply.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, _P, _P, _P, _P, _P]
    lib.selscan_ehh.restype = ctypes.c_int
    lib.selscan_ehh.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                ctypes.c_int64, ctypes.POINTER(selscan_params),
                                ctypes.POINTER(selscan_ehh_out), ctypes.c_int64, _P,
                                ctypes.c_size_t, _P]
    lib.selscan_ehh_noalloc.restype = ctypes.c_int
    lib.selscan_ehh_noalloc.argtypes = [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P,
                                        _P, ctypes.c_int64, ctypes.POINTER(selscan_params),
                                        ctypes.POINTER(selscan_ehh_out), ctypes.c_int64, _P]
    lib.selscan_pack.restype = ctypes.c_int
    lib.selscan_pack.argtypes = [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P,
                                 ctypes.c_int64, _P]
    lib.selscan_batch_item_bytes.restype = ctypes.c_size_t
    lib.selscan_batch_item_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32]
    lib.selscan_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.selscan_batch_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                  ctypes.c_int32]
    lib.selscan_batch_prepare.restype = ctypes.c_int
    lib.selscan_batch_prepare.argtypes = [ctypes.POINTER(selscan_scan), _P]
    lib.selscan_batch_run.restype = ctypes.c_int
    lib.selscan_batch_run.argtypes = [ctypes.POINTER(selscan_scan), ctypes.c_int32, _P, _P, _P,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P,
                                      ctypes.c_size_t, _P]
    lib.selscan_read_tped.restype = ctypes.c_int
    lib.selscan_read_tped.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int64), _P, ctypes.c_int64, _P, _P,
                                      ctypes.POINTER(ctypes.c_int64)]
    lib.selscan_normalize_workspace_bytes.restype = ctypes.c_size_t
    lib.selscan_normalize_workspace_bytes.argtypes = [ctypes.c_int32]
    lib.selscan_normalize.restype = ctypes.c_int
    lib.selscan_normalize.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      _P, _P, _P, _P, _P, ctypes.c_size_t, _P]
    lib.selscan_launch_count.restype = ctypes.c_int32
    lib.selscan_launch_count.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P]
    lib.selscan_sweep_work.restype = ctypes.c_int
    lib.selscan_sweep_work.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.selscan_default_schedule.restype = ctypes.c_int32
    lib.selscan_default_schedule.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]
    lib.selscan_batch_finalize.restype = ctypes.c_int
    lib.selscan_batch_finalize.argtypes = [ctypes.POINTER(selscan_scan), _P]
    lib.selscan_strerror.restype = ctypes.c_char_p
    lib.selscan_strerror.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


class SelscanError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {selscan_strerror(code)} ({code})")


def selscan_strerror(code: int) -> str:
    return load_library().selscan_strerror(code).decode()


def selscan_default_params(**overrides) -> selscan_params:
    p = selscan_params()
    load_library().selscan_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "ehh_cut":
            p.ehh_cut_num, p.ehh_cut_den = int(v[0]), int(v[1])
        elif k == "maf":
            p.maf_num, p.maf_den = int(v[0]), int(v[1])
        else:
            setattr(p, k, int(v))
    return p


def make_launch(schedule: int = SCHED_DEFAULT, warps_per_cta: int = 0, ctas_per_sm: int = 0,
                smem_entries: int = 0, probe_steps: int = 0, window_rows: int = 0,
                cores_per_fetch: int = 0, min_ctas_per_sm: int = 0, big_group_entries: int = 0,
                sweep_warmup: int = 0, sweep_stage_cores: int = 0, sweep_threads: int = 0,
                sweep_split_tile: int = 0, sweep_ctas_per_sm: int = 0,
                events=None) -> selscan_launch:
    """events: optional (begin, end) torch.cuda.Event pair bracketing the walk kernels,
    or (begin, end, sort_done) with an event recorded after the first stage's sort."""
    L = selscan_launch(schedule, warps_per_cta, ctas_per_sm, smem_entries, probe_steps,
                       window_rows, cores_per_fetch, min_ctas_per_sm)
    L.big_group_entries = big_group_entries
    L.sweep_warmup = sweep_warmup
    L.sweep_stage_cores = sweep_stage_cores
    L.sweep_threads = sweep_threads
    L.sweep_split_tile = sweep_split_tile
    L.sweep_ctas_per_sm = sweep_ctas_per_sm
    if events is not None:
        L.walk_begin_event = ctypes.c_void_p(events[0].cuda_event)
        L.walk_end_event = ctypes.c_void_p(events[1].cuda_event)
        if len(events) > 2:
            L.sweep_done_event = ctypes.c_void_p(events[2].cuda_event)
    return L


def selscan_read_tped(path: str, ld: Optional[int] = None):
    """TPED file -> (packed rows uint64 [m, ld], positions int64 [m], map float64 [m], n)
    on the host, ready for to_device / selscan_ihs."""
    import numpy as np
    lib = load_library()
    n, m, bad = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.selscan_read_tped(path.encode(), ctypes.byref(n), ctypes.byref(m), None, 0, None,
                               None, ctypes.byref(bad))
    if rc != OK:
        raise SelscanError(rc, f"selscan_read_tped: {path}, marker line {bad.value}")
    ld = ld or (n.value + 63) // 64
    rows = np.zeros((m.value, ld), dtype=np.uint64)
    pos = np.zeros(m.value, dtype=np.int64)
    gmap = np.zeros(m.value, dtype=np.float64)
    rc = lib.selscan_read_tped(path.encode(), ctypes.byref(n), ctypes.byref(m), rows.ctypes.data, ld,
                               pos.ctypes.data, gmap.ctypes.data, ctypes.byref(bad))
    if rc != OK:
        raise SelscanError(rc, f"selscan_read_tped: {path}, marker line {bad.value}")
    return rows, pos, gmap, n.value


def selscan_normalize(score: torch.Tensor, status: torch.Tensor, n1: torch.Tensor, n: int,
                      nbins: int, stream=None) -> Dict[str, torch.Tensor]:
    """Standardised scores (Eq. 7 / Eq. 11) of lnratio/status/n1 device tensors
    (nbins = 1 for XPEHH's genome-wide normalisation)."""
    lib = load_library()
    m = score.numel()
    dev = score.device
    out = dict(score=torch.empty(m, dtype=torch.float64, device=dev),
               count=torch.empty(nbins, dtype=torch.int64, device=dev),
               mean=torch.empty(nbins, dtype=torch.float64, device=dev),
               sd=torch.empty(nbins, dtype=torch.float64, device=dev))
    nb = int(lib.selscan_normalize_workspace_bytes(nbins))
    if nb == 0:
        raise SelscanError(ERR_INVALID_ARG, "selscan_normalize_workspace_bytes")
    ws = _workspace(nb, dev, None)
    rc = lib.selscan_normalize(_ptr(score), _ptr(status), _ptr(n1), m, n, nbins, _ptr(out["score"]),
                               _ptr(out["count"]), _ptr(out["mean"]), _ptr(out["sd"]), _ptr(ws),
                               ws.numel(), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_normalize")
    out["_workspace"] = ws
    return out


def selscan_normalize_bin_sums(score: torch.Tensor, status: torch.Tensor, n1: torch.Tensor, n: int,
                               nbins: int, pass_: int, bin_mean: Optional[torch.Tensor] = None,
                               stream=None, workspace: Optional[torch.Tensor] = None):
    """One shard's per-bin sums: pass 0 -> (count int64 [nbins], sum of scores);
    pass 1 -> (None, sum of squared deviations about bin_mean)."""
    lib = load_library()
    dev = score.device
    cnt = torch.empty(nbins, dtype=torch.int64, device=dev) if pass_ == 0 else None
    sm = torch.empty(nbins, dtype=torch.float64, device=dev)
    ws = _workspace(int(lib.selscan_normalize_workspace_bytes(nbins)), dev, workspace)
    rc = lib.selscan_normalize_bin_sums(_ptr(score), _ptr(status), _ptr(n1), score.numel(), n, nbins,
                                        pass_, _ptr(bin_mean), _ptr(cnt), _ptr(sm), _ptr(ws),
                                        ws.numel(), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_normalize_bin_sums")
    return cnt, sm


def selscan_normalize_finish(nbins: int, pass_: int, bin_count: torch.Tensor, bin_sum: torch.Tensor,
                             stream=None) -> torch.Tensor:
    """Bin means (pass 0) or sample SDs (pass 1) from totals over all shards."""
    out = torch.empty(nbins, dtype=torch.float64, device=bin_sum.device)
    rc = load_library().selscan_normalize_finish(
        nbins, pass_, _ptr(bin_count), _ptr(bin_sum), _ptr(out) if pass_ == 0 else None,
        _ptr(out) if pass_ == 1 else None, _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_normalize_finish")
    return out


def selscan_normalize_apply(score: torch.Tensor, status: torch.Tensor, n1: torch.Tensor, n: int,
                            nbins: int, bin_count: torch.Tensor, bin_mean: torch.Tensor,
                            bin_sd: torch.Tensor, stream=None) -> torch.Tensor:
    """Standardised scores of one shard from the genome-wide bin statistics."""
    out = torch.empty(score.numel(), dtype=torch.float64, device=score.device)
    rc = load_library().selscan_normalize_apply(_ptr(score), _ptr(status), _ptr(n1), score.numel(),
                                                n, nbins, _ptr(bin_count), _ptr(bin_mean),
                                                _ptr(bin_sd), _ptr(out), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_normalize_apply")
    return out


def selscan_default_schedule(n_total: int, m: int, mode: int) -> int:
    """Schedule a default launch takes for this scan shape (-1: bad arguments)."""
    return int(load_library().selscan_default_schedule(n_total, m, mode))


def selscan_sweep_work(n_total: int, m: int, mode: int,
                       launch: Optional[selscan_launch] = None):
    """(marker passes, elements per pass) of the sorting kernels of a sweep
    call, or None if the launch does not take the sweep schedule."""
    mp, el = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = load_library().selscan_sweep_work(n_total, m, mode,
                                           ctypes.byref(launch) if launch is not None else None,
                                           ctypes.byref(mp), ctypes.byref(el))
    return None if rc != OK else (int(mp.value), int(el.value))


def selscan_launch_count(n_total: int, m: int, mode: int,
                         launch: Optional[selscan_launch] = None) -> int:
    """Kernel launches of one scan call with this launch shape."""
    return int(load_library().selscan_launch_count(
        n_total, m, mode, ctypes.byref(launch) if launch is not None else None))


def selscan_workspace_bytes(n_total: int, m: int, mode: int,
                            launch: Optional[selscan_launch] = None) -> int:
    lib = load_library()
    return int(lib.selscan_workspace_bytes(n_total, m, mode,
                                           ctypes.byref(launch) if launch is not None else None))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device, workspace: Optional[torch.Tensor]):
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes or workspace.data_ptr() % 256:
            raise SelscanError(ERR_WORKSPACE, "workspace")
        return workspace
    ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws[off:off + max(nbytes, 256)]


def _as_rows(hap: torch.Tensor) -> torch.Tensor:
    if hap.dim() != 2 or hap.element_size() != 8 or not hap.is_cuda or not hap.is_contiguous():
        raise ValueError("hap must be a contiguous 2-D 64-bit CUDA tensor [m, ld]")
    return hap


def _ihs_outputs(k: int, dev) -> Dict[str, torch.Tensor]:
    return dict(status=torch.empty(k, dtype=torch.int8, device=dev),
                n1=torch.empty(k, dtype=torch.int32, device=dev),
                ihh1=torch.empty(k, dtype=torch.float64, device=dev),
                ihh0=torch.empty(k, dtype=torch.float64, device=dev),
                lnratio=torch.empty(k, dtype=torch.float64, device=dev),
                stop=torch.empty((k, 4), dtype=torch.int32, device=dev),
                digest=torch.empty((k, 4), dtype=torch.int64, device=dev),
                error=torch.zeros(1, dtype=torch.int32, device=dev))


def _xpehh_outputs(k: int, dev) -> Dict[str, torch.Tensor]:
    return dict(status=torch.empty(k, dtype=torch.int8, device=dev),
                n1=torch.empty(k, dtype=torch.int32, device=dev),
                ihhA=torch.empty(k, dtype=torch.float64, device=dev),
                ihhB=torch.empty(k, dtype=torch.float64, device=dev),
                lnratio=torch.empty(k, dtype=torch.float64, device=dev),
                stop=torch.empty((k, 2), dtype=torch.int32, device=dev),
                digest=torch.empty((k, 6), dtype=torch.int64, device=dev),
                error=torch.zeros(1, dtype=torch.int32, device=dev))


def selscan_ihs(hap: torch.Tensor, n: int, pos: torch.Tensor, gmap: torch.Tensor,
                params: Optional[selscan_params] = None, launch: Optional[selscan_launch] = None,
                stream=None, workspace: Optional[torch.Tensor] = None,
                out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """iHS at every marker; returns device tensors (valid after stream sync)."""
    return selscan_ihs_range(hap, n, pos, gmap, 0, hap.shape[0], params, launch, stream,
                             workspace, out)


def selscan_ihs_range(hap: torch.Tensor, n: int, pos: torch.Tensor, gmap: torch.Tensor, k0: int,
                      k1: int, params: Optional[selscan_params] = None,
                      launch: Optional[selscan_launch] = None, stream=None,
                      workspace: Optional[torch.Tensor] = None,
                      out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """iHS at the cores [k0, k1) (outputs of k1 - k0 entries); the whole
    matrix is read by the walks."""
    lib = load_library()
    hap = _as_rows(hap)
    m, ld = hap.shape
    dev = hap.device
    if out is None:
        out = _ihs_outputs(max(k1 - k0, 0), dev)
    p = params if params is not None else selscan_default_params()
    ws = _workspace(selscan_workspace_bytes(n, max(k1 - k0, 1), MODE_IHS, launch), dev, workspace)
    o = selscan_ihs_out(*(_ptr(out[f]) for f in ("status", "n1", "ihh1", "ihh0", "lnratio",
                                                  "stop", "digest", "error")))
    rc = lib.selscan_ihs_range(_ptr(hap), ld, n, m, k0, k1, _ptr(pos), _ptr(gmap), ctypes.byref(p),
                               ctypes.byref(o), _ptr(ws), ws.numel(),
                               ctypes.byref(launch) if launch is not None else None,
                               _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_ihs_range" if (k0, k1) != (0, m) else "selscan_ihs")
    out["_workspace"] = ws
    return out


def selscan_xpehh(hap: torch.Tensor, nA: int, nB: int, pos: torch.Tensor, gmap: torch.Tensor,
                  params: Optional[selscan_params] = None,
                  launch: Optional[selscan_launch] = None, stream=None,
                  workspace: Optional[torch.Tensor] = None,
                  out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """XPEHH at every marker; rows hold W_A words of A then W_B words of B."""
    return selscan_xpehh_range(hap, nA, nB, pos, gmap, 0, hap.shape[0], params, launch, stream,
                               workspace, out)


def selscan_xpehh_range(hap: torch.Tensor, nA: int, nB: int, pos: torch.Tensor,
                        gmap: torch.Tensor, k0: int, k1: int,
                        params: Optional[selscan_params] = None,
                        launch: Optional[selscan_launch] = None, stream=None,
                        workspace: Optional[torch.Tensor] = None,
                        out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """XPEHH at the cores [k0, k1) (outputs of k1 - k0 entries)."""
    lib = load_library()
    hap = _as_rows(hap)
    m, ld = hap.shape
    dev = hap.device
    if out is None:
        out = _xpehh_outputs(max(k1 - k0, 0), dev)
    p = params if params is not None else selscan_default_params()
    ws = _workspace(selscan_workspace_bytes(nA + nB, max(k1 - k0, 1), MODE_XPEHH, launch), dev,
                    workspace)
    o = selscan_xpehh_out(*(_ptr(out[f]) for f in ("status", "n1", "ihhA", "ihhB", "lnratio",
                                                    "stop", "digest", "error")))
    rc = lib.selscan_xpehh_range(_ptr(hap), ld, nA, nB, m, k0, k1, _ptr(pos), _ptr(gmap),
                                 ctypes.byref(p), ctypes.byref(o), _ptr(ws), ws.numel(),
                                 ctypes.byref(launch) if launch is not None else None,
                                 _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_xpehh_range" if (k0, k1) != (0, m) else "selscan_xpehh")
    out["_workspace"] = ws
    return out


def selscan_ehh(hap: torch.Tensor, n: int, pos: torch.Tensor, gmap: torch.Tensor, locus: int,
                capacity: int, params: Optional[selscan_params] = None, stream=None,
                workspace: Optional[torch.Tensor] = None) -> Dict[str, torch.Tensor]:
    """S(i) of the six walks around one locus: [allele 1, allele 0, whole] x [down, up]."""
    lib = load_library()
    hap = _as_rows(hap)
    m, ld = hap.shape
    dev = hap.device
    out = dict(S=torch.zeros((3, 2, max(capacity, 0)), dtype=torch.int64, device=dev),
               len=torch.empty((3, 2), dtype=torch.int64, device=dev),
               stop=torch.empty((3, 2), dtype=torch.int32, device=dev),
               status=torch.empty((3, 2), dtype=torch.int8, device=dev),
               ihh=torch.empty((3, 2), dtype=torch.float64, device=dev),
               denom=torch.empty(3, dtype=torch.int64, device=dev),
               error=torch.zeros(1, dtype=torch.int32, device=dev))
    p = params if params is not None else selscan_default_params()
    ws = _workspace(selscan_workspace_bytes(n, m, MODE_EHH, None), dev, workspace)
    o = selscan_ehh_out(*(_ptr(out[f]) if out[f].numel() else None
                          for f in ("S", "len", "stop", "status", "ihh", "denom", "error")))
    rc = lib.selscan_ehh(_ptr(hap), ld, n, m, _ptr(pos), _ptr(gmap), locus, ctypes.byref(p),
                         ctypes.byref(o), capacity, _ptr(ws), ws.numel(), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_ehh")
    return out


def selscan_ehh_noalloc(hap: torch.Tensor, n: int, pos: torch.Tensor, gmap: torch.Tensor,
                        locus: int, capacity: int, params: Optional[selscan_params] = None,
                        stream=None) -> Dict[str, torch.Tensor]:
    """selscan_ehh without a workspace: the library's fixed device scratch is
    used instead (n <= EHH_NOALLOC_MAX_N; calls on one GPU must not overlap).
    The output tensors are still allocated here, by the caller's side."""
    lib = load_library()
    hap = _as_rows(hap)
    m, ld = hap.shape
    dev = hap.device
    out = dict(S=torch.zeros((3, 2, max(capacity, 0)), dtype=torch.int64, device=dev),
               len=torch.empty((3, 2), dtype=torch.int64, device=dev),
               stop=torch.empty((3, 2), dtype=torch.int32, device=dev),
               status=torch.empty((3, 2), dtype=torch.int8, device=dev),
               ihh=torch.empty((3, 2), dtype=torch.float64, device=dev),
               denom=torch.empty(3, dtype=torch.int64, device=dev),
               error=torch.zeros(1, dtype=torch.int32, device=dev))
    p = params if params is not None else selscan_default_params()
    o = selscan_ehh_out(*(_ptr(out[f]) if out[f].numel() else None
                          for f in ("S", "len", "stop", "status", "ihh", "denom", "error")))
    rc = lib.selscan_ehh_noalloc(_ptr(hap), ld, n, m, _ptr(pos), _ptr(gmap), locus,
                                 ctypes.byref(p), ctypes.byref(o), capacity, _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_ehh_noalloc")
    return out


def selscan_pack(hap01: torch.Tensor, n: int, hap_major: bool = False, ld: Optional[int] = None,
                 stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """uint8 0/1 matrix ([m, n], or [n, m] if hap_major) -> packed rows [m, ld] (int64 bits),
    written to ``out`` (a contiguous int64 [m, ld] CUDA tensor) if given."""
    lib = load_library()
    if hap01.dtype != torch.uint8 or not hap01.is_cuda or not hap01.is_contiguous():
        raise ValueError("hap01 must be a contiguous uint8 CUDA tensor")
    m = hap01.shape[1] if hap_major else hap01.shape[0]
    W = (n + 63) // 64
    ld = (W if out is None else out.shape[1]) if ld is None else ld
    if out is not None:
        if (out.dtype != torch.int64 or not out.is_cuda or not out.is_contiguous()
                or tuple(out.shape) != (m, ld)):
            raise ValueError("out must be a contiguous int64 CUDA tensor [m, ld]")
        rows = out
    else:
        rows = torch.empty((m, ld), dtype=torch.int64, device=hap01.device)
    rc = lib.selscan_pack(_ptr(hap01), n, m, 1 if hap_major else 0, _ptr(rows), ld, _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_pack")
    return rows


def selscan_batch_item_bytes(m: int, mode: int) -> int:
    return int(load_library().selscan_batch_item_bytes(m, mode))


def selscan_batch_workspace_bytes(max_n_total: int, max_ld: int, max_scans: int,
                                  max_units: int) -> int:
    return int(load_library().selscan_batch_workspace_bytes(max_n_total, max_ld, max_scans,
                                                            max_units))


def selscan_batch_prepare(scan: selscan_scan, stream=None) -> None:
    rc = load_library().selscan_batch_prepare(ctypes.byref(scan), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_batch_prepare")


def selscan_batch_run(scans, unit_scan, unit_c0, unit_c1, max_n_total: int, max_ld: int,
                      workspace: torch.Tensor, stream=None) -> None:
    """One tick over core ranges of several scans (host-side arrays)."""
    import numpy as np
    arr = (selscan_scan * len(scans))(*scans)
    us = np.ascontiguousarray(unit_scan, dtype=np.int32)
    c0 = np.ascontiguousarray(unit_c0, dtype=np.int64)
    c1 = np.ascontiguousarray(unit_c1, dtype=np.int64)
    rc = load_library().selscan_batch_run(arr, len(scans), us.ctypes.data, c0.ctypes.data,
                                          c1.ctypes.data, len(us), max_n_total, max_ld,
                                          _ptr(workspace), workspace.numel(), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_batch_run")


def selscan_batch_finalize(scan: selscan_scan, stream=None) -> None:
    rc = load_library().selscan_batch_finalize(ctypes.byref(scan), _stream(stream))
    if rc != OK:
        raise SelscanError(rc, "selscan_batch_finalize")


def check(out: Dict[str, torch.Tensor]) -> None:
    """Synchronise on the device error word and raise if a device check failed."""
    e = int(out["error"].item())
    if e != OK:
        raise SelscanError(e, "device")


def to_device(rows, pos, gmap, device="cuda"):
    """numpy packed rows / positions / map -> CUDA tensors of the ABI's types."""
    import numpy as np
    r = torch.from_numpy(np.ascontiguousarray(rows).view(np.int64)).to(device)
    p = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.int64)).to(device)
    g = torch.from_numpy(np.ascontiguousarray(gmap, dtype=np.float64)).to(device)
    return r, p, g
