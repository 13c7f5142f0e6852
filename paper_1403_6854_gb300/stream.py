"""Scans of host-resident data sets, each upload overlapped with the scan before it.

A caller with many data sets in host memory (replicate simulations, several
chromosomes, one population pair after another) pays for three things per data
set: the upload of its packed matrix, positions and map, the scan, and the read
of its per-core results.  Run one call at a time, the copies add to every scan.
``scan_host_stream`` keeps two device copies of the inputs and of the outputs:
while scan k runs on the compute stream, data set k + 1 is uploaded on an upload
stream and the results of scan k - 1 are read back on a download stream, with
CUDA events as the only ordering between the three.  The scans themselves are
the library's ``selscan_ihs`` / ``selscan_xpehh`` calls on device buffers, so
every result equals that of the same call on device-resident inputs bit for bit.

iHS inputs may also be unpacked 0/1 bytes (haplotype-major [n, m] or
marker-major [m, n], only bit 0 of each byte counts): they are uploaded as
bytes and packed on the device (``selscan_pack``) on the upload stream, so
the upload and packing of data set k + 1 run beside scan k.

Host inputs should be in pinned memory (``tensor.pin_memory()``); pageable
memory works but its copies do not overlap.
"""
from __future__ import annotations

from typing import Dict, Iterable, Iterator, Optional, Sequence, Tuple

import torch

from . import (MODE_IHS, MODE_XPEHH, SelscanError, _ihs_outputs, _workspace, _xpehh_outputs,
               selscan_default_params, selscan_ihs, selscan_pack, selscan_workspace_bytes,
               selscan_xpehh)

LAYOUTS = ("rows", "hap_major", "marker_major")

IHS_FIELDS = ("status", "n1", "ihh1", "ihh0", "lnratio", "stop")
XPEHH_FIELDS = ("status", "n1", "ihhA", "ihhB", "lnratio", "stop")


def scan_host_stream(inputs: Iterable[Tuple[torch.Tensor, torch.Tensor, torch.Tensor]],
                     mode: int, n: int, nB: int = 0, max_m: int = 0, params=None, launch=None,
                     fields: Optional[Sequence[str]] = None,
                     workspace: Optional[torch.Tensor] = None,
                     layout: str = "rows") -> Iterator[Dict[str, torch.Tensor]]:
    """Scan each (rows [m, ld] 64-bit, pos [m] int64, gmap [m] float64) host triple in
    turn on the current CUDA device and yield its results in host tensors (the
    ``fields`` of the scan's output dict, trimmed to m entries), in input order.

    mode: MODE_IHS (n haplotypes) or MODE_XPEHH (n = nA, nB).  All inputs share n,
    nB and the row stride ld; their marker counts may differ up to ``max_m`` (default:
    the first input's).  The yielded tensors live in a pinned ring of two result
    sets: a result stays valid until the next one is requested (the read-back of
    the scan after next then reuses its memory), so copy it to keep it longer.
    ``workspace``: an optional device workspace (256-byte aligned), used by every
    scan of the stream and replaced by a larger one if an input needs more.  A
    device-side error (unsorted positions, a timed-out wait) raises SelscanError
    when the result of that scan is reached.  Closing the generator early waits
    for its copies in flight.

    layout: "rows" (the default: each input's first tensor is the packed matrix),
    or, for iHS, "hap_major" (uint8 [n, m]) / "marker_major" (uint8 [m, n]) 0/1
    bytes, packed on the device into rows of (n + 63) // 64 words.
    """
    if mode not in (MODE_IHS, MODE_XPEHH):
        raise ValueError("mode must be MODE_IHS or MODE_XPEHH")
    if mode == MODE_XPEHH and nB < 1:
        raise ValueError("XPEHH needs nB >= 1")
    if layout not in LAYOUTS:
        raise ValueError(f"layout must be one of {LAYOUTS}")
    if layout != "rows" and mode != MODE_IHS:
        raise ValueError("byte layouts are packed for iHS scans only")
    hap_major = layout == "hap_major"
    fields = tuple(fields) if fields is not None else (IHS_FIELDS if mode == MODE_IHS
                                                       else XPEHH_FIELDS)
    p = params if params is not None else selscan_default_params()
    it = iter(inputs)
    first = next(it, None)
    if first is None:
        return
    if layout == "rows":
        m0, ld = first[0].shape
    else:
        m0 = first[0].shape[1] if hap_major else first[0].shape[0]
        ld = (n + 63) // 64
    cap = max(int(max_m), int(m0))
    n_total = n + (nB if mode == MODE_XPEHH else 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    cs = torch.cuda.current_stream(dev)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    # two device input sets, two device output sets, two pinned result sets; all
    # allocated (on the compute stream) before any stream uses them, kept to the end
    d_in = [(torch.empty((cap, ld), dtype=torch.int64, device=dev),
             torch.empty(cap, dtype=torch.int64, device=dev),
             torch.empty(cap, dtype=torch.float64, device=dev)) for _ in range(2)]
    # byte layouts: the uploaded bytes of each slot, packed into its rows
    d_bytes = ([torch.empty(n * cap, dtype=torch.uint8, device=dev) for _ in range(2)]
               if layout != "rows" else None)
    mk = _ihs_outputs if mode == MODE_IHS else _xpehh_outputs
    d_out = [mk(cap, dev) for _ in range(2)]
    h_out = [{f: torch.empty(d_out[0][f].shape, dtype=d_out[0][f].dtype).pin_memory()
              for f in fields + ("error",)} for _ in range(2)]
    ws = workspace
    up_done = [torch.cuda.Event() for _ in range(2)]
    scan_done = [torch.cuda.Event() for _ in range(2)]
    read_done = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]                 # slot s holds a scan whose buffers may be in use

    def upload(slot: int, item) -> int:
        rows, pos, gmap = item
        if layout == "rows":
            m = rows.shape[0]
            if rows.dim() != 2 or rows.shape[1] != ld or rows.element_size() != 8:
                raise ValueError("every input's rows must be [m, ld] 64-bit with one ld")
        else:
            m = rows.shape[1] if hap_major else rows.shape[0]
            if (rows.dim() != 2 or rows.dtype != torch.uint8 or not rows.is_contiguous()
                    or rows.shape[0 if hap_major else 1] != n):
                raise ValueError("byte inputs must be contiguous uint8 [n, m] (hap_major) "
                                 "or [m, n] (marker_major)")
        if m > cap or pos.shape[0] != m or gmap.shape[0] != m:
            raise ValueError(f"marker count {m} above max_m {cap} or inconsistent arrays")
        if used[slot]:                    # the scan before last read this input set
            up.wait_event(scan_done[slot])
        with torch.cuda.stream(up):
            r, ps, g = d_in[slot]
            if layout == "rows":
                r[:m].copy_(rows.view(torch.int64), non_blocking=True)
            else:
                b = d_bytes[slot][:n * m].view(rows.shape)
                b.copy_(rows, non_blocking=True)
                selscan_pack(b, n, hap_major=hap_major, stream=up, out=r[:m])
            ps[:m].copy_(pos, non_blocking=True)
            g[:m].copy_(gmap, non_blocking=True)
        up_done[slot].record(up)
        return m

    try:
        k = 0
        m_cur = upload(0, first)
        pending = None                    # (slot, m) of the scan whose results are in flight
        item = first
        while item is not None:
            s = k & 1
            cs.wait_event(up_done[s])
            if used[s]:                   # its outputs were read back before reuse
                cs.wait_event(read_done[s])
            need = selscan_workspace_bytes(n_total, m_cur, mode, launch)
            if ws is None or ws.numel() < need:
                ws = _workspace(need, dev, None)
            r, ps, g = d_in[s]
            out = {f: t[:m_cur] for f, t in d_out[s].items() if f != "error"}
            out["error"] = d_out[s]["error"]
            if mode == MODE_IHS:
                selscan_ihs(r[:m_cur], n, ps[:m_cur], g[:m_cur], params=p, launch=launch,
                            stream=cs, workspace=ws, out=out)
            else:
                selscan_xpehh(r[:m_cur], n, nB, ps[:m_cur], g[:m_cur], params=p, launch=launch,
                              stream=cs, workspace=ws, out=out)
            scan_done[s].record(cs)
            used[s] = True
            nxt = next(it, None)
            m_next = upload(s ^ 1, nxt) if nxt is not None else 0
            # read this scan's results back behind it
            down.wait_event(scan_done[s])
            with torch.cuda.stream(down):
                for f in fields:
                    h_out[s][f][:m_cur].copy_(out[f], non_blocking=True)
                h_out[s]["error"].copy_(out["error"], non_blocking=True)
            read_done[s].record(down)
            if pending is not None:
                yield _finish(*pending, h_out, read_done, fields)
            pending = (s, m_cur)
            item, m_cur = nxt, m_next
            k += 1
        yield _finish(*pending, h_out, read_done, fields)
    finally:
        # no copy may still touch the buffers once they are released
        up.synchronize()
        down.synchronize()


def _finish(slot: int, m: int, h_out, read_done, fields) -> Dict[str, torch.Tensor]:
    read_done[slot].synchronize()
    e = int(h_out[slot]["error"][0])
    if e != 0:
        raise SelscanError(e, "device")
    return {f: h_out[slot][f][:m] for f in fields}
