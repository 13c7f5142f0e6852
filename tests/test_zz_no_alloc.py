"""selscan_ehh_noalloc: the allocation-free single-locus report.

Some callers cannot allocate device memory while they run (their memory
belongs to another framework's pool, or everything is reserved at start-up),
so this entry point takes no workspace and uses a fixed array inside the
library instead.  Its results must equal those of selscan_ehh, which uses a
caller workspace, on consecutive calls that find the previous call's
leftovers in the shared array, including calls whose sample size (and with
it the slices' size and offsets in the array) changes from one call to the
next.  A 5,000-haplotype locus is also checked against the CPU oracle.  This
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import IHH_RTOL, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


def call_noalloc_abi(sg, hap, n, pos, gmap, locus, cap):
    """Call selscan_ehh_noalloc directly through the C ABI (ctypes)."""
    lib = sg.load_library()
    dev = hap.device
    out = dict(S=torch.zeros((3, 2, cap), dtype=torch.int64, device=dev),
               len=torch.empty((3, 2), dtype=torch.int64, device=dev),
               stop=torch.empty((3, 2), dtype=torch.int32, device=dev),
               status=torch.empty((3, 2), dtype=torch.int8, device=dev),
               ihh=torch.empty((3, 2), dtype=torch.float64, device=dev),
               denom=torch.empty(3, dtype=torch.int64, device=dev),
               error=torch.zeros(1, dtype=torch.int32, device=dev))
    o = sg.selscan_ehh_out(*(ctypes.c_void_p(out[f].data_ptr())
                             for f in ("S", "len", "stop", "status", "ihh", "denom", "error")))
    p = sg.selscan_default_params()
    rc = lib.selscan_ehh_noalloc(ctypes.c_void_p(hap.data_ptr()), hap.shape[1], n, hap.shape[0],
                                 ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(gmap.data_ptr()),
                                 locus, ctypes.byref(p), ctypes.byref(o), cap,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, sg.selscan_strerror(rc)
    torch.cuda.synchronize()
    assert int(out["error"].item()) == 0
    return to_np(out)


def assert_same(a, b):
    for f in ("len", "stop", "status", "denom"):
        assert np.array_equal(a[f], b[f]), f
    for w in range(3):
        for d in range(2):
            k = min(int(a["len"][w, d]), a["S"].shape[2])
            assert np.array_equal(a["S"][w, d, :k], b["S"][w, d, :k])
    np.testing.assert_allclose(a["ihh"], b["ihh"], rtol=IHH_RTOL, atol=0)


def wide_data():
    """5,000 haplotypes on 3,000 markers: slices near the array's size."""
    spec = synth.ScanSpec("wide", "ihs", 3000, 750_000, 7, [synth.PopSpec(5000, 200)])
    return synth.generate(spec)


def test_noalloc_equals_workspace_entry_point_on_consecutive_calls(sg):
    """Calls in the order wide, small, wide, small, wide: each one equals a
    fresh selscan_ehh on the same locus, whatever the previous call left in
    the shared array."""
    cap = 2048
    wide = wide_data()
    small = synth.generate(synth.spec("chr22"))
    sets = []
    for d in (wide, small):
        hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
        sets.append((hap, d.spec.pops[0].n, pos, gmap))
    sequence = [(0, 1500), (1, 11_000), (0, 1517), (1, 11_090), (0, 1500)]
    for which, locus in sequence:
        hap, n, pos, gmap = sets[which]
        got = call_noalloc_abi(sg, hap, n, pos, gmap, locus, cap)
        ref = sg.selscan_ehh(hap, n, pos, gmap, locus, cap)
        sg.check(ref)
        assert_same(got, to_np(ref))


def test_noalloc_wide_locus_matches_the_oracle(sg):
    """The 5,000-haplotype case against the CPU oracle's literal string
    enumeration: every S(i) recorded, lengths, stops, status and iHH."""
    cap = 2048
    d = wide_data()
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
    for locus in (1500, 1517):
        got = call_noalloc_abi(sg, hap, 5000, pos, gmap, locus, cap)
        ref = oracle.ehh(d.rows, 5000, d.pos, d.gmap, locus, cap)
        assert_same(got, ref)


def test_noalloc_refuses_samples_above_its_limit(sg):
    lib = sg.load_library()
    fake = ctypes.c_void_p(0x1000)
    o = sg.selscan_ehh_out(*([fake] * 7))
    p = sg.selscan_default_params()
    n = sg.EHH_NOALLOC_MAX_N + 1
    rc = lib.selscan_ehh_noalloc(fake, (n + 63) // 64, n, 10, fake, fake, 0, ctypes.byref(p),
                                 ctypes.byref(o), 4, None)
    assert rc == sg.ERR_INVALID_ARG
