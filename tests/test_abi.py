"""C ABI library: builds for sm_103a, loads, exports every declared symbol,
and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "selscan.h")


@pytest.fixture(scope="module")
def sg():
    from paper_1403_6854_gb300 import _build
    _build.build()
    import paper_1403_6854_gb300 as sg
    sg.load_library()
    return sg


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(selscan_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("selscan_ihs", "selscan_xpehh", "selscan_ehh", "selscan_pack",
              "selscan_workspace_bytes", "selscan_strerror", "selscan_default_params"):
        assert n in names


def test_library_exports_every_declared_symbol(sg):
    lib = sg.load_library()
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", sg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (selscan_\w+)", out))
    assert exported == set(declared())
    assert set(sg.EXPORTS) == set(declared())


def test_built_for_sm103a_only(sg):
    from paper_1403_6854_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_defaults(sg):
    assert sg.selscan_strerror(0) == "ok"
    assert "workspace" in sg.selscan_strerror(sg.ERR_WORKSPACE)
    assert sg.selscan_strerror(12345) == "unknown error code"
    p = sg.selscan_default_params()
    assert (p.ehh_cut_num, p.ehh_cut_den, p.maf_num, p.maf_den) == (1, 20, 1, 20)
    assert (p.gap_scale_bp, p.max_gap_bp, p.include_crossing_term) == (20000, 200000, 0)


def test_workspace_bytes(sg):
    a = sg.selscan_workspace_bytes(100, 2000, sg.MODE_IHS)
    b = sg.selscan_workspace_bytes(100, 4000, sg.MODE_IHS)
    c = sg.selscan_workspace_bytes(5000, 2000, sg.MODE_IHS)
    assert 0 < a < b and a < c
    assert sg.selscan_workspace_bytes(1, 10, sg.MODE_IHS) == 0
    assert sg.selscan_workspace_bytes(414, 100, sg.MODE_XPEHH) > 0
    assert sg.selscan_workspace_bytes(100, 100, sg.MODE_EHH) > 0


def test_host_side_argument_errors(sg):
    lib = sg.load_library()
    p = sg.selscan_default_params()
    o = sg.selscan_ihs_out()
    fake = ctypes.c_void_p(0x1000)
    # null pointers
    assert lib.selscan_ihs(None, 2, 100, 10, fake, fake, ctypes.byref(p), ctypes.byref(o), fake,
                           1 << 20, None, None) == sg.ERR_INVALID_ARG
    # n < 2 and ld < W, before any device work
    o2 = sg.selscan_ihs_out(*([fake] * 8))
    assert lib.selscan_ihs(fake, 2, 1, 10, fake, fake, ctypes.byref(p), ctypes.byref(o2), fake,
                           1 << 20, None, None) == sg.ERR_INVALID_ARG
    assert lib.selscan_ihs(fake, 1, 100, 10, fake, fake, ctypes.byref(p), ctypes.byref(o2), fake,
                           1 << 20, None, None) == sg.ERR_INVALID_ARG
    assert lib.selscan_ihs(fake, 2000, 70000, 10, fake, fake, ctypes.byref(p), ctypes.byref(o2),
                           fake, 1 << 30, None, None) == sg.ERR_INVALID_ARG
    # a zero denominator
    bad = sg.selscan_default_params(ehh_cut=(1, 0))
    assert lib.selscan_ihs(fake, 2, 100, 10, fake, fake, ctypes.byref(bad), ctypes.byref(o2), fake,
                           1 << 20, None, None) == sg.ERR_INVALID_ARG
    # workspace too small / misaligned
    assert lib.selscan_ihs(fake, 2, 100, 10, fake, fake, ctypes.byref(p), ctypes.byref(o2), fake,
                           16, None, None) == sg.ERR_WORKSPACE
    assert lib.selscan_ihs(fake, 2, 100, 10, fake, fake, ctypes.byref(p), ctypes.byref(o2),
                           ctypes.c_void_p(0x1008), 1 << 30, None, None) == sg.ERR_WORKSPACE
    ox = sg.selscan_xpehh_out(*([fake] * 8))
    assert lib.selscan_xpehh(fake, 2, 1, 5, 10, fake, fake, ctypes.byref(p), ctypes.byref(ox),
                             fake, 1 << 20, None, None) == sg.ERR_INVALID_ARG
    oe = sg.selscan_ehh_out(*([fake] * 7))
    assert lib.selscan_ehh(fake, 2, 100, 10, fake, fake, 10, ctypes.byref(p), ctypes.byref(oe), 4,
                           fake, 1 << 20, None) == sg.ERR_INVALID_ARG
    assert lib.selscan_pack(fake, 100, 10, 2, fake, 2, None) == sg.ERR_INVALID_ARG


def test_batch_limits(sg):
    """Tick limits of the batch ABI, rejected before any device work."""
    lib = sg.load_library()
    assert sg.selscan_batch_workspace_bytes(100, 2, 64, 256) > 0
    assert sg.selscan_batch_workspace_bytes(100, 2, 65, 1) == 0
    assert sg.selscan_batch_workspace_bytes(100, 2, 1, 257) == 0
    assert sg.selscan_batch_item_bytes(1000, sg.MODE_IHS) >= 1000 * 4 * 9
    assert sg.selscan_batch_item_bytes(0, sg.MODE_IHS) == 0
    scans = (sg.selscan_scan * 65)()
    us = (ctypes.c_int32 * 257)()
    c = (ctypes.c_int64 * 257)()
    fake = ctypes.c_void_p(0x1000)
    assert lib.selscan_batch_run(scans, 65, us, c, c, 1, 100, 2, fake, 1 << 30,
                                 None) == sg.ERR_INVALID_ARG
    assert lib.selscan_batch_run(scans, 1, us, c, c, 257, 100, 2, fake, 1 << 30,
                                 None) == sg.ERR_INVALID_ARG
    # a scan that fails its checks (all-zero struct) launches nothing
    assert lib.selscan_batch_prepare(scans, None) == sg.ERR_INVALID_ARG


def test_default_schedule_rule(sg):
    """A default launch sorts once m >= 32768 + 4 n (at most 16383 haplotypes);
    host-only, so it runs without a GPU."""
    I, X = sg.MODE_IHS, sg.MODE_XPEHH
    assert sg.selscan_default_schedule(5000, 52768, I) == sg.SCHED_SWEEP
    assert sg.selscan_default_schedule(5000, 52767, I) == sg.SCHED_IN_ORDER
    assert sg.selscan_default_schedule(100, 33168, I) == sg.SCHED_SWEEP
    assert sg.selscan_default_schedule(100, 33167, I) == sg.SCHED_IN_ORDER
    assert sg.selscan_default_schedule(204, 22147, I) == sg.SCHED_IN_ORDER      # chr22-shaped
    assert sg.selscan_default_schedule(414, 22147, X) == sg.SCHED_IN_ORDER
    assert sg.selscan_default_schedule(2500 + 2500, 1_000_000, X) == sg.SCHED_SWEEP
    assert sg.selscan_default_schedule(16383, 10_000_000, I) == sg.SCHED_SWEEP
    assert sg.selscan_default_schedule(16384, 10_000_000, I) == sg.SCHED_IN_ORDER
    for bad in ((1, 100000, I), (100, 0, I), (100, 100000, 7)):
        assert sg.selscan_default_schedule(*bad) == -1


def test_sweep_plan_shape_on_host(sg):
    """Host-side plan of the default launch (152 SMs when no GPU answers): the
    5,000 x 1M scan is one sweep stage (validate, select, sweep, split walk,
    bucket x3, second pass, finalize) with its slots under the 24 GiB budget;
    a chr22-shaped scan takes the per-step walk."""
    I = sg.MODE_IHS
    assert sg.selscan_launch_count(5000, 1_000_000, I) == 9
    assert sg.selscan_launch_count(204, 22147, I) == 4
    ws = sg.selscan_workspace_bytes(5000, 1_000_000, I)
    assert 20 << 30 < ws < 26 << 30
    # 64-core stages of chunks of about 4,400 cores (152 SMs: 228 chunks per
    # direction) take about 69 stages, two launches each
    k = sg.selscan_launch_count(5000, 1_000_000, I, sg.make_launch(sg.SCHED_SWEEP, sweep_stage_cores=64))
    assert (k - 7) % 2 == 0 and 60 <= (k - 7) // 2 <= 80


def test_single_locus_report_refuses_a_row_stride_beyond_shared_memory(sg):
    """Both single-locus entry points stage rows of ld words in each walk's
    marker window: a padded stride above about 1,040 words would exceed one
    CTA's shared memory, and both refuse it as unsupported before any device
    work (fake device pointers are never touched)."""
    lib = sg.load_library()
    p = sg.selscan_default_params()
    fake = ctypes.c_void_p(0x1000)
    oe = sg.selscan_ehh_out(*([fake] * 7))
    for ld, want in ((1100, sg.ERR_UNSUPPORTED), (4096, sg.ERR_UNSUPPORTED)):
        assert lib.selscan_ehh(fake, ld, 100, 10, fake, fake, 3, ctypes.byref(p), ctypes.byref(oe),
                               4, fake, 1 << 30, None) == want
        assert lib.selscan_ehh_noalloc(fake, ld, 100, 10, fake, fake, 3, ctypes.byref(p),
                                       ctypes.byref(oe), 4, None) == want
    # arguments are checked the same way by both
    bad = sg.selscan_default_params(ehh_cut=(1, 0))
    assert lib.selscan_ehh_noalloc(fake, 2, 100, 10, fake, fake, 3, ctypes.byref(bad),
                                   ctypes.byref(oe), 4, None) == sg.ERR_INVALID_ARG
    assert lib.selscan_ehh_noalloc(fake, 2, 100, 10, fake, fake, 10, ctypes.byref(p),
                                   ctypes.byref(oe), 4, None) == sg.ERR_INVALID_ARG


def test_peak_library_exports_its_header(sg):
    """The integer-peak measurement library exports exactly what
    include/selscan_peak.h declares and refuses bad arguments on the host."""
    from paper_1403_6854_gb300 import peak
    src = open(os.path.join(ROOT, "include", "selscan_peak.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(selscan_peak_[a-z_]+)\s*\(", src))
    out = subprocess.run(["nm", "-D", "--defined-only", peak.PEAK_LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    assert set(re.findall(r"\bT (selscan_\w+)", out)) == names == set(peak.EXPORTS)
    lib = peak.load_library()
    r = peak.selscan_peak_result()
    assert lib.selscan_peak_int(7, 10, ctypes.c_void_p(0x1000), 1 << 30, ctypes.byref(r)) == -1
    assert lib.selscan_peak_int(0, 0, ctypes.c_void_p(0x1000), 1 << 30, ctypes.byref(r)) == -1


def test_sweep_work_on_host(sg):
    """Host-only count of the sorting kernels' work: a chunk's passes are its
    cores plus its warm-up (clipped at the chromosome ends), both directions;
    None for a launch that does not sort."""
    I = sg.MODE_IHS
    passes, elements = sg.selscan_sweep_work(5000, 1_000_000, I)
    assert elements >= 5000 and elements % 64 == 0
    # 2 x (m markers) plus at most two warm-ups per chunk and direction
    assert 2_000_000 < passes < 2_000_000 + 2 * 228 * 1536 + 1
    L = sg.make_launch(sg.SCHED_SWEEP, sweep_warmup=1024)
    p2, _ = sg.selscan_sweep_work(5000, 1_000_000, I, L)
    assert p2 < passes
    # more sorting CTAs per SM: more chunks, each with its own warm-up
    p1, _ = sg.selscan_sweep_work(5000, 1_000_000, I, sg.make_launch(sg.SCHED_SWEEP, sweep_ctas_per_sm=1))
    p4, _ = sg.selscan_sweep_work(5000, 1_000_000, I, sg.make_launch(sg.SCHED_SWEEP, sweep_ctas_per_sm=4))
    assert p1 < passes < p4
    assert sg.selscan_sweep_work(204, 22147, I) is None          # per-step default
    assert sg.selscan_sweep_work(204, 22147, I, sg.make_launch(sg.SCHED_SWEEP)) is not None
