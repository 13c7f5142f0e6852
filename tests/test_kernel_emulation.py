"""The sorting kernel and the split walk, compiled for the host and run there
(tests/emu: one OS thread per CUDA thread, shuffles and barriers emulated),
against the oracle: every walk that stays inside its chunk's history has the
oracle's stop index and S digest (the exact sequence of S(i), Eq. 3-5 and the
Section 1.2 rules), and iHH to rounding.  No GPU needed: this checks the
kernels' logic (sort order, run lengths, first windows, split terms, step
rules) on the CPU suite, for iHS and XPEHH, narrow and 256-thread sorts,
several stages and hand-offs past the history."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (mode, nA, nB, m, threads, warm-up, stage cores)
SHAPES = [("ihs", 100, 0, 600, 32, 160, 64),
          ("ihs", 300, 0, 500, 64, 200, 100),
          ("xpehh", 120, 80, 450, 64, 150, 70),
          ("ihs", 700, 0, 260, 256, 100, 60)]


@pytest.fixture(scope="module")
def runner(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    import importlib.util
    spec = importlib.util.spec_from_file_location("emu_extract", os.path.join(HERE, "emu", "extract.py"))
    ex = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ex)
    d = tmp_path_factory.mktemp("emu")
    ex.build(str(d / "kernels_host.h"))
    exe = str(d / "run_scan")
    cmd = [gxx, "-std=c++17", "-O2", "-pthread", "-I", os.path.join(HERE, "emu"),
           "-I", os.path.join(ROOT, "include"), "-I", str(d), os.path.join(HERE, "emu", "run_scan.cpp"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


@pytest.mark.timeout(600)
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_kernels_on_host_match_oracle(runner, shape):
    exe, d = runner
    mode, nA, nB, m, T, L, R = SHAPES[shape]
    n = nA + nB
    pops = [synth.PopSpec(nA, 12)] + ([synth.PopSpec(nB, 15)] if mode == "xpehh" else [])
    data = synth.generate(synth.ScanSpec(f"emu{shape}", mode, m, 250 * m, 900 + shape, pops))
    W = data.rows.shape[1]
    WA = (nA + 63) // 64
    if mode == "ihs":
        n1 = synth.unpack(data.rows, nA).sum(1)
        status = np.where(20 * np.minimum(n1, n - n1) < n, 1, 0).astype(np.int8)   # MAF below 1/20
    else:
        status = np.zeros(m, np.int8)
    files = {}
    for k, arr in (("rows", data.rows.astype(np.uint64)), ("st", status),
                   ("pos", data.pos.astype(np.int64)), ("gm", data.gmap.astype(np.float64))):
        files[k] = str(d / f"{shape}_{k}.bin")
        arr.tofile(files[k])
    per = max(L, 256)
    nch = max(1, (m + per - 1) // per)
    B = (m + nch - 1) // nch
    out = str(d / f"{shape}_out.bin")
    args = [exe, str(n), str(nA), str(nB), str(W), str(WA), str(m), str(L), str(R), str(T), str(nch),
            str(B), files["rows"], files["st"], files["pos"], files["gm"], out]
    r = subprocess.run(args, capture_output=True, text=True, timeout=500)
    assert r.returncode == 0, r.stdout[-500:] + r.stderr[-2000:]
    ipc = 2 if nB else 4
    items = m * ipc
    raw = open(out, "rb").read()
    istat = np.frombuffer(raw, np.int8, items, 0).reshape(m, ipc)
    stop = np.frombuffer(raw, np.int32, items, items).reshape(m, ipc)
    ihh = np.frombuffer(raw, np.float64, items * 2, 5 * items)
    dig = np.frombuffer(raw, np.uint64, items * 3, 21 * items)
    if nB:
        ref = oracle.xpehh(data.rows, nA, nB, data.pos, data.gmap)
        dig = dig.reshape(m, 2, 3)
        rdig = ref["digest"].reshape(m, 2, 3)
    else:
        ref = oracle.ihs(data.rows, nA, data.pos, data.gmap)
        dig = dig[:items].reshape(m, 4)
        rdig = ref["digest"].reshape(m, 4)
    walked = istat != 0x7F                 # walks handed past the history are not written
    assert walked.sum() > items // 4
    np.testing.assert_array_equal(stop[walked], ref["stop"].reshape(m, ipc)[walked])
    np.testing.assert_array_equal(dig[walked], rdig[walked])
    if not nB:
        # iHH_1 of a core = its allele-1 walks down and up, where both were walked here
        ih = ihh[:items].reshape(m, 4)
        both = walked[:, 0] & walked[:, 1] & (ref["status"] == 0)
        np.testing.assert_allclose(ih[both, 0] + ih[both, 1], ref["ihh1"][both], rtol=1e-12, atol=0)
