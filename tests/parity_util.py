"""Shared helpers for the GPU-vs-oracle parity tests (test code only)."""
import numpy as np

# tolerances: integers bit-exact; iHH relative 1e-12; ln ratios absolute 1e-9
IHH_RTOL = 1e-12
LN_ATOL = 1e-9


def to_np(out):
    r = {}
    for k, v in out.items():
        if k.startswith("_") or k == "error":
            continue
        a = v.detach().cpu().numpy()
        if k in ("digest", "S", "denom"):
            a = a.view(np.uint64)
        r[k] = a
    return r


def assert_ihs_equal(got, ref, idx=None, fields=("ihh1", "ihh0")):
    sel = slice(None) if idx is None else idx
    g = {k: v[sel] for k, v in got.items()}
    bad = np.flatnonzero(g["status"] != ref["status"])
    assert bad.size == 0, f"status differs at {bad[:10]}: {g['status'][bad[:10]]} vs {ref['status'][bad[:10]]}"
    assert np.array_equal(g["n1"], ref["n1"]), "n1"
    bad = np.flatnonzero(np.any(g["stop"] != ref["stop"], axis=1))
    assert bad.size == 0, f"stop differs at {bad[:10]}: {g['stop'][bad[:3]]} vs {ref['stop'][bad[:3]]}"
    bad = np.flatnonzero(np.any(g["digest"] != ref["digest"], axis=1))
    assert bad.size == 0, f"digest differs at {bad[:10]}"
    for f in fields:
        np.testing.assert_allclose(g[f], ref[f], rtol=IHH_RTOL, atol=0, err_msg=f)
    assert np.array_equal(np.isnan(g["lnratio"]), np.isnan(ref["lnratio"])), "NaN pattern"
    ok = ~np.isnan(ref["lnratio"])
    np.testing.assert_allclose(g["lnratio"][ok], ref["lnratio"][ok], rtol=0, atol=LN_ATOL)


def assert_xpehh_equal(got, ref, idx=None):
    assert_ihs_equal(got, ref, idx, fields=("ihhA", "ihhB"))


def assert_bitwise_equal(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=a[k].dtype.kind == "f"), k
