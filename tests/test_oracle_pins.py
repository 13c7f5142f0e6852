"""Pins for the CPU oracle against facts the paper and the mathematics fix.

* hand-computed worked examples (Section 1.1 example, Eq. 1/3/4/5) stored in
  tests/golden/ with their derivations;
* brute-force pair counting: S(i) is the number of unordered haplotype pairs
  that agree on every marker x_0..x_i (a second definition of
  sum_h C(n_h, 2), independent of string enumeration);
* closed forms for the trapezoid (Eq. 4) and the Section 1.2 rules
  (truncation, gap scaling, gap abort, edge abort, MAF filter);
* invariants (EHH_c(x_0) = 1, S non-increasing, Eq. 2 decomposition
  S_whole = S_1 + S_0) and exact symmetries (marker reversal, haplotype
  permutation, allele relabelling, population swap, A = B).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def pack(h):
    return synth.pack(np.asarray(h, dtype=np.uint8))


# ------------------------------------------------------------- golden cases
def test_worked_example_ihs():
    g = load("worked_example_ihs.json")
    rows = pack(g["hap"])
    r = oracle.ihs(rows, 6, g["pos"], g["gmap"], cores=[g["core"]])
    e = g["expect_ihs"]
    assert r["status"][0] == e["status"]
    assert r["n1"][0] == e["n1"]
    assert r["stop"][0].tolist() == e["stop"]
    assert r["digest"][0].tolist() == e["digest"]
    assert r["ihh1"][0] == pytest.approx(e["ihh1"], rel=1e-14)
    assert r["ihh0"][0] == pytest.approx(e["ihh0"], rel=1e-14)
    assert r["lnratio"][0] == pytest.approx(e["lnratio"], abs=1e-14)


def test_worked_example_ehh_trace():
    g = load("worked_example_ihs.json")
    rows = pack(g["hap"])
    r = oracle.ehh(rows, 6, g["pos"], g["gmap"], g["core"], capacity=8)
    e = g["expect_ehh"]
    assert r["denom"].tolist() == e["denom"]
    for w, name in enumerate(("allele1", "allele0", "whole")):
        want = e["S"][name]
        for d in range(2):
            assert r["len"][w, d] == len(want)
            assert r["S"][w, d, :len(want)].tolist() == want
            assert r["stop"][w, d] == e["stop"][name]
            assert r["status"][w, d] == oracle.OK
            assert r["ihh"][w, d] == pytest.approx(e["ihh"][name], rel=1e-14)
    # the paper's sets at x_1: C(x_1) = {11,10,00,01}, H_1 = {11,10}, H_0 = {00,01}
    hap = np.array(g["hap"])
    c = g["core"]
    strings = {f"{hap[c, h]}{hap[c + 1, h]}" for h in range(6)}
    assert strings == {"11", "10", "00", "01"}
    assert {s for s in strings if s[0] == "1"} == {"11", "10"}
    assert {s for s in strings if s[0] == "0"} == {"00", "01"}


def test_worked_example_xpehh():
    g = load("worked_example_xpehh.json")
    nA, nB = g["nA"], g["nB"]
    hap = np.array(g["hap"], dtype=np.uint8)
    rows = np.concatenate([pack(hap[:, :nA]), pack(hap[:, nA:])], axis=1)
    r = oracle.xpehh(rows, nA, nB, g["pos"], g["gmap"], cores=[g["core"]])
    e = g["expect"]
    assert r["status"][0] == e["status"]
    assert r["n1"][0] == e["n1"]
    assert r["stop"][0].tolist() == e["stop"]
    assert r["digest"][0].tolist() == e["digest"]
    assert r["ihhA"][0] == pytest.approx(e["ihhA"], rel=1e-14)
    assert r["ihhB"][0] == pytest.approx(e["ihhB"], rel=1e-14)
    assert r["lnratio"][0] == pytest.approx(e["lnratio"], abs=1e-14)


# ------------------------------------------------------- brute-force pairs
def brute_S(hap, members, j, d, i):
    """Number of unordered pairs among `members` equal on x_0..x_i."""
    xs = [j + (d * 2 - 1) * k for k in range(i + 1)]
    sub = hap[np.ix_(xs, members)]
    cnt = 0
    for a in range(len(members)):
        for b in range(a + 1, len(members)):
            cnt += int(np.array_equal(sub[:, a], sub[:, b]))
    return cnt


@pytest.mark.parametrize("seed", range(6))
def test_trace_equals_brute_force_pairs(seed):
    n, m = 14, 16
    hap, pos, gmap = synth.tiny_mosaic(n, m, seed, founders=3, switch=0.08, flip=0.02)
    rows = pack(hap)
    cap = m + 2
    for j in range(m):
        r = oracle.ehh(rows, n, pos, gmap, j, capacity=cap)
        carriers = {0: [h for h in range(n) if hap[j, h] == 1],
                    1: [h for h in range(n) if hap[j, h] == 0],
                    2: list(range(n))}
        for w in range(3):
            N = len(carriers[w])
            D = N * (N - 1) // 2
            assert r["denom"][w] == D
            for d in range(2):
                L = r["len"][w, d]
                if D == 0:
                    assert r["status"][w, d] == oracle.UNDEFINED
                    continue
                edge = j if d == 0 else m - 1 - j
                for i in range(L):
                    assert r["S"][w, d, i] == brute_S(hap, carriers[w], j, d, i)
                # stop: first i >= 1 with 20 S < D (strict, cutoff 1/20), else edge
                first = next((i for i in range(1, edge + 1)
                              if 20 * brute_S(hap, carriers[w], j, d, i) < D), None)
                if first is None:
                    assert r["status"][w, d] == oracle.ABORT_EDGE
                    assert r["stop"][w, d] == edge + 1
                    assert L == edge + 1
                else:
                    assert r["status"][w, d] == oracle.OK
                    assert r["stop"][w, d] == first
                    assert L == first + 1


@pytest.mark.parametrize("seed", range(4))
def test_xpehh_pooled_stop_and_digest_brute_force(seed):
    nA, nB, m = 8, 7, 14
    hap, pos, gmap = synth.tiny_mosaic(nA + nB, m, 100 + seed, founders=2, switch=0.1, flip=0.02)
    rows = np.concatenate([pack(hap[:, :nA]), pack(hap[:, nA:])], axis=1)
    r = oracle.xpehh(rows, nA, nB, pos, gmap)
    A, B, P = list(range(nA)), list(range(nA, nA + nB)), list(range(nA + nB))
    DP = (nA + nB) * (nA + nB - 1) // 2
    for j in range(m):
        for d in range(2):
            edge = j if d == 0 else m - 1 - j
            first = next((i for i in range(1, edge + 1) if 20 * brute_S(hap, P, j, d, i) < DP),
                         None)
            last = edge if first is None else first
            dig = [0, 0, 0]
            for i in range(last + 1):
                for q, mem in enumerate((A, B, P)):
                    dig[q] = (dig[q] + (i + 1) * brute_S(hap, mem, j, d, i)) % (1 << 64)
            assert r["digest"][j, 3 * d:3 * d + 3].tolist() == dig
            assert r["stop"][j, d] == (edge + 1 if first is None else first)


# ------------------------------------------------------------ closed forms
DELTA = 1.0 / 128.0  # dyadic map step: every map difference and sum is exact


def line_case(k, m=None, n_other=3, gap_at=None, gap_bp=None, spacing=1000):
    """Two carriers of allele 1 at core 0 agree on markers 0..k-1 and differ
    at marker k; n_other carriers of allele 0 are all distinct at marker 1."""
    m = m or k + 2
    n = 2 + n_other
    hap = np.zeros((m, n), dtype=np.uint8)
    hap[0, :2] = 1
    hap[1:k, :2] = 1
    if k < m:
        hap[k, 0] = 1
        hap[k, 1] = 0
    pos = np.arange(m, dtype=np.int64) * spacing + 1
    if gap_at is not None:
        pos[gap_at:] += gap_bp - spacing
    gmap = np.arange(m, dtype=np.float64) * DELTA
    return hap, pos, gmap


@pytest.mark.parametrize("k", [1, 2, 3, 7, 12])
def test_identical_then_split_closed_form(k):
    hap, pos, gmap = line_case(k)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    # allele-1 walk upward: EHH_1 = 1 for i < k, 0 at i = k -> iHH = (k - 1) delta (c1)
    assert r["stop"][0, 1] == k and r["status"][0, 1] == oracle.OK
    assert r["ihh"][0, 1] == (k - 1) * DELTA
    assert r["S"][0, 1, :k + 1].tolist() == [1] * k + [0]
    # with the crossing term: + 1/2 (1 + 0) delta
    r2 = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64,
                    p=oracle.params(include_crossing_term=1))
    assert r2["ihh"][0, 1] == (k - 0.5) * DELTA
    assert r2["stop"][0, 1] == k
    # downward from marker 0: the array end is reached at once
    assert r["status"][0, 0] == oracle.ABORT_EDGE and r["stop"][0, 0] == 1
    assert r["ihh"][0, 0] == 0.0


def test_held_to_edge_closed_form():
    m = 9
    hap, pos, gmap = line_case(k=m, m=m)  # never split: EHH_1 = 1 to the end
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    assert r["status"][0, 1] == oracle.ABORT_EDGE
    assert r["stop"][0, 1] == m
    assert r["ihh"][0, 1] == (m - 1) * DELTA


@pytest.mark.parametrize("gap_bp,factor", [(20_000, 1.0), (20_001, 20_000 / 20_001),
                                           (40_000, 0.5), (200_000, 0.1)])
def test_gap_scaling(gap_bp, factor):
    k = 6
    hap, pos, gmap = line_case(k, gap_at=3, gap_bp=gap_bp)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    assert r["status"][0, 1] == oracle.OK
    want = (k - 2) * DELTA + DELTA * factor
    assert r["ihh"][0, 1] == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("gap_bp,aborts", [(200_000, False), (200_001, True)])
def test_gap_abort_boundary(gap_bp, aborts):
    k = 6
    hap, pos, gmap = line_case(k, gap_at=3, gap_bp=gap_bp)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    if aborts:
        assert r["status"][0, 1] == oracle.ABORT_GAP and r["stop"][0, 1] == 3
        assert r["ihh"][0, 1] == 2 * DELTA  # steps 1, 2 summed before the gap
    else:
        assert r["status"][0, 1] == oracle.OK and r["stop"][0, 1] == k


@pytest.mark.parametrize("k", [2, 7])
def test_physical_map_closed_form(k):
    """use_physical_map: g is the physical distance (position units); the map's
    values are ignored (a constant map here would give iHH = 0 otherwise)."""
    hap, pos, gmap = line_case(k, spacing=1000)
    flat = np.full_like(gmap, 5.0)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, flat, 0, capacity=64,
                   p=oracle.params(use_physical_map=1))
    assert r["status"][0, 1] == oracle.OK and r["stop"][0, 1] == k
    assert r["ihh"][0, 1] == (k - 1) * 1000.0


@pytest.mark.parametrize("gap_bp", [20_000, 20_001, 40_000, 150_000])
def test_physical_map_gap_scaling(gap_bp):
    """A step longer than the 20 kbp scale contributes g = b * 20000 / b, i.e.
    the scale itself; shorter steps contribute b."""
    k = 6
    hap, pos, gmap = line_case(k, gap_at=3, gap_bp=gap_bp)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64,
                   p=oracle.params(use_physical_map=1))
    assert r["status"][0, 1] == oracle.OK
    want = (k - 2) * 1000.0 + min(gap_bp, 20_000)
    assert r["ihh"][0, 1] == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("seed", [3, 4])
def test_physical_map_equals_map_of_positions(seed):
    """Physical mode equals genetic mode run with the positions as the map
    (both integrate the same doubles), whatever map is passed."""
    hap, pos, gmap = synth.tiny_mosaic(40, 90, seed, founders=3, switch=0.08, flip=0.02)
    rows = pack(hap)
    as_map = pos.astype(np.float64)
    gen = oracle.ihs(rows, 40, pos, as_map)
    phys = oracle.ihs(rows, 40, pos, gmap[::-1].copy(), p=oracle.params(use_physical_map=1))
    for f in ("status", "n1", "stop", "digest", "ihh1", "ihh0"):
        assert np.array_equal(gen[f], phys[f]), f
    ok = ~np.isnan(gen["lnratio"])
    assert np.array_equal(gen["lnratio"][ok], phys["lnratio"][ok])


def test_gap_after_stop_is_not_seen():
    k = 3
    hap, pos, gmap = line_case(k, m=8, gap_at=5, gap_bp=500_000)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    assert r["status"][0, 1] == oracle.OK and r["stop"][0, 1] == k


def test_gap_on_the_crossing_step_aborts():
    # the gap test comes before that step's EHH (reading c5)
    k = 4
    hap, pos, gmap = line_case(k, gap_at=k, gap_bp=300_000)
    r = oracle.ehh(pack(hap), hap.shape[1], pos, gmap, 0, capacity=64)
    assert r["status"][0, 1] == oracle.ABORT_GAP and r["stop"][0, 1] == k


@pytest.mark.parametrize("minor,reported", [(5, True), (4, False)])
def test_maf_boundary(minor, reported):
    n, m = 100, 5
    hap = np.zeros((m, n), dtype=np.uint8)
    hap[2, :minor] = 1
    pos = np.arange(m, dtype=np.int64) * 1000 + 1
    gmap = np.arange(m, dtype=np.float64) * DELTA
    r = oracle.ihs(pack(hap), n, pos, gmap, cores=[2])
    assert r["n1"][0] == minor
    if reported:
        assert r["status"][0] != oracle.MAF_FILTERED
    else:
        assert r["status"][0] == oracle.MAF_FILTERED and np.isnan(r["lnratio"][0])
        assert r["stop"][0].tolist() == [0, 0, 0, 0]


def xpehh_rows(hapA, hapB):
    return np.concatenate([pack(hapA), pack(hapB)], 1)


@pytest.mark.parametrize("derived_a,derived_b,filtered", [
    (5, 0, False),    # pooled minor 5 of 100: 5/100 >= 1/20, reported; B alone is monomorphic
    (2, 3, False),    # pooled minor 5: reported, though A alone (2/50 < 1/20) would be filtered
    (4, 0, True),     # pooled minor 4 of 100: filtered, though A alone (4/50) would pass
    (50, 46, True),   # pooled derived 96: minor 4, filtered (the minor allele is the ancestral one)
    (45, 50, False),  # pooled derived 95: minor 5, reported
])
def test_xpehh_maf_filter_tests_the_pooled_sample(derived_a, derived_b, filtered):
    """Reading c9: the paper states the MAF filter for iHS only (Section 1.2).
    With xpehh_maf_filter set, the oracle applies that rule to the pooled
    sample A + B at the core (minor count vs n_A + n_B), not to either
    population alone; without it every marker is reported.  n_A = n_B = 50,
    cutoff 1/20: a pooled minor count of 5 is reported and 4 is filtered,
    including cases where a per-population reading would decide the other
    way."""
    nA = nB = 50
    m = 6
    hA = np.zeros((m, nA), dtype=np.uint8)
    hB = np.zeros((m, nB), dtype=np.uint8)
    hA[3, :derived_a] = 1
    hB[3, :derived_b] = 1
    # the flanking markers split every pair, so walks end after one step
    rng = np.random.default_rng(derived_a * 100 + derived_b)
    for k in (0, 1, 2, 4, 5):
        hA[k] = rng.integers(0, 2, nA)
        hB[k] = rng.integers(0, 2, nB)
    pos = np.arange(m, dtype=np.int64) * 1000 + 1
    gmap = np.arange(m, dtype=np.float64) * DELTA
    rows = xpehh_rows(hA, hB)
    on = oracle.xpehh(rows, nA, nB, pos, gmap, cores=[3], p=oracle.params(xpehh_maf_filter=1))
    off = oracle.xpehh(rows, nA, nB, pos, gmap, cores=[3], p=oracle.params(xpehh_maf_filter=0))
    assert on["n1"][0] == off["n1"][0] == derived_a + derived_b
    assert off["status"][0] != oracle.MAF_FILTERED
    if filtered:
        assert on["status"][0] == oracle.MAF_FILTERED and np.isnan(on["lnratio"][0])
        assert on["stop"][0].tolist() == [0, 0] and on["digest"][0].tolist() == [0] * 6
    else:
        assert on["status"][0] == off["status"][0] != oracle.MAF_FILTERED
        assert on["stop"][0].tolist() == off["stop"][0].tolist()
        assert on["digest"][0].tolist() == off["digest"][0].tolist()
    # the filter also follows the cutoff parameter: at 1/10 a pooled minor count
    # of 5 is filtered
    tight = oracle.xpehh(rows, nA, nB, pos, gmap, cores=[3],
                         p=oracle.params(xpehh_maf_filter=1, maf=(1, 10)))
    assert tight["status"][0] == oracle.MAF_FILTERED


def test_ehh_exactly_at_cutoff_continues():
    # Reading c2 (strict "<"): 16 carriers walking down from core marker 4;
    # x_1 splits them 4 + 12, so S(1) = 6 + 66 = 72 and EHH_1(x_1) = 72/120,
    # exactly the cutoff 3/5 -> the walk continues; x_2 splits the 12 into
    # 6 + 6, S(2) = 6 + 15 + 15 = 36 < 72 -> stop at i = 2.
    n = 16
    hap = np.zeros((6, n), dtype=np.uint8)
    hap[4, :] = 1                               # core at marker 4
    hap[3, 4:] = 1                              # x_1
    hap[2, 4:10] = 1                            # x_2
    pos = np.arange(6, dtype=np.int64) * 1000 + 1
    gmap = np.arange(6, dtype=np.float64) * DELTA
    p = oracle.params(ehh_cut=(3, 5))
    r = oracle.ehh(pack(hap), n, pos, gmap, 4, capacity=16, p=p)
    S = r["S"][0, 0].tolist()
    assert S[:3] == [120, 72, 36]               # 72/120 = 3/5: equal, continue
    assert r["stop"][0, 0] == 2 and r["status"][0, 0] == oracle.OK
    # and with a cutoff a hair above 3/5 the walk stops at step 1
    r = oracle.ehh(pack(hap), n, pos, gmap, 4, capacity=16, p=oracle.params(ehh_cut=(601, 1000)))
    assert r["stop"][0, 0] == 1


def test_flat_map_gives_undefined():
    n, m = 10, 12
    hap, pos, _ = synth.tiny_mosaic(n, m, 3, founders=2, switch=0.05, flip=0.0)
    gmap = np.zeros(m)
    r = oracle.ihs(pack(hap), n, pos, gmap)
    walked = r["status"] != oracle.MAF_FILTERED
    assert np.all(r["ihh1"][walked] == 0.0) and np.all(r["ihh0"][walked] == 0.0)
    assert np.all(np.isin(r["status"][walked], [oracle.UNDEFINED, oracle.ABORT_EDGE,
                                                oracle.ABORT_GAP]))


def test_every_pair_split_at_x1_gives_undefined():
    # carriers of allele 1 all distinct after one step: only possible with 2
    # carriers, so: 2 carriers differing at x_1 in both directions
    n, m = 6, 5
    hap = np.zeros((m, n), dtype=np.uint8)
    hap[2, :2] = 1
    hap[1, 0] = 1
    hap[3, 0] = 1
    hap[1, 2:] = [0, 1, 0, 1]
    hap[3, 2:] = [0, 1, 1, 0]
    hap[0, 2:] = [0, 0, 1, 1]
    hap[4, 2:] = [1, 0, 1, 0]
    pos = np.arange(m, dtype=np.int64) * 1000 + 1
    gmap = np.arange(m, dtype=np.float64) * DELTA
    r = oracle.ihs(pack(hap), n, pos, gmap, cores=[2])
    assert r["stop"][0, :2].tolist() == [1, 1]
    assert r["ihh1"][0] == 0.0
    assert r["status"][0] == oracle.UNDEFINED and np.isnan(r["lnratio"][0])


def test_single_carrier_is_undefined():
    n, m = 6, 5
    hap = np.zeros((m, n), dtype=np.uint8)
    hap[2, 0] = 1
    pos = np.arange(m, dtype=np.int64) * 1000 + 1
    gmap = np.arange(m, dtype=np.float64) * DELTA
    r = oracle.ihs(pack(hap), n, pos, gmap, cores=[2], p=oracle.params(maf=(0, 1)))
    assert r["stop"][0, :2].tolist() == [0, 0]
    assert r["status"][0] >= oracle.UNDEFINED


# -------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(3))
def test_invariants(seed):
    n, m = 24, 40
    hap, pos, gmap = synth.tiny_mosaic(n, m, 50 + seed, founders=3, switch=0.05, flip=0.01)
    rows = pack(hap)
    for j in range(0, m, 3):
        r = oracle.ehh(rows, n, pos, gmap, j, capacity=m + 1)
        for w in range(3):
            D = int(r["denom"][w])
            for d in range(2):
                L = int(r["len"][w, d])
                if D == 0:
                    continue
                S = r["S"][w, d, :L].astype(np.int64)
                if w < 2:
                    assert S[0] == D           # EHH_c(x_0) = 1
                assert np.all(S <= D) and np.all(S >= 0)   # 0 <= EHH <= 1
                assert np.all(np.diff(S) <= 0)             # non-increasing
                assert r["ihh"][w, d] >= 0.0
                edge = j if d == 0 else m - 1 - j
                assert r["stop"][w, d] <= edge + 1
        # Eq. 2: C(x_i) is the union of H_1(x_i) and H_0(x_i)
        for d in range(2):
            L = int(min(r["len"][:, d]))
            if r["denom"][0] and r["denom"][1]:
                assert np.array_equal(r["S"][2, d, :L], r["S"][0, d, :L] + r["S"][1, d, :L])


# -------------------------------------------------------------- symmetries
def _ihs_all(hap, pos, gmap, **kw):
    return oracle.ihs(pack(hap), hap.shape[1], pos, gmap, p=oracle.params(maf=(0, 1)), **kw)


@pytest.mark.parametrize("seed", range(3))
def test_marker_reversal_swaps_directions(seed):
    n, m = 20, 30
    hap, pos, gmap = synth.tiny_mosaic(n, m, 200 + seed, founders=3, switch=0.06, flip=0.01)
    a = _ihs_all(hap, pos, gmap)
    rpos = (pos[-1] + 1 - pos)[::-1].copy()
    rgmap = (gmap[-1] - gmap)[::-1].copy()
    b = _ihs_all(hap[::-1].copy(), rpos, rgmap)
    for k in range(m):
        kk = m - 1 - k
        assert a["status"][k] == b["status"][kk]
        assert a["stop"][k].tolist() == b["stop"][kk][[1, 0, 3, 2]].tolist()
        assert a["digest"][k].tolist() == b["digest"][kk][[1, 0, 3, 2]].tolist()
        assert a["ihh1"][k] == b["ihh1"][kk] and a["ihh0"][k] == b["ihh0"][kk]


@pytest.mark.parametrize("seed", range(3))
def test_haplotype_permutation_invariance(seed):
    n, m = 20, 30
    hap, pos, gmap = synth.tiny_mosaic(n, m, 300 + seed, founders=3, switch=0.06, flip=0.01)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    a = _ihs_all(hap, pos, gmap)
    b = _ihs_all(hap[:, perm].copy(), pos, gmap)
    for f in ("status", "n1", "stop", "digest", "ihh1", "ihh0"):
        assert np.array_equal(a[f], b[f])
    assert np.array_equal(a["lnratio"], b["lnratio"], equal_nan=True)


@pytest.mark.parametrize("seed", range(3))
def test_allele_relabel_negates_ihs(seed):
    n, m = 20, 30
    hap, pos, gmap = synth.tiny_mosaic(n, m, 400 + seed, founders=3, switch=0.06, flip=0.01)
    a = _ihs_all(hap, pos, gmap)
    b = _ihs_all((1 - hap).astype(np.uint8), pos, gmap)
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["ihh1"], b["ihh0"]) and np.array_equal(a["ihh0"], b["ihh1"])
    assert np.array_equal(a["stop"], b["stop"][:, [2, 3, 0, 1]])
    ok = a["status"] == oracle.OK
    assert np.allclose(a["lnratio"][ok], -b["lnratio"][ok], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_population_swap_negates_xpehh(seed):
    nA, nB, m = 9, 13, 25
    hap, pos, gmap = synth.tiny_mosaic(nA + nB, m, 500 + seed, founders=3, switch=0.06, flip=0.01)
    A, B = pack(hap[:, :nA]), pack(hap[:, nA:])
    a = oracle.xpehh(np.concatenate([A, B], 1), nA, nB, pos, gmap)
    b = oracle.xpehh(np.concatenate([B, A], 1), nB, nA, pos, gmap)
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["ihhA"], b["ihhB"]) and np.array_equal(a["ihhB"], b["ihhA"])
    assert np.array_equal(a["stop"], b["stop"])
    ok = a["status"] == oracle.OK
    assert np.allclose(a["lnratio"][ok], -b["lnratio"][ok], rtol=0, atol=1e-15)


def test_identical_populations_give_zero_xpehh():
    n, m = 12, 25
    hap, pos, gmap = synth.tiny_mosaic(n, m, 600, founders=4, switch=0.25, flip=0.05)
    A = pack(hap)
    r = oracle.xpehh(np.concatenate([A, A], 1), n, n, pos, gmap)
    assert np.array_equal(r["ihhA"], r["ihhB"])
    ok = r["status"] == oracle.OK
    assert ok.any()
    assert np.all(r["lnratio"][ok] == 0.0)


def test_ihs_items_match_single_locus_trace():
    n, m = 18, 30
    hap, pos, gmap = synth.tiny_mosaic(n, m, 700, founders=3, switch=0.06, flip=0.01)
    rows = pack(hap)
    a = oracle.ihs(rows, n, pos, gmap, p=oracle.params(maf=(0, 1)))
    for j in range(m):
        r = oracle.ehh(rows, n, pos, gmap, j, capacity=m + 1)
        assert a["stop"][j].tolist() == [r["stop"][0, 0], r["stop"][0, 1], r["stop"][1, 0],
                                         r["stop"][1, 1]]
        assert a["ihh1"][j] == r["ihh"][0, 0] + r["ihh"][0, 1]
        assert a["ihh0"][j] == r["ihh"][1, 0] + r["ihh"][1, 1]


def test_cutoff_parameter_on_worked_example():
    # with cutoff 1/2 the allele-1 walk of the worked example stops at x_1
    # (EHH_1(x_1) = 1/3 < 1/2) and its sum is empty; allele 0 likewise
    g = load("worked_example_ihs.json")
    r = oracle.ihs(pack(g["hap"]), 6, g["pos"], g["gmap"], cores=[g["core"]],
                   p=oracle.params(ehh_cut=(1, 2)))
    assert r["stop"][0].tolist() == [1, 1, 1, 1]
    assert r["status"][0] == oracle.UNDEFINED
    r = oracle.ihs(pack(g["hap"]), 6, g["pos"], g["gmap"], cores=[g["core"]],
                   p=oracle.params(ehh_cut=(1, 2), include_crossing_term=1))
    # crossing term only: 1/2 (1 + 1/3) 0.01 per direction for both alleles
    assert r["ihh1"][0] == pytest.approx(2 * 0.5 * (4 / 3) * 0.01, rel=1e-14)
    assert r["lnratio"][0] == pytest.approx(0.0, abs=1e-15)


def test_bad_arguments_rejected():
    rows = pack(np.zeros((3, 4), dtype=np.uint8))
    pos = np.array([1, 2, 3])
    gmap = np.zeros(3)
    with pytest.raises(ValueError):
        oracle.ihs(rows, 1, pos, gmap)
    with pytest.raises(ValueError):
        oracle.ihs(rows, 4, pos, gmap, p=oracle.params(ehh_cut=(1, 0)))
    with pytest.raises(ValueError):
        oracle.xpehh(rows, 1, 4, pos, gmap)


# ------------------------------------------------------------ standardisation (Eq. 7, Eq. 11)
def test_normalize_two_scores_per_bin():
    """Two scores a < b in a bin: mean (a+b)/2, sample SD (b-a)/sqrt(2), so the
    standardised scores are -+1/sqrt(2) whatever a and b are."""
    n, nbins = 100, 10
    n1 = np.array([12, 17, 55, 58, 91, 99])          # bins 1, 1, 5, 5, 9, 9
    score = np.array([-3.0, 5.0, 0.25, 0.5, 7.0, -7.0])
    st = np.zeros(6, dtype=np.int8)
    r = oracle.normalize(score, st, n1, n, nbins)
    want = np.array([-1, 1, -1, 1, 1, -1]) / np.sqrt(2.0)
    np.testing.assert_allclose(r["score"], want, rtol=1e-15)
    assert r["count"].tolist() == [0, 2, 0, 0, 0, 2, 0, 0, 0, 2]


def test_normalize_bin_edges_and_undefined():
    n, nbins = 100, 10
    # 9/100 -> bin 0; 10/100 -> bin 1 (floor at the edge); 100/100 -> bin 9 (clamped)
    n1 = np.array([9, 10, 100, 100, 50, 50, 50, 30])
    st = np.array([0, 0, 0, 0, 0, 0, 2, 0], dtype=np.int8)      # one UNDEFINED marker
    score = np.array([1.0, 2.0, 3.0, 3.0, 1.0, 4.0, 9.0, 6.0])
    r = oracle.normalize(score, st, n1, n, nbins)
    assert r["count"].tolist() == [1, 1, 0, 1, 0, 2, 0, 0, 0, 2]
    assert np.isnan(r["score"][[0, 1, 7]]).all()        # singleton bins: no SD
    assert np.isnan(r["score"][[2, 3]]).all()           # constant bin: SD 0
    assert np.isnan(r["score"][6])                      # not OK
    np.testing.assert_allclose(r["score"][[4, 5]], [-1 / np.sqrt(2), 1 / np.sqrt(2)], rtol=1e-15)


@pytest.mark.parametrize("seed", [1, 2])
def test_normalize_invariants(seed):
    """Within every bin the standardised scores have mean 0 and sample SD 1,
    and a positive affine map of the raw scores leaves them unchanged."""
    rng = np.random.default_rng(seed)
    m, n = 5000, 700
    n1 = rng.integers(35, 666, size=m)
    st = np.where(rng.random(m) < 0.9, 0, 3).astype(np.int8)
    score = rng.normal(0.3, 1.7, size=m) + 0.01 * n1
    for nbins in (1, 7, 50):
        r = oracle.normalize(score, st, n1, n, nbins)
        bins = np.zeros(m, int) if nbins == 1 else np.minimum(nbins - 1, (n1 * nbins) // n)
        for b in range(nbins):
            v = r["score"][(st == 0) & (bins == b)]
            if v.size >= 2:
                assert abs(v.mean()) < 1e-12 and abs(v.std(ddof=1) - 1.0) < 1e-12
        r2 = oracle.normalize(2.5 * score - 11.0, st, n1, n, nbins)
        np.testing.assert_allclose(r2["score"], r["score"], rtol=0, atol=1e-12)
