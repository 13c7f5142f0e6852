"""TPED reader (host code of the C ABI): synthetic matrices written as TPED
read back bit for bit; malformed files are refused with the marker line."""
import os

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


def write_tped(path, hap, pos, gmap, chrom="22"):
    with open(path, "w") as f:
        for k in range(hap.shape[0]):
            f.write(f"{chrom} rs{k} {float(gmap[k])!r} {int(pos[k])} " + " ".join(map(str, hap[k])) + "\n")


@pytest.mark.parametrize("n,m", [(1, 3), (64, 50), (65, 40), (203, 120)])
def test_round_trip(sg, tmp_path, n, m):
    hap, pos, gmap = synth.tiny_mosaic(n, m, n + m, founders=3, switch=0.1, flip=0.05)
    path = os.path.join(tmp_path, "x.tped")
    write_tped(path, hap, pos, gmap)
    rows, p, g, nn = sg.selscan_read_tped(path)
    assert nn == n
    assert np.array_equal(rows, synth.pack(hap))
    assert np.array_equal(p, pos) and np.array_equal(g, gmap)
    rows2, _, _, _ = sg.selscan_read_tped(path, ld=(n + 63) // 64 + 3)   # wider stride
    assert np.array_equal(rows2[:, :(n + 63) // 64], rows) and not rows2[:, (n + 63) // 64:].any()


def test_blank_lines_and_tabs(sg, tmp_path):
    path = os.path.join(tmp_path, "t.tped")
    with open(path, "w") as f:
        f.write("1\ta\t0.5\t100\t1\t0\t1\n\n1 b 0.75 250   0 0 1\r\n")
    rows, p, g, n = sg.selscan_read_tped(path)
    assert n == 3 and rows[:, 0].tolist() == [0b101, 0b100]
    assert p.tolist() == [100, 250] and g.tolist() == [0.5, 0.75]


@pytest.mark.parametrize("text,line", [("1 a 0.5 100 1 0 2\n", 1),            # allele 2
                                       ("1 a 0.5 100 1 0\n1 b 0.6 200 1\n", 2),   # width changes
                                       ("1 a x 100 1 0\n", 1),                   # bad map value
                                       ("1 a 0.5\n", 1),                         # no alleles
                                       ("", 0)])                                # empty file
def test_malformed(sg, tmp_path, text, line):
    path = os.path.join(tmp_path, "bad.tped")
    with open(path, "w") as f:
        f.write(text)
    with pytest.raises(sg.SelscanError) as e:
        sg.selscan_read_tped(path)
    assert f"marker line {line}" in str(e.value)


def test_missing_file(sg, tmp_path):
    with pytest.raises(sg.SelscanError):
        sg.selscan_read_tped(os.path.join(tmp_path, "none.tped"))
