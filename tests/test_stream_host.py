"""Host-side argument checks of paper_1403_6854_gb300.stream (no GPU needed)."""
import pytest


def test_stream_argument_checks():
    import paper_1403_6854_gb300 as sg
    from paper_1403_6854_gb300.stream import scan_host_stream
    with pytest.raises(ValueError):
        next(scan_host_stream([], 7, 10))
    with pytest.raises(ValueError):
        next(scan_host_stream([], sg.MODE_XPEHH, 10, 0))
    assert list(scan_host_stream([], sg.MODE_IHS, 10)) == []


def test_stream_layout_checks():
    import paper_1403_6854_gb300 as sg
    from paper_1403_6854_gb300.stream import scan_host_stream
    with pytest.raises(ValueError):
        next(scan_host_stream([], sg.MODE_IHS, 10, layout="bits"))
    with pytest.raises(ValueError):
        next(scan_host_stream([], sg.MODE_XPEHH, 10, 12, layout="hap_major"))
