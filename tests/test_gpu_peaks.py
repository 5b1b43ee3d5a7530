"""The integer-pipe and L2 microbenchmarks behind the enumeration's roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_int_peaks_are_plausible():
    import paper_2403_07858_gb300 as gbc
    gbc.build()
    pk = gbc.measure_int_peaks(0)
    # 152 SMs at about 2 GHz: between 1e11 and 1e14 words/s for the AND + POPC
    # + ADD loop, and an L2 stream between 1e11 and 1e14 bytes/s
    assert 1e11 < pk["and_popc_words_per_s"] < 1e14, pk
    assert 1e11 < pk["l2_bytes_per_s"] < 1e14, pk
