"""Host side of the launch-shape table (no device work): import/export round
trip and rejection of shapes that cannot launch."""
import pytest

import paper_1407_3383_gb300 as G


def test_tune_table_round_trip():
    G.ntt_tune_import("8 20 0 3 1\n4 15 0 4 2\n")
    assert G.ntt_tune_get(8, 20) == (0, 3, 1)
    assert G.ntt_tune_get(4, 15) == (0, 4, 2)
    text = G.ntt_tune_export()
    assert "8 20 0 3 1" in text and "4 15 0 4 2" in text
    G.ntt_tune_reset()
    assert G.ntt_tune_export() == ""


def test_tune_rejects_bad_shapes():
    with pytest.raises(G.NttError):
        G.ntt_tune_import("4 16 0 9 3\n")     # 512 columns per block
    with pytest.raises(G.NttError):
        G.ntt_tune_import("5 16 0 4 3\n")     # no 5-byte words


def test_default_shapes():
    G.ntt_tune_reset()
    # one-block sizes: 16 products per block for short vectors, 8 / 4 / 2 for
    # tiles of 2^9 / 2^10 / 2^11 words (a block's column phase runs at least
    # 512 lines), 1 from 2^12 on
    assert G.ntt_tune_get(4, 8)[0] == 4
    for wb in (4, 8):
        assert [G.ntt_tune_get(wb, k)[0] for k in (9, 10, 11, 12, 13)] == [3, 2, 1, 0, 0]
    # the one-block limit is 2^13 for both word sizes: 2^14 takes the two
    # global passes (columns per block logw >= 1)
    assert G.ntt_tune_get(4, 14)[1] >= 1 and G.ntt_tune_get(8, 14)[1] >= 1
    # n = 2^16 .. 2^24 above the one-block limit: the direct kernels (logw = 0)
    for k in range(16, 25):
        assert G.ntt_tune_get(4, k)[1] == 0 and G.ntt_tune_get(8, k)[1] == 0
    assert G.ntt_tune_get(4, 15)[1] >= 1

