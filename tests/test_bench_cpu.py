"""Host-side arithmetic of bench.py (no GPU): the attention pair count behind the
roofline's algorithmic exponentials, full and windowed, against the oracle's
window mask counted element by element."""
import numpy as np

import bench
import oracle


def test_attention_pairs_full():
    sizes = np.array([1, 17, 300, 0, 2500])
    assert bench.attention_pairs(sizes, 0) == float((sizes.astype(np.int64) ** 2).sum())


def test_attention_pairs_windowed_match_mask():
    for w in (1, 2, 4):
        sizes = np.array([1, 127, 128, 129, 700, 1300])
        expect = sum(int(oracle.window_mask(int(n), w).sum()) for n in sizes)
        assert bench.attention_pairs(sizes, w) == expect
    # a window reaching every block is full attention
    assert bench.attention_pairs(np.array([700]), 6) == 700 ** 2
