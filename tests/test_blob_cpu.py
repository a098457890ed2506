"""The weight-blob reader (synth.unpack_blob) against the writer (synth.pack_blob)."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("cfg,seed", [(synth.SMALL, 0), (synth.PAPER, 4), (synth.FULL, 1)])
def test_unpack_inverts_pack(cfg, seed):
    w = synth.make_weights(cfg, seed, perturbed=True)
    blob = synth.pack_blob(cfg, w)
    c2, w2 = synth.unpack_blob(blob)
    assert c2 == cfg
    assert set(w2) == set(w)
    for k in w:
        np.testing.assert_array_equal(np.asarray(w[k], np.float32), w2[k])
    assert synth.pack_blob(c2, w2) == blob


def test_unpack_rejects_bad_blobs():
    blob = synth.pack_blob(synth.SMALL, synth.make_weights(synth.SMALL, 0))
    with pytest.raises(ValueError):
        synth.unpack_blob(b"XXXX" + blob[4:])
    with pytest.raises(ValueError):
        synth.unpack_blob(blob + b"\0\0\0\0")
