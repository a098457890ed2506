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


def test_error_budget_tool_reads_blob_weights(tmp_path):
    """tests/lowp_budget.py --blob: a blob of the seeded precision-workload model gives the
    seeded weights back."""
    from tests import lowp_budget
    cfg, wseed, _, _ = synth.workload("prec64")
    w = synth.make_weights(cfg, wseed)
    path = tmp_path / "m.blob"
    path.write_bytes(synth.pack_blob(cfg, w))
    c1, w1 = lowp_budget._weights(str(path))
    c0, w0 = lowp_budget._weights("")
    assert c1 == c0 == cfg
    for k in w0:
        np.testing.assert_array_equal(np.asarray(w0[k], np.float32), w1[k])
