"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and rejects malformed blobs and arguments without touching a GPU."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

import synth
from paper_2601_17554_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mlpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlpf_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_match_binding():
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.mlpf_abi_version() == 105


def load_status(lib, blob):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    st = lib.mlpf_load_weights(buf, len(blob), 0, ctypes.byref(h))
    assert not h.value or st == 0
    if h.value:
        lib.mlpf_free(h)
    return st, lib.mlpf_last_error().decode()


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(synth.SMALL, synth.make_weights(synth.SMALL, 0))


def test_rejects_bad_magic(lib, blob):
    st, msg = load_status(lib, b"XLPF" + blob[4:])
    assert st == _lib.MLPF_E_FORMAT and "magic" in msg


def test_rejects_bad_version(lib, blob):
    st, msg = load_status(lib, blob[:4] + struct.pack("<i", 7) + blob[8:])
    assert st == _lib.MLPF_E_FORMAT and "version" in msg


def test_rejects_truncated(lib, blob):
    for cut in (60, 1000, len(blob) - 4):
        st, msg = load_status(lib, blob[:cut])
        assert st == _lib.MLPF_E_FORMAT and "truncated" in msg, (cut, msg)


def test_rejects_trailing_bytes(lib, blob):
    st, msg = load_status(lib, blob + b"\0" * 8)
    assert st == _lib.MLPF_E_FORMAT


def test_rejects_bad_config(lib, blob):
    hdr = list(struct.unpack("<10i", blob[8:48]))
    hdr[2] = 5  # 64 / 5 heads
    st, _ = load_status(lib, blob[:8] + struct.pack("<10i", *hdr) + blob[48:])
    assert st == _lib.MLPF_E_FORMAT


def test_rejects_wrong_tensor_name(lib, blob):
    i = blob.index(b"emb.b1")
    st, msg = load_status(lib, blob[:i] + b"emb.b9" + blob[i + 6:])
    assert st == _lib.MLPF_E_FORMAT and "unexpected tensor" in msg


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.mlpf_load_weights(None, 100, 0, ctypes.byref(h)) == _lib.MLPF_E_INVALID
    assert lib.mlpf_load_weights(b"MLPF", 4, 0, ctypes.byref(h)) == _lib.MLPF_E_INVALID
    st = lib.mlpf_forward(None, 1, None, None, 1, 10, 10, None, None, None, None, None)
    assert st == _lib.MLPF_E_INVALID
    lib.mlpf_free(None)
    assert lib.mlpf_last_launch_count(None) == -1


def test_blob_round_trip_layout():
    """The blob header and tensor records follow the documented layout."""
    cfg = synth.SMALL
    w = synth.make_weights(cfg, 0, perturbed=True)
    b = synth.pack_blob(cfg, w)
    assert b[:4] == b"MLPF" and struct.unpack("<i", b[4:8])[0] == 1
    hdr = struct.unpack("<10i", b[8:48])
    assert hdr[:9] == (42, 64, 4, 256, 1, 1, 6, 5, 0)
    off = 48
    for name, shape, _ in synth.tensor_specs(cfg):
        nm = b[off:off + 48].rstrip(b"\0").decode()
        nd, s0, s1 = struct.unpack("<3i", b[off + 48:off + 60])
        assert nm == name and nd == len(shape)
        n = int(np.prod(shape))
        data = np.frombuffer(b[off + 60:off + 60 + 4 * n], np.float32)
        np.testing.assert_array_equal(data, w[name].ravel())
        off += 60 + 4 * n
    assert off == len(b)
