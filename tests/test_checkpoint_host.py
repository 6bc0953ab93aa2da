"""Checkpoint files on the host (no GPU): round trip, integrity check, errors.

The file's trailer is checked against zlib.crc32 over header and payload (an
independent implementation of the same IEEE 802.3 CRC-32).
"""
import os
import struct
import zlib

import numpy as np
import pytest

H = pytest.importorskip("paper_2601_20550_gb300.heom")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


def test_round_trip_and_crc(tmp_path):
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, 7, 5)) + 1j * rng.standard_normal((3, 7, 5))
    p = str(tmp_path / "a.ckpt")
    H.heom_ckpt_write(p, a)
    assert not os.path.exists(p + ".tmp")
    assert H.heom_ckpt_verify(p) == a.nbytes
    b = H.heom_ckpt_read(p, np.zeros_like(a))
    assert np.array_equal(a, b)
    raw = open(p, "rb").read()
    assert raw[:8] == b"HEOMCKPT"
    assert struct.unpack("<Q", raw[16:24])[0] == a.nbytes
    assert struct.unpack("<I", raw[-4:])[0] == zlib.crc32(raw[:-4])
    assert raw[88:-4] == a.tobytes()
    # an empty payload is a valid checkpoint
    H.heom_ckpt_write(p, np.zeros(0))
    assert H.heom_ckpt_verify(p) == 0


@pytest.mark.parametrize("damage", ["flip_payload", "flip_header", "truncate", "magic", "missing"])
def test_damaged_file_is_rejected_and_buffer_kept(tmp_path, damage):
    a = np.arange(1000, dtype=np.float64)
    p = str(tmp_path / "a.ckpt")
    H.heom_ckpt_write(p, a)
    raw = bytearray(open(p, "rb").read())
    if damage == "flip_payload":
        raw[88 + 4000] ^= 0x10
    elif damage == "flip_header":
        raw[40] ^= 0x01          # inside the tag
    elif damage == "truncate":
        raw = raw[:-100]
    elif damage == "magic":
        raw[0:8] = b"NOTACKPT"
    if damage == "missing":
        os.remove(p)
    else:
        open(p, "wb").write(bytes(raw))
    out = np.full(1000, -7.0)
    with pytest.raises(H.HeomError) as ei:
        H.heom_ckpt_read(p, out)
    assert ei.value.status == -8, str(ei.value)
    assert np.all(out == -7.0)
    with pytest.raises(H.HeomError) as ei:
        H.heom_ckpt_verify(p)
    assert ei.value.status == -8


def test_size_mismatch_is_an_argument_error(tmp_path):
    p = str(tmp_path / "a.ckpt")
    H.heom_ckpt_write(p, np.zeros(10))
    with pytest.raises(H.HeomError) as ei:
        H.heom_ckpt_read(p, np.zeros(11))
    assert ei.value.status == -1
