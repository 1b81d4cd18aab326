"""Index files on the host (no GPU): the library's CRC-32 against zlib's, and the
loader's header checks, which run before any device call (a missing, foreign,
truncated or corrupted header is rejected with PEOS_E_INVAL)."""
import os
import struct
import zlib

import numpy as np
import pytest

HEADER = struct.Struct("<8sIIqiiiiiQQiiI")
ENTRY = struct.Struct("<IIQ")


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


def test_crc32_matches_zlib(P):
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 64, 1000, 1 << 17):
        data = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert P.crc32(data) == zlib.crc32(data), n
    assert P.crc32(b"123456789") == 0xCBF43926  # the check value of CRC-32/ISO-HDLC


def _header(nsec=2, kind=0, n=10, R=4, L=2, m=16, d=8, entry=0, rec=128, node=48, sbits=32):
    return HEADER.pack(b"PEOSIDX1", 4, kind, n, R, L, m, d, entry, 7, rec, node, sbits, nsec)


def _file(path, head, table, crc=None):
    body = head + b"".join(ENTRY.pack(*t) for t in table)
    c = zlib.crc32(body) if crc is None else crc
    with open(path, "wb") as f:
        f.write(body + struct.pack("<I", c))
    return str(path)


def test_header_rejections(P, tmp_path):
    with pytest.raises(P.PeosError, match="cannot open"):
        P.load_codes(str(tmp_path / "missing.idx"))
    p = tmp_path / "short.idx"
    p.write_bytes(b"PEOSIDX1\x01\x00")
    with pytest.raises(P.PeosError, match="truncated header"):
        P.load_codes(str(p))
    p = tmp_path / "foreign.idx"
    p.write_bytes(b"NOTANIDX" + bytes(200))
    with pytest.raises(P.PeosError, match="not a PEOs index"):
        P.load_codes(str(p))
    table = [(1, 0, 960), (2, 0, 1920)]
    good = _header()
    with pytest.raises(P.PeosError, match="header checksum"):
        P.load_codes(_file(tmp_path / "crc.idx", good, table, crc=12345))
    with pytest.raises(P.PeosError, match="truncated section table"):
        P.load_codes(_file(tmp_path / "tab.idx", _header(nsec=5), table))
    with pytest.raises(P.PeosError, match="unsupported version"):
        P.load_codes(_file(tmp_path / "ver.idx", HEADER.pack(b"PEOSIDX1", 9, *HEADER.unpack(good)[2:]), table))
    with pytest.raises(P.PeosError, match="bad shape"):
        P.load_codes(_file(tmp_path / "shape.idx", _header(L=3), table))
    with pytest.raises(P.PeosError, match="bad shape"):  # sizes that would overflow are refused
        P.load_codes(_file(tmp_path / "huge.idx", _header(n=1 << 50), table))
    with pytest.raises(P.PeosError, match="bad L / m"):
        P.load_codes(_file(tmp_path / "m.idx", _header(m=200), table))
    with pytest.raises(P.PeosError, match="bad strides"):
        P.load_codes(_file(tmp_path / "stride.idx", _header(rec=97), table))
    with pytest.raises(P.PeosError, match="bad scalar width"):
        P.load_codes(_file(tmp_path / "sbits.idx", _header(sbits=12), table))
    with pytest.raises(P.PeosError, match="bad strides"):  # an 8-bit record is 96 bytes here, not 128
        P.load_codes(_file(tmp_path / "sb8.idx", _header(sbits=8), table))
    with pytest.raises(P.PeosError, match="unknown kind"):
        P.load_codes(_file(tmp_path / "kind.idx", _header(kind=5), table))
    # sections are checked against the shape before anything is allocated on a device
    with pytest.raises(P.PeosError, match="section size"):
        P.load_codes(_file(tmp_path / "size.idx", good, [(1, 0, 1000), (2, 0, 1920)]))
    with pytest.raises(P.PeosError, match="unknown section"):
        P.load_codes(_file(tmp_path / "sec.idx", good, [(9, 0, 0), (2, 0, 1920)]))
    assert os.path.exists(tmp_path / "kind.idx")
