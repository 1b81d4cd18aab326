"""Index files on the GPU: a saved and reloaded codes handle (PEOs codes with and without
the dimension permutation of Appendix D.1, SimHash bits) holds the same bytes and gives
the same searches; the file's checksums are zlib's CRC-32 of its parts, and a flipped or
missing byte anywhere is rejected without leaving the device unusable.  The graph comes
back out of the edge records."""
import struct
import zlib

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HEADER = struct.Struct("<8sIIqiiiiiQQiiI")
ENTRY = struct.Struct("<IIQ")
SEC_PERM = 6


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def env(P, sift20k):
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    Q = torch.from_numpy(case.Q).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    cfg = case.cfg
    perm = P.dim_permutation(G, X, cfg.L)
    handles = {"plain": P.build_codes(G, X, cfg.L, cfg.m, cfg.proj_seed),
               "perm": P.build_codes(G, X, cfg.L, cfg.m, cfg.proj_seed, perm=perm),
               "simhash": P.build_simhash(G, X, 128, 5)}
    return case, X, Q, G, perm, handles


def _parse(raw: bytes):
    h = HEADER.unpack_from(raw, 0)
    nsec = h[-1]
    table = [ENTRY.unpack_from(raw, HEADER.size + i * ENTRY.size) for i in range(nsec)]
    off = HEADER.size + nsec * ENTRY.size
    (hc,) = struct.unpack_from("<I", raw, off)
    return h, table, hc, off + 4


def _searches(P, G, codes, X, Q, kind):
    out = []
    frames = (0,) if kind == "simhash" else (0, 1)
    for frame in frames:
        ids, dists, cnt = P.search(G, codes, X, Q, 10, 48, eps=0.2, routing=2 if kind == "simhash" else 1,
                                   frame=frame, counters=True)
        out.append((ids.cpu().numpy(), dists.cpu().numpy().view(np.uint32), cnt.cpu().numpy()))
    return out


@pytest.mark.parametrize("kind", ["plain", "perm", "simhash"])
def test_roundtrip(P, env, kind, tmp_path):
    case, X, Q, G, perm, handles = env
    codes = handles[kind]
    path = str(tmp_path / f"{kind}.idx")
    codes.save(path)
    raw = open(path, "rb").read()
    h, table, hc, off = _parse(raw)
    assert h[0] == b"PEOSIDX1" and h[1] == 4 and h[2] == (1 if kind == "simhash" else 0) and h[-2] == 32
    assert hc == zlib.crc32(raw[:off - 4])
    for sid, crc, nbytes in table:  # sections follow the table back to back
        assert crc == zlib.crc32(raw[off:off + nbytes]), sid
        if sid == SEC_PERM:
            assert np.array_equal(np.frombuffer(raw[off:off + nbytes], dtype=np.int32), perm.cpu().numpy())
        off += nbytes
    assert off == len(raw)
    assert (SEC_PERM in [t[0] for t in table]) == (kind == "perm")

    back = P.load_codes(path)
    a, b = codes.info(), back.info()
    for f in ("n", "R", "L", "m", "d", "entry", "record_stride", "node_proj_stride", "kind"):
        assert a[f] == b[f], f
    assert bool(b["perm"]) == (kind == "perm")
    ea, eb = codes.arrays(), back.arrays()
    for name in ea:
        assert np.array_equal(np.asarray(ea[name]), np.asarray(eb[name])), name
    # every device array, Wt and the row norms included, comes back byte for byte
    path2 = str(tmp_path / f"{kind}_again.idx")
    back.save(path2)
    assert open(path2, "rb").read() == raw
    # the graph comes back out of the records: searching the file alone gives the same
    G2 = back.graph()
    assert np.array_equal(G2.nbrs.cpu().numpy(), case.nbrs) and G2.entry == case.entry
    for x, y in zip(_searches(P, G, codes, X, Q, kind), _searches(P, G2, back, X, Q, kind)):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
    back.free()


def test_damaged_files_are_rejected(P, env, tmp_path):
    case, X, Q, G, perm, handles = env
    path = str(tmp_path / "good.idx")
    handles["perm"].save(path)
    raw = open(path, "rb").read()
    h, table, hc, off = _parse(raw)
    bad = str(tmp_path / "bad.idx")

    def rejected(data, match):
        with open(bad, "wb") as f:
            f.write(data)
        with pytest.raises(P.PeosError, match=match):
            P.load_codes(bad)

    for sid, crc, nbytes in table:  # one flipped bit in the middle of every section
        b = bytearray(raw)
        b[off + nbytes // 2] ^= 0x10
        rejected(bytes(b), "section checksum")
        off += nbytes
    b = bytearray(raw)
    b[48] ^= 0x01  # inside the seed (bytes 44..51)
    rejected(bytes(b), "header checksum")
    b = bytearray(raw)
    b[HEADER.size + 1] ^= 0x01  # a section id in the table
    rejected(bytes(b), "header checksum")
    rejected(raw[:-1], "truncated")
    rejected(raw[:len(raw) // 2], "truncated")
    rejected(raw[:HEADER.size + 3], "truncated section table")
    # a permutation section that is not a permutation, with checksums made to match
    h, table, hc, off = _parse(raw)
    b = bytearray(raw)
    pos, k = off, 0
    for k, (sid, crc, nbytes) in enumerate(table):
        if sid == SEC_PERM:
            break
        pos += nbytes
    p = np.frombuffer(raw[pos:pos + table[k][2]], dtype=np.int32).copy()
    p[1] = p[0]
    b[pos:pos + p.nbytes] = p.tobytes()
    ent = HEADER.size + k * ENTRY.size
    b[ent:ent + ENTRY.size] = ENTRY.pack(SEC_PERM, zlib.crc32(p.tobytes()), p.nbytes)
    b[off - 4:off] = struct.pack("<I", zlib.crc32(bytes(b[:off - 4])))
    rejected(bytes(b), "not a permutation")
    # the device is still usable and the good file still loads
    good = P.load_codes(path)
    ids = P.search(G, good, X, Q, 10, 32, routing=1)[0].cpu().numpy()
    want = P.search(G, handles["perm"], X, Q, 10, 32, routing=1)[0].cpu().numpy()
    assert np.array_equal(ids, want)
