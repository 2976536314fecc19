"""PDB table files (host-only calls, no GPU): the table bytes and the pattern come back as
written, and a damaged, truncated or foreign file is refused.  The tables are the oracle's
(Background: PDBs; an interface for reusing tables built once)."""
import os

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


def test_round_trip_of_an_oracle_table(P, orc, tmp_path):
    tiles = [1, 2, 3, 4]
    table = orc.pdb_build(3, tiles)
    path = tmp_path / "pdb_1234.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP3, tiles, table)
    assert os.path.getsize(path) == 128 + len(table)
    dom, t, div, back = P.cbdfs_pdb_file_read(path)
    assert dom == P.DOM_STP3 and t == tiles and div == 1
    assert back.dtype == np.uint8 and np.array_equal(back, table)


def test_round_trip_of_a_div_table(P, orc, tmp_path):
    tiles = [5, 6, 7, 8]
    table = orc.pdb_div(orc.pdb_build(3, tiles), 7)
    path = tmp_path / "pdb_div7.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP3, tiles, table, div=7)
    dom, t, div, back = P.cbdfs_pdb_file_read(path)
    assert (dom, t, div) == (P.DOM_STP3, tiles, 7) and np.array_equal(back, table)


def test_damaged_files_are_refused(P, tmp_path):
    table = (W.splitmix64_array(5, 3360) % np.uint64(40)).astype(np.uint8)  # 16 * 15 * 14 ranks
    path = tmp_path / "pdb.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP4, [1, 2, 3], table)
    raw = bytearray(path.read_bytes())
    # one flipped table byte: the hash no longer matches
    bad = bytearray(raw)
    bad[128 + 777] ^= 1
    (tmp_path / "flip.bin").write_bytes(bytes(bad))
    with pytest.raises(P.CbdfsError) as e:
        P.cbdfs_pdb_file_read(tmp_path / "flip.bin")
    assert e.value.status == P.CBDFS_EINVAL and "hash" in str(e.value)
    # truncated
    (tmp_path / "short.bin").write_bytes(bytes(raw[:-10]))
    with pytest.raises(P.CbdfsError) as e:
        P.cbdfs_pdb_file_read(tmp_path / "short.bin")
    assert e.value.status == P.CBDFS_EINVAL
    # not a PDB file
    (tmp_path / "other.bin").write_bytes(b"x" * 200)
    with pytest.raises(P.CbdfsError) as e:
        P.cbdfs_pdb_file_read(tmp_path / "other.bin")
    assert e.value.status == P.CBDFS_EINVAL
    # no file
    with pytest.raises(P.CbdfsError) as e:
        P.cbdfs_pdb_file_read(tmp_path / "missing.bin")
    assert e.value.status == P.CBDFS_ENOTFOUND
    # the intact file still reads
    assert np.array_equal(P.cbdfs_pdb_file_read(path)[3], table)


def test_bad_arguments(P, tmp_path):
    with pytest.raises(P.CbdfsError):
        P.cbdfs_pdb_file_write(tmp_path / "x.bin", 7, [1, 2], np.zeros(4, np.uint8))  # no such domain
    with pytest.raises(P.CbdfsError):
        P.cbdfs_pdb_file_write(tmp_path / "x.bin", P.DOM_STP3, [], np.zeros(4, np.uint8))  # no tiles


def test_header_layout_is_the_documented_one(P, tmp_path):
    # "CBDFSPDB", version, domain, k, 16 tiles, DIV factor, entry count, FNV-1a 64 of the table
    import struct
    table = np.arange(1120, dtype=np.uint64).astype(np.uint8)  # ceil(16 * 15 * 14 / 3)
    path = tmp_path / "layout.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP4, [10, 11, 15], table, div=3)
    raw = path.read_bytes()
    magic, version, dom, k = struct.unpack_from("<8sIii", raw, 0)
    tiles = struct.unpack_from("<16i", raw, 20)
    div, entries, h = struct.unpack_from("<IQQ", raw, 84)
    assert (magic, version, dom, k) == (b"CBDFSPDB", 1, P.DOM_STP4, 3)
    assert tiles == (10, 11, 15) + (0,) * 13 and div == 3 and entries == 1120
    fnv = 14695981039346656037
    for b in table.tobytes():
        fnv = ((fnv ^ b) * 1099511628211) % (1 << 64)
    assert h == fnv
    assert raw[128:] == table.tobytes() and len(raw) == 128 + 1120


def _fnv(data):
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) % (1 << 64)
    return h


def test_headers_that_no_table_has_are_refused(P, orc, tmp_path):
    # a header whose hash matches its bytes but whose domain, DIV factor or entry count is not
    # that of any table for its pattern is refused, so a reader sizing its buffer from the
    # header never reads past what the pattern implies
    import struct
    table = orc.pdb_build(3, [1, 2, 3])  # 9 * 8 * 7 = 504 ranks
    path = tmp_path / "good.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP3, [1, 2, 3], table)
    raw = path.read_bytes()
    assert len(raw) == 128 + 504

    def patched(name, domain=None, div=None, body=None):
        hd = bytearray(raw[:128])
        body = raw[128:] if body is None else body
        if domain is not None:
            struct.pack_into("<i", hd, 12, domain)
        if div is not None:
            struct.pack_into("<I", hd, 84, div)
        struct.pack_into("<QQ", hd, 88, len(body), _fnv(body))
        (tmp_path / name).write_bytes(bytes(hd) + body)
        return tmp_path / name

    for f in (patched("short_table.bin", body=raw[128:128 + 400]),  # 400 entries, hash of 400
              patched("domain.bin", domain=5),
              patched("div0.bin", div=0),
              patched("div2.bin", div=2)):                             # 504 entries but DIV 2 has 252
        with pytest.raises(P.CbdfsError) as e:
            P.cbdfs_pdb_file_read(f)
        assert e.value.status == P.CBDFS_EINVAL
    # a DIV-2 header with 252 entries is a valid file
    ok = patched("div2_ok.bin", div=2, body=bytes(orc.pdb_div(table, 2)))
    assert P.cbdfs_pdb_file_read(ok)[2] == 2
    # the writer refuses an entry count the pattern does not imply
    with pytest.raises(P.CbdfsError):
        P.cbdfs_pdb_file_write(tmp_path / "x.bin", P.DOM_STP3, [1, 2, 3], table[:500])
