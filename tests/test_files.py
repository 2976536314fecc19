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
    table = (W.splitmix64_array(5, 10_000) % np.uint64(40)).astype(np.uint8)
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
    table = np.arange(1000, dtype=np.uint64).astype(np.uint8)
    path = tmp_path / "layout.bin"
    P.cbdfs_pdb_file_write(path, P.DOM_STP4, [10, 11, 15], table, div=3)
    raw = path.read_bytes()
    magic, version, dom, k = struct.unpack_from("<8sIii", raw, 0)
    tiles = struct.unpack_from("<16i", raw, 20)
    div, entries, h = struct.unpack_from("<IQQ", raw, 84)
    assert (magic, version, dom, k) == (b"CBDFSPDB", 1, P.DOM_STP4, 3)
    assert tiles == (10, 11, 15) + (0,) * 13 and div == 3 and entries == 1000
    fnv = 14695981039346656037
    for b in table.tobytes():
        fnv = ((fnv ^ b) * 1099511628211) % (1 << 64)
    assert h == fnv
    assert raw[128:] == table.tobytes() and len(raw) == 128 + 1000
