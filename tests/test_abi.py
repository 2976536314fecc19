"""CPU checks of the product library: it loads, exports every symbol include/cbdfs.h
declares, and its host-side domain code agrees with the oracle's."""
import ctypes
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_cbdfs_build", os.path.join(ROOT, "paper_2507_11916_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2507_11916_b300 as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "cbdfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "heur_submit_batch" in names and "cbdfs_solve" in names and "pdb_build" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.EXPORTED) == names


def test_no_gpu_means_a_device_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.CbdfsError) as e:
        lib.cbdfs_create(0)
    assert e.value.status == lib.CBDFS_EDEVICE


def test_stp_moves_match_oracle(lib, orc):
    for side, dom in ((3, lib.DOM_STP3), (4, lib.DOM_STP4)):
        goal = W.stp_goal(side)
        for i in range(30):
            walk = W.stp_walk(side, 80, 300 + i)
            assert lib.cbdfs_apply_moves(dom, goal, walk) == orc.stp_apply_walk(side, walk)
            s = orc.stp_apply_walk(side, walk)
            assert lib.cbdfs_manhattan(dom, s) == orc.stp_md(s, side)
    # an illegal move (blank off the board) is rejected
    with pytest.raises(lib.CbdfsError):
        lib.cbdfs_apply_moves(lib.DOM_STP3, W.stp_goal(3), [W.DIR_UP])


def test_rc_moves_match_oracle(lib, orc):
    for i in range(200):
        seq = W.rc_scramble(20, 900 + i)
        assert lib.cbdfs_apply_moves(lib.DOM_RC3, W.rc_goal(), seq) == orc.rc_apply_seq(seq)
    for s in W.random_rc_states(50, 4):
        st = (int(s[0]), int(s[1]))
        for m in range(18):
            assert lib.cbdfs_apply_moves(lib.DOM_RC3, st, [m]) == orc.rc_apply(st, m)


def test_search_defaults(lib):
    d = lib.cbdfs_search_defaults()
    assert d["bts_n0"] == 10000 and d["timeout_us"] == 4000 and d["complete_final"] == 1
