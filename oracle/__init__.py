"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct CPU statement of what the batched CB-DFS hot path of
"A Parallel CPU-GPU Framework for Batching Heuristic Operations in Depth-First Heuristic
Search" (arXiv 2507.11916) computes.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import it.  It shares no code with the product package:
the search, domain and pattern-database parts live in `oracle.c` (built here with gcc), the
network parts are float64 numpy below.

Section map (paper sections, equations and algorithms):
  * domains, Manhattan distance, BFS ............ oracle.c (Background; Experimental Setup)
  * pattern databases ............................ oracle.c `or_pdb_build` (Background,
    Heuristics: an abstraction of the state space; additive costs)
  * CB-DFS ....................................... oracle.c `or_cbdfs` (Background: IDA*
    and BTS both repeat a cost-bounded DFS; Algorithm 3's expansion test, read as
    g + h <= bound as in the theorem's proof)
  * IDA* driver .................................. `ida_star` (Algorithm 1: bound = h(start),
    then CB-DFS and UpdateThreshold until a solution; the next threshold is the lowest
    f-cost left unexpanded, Background, AIDA*)
  * BTS driver ................................... `bts` (Background: BTS; Batch BTS
    enhancements: node limit, initial limit 10,000, initial bound h(root)+1).
    Parity unpinned against the paper for the bound-search schedule (the paper gives only
    the two constants and the requirement of exponential growth).
  * real-valued heuristics ....................... oracle.c `or_cbdfs_real`, `ida_star_real`,
    `bts_real`, `h_real`, `bound_test_real` (section "Regression-Based Neural Heuristics":
    real h, real f-costs and thresholds; Experimental Setup: the regression model's
    predictions minus 2.2).  `bts_real`'s binary search over real bounds is this oracle's
    reading (parity unpinned against the paper beyond the costs and the integer case).
  * DIV-compressed PDBs ........................... `pdb_div`, `pdb_div_h` (Background: DIV
    groups k adjacent entries by dividing the index by k and keeps the smallest; PDB
    Comparison: h_DIV of the network's size is the plain-heuristic comparator)
  * network heuristic ............................ `mlp_forward`, `h_regression`,
    `h_classifier` (Experimental Setup: a classifier heuristic and a regression heuristic;
    Background, Heuristics: classes are integer h values), `h_quantile` (Related Work: the
    classification quantile of ordered classes, lowered for admissibility), `h_combo` (the
    minimum over an ensemble; sums of such minima with MD, Experimental Setup)
  * training ..................................... `train_forward_backward`, `adam_step`
    (Experimental Setup: the models are trained from PDB values).  Not from the paper:
    float64 cross-entropy / MSE back-propagation and Adam as published by Kingma & Ba.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")

DOM_STP3, DOM_STP4, DOM_RC3 = 0, 1, 2
H_ZERO, H_MD, H_PDB, H_CALLBACK = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_oracle.so with gcc (no GPU code involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OrResult(ctypes.Structure):
    _fields_ = [("expanded", ctypes.c_int64), ("generated", ctypes.c_int64),
                ("minf", ctypes.c_int64), ("found", ctypes.c_int), ("cost", ctypes.c_int),
                ("cut", ctypes.c_int), ("path_len", ctypes.c_int),
                ("path", ctypes.c_int * 256)]


HEUR_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p)


class OrResultReal(ctypes.Structure):
    _fields_ = [("expanded", ctypes.c_int64), ("generated", ctypes.c_int64),
                ("minf", ctypes.c_double), ("found", ctypes.c_int), ("cost", ctypes.c_int),
                ("cut", ctypes.c_int), ("path_len", ctypes.c_int),
                ("path", ctypes.c_int * 256)]


HEUR_REAL_CB = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        u64p = ctypes.POINTER(ctypes.c_uint64)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_stp_md.argtypes = [ctypes.c_uint64, ctypes.c_int]
        L.or_stp_apply.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u64p]
        L.or_stp_apply_walk.argtypes = [ctypes.c_int, ip, ctypes.c_int, u64p]
        L.or_perm_rank.argtypes = [ip, ctypes.c_int]
        L.or_perm_rank.restype = ctypes.c_int64
        L.or_stp3_bfs.argtypes = [ctypes.c_void_p, ip]
        L.or_stp3_bfs.restype = ctypes.c_int64
        L.or_rc_apply.argtypes = [u64p, ctypes.c_int, u64p]
        L.or_rc_apply_seq.argtypes = [ip, ctypes.c_int, u64p]
        L.or_rc_invariants.argtypes = [u64p]
        L.or_rc_bfs_counts.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.or_npk.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_npk.restype = ctypes.c_int64
        L.or_pdb_rank.argtypes = [ip, ctypes.c_int, ctypes.c_int]
        L.or_pdb_rank.restype = ctypes.c_int64
        L.or_pdb_build.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.c_void_p]
        L.or_pdb_build.restype = ctypes.c_int64
        L.or_pdb_ball.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p]
        L.or_pdb_ball.restype = ctypes.c_int64
        L.or_rc_corner_index.argtypes = [u64p]
        L.or_rc_corner_index.restype = ctypes.c_int64
        L.or_rc_corner_ball.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        L.or_rc_corner_ball.restype = ctypes.c_int64
        L.or_rc_corner_pdb.argtypes = [ctypes.c_void_p]
        L.or_pdb_h.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ip, ip,
                               ctypes.c_void_p]
        L.or_cbdfs.argtypes = [ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ip, ip, ctypes.c_void_p,
                               HEUR_CB, ctypes.c_void_p, ctypes.POINTER(OrResult)]
        L.or_heuristic.argtypes = [ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, ip, ip,
                                   ctypes.c_void_p]
        assert L.or_result_size() == ctypes.sizeof(OrResult)
        L.or_cbdfs_real.argtypes = [ctypes.c_int, u64p, ctypes.c_double, ctypes.c_int64,
                                    ctypes.c_int, HEUR_REAL_CB, ctypes.c_void_p,
                                    ctypes.POINTER(OrResultReal)]
        assert L.or_result_real_size() == ctypes.sizeof(OrResultReal)
    return _lib


def _ints(xs):
    xs = list(xs)
    return (ctypes.c_int * max(1, len(xs)))(*xs)


def _words(state):
    if isinstance(state, (int, np.integer)):
        state = [int(state)]
    return (ctypes.c_uint64 * 2)(*(list(int(w) for w in state) + [0] * (2 - len(state))))


# ---------------------------------------------------------------------------------------
# domains
# ---------------------------------------------------------------------------------------

def stp_goal(side: int) -> int:
    return sum(t << (4 * t) for t in range(side * side))


def stp_md(state: int, side: int) -> int:
    return lib().or_stp_md(ctypes.c_uint64(int(state)), side)


def stp_apply(state: int, side: int, d: int):
    out = ctypes.c_uint64()
    ok = lib().or_stp_apply(ctypes.c_uint64(int(state)), side, d, ctypes.byref(out))
    return out.value if ok else None


def stp_apply_walk(side: int, dirs) -> int:
    out = ctypes.c_uint64()
    ok = lib().or_stp_apply_walk(side, _ints(dirs), len(dirs), ctypes.byref(out))
    if not ok:
        raise ValueError("illegal move in walk")
    return out.value


def perm_rank(perm) -> int:
    return lib().or_perm_rank(_ints(perm), len(perm))


def stp3_bfs():
    """(dist array indexed by perm_rank of the cells, number reached, max distance)."""
    dist = np.empty(362880, dtype=np.int8)
    md = ctypes.c_int()
    n = lib().or_stp3_bfs(dist.ctypes.data, ctypes.byref(md))
    return dist, n, md.value


def rc_goal():
    return (sum((c * 3) << (5 * c) for c in range(8)), sum((e * 2) << (5 * e) for e in range(12)))


def rc_apply(state, move):
    out = (ctypes.c_uint64 * 2)()
    lib().or_rc_apply(_words(state), move, out)
    return (out[0], out[1])


def rc_apply_seq(moves):
    out = (ctypes.c_uint64 * 2)()
    lib().or_rc_apply_seq(_ints(moves), len(moves), out)
    return (out[0], out[1])


def rc_invariants(state) -> int:
    return lib().or_rc_invariants(_words(state))


def rc_bfs_counts(maxdepth: int):
    distinct = np.zeros(maxdepth + 1, dtype=np.int64)
    tree = np.zeros(maxdepth + 1, dtype=np.int64)
    assert lib().or_rc_bfs_counts(maxdepth, distinct.ctypes.data, tree.ctypes.data) == 0
    return distinct, tree


# ---------------------------------------------------------------------------------------
# pattern databases
# ---------------------------------------------------------------------------------------

PATTERNS_663 = ([1, 2, 3, 5, 6, 7], [4, 8, 9, 12, 13, 14], [10, 11, 15])


def npk(n: int, k: int) -> int:
    return lib().or_npk(n, k)


def pdb_rank(pos, n: int) -> int:
    return lib().or_pdb_rank(_ints(pos), len(pos), n)


def pdb_build(side: int, tiles) -> np.ndarray:
    """uint8 table indexed by the lexicographic rank of the pattern tiles' cells."""
    table = np.empty(npk(side * side, len(tiles)), dtype=np.uint8)
    r = lib().or_pdb_build(side, _ints(tiles), len(tiles), table.ctypes.data)
    if r < 0:
        raise MemoryError("pdb_build")
    return table


def pdb_ball(side: int, tiles, maxd: int, cap: int = 1 << 24):
    """(ranks, values) of every placement of the pattern within distance maxd of the goal,
    from the same search as pdb_build stopped after level maxd: the entries of the full
    table that are <= maxd, without building the table."""
    ranks = np.empty(cap, dtype=np.int64)
    vals = np.empty(cap, dtype=np.uint8)
    m = lib().or_pdb_ball(side, _ints(tiles), len(tiles), maxd, cap, ranks.ctypes.data, vals.ctypes.data)
    if m < 0:
        raise MemoryError("pdb_ball: more than cap states within the distance")
    return ranks[:m].copy(), vals[:m].copy()


RC_CORNER_ENTRIES = 40320 * 2187  # 8! corner placements x 3^7 twists


def rc_corner_index(state) -> int:
    """The 8-corner PDB's index of a cube state (oracle.c `or_rc_corner_index`)."""
    return int(lib().or_rc_corner_index(_words(state)))


def rc_corner_ball(maxd: int, cap: int = 1 << 24):
    """(indices, distances) of every corner configuration within maxd face turns of the
    solved one, sorted by index: the 8-corner PDB's entries up to maxd."""
    idx = np.empty(cap, np.int64)
    val = np.empty(cap, np.uint8)
    n = lib().or_rc_corner_ball(maxd, cap, idx.ctypes.data, val.ctypes.data)
    if n < 0:
        raise ValueError("ball larger than cap")
    return idx[:n].copy(), val[:n].copy()


def rc_corner_pdb() -> np.ndarray:
    """The full 8-corner table (oracle.c `or_rc_corner_pdb`; 88 MB, about half a minute)."""
    t = np.empty(RC_CORNER_ENTRIES, np.uint8)
    if lib().or_rc_corner_pdb(t.ctypes.data) < 0:
        raise MemoryError("corner PDB queue")
    return t


class PDB:
    """An additive PDB: one table per pattern; h = sum of the table entries."""

    def __init__(self, side, patterns, tables):
        self.side = side
        self.patterns = [list(p) for p in patterns]
        self.tables = [np.ascontiguousarray(t, dtype=np.uint8) for t in tables]
        self._k = _ints(len(p) for p in self.patterns)
        self._tiles = _ints(t for p in self.patterns for t in p)
        self._ptrs = (ctypes.c_void_p * len(self.tables))(*(t.ctypes.data for t in self.tables))

    def h(self, state: int) -> int:
        return lib().or_pdb_h(ctypes.c_uint64(int(state)), self.side, len(self.patterns),
                              self._k, self._tiles, self._ptrs)

    def hs(self, states) -> np.ndarray:
        return np.array([self.h(int(s)) for s in states], dtype=np.int64)


def pdb_div(table, k: int) -> np.ndarray:
    """DIV compression (Background: k adjacent entries are grouped by dividing the index by
    k, and each group keeps its smallest entry so that the heuristic stays admissible):
    entry j of the result = min(table[j*k], ..., table[j*k + k - 1]) over the entries that
    exist; ceil(len / k) entries."""
    t = np.asarray(table, np.uint8)
    m = -(-len(t) // k)
    pad = np.full(m * k, 255, np.uint8)
    pad[:len(t)] = t
    return pad.reshape(m, k).min(axis=1)


def pdb_div_h(side, patterns, div_tables, k, state) -> int:
    """h of an additive PDB whose tables are DIV-compressed by k: sum over patterns of
    div_table[rank // k]; the goal gets 0."""
    n = side * side
    if int(state) == stp_goal(side):
        return 0
    where = {}
    for p in range(n):
        where[(int(state) >> (4 * p)) & 15] = p
    return int(sum(int(t[pdb_rank([where[x] for x in pat], n) // k]) for pat, t in zip(patterns, div_tables)))


# ---------------------------------------------------------------------------------------
# search
# ---------------------------------------------------------------------------------------

class Heur:
    """What CB-DFS uses for h: kind H_ZERO / H_MD / H_PDB, or a Python callable."""

    def __init__(self, kind=H_ZERO, pdb: PDB | None = None, fn=None):
        self.kind = H_CALLBACK if fn is not None else kind
        self.pdb = pdb
        self.fn = fn
        self._cache = {}

        def _cb(ptr, _user):
            key = (ptr[0], ptr[1])
            v = self._cache.get(key)
            if v is None:
                v = int(self.fn(key))
                self._cache[key] = v
            return v

        self._cb = HEUR_CB(_cb) if fn is not None else ctypes.cast(None, HEUR_CB)

    def args(self):
        if self.kind == H_PDB:
            p = self.pdb
            return (H_PDB, len(p.patterns), p._k, p._tiles, p._ptrs)
        return (self.kind, 0, None, None, None)


def cbdfs(domain, start, bound, heur: Heur, limit=-1, complete=True) -> OrResult:
    """One cost-bounded DFS (see oracle.c `or_cbdfs`)."""
    res = OrResult()
    kind, npat, pk, pt, tabs = heur.args()
    lib().or_cbdfs(domain, _words(start), int(bound), int(limit), int(complete), kind, npat,
                   pk, pt, tabs, heur._cb, None, ctypes.byref(res))
    return res


def heuristic(domain, state, heur: Heur) -> int:
    if heur.kind == H_CALLBACK:
        w = _words(state)
        if (domain == DOM_RC3 and (w[0], w[1]) == rc_goal()) or \
                (domain != DOM_RC3 and w[0] == stp_goal(3 if domain == DOM_STP3 else 4)):
            return 0
        return int(heur.fn((w[0], w[1])))
    kind, npat, pk, pt, tabs = heur.args()
    return lib().or_heuristic(domain, _words(state), kind, npat, pk, pt, tabs)


def ida_star(domain, start, heur: Heur, complete=True, max_iters=1000):
    """Algorithm 1 run serially: bound = h(start); repeat CB-DFS(bound) and raise the bound
    to the lowest f-cost that the iteration left unexpanded, until a goal is found.
    Returns dict(cost, iters=[(bound, expanded, generated)], path)."""
    bound = heuristic(domain, start, heur)
    iters = []
    for _ in range(max_iters):
        r = cbdfs(domain, start, bound, heur, -1, complete)
        iters.append((bound, r.expanded, r.generated))
        if r.found:
            return dict(cost=r.cost, iters=iters, path=list(r.path[:r.path_len]))
        if r.minf < 0:
            return dict(cost=None, iters=iters, path=None)
        bound = int(r.minf)
    raise RuntimeError("iteration cap reached")


BTS_C1, BTS_C2, BTS_N0 = 2, 8, 10000


def bts(domain, start, heur: Heur, c1=BTS_C1, c2=BTS_C2, n0=BTS_N0, max_searches=100000):
    """Budgeted Tree Search as a driver over CB-DFS with an expansion limit.

    Paper facts (Background: BTS; Batch BTS enhancements): BTS repeats CB-DFS with a node
    expansion limit and searches over cost bounds so that the expansions of successive
    iterations grow exponentially; Batch BTS starts from a node count of 10,000 and a first
    bound of h(root)+1.  The schedule below is this oracle's reading (parity unpinned
    against the paper, which gives no other constants).  Every search runs in complete
    mode, so an uncut search that reaches a goal reports the least goal cost in its tree,
    which is optimal for an admissible h.

    N is the growth base (n0 at first).  A round looks for a bound whose search expands
    between c1*N and c2*N nodes:
      1. try the IDA* next bound (h(root)+1 in the first round) with limit c2*N;
         accept it if uncut with >= c1*N expansions; if it is cut, run that bound without a
         limit and accept it;
      2. if it was uncut but small, try next + 2^j (j = 0, 1, ...) with limit c2*N until a
         bound is cut or expands >= c1*N, then binary-search the least such bound above the
         last small one; accept it if uncut, else run it without a limit and accept it;
      3. an uncut search that reaches a goal ends the run; an uncut search with no f above
         its bound (finite tree, no goal) ends it with no solution.
    Accepting a search sets N to its expansions and `next` to its least f above the bound.
    Returns dict(cost, searches=[(bound, limit, expanded, generated, cut, found)])."""
    searches = []

    def run(b, limit):
        r = cbdfs(domain, start, b, heur, limit, True)
        searches.append((b, limit, r.expanded, r.generated, r.cut, r.found))
        if len(searches) > max_searches:
            raise RuntimeError("search cap reached")
        return r

    class Done(Exception):
        pass

    def ends(r):
        if not r.cut and r.found:
            raise Done(r.cost)
        if not r.cut and r.minf < 0:
            raise Done(None)

    N = n0
    nxt = heuristic(domain, start, heur) + 1
    try:
        while True:
            limit = c2 * N
            r = run(nxt, limit)
            ends(r)
            if r.cut:
                r = run(nxt, -1)
                ends(r)
                N, nxt = max(r.expanded, 1), r.minf
                continue
            if r.expanded >= c1 * N:
                N, nxt = r.expanded, r.minf
                continue
            lo, j = nxt, 0
            while True:
                b = nxt + (1 << j)
                r = run(b, limit)
                ends(r)
                if r.cut or r.expanded >= c1 * N:
                    hi, hi_r = b, r
                    break
                lo, j = b, j + 1
            while hi - lo > 1:
                mid = (lo + hi) // 2
                r = run(mid, limit)
                ends(r)
                if r.cut or r.expanded >= c1 * N:
                    hi, hi_r = mid, r
                else:
                    lo = mid
            if hi_r.cut:
                hi_r = run(hi, -1)
                ends(hi_r)
            N, nxt = max(hi_r.expanded, 1), hi_r.minf
    except Done as d:
        return dict(cost=d.args[0], searches=searches)


# ---------------------------------------------------------------------------------------
# real-valued heuristics (section "Regression-Based Neural Heuristics": a regression
# network's h is real, so f-costs are real and IDA*'s thresholds move by small steps; BTS's
# search over bounds does not depend on how far apart f-costs lie)
# ---------------------------------------------------------------------------------------

class HeurReal:
    """A real-valued h: a callable on the packed words (a tuple of two ints), cached per
    state.  The goal gets 0 without a call."""

    def __init__(self, fn):
        self.fn = fn
        self._cache = {}

        def _cb(ptr, _user):
            key = (ptr[0], ptr[1])
            v = self._cache.get(key)
            if v is None:
                v = float(self.fn(key))
                self._cache[key] = v
            return v

        self._cb = HEUR_REAL_CB(_cb)

    def h(self, domain, state) -> float:
        w = _words(state)
        if (domain == DOM_RC3 and (w[0], w[1]) == rc_goal()) or \
                (domain != DOM_RC3 and w[0] == stp_goal(3 if domain == DOM_STP3 else 4)):
            return 0.0
        return float(self.fn((w[0], w[1])))


def cbdfs_real(domain, start, bound, heur: HeurReal, limit=-1, complete=True) -> OrResultReal:
    """One cost-bounded DFS with f = g + h and the bound in float64 (oracle.c
    `or_cbdfs_real`; the same tree rules as `cbdfs`).  minf < 0: no f above the bound."""
    res = OrResultReal()
    lib().or_cbdfs_real(domain, _words(start), float(bound), int(limit), int(complete),
                        heur._cb, None, ctypes.byref(res))
    return res


def ida_star_real(domain, start, heur: HeurReal, complete=True, max_iters=100000):
    """Algorithm 1 with a real-valued h: bound = h(start), then the least f above each
    iteration's bound.  Returns dict(cost, iters=[(bound, expanded, generated)], path)."""
    bound = heur.h(domain, start)
    iters = []
    for _ in range(max_iters):
        r = cbdfs_real(domain, start, bound, heur, -1, complete)
        iters.append((bound, r.expanded, r.generated))
        if r.found:
            return dict(cost=r.cost, iters=iters, path=list(r.path[:r.path_len]))
        if r.minf < 0:
            return dict(cost=None, iters=iters, path=None)
        bound = r.minf
    raise RuntimeError("iteration cap reached")


def bts_real(domain, start, heur: HeurReal, c1=None, c2=None, n0=None, max_searches=100000):
    """`bts` with real bounds.  The same schedule (first bound h(root)+1; the IDA* next
    bound, then next + 2^j, then a binary search between the last small bound lo and the
    first big one hi), with one change that the real line needs: the binary search runs
    while some f-cost lies strictly between lo and hi -- lo's least f above its bound,
    minf(lo), is below hi -- and probes mid = max((lo+hi)/2, minf(lo)), so that every probe
    can change the tree.  (With integer f-costs this accepts the same bound as `bts`: the
    least big bound.)  Returns dict(cost, searches=[(bound, limit, expanded, generated, cut,
    found)])."""
    c1 = BTS_C1 if c1 is None else c1
    c2 = BTS_C2 if c2 is None else c2
    n0 = BTS_N0 if n0 is None else n0
    searches = []

    def run(b, limit):
        r = cbdfs_real(domain, start, b, heur, limit, True)
        searches.append((b, limit, r.expanded, r.generated, r.cut, r.found))
        if len(searches) > max_searches:
            raise RuntimeError("search cap reached")
        return r

    class Done(Exception):
        pass

    def ends(r):
        if not r.cut and r.found:
            raise Done(r.cost)
        if not r.cut and r.minf < 0:
            raise Done(None)

    N = n0
    nxt = heur.h(domain, start) + 1.0
    try:
        while True:
            limit = c2 * N
            r = run(nxt, limit)
            ends(r)
            if r.cut:
                r = run(nxt, -1)
                ends(r)
                N, nxt = max(r.expanded, 1), r.minf
                continue
            if r.expanded >= c1 * N:
                N, nxt = r.expanded, r.minf
                continue
            lo, lo_minf, j = nxt, r.minf, 0
            while True:
                b = nxt + float(1 << j)
                r = run(b, limit)
                ends(r)
                if r.cut or r.expanded >= c1 * N:
                    hi, hi_r = b, r
                    break
                lo, lo_minf, j = b, r.minf, j + 1
            while lo_minf < hi:
                mid = max((lo + hi) / 2.0, lo_minf)
                if mid >= hi:
                    mid = lo_minf
                r = run(mid, limit)
                ends(r)
                if r.cut or r.expanded >= c1 * N:
                    hi, hi_r = mid, r
                else:
                    lo, lo_minf = mid, r.minf
            if hi_r.cut:
                hi_r = run(hi, -1)
                ends(hi_r)
            N, nxt = max(hi_r.expanded, 1), hi_r.minf
    except Done as d:
        return dict(cost=d.args[0], searches=searches)


# ---------------------------------------------------------------------------------------
# the network heuristic (float64)
# ---------------------------------------------------------------------------------------

def one_hot(domain: int, states) -> np.ndarray:
    """Float64 one-hot encoding.  STP: index tile*N + cell (blank included), width N*N.
    RC: corner cubie c at c*24 + (slot*3 + twist), edge cubie e at 192 + e*24 +
    (slot*2 + flip), width 480."""
    states = np.asarray(states, dtype=np.uint64)
    if domain == DOM_RC3:
        states = states.reshape(-1, 2)
        n = states.shape[0]
        X = np.zeros((n, 480))
        rows = np.arange(n)
        for c in range(8):
            f = ((states[:, 0] >> np.uint64(5 * c)) & np.uint64(31)).astype(np.int64)
            X[rows, c * 24 + f] = 1.0
        for e in range(12):
            f = ((states[:, 1] >> np.uint64(5 * e)) & np.uint64(31)).astype(np.int64)
            X[rows, 192 + e * 24 + f] = 1.0
        return X
    side = 3 if domain == DOM_STP3 else 4
    N = side * side
    states = states.reshape(-1)
    n = states.shape[0]
    X = np.zeros((n, N * N))
    rows = np.arange(n)
    for p in range(N):
        t = ((states >> np.uint64(4 * p)) & np.uint64(15)).astype(np.int64)
        X[rows, t * N + p] = 1.0
    return X


def bf16_round(a) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32.  NaN not handled."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32)


def _e4m3_grid() -> np.ndarray:
    """All finite non-negative E4M3 (OCP FP8, bias 7, max 448) values, ascending."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue  # NaN encoding
            if e == 0:
                vals.append(m / 8 * 2.0 ** -6)
            else:
                vals.append((1 + m / 8) * 2.0 ** (e - 7))
    return np.array(sorted(vals))


_E4M3 = None


def e4m3_round(x) -> np.ndarray:
    """Round float32 values to the nearest E4M3 value (ties to the even code), saturating
    at +-448.  The input is taken as float32 and the decision made exactly."""
    global _E4M3
    if _E4M3 is None:
        _E4M3 = _e4m3_grid()
    g = _E4M3
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    s = np.sign(x)
    a = np.minimum(np.abs(x), 448.0)
    i = np.clip(np.searchsorted(g, a), 1, len(g) - 1)
    lo, hi = g[i - 1], g[i]
    pick_hi = (hi - a) < (a - lo)
    tie = (hi - a) == (a - lo)
    even_hi = (i % 2) == 0  # codes are consecutive, index parity = mantissa LSB parity
    pick_hi = pick_hi | (tie & even_hi)
    r = np.where(pick_hi, hi, lo)
    r = np.where(a == 0, 0.0, r)
    return (s * r).astype(np.float32)


def fp8_weight_scale(W) -> np.float32:
    """Per-tensor scale: amax / 448, computed in float32."""
    return np.float32(np.max(np.abs(np.asarray(W, dtype=np.float32)))) / np.float32(448.0)


def quantise_weights(Ws, prec: str):
    """The weights a precision evaluates, widened back to float32: 'fp32' unchanged,
    'bf16' rounded to bfloat16, 'fp8' as scale * E4M3(W / scale)."""
    if prec == "fp32":
        return [np.asarray(W, np.float32) for W in Ws]
    if prec == "bf16":
        return [bf16_round(W) for W in Ws]
    if prec == "fp8":
        out = []
        for W in Ws:
            s = fp8_weight_scale(W)
            q = e4m3_round(np.asarray(W, np.float32) / s)
            out.append((q.astype(np.float64) * float(s)).astype(np.float32))
        return out
    raise ValueError(prec)


def mlp_forward(Ws, bs, X, return_hidden=False, act_scales=None, bf16_acts=False,
                store_last=False):
    """z_l = a_{l-1} W_l^T + b_l with ReLU on every layer but the last, in float64.

    The arithmetic stays float64; the options below only round the values a low-precision
    network stores between its layers (the storage formats of Experimental Setup's h_M run
    in BF16 or FP8 here), each stored value rounded once from its float64 value:

    act_scales: E4M3 storage of the activations that feed a following hidden layer: hidden
        layer l's output (l < L-2) becomes s_l * E4M3(float32(a) * float32(1/s_l)).
    bf16_acts: BF16 storage of those activations instead (when act_scales is None):
        a -> bfloat16(float32(a)), round to nearest, ties to even.
    store_last: the last hidden layer's output, which feeds the float32 last layer, is
        stored in BF16 too (a network whose last layer runs as a separate step reads it
        from memory); without it that output is not rounded (the last layer reads the
        accumulator)."""
    a = np.asarray(X, dtype=np.float64)
    hidden = []
    L = len(Ws)
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if l < L - 1:
            a = np.maximum(z, 0.0)
            if l < L - 2 and act_scales is not None:
                inv = np.float32(1.0) / np.float32(act_scales[l])
                q = e4m3_round(a.astype(np.float32) * inv)
                a = q.astype(np.float64) * float(np.float32(act_scales[l]))
            elif (l < L - 2 and bf16_acts) or (l == L - 2 and store_last):
                a = bf16_round(a.astype(np.float32)).astype(np.float64)
            hidden.append(a)
        else:
            a = z
    return (a, hidden) if return_hidden else a


def is_goal_states(domain, states) -> np.ndarray:
    states = np.asarray(states, dtype=np.uint64)
    if domain == DOM_RC3:
        g = rc_goal()
        s = states.reshape(-1, 2)
        return (s[:, 0] == np.uint64(g[0])) & (s[:, 1] == np.uint64(g[1]))
    return states.reshape(-1) == np.uint64(stp_goal(3 if domain == DOM_STP3 else 4))


def md_states(domain, states) -> np.ndarray:
    side = 3 if domain == DOM_STP3 else 4
    return np.array([stp_md(int(s), side) for s in np.asarray(states).reshape(-1)], np.int64)


def h_regression(y, md=None, goal=None) -> np.ndarray:
    """h = max(max(rint(y), 0), MD), rint rounding half to even, clamped to 255;
    the goal gets 0."""
    h = np.maximum(np.rint(np.asarray(y, np.float64).reshape(-1)), 0.0)
    h = np.minimum(h, 255.0).astype(np.int64)
    if md is not None:
        h = np.maximum(h, np.asarray(md, np.int64))
    h = np.minimum(h, 255)
    if goal is not None:
        h = np.where(goal, 0, h)
    return h


def h_classifier(logits, md=None, goal=None) -> np.ndarray:
    """h = the class with the largest logit (lowest index on ties); optional max with MD;
    the goal gets 0."""
    logits = np.asarray(logits, np.float64)
    h = np.argmax(logits, axis=1).astype(np.int64)
    if md is not None:
        h = np.maximum(h, np.asarray(md, np.int64))
    h = np.minimum(h, 255)
    if goal is not None:
        h = np.where(goal, 0, h)
    return h


def h_real(y, offset, md=None, goal=None) -> np.ndarray:
    """The real-valued regression heuristic (Experimental Setup: the regression model's
    predictions minus 2.2, for admissibility): h = max(y + offset, 0), max'ed with MD when
    given; the goal gets 0."""
    h = np.maximum(np.asarray(y, np.float64).reshape(-1) + offset, 0.0)
    if md is not None:
        h = np.maximum(h, np.asarray(md, np.float64))
    if goal is not None:
        h = np.where(goal, 0.0, h)
    return h


def bound_test_real(g, h, bound, dtype=np.float64):
    """The bound test with real h: mask_i = (g_i + h_i <= bound) with the sum and the
    comparison in `dtype`; minf = least g_i + h_i above the bound (inf if none)."""
    f = np.asarray(g, dtype) + np.asarray(h, dtype)
    ok = f <= dtype(bound)
    n = len(f)
    words = np.zeros((n + 31) // 32, dtype=np.uint64)
    for i in np.nonzero(ok)[0]:
        words[i // 32] |= np.uint64(1) << np.uint64(i % 32)
    above = f[~ok]
    minf = float(above.min()) if above.size else float("inf")
    return words.astype(np.uint32), minf


def h_quantile(logits, q, md=None, goal=None) -> np.ndarray:
    """The classifier quantile (Related Work: ordered classes let the quantile of the
    predicted class be lowered for admissibility): with p = softmax(logits), h = the smallest
    class c with p_0 + ... + p_c >= q (the last class if no partial sum reaches q); optional
    max with MD; the goal gets 0."""
    y = np.asarray(logits, np.float64)
    p = np.exp(y - y.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    cdf = np.cumsum(p, axis=1)
    C = y.shape[1]
    h = np.array([next((c for c in range(C) if cdf[i, c] >= q), C - 1) for i in range(len(y))], np.int64)
    if md is not None:
        h = np.maximum(h, np.asarray(md, np.int64))
    h = np.minimum(h, 255)
    if goal is not None:
        h = np.where(goal, 0, h)
    return h


def h_combo(member_h, group_sizes, md=None, goal=None) -> np.ndarray:
    """A composite heuristic (Related Work: the minimum over an ensemble keeps a learned
    heuristic admissible; Experimental Setup: the 15-puzzle h_M adds ensembles trained on PDB
    minus MD to MD): member_h[m] are the members' h arrays, group after group; h = [md] + the
    sum over groups of the minimum over the group's members, clamped to 255; the goal gets 0."""
    hs = [np.asarray(h, np.int64) for h in member_h]
    total = np.zeros_like(hs[0]) if md is None else np.asarray(md, np.int64).copy()
    m = 0
    for k in group_sizes:
        total = total + np.min(np.stack(hs[m:m + k]), axis=0)
        m += k
    total = np.minimum(total, 255)
    if goal is not None:
        total = np.where(goal, 0, total)
    return total


def quantile_margin(logits, q, width) -> np.ndarray:
    """True where a partial sum of softmax(logits) lies within `width` (absolute, per row or
    scalar) of q: a logit error of that size may move the quantile class."""
    y = np.asarray(logits, np.float64)
    p = np.exp(y - y.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    cdf = np.cumsum(p, axis=1)
    w = np.broadcast_to(np.asarray(width, np.float64).reshape(-1, 1) if np.ndim(width) else width, cdf.shape)
    return (np.abs(cdf - q) < w).any(axis=1)


def regression_margin(y, width=1e-2) -> np.ndarray:
    """True where y lies within `width` of a half-integer rounding boundary."""
    y = np.asarray(y, np.float64).reshape(-1)
    return np.abs(y - (np.floor(y) + 0.5)) < width


def classifier_margin(logits, width=1e-2) -> np.ndarray:
    """True where the two largest logits differ by less than `width`."""
    s = np.sort(np.asarray(logits, np.float64), axis=1)
    return (s[:, -1] - s[:, -2]) < width


def bound_test(g, h, bound):
    """mask_i = (g_i + h_i <= bound), packed 32 per uint32 word (bit i%32 of word i/32);
    minf = least g_i + h_i above the bound (0xFFFFFFFF if none)."""
    f = np.asarray(g, np.int64) + np.asarray(h, np.int64)
    ok = f <= bound
    n = len(f)
    words = np.zeros((n + 31) // 32, dtype=np.uint64)
    for i in np.nonzero(ok)[0]:
        words[i // 32] |= np.uint64(1) << np.uint64(i % 32)
    above = f[~ok]
    minf = int(above.min()) if above.size else 0xFFFFFFFF
    return words.astype(np.uint32), minf


# ---------------------------------------------------------------------------------------
# training (float64)
# ---------------------------------------------------------------------------------------

def train_forward_backward(Ws, bs, X, labels, loss="ce", bf16_storage=False):
    """Loss and gradients of the mean loss over the batch.
    loss='ce': softmax cross-entropy against integer labels;
    loss='mse': 0.5*(y - label)^2 on a single output.

    bf16_storage: emulate a step that stores the hidden activations and the hidden layers'
    dZ in bfloat16 (each rounded from its float32 value); the last layer, the loss and its
    dZ stay unrounded.  The ReLU masks then come from the stored activations."""
    def rnd(x):
        return bf16_round(np.asarray(x, np.float32)).astype(np.float64) if bf16_storage else x

    Ws = [np.asarray(W, np.float64) for W in Ws]
    bs = [np.asarray(b, np.float64) for b in bs]
    acts = [np.asarray(X, np.float64)]
    zs = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = acts[-1] @ W.T + b
        zs.append(z)
        acts.append(rnd(np.maximum(z, 0.0)) if l < len(Ws) - 1 else z)
    out = acts[-1]
    B = out.shape[0]
    labels = np.asarray(labels)
    if loss == "ce":
        m = out.max(axis=1, keepdims=True)
        e = np.exp(out - m)
        p = e / e.sum(axis=1, keepdims=True)
        L = float(np.mean(-np.log(p[np.arange(B), labels.astype(np.int64)])))
        dz = p.copy()
        dz[np.arange(B), labels.astype(np.int64)] -= 1.0
        dz /= B
    elif loss == "mse":
        r = out[:, 0] - labels.astype(np.float64)
        L = float(np.mean(0.5 * r * r))
        dz = (r / B)[:, None]
    else:
        raise ValueError(loss)
    gW = [None] * len(Ws)
    gb = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gW[l] = dz.T @ acts[l]
        gb[l] = dz.sum(axis=0)
        if l > 0:
            da = dz @ Ws[l]
            dz = rnd(da * (acts[l] > 0))
    return L, gW, gb


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, with bias correction); returns (w, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
