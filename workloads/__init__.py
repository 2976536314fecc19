"""Seeded synthetic inputs, shared by the oracle-side tests and the CUDA-side tests and bench.

This module holds random draws and the packed-state format only. It holds no heuristic,
search, pattern-database or network arithmetic, so neither side of a parity test can borrow
the other's answer from here.

What it produces:

* a counter-based splitmix64 generator (Steele, Lea & Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014), scalar and vectorised;
* sliding-tile random walks as blank-move direction sequences (only the blank position is
  tracked, so the walk is legal and never undoes its previous move), and Rubik's-cube
  scrambles as face-turn sequences that never turn one face twice in a row and take two
  opposite faces in one order only.  Each side of a test applies these sequences with its
  own domain code;
* uniformly random reachable packed states (sliding-tile and cube) for kernel inputs;
* network weights with the stated init laws, drawn in float64 and stored as float32.

Packed formats (the library's public ABI, restated here so both sides agree):

* sliding-tile puzzle, N = side*side cells: nibble p (bits 4p..4p+3) of one uint64 holds
  the tile at cell p, 0 = blank.  The goal puts tile t on cell t (blank on cell 0).
* Rubik's cube: two uint64 words.  Word 0 holds, for corner cubie c = 0..7, the 5-bit
  field (bits 5c..5c+4) slot*3 + twist; word 1 holds, for edge cubie e = 0..11, the 5-bit
  field slot*2 + flip.  Slots and cubies share one numbering (URF UFL ULB UBR DFR DLF DBL
  DRB for corners; UR UF UL UB DR DF DL DB FR FL BL BR for edges), so the solved cube has
  every cubie in its own slot with zero twist and flip.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15

# blank-move directions for the sliding-tile puzzle: the blank moves up, left, right, down
DIR_UP, DIR_LEFT, DIR_RIGHT, DIR_DOWN = 0, 1, 2, 3
# cube faces in the library's numbering; opposite(f) = (f + 3) % 6
FACES = "URFDLB"


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Scalar splitmix64 stream: state += gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return _mix64(self.state)

    def below(self, k: int) -> int:
        """An integer in [0, k): the next draw modulo k."""
        return self.next() % k

    def uniform(self) -> float:
        """A double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def seed_for(tag: int, index: int) -> int:
    """Per-instance seed: one splitmix64 mix of (tag << 32 | index)."""
    return _mix64(((tag & 0xFFFFFFFF) << 32 | (index & 0xFFFFFFFF)) & MASK64)


def splitmix64_array(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based draws: element i is the (offset+i+1)-th output of SplitMix64(seed)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


# ---------------------------------------------------------------------------------------
# sliding-tile puzzle
# ---------------------------------------------------------------------------------------

def stp_goal(side: int) -> int:
    return sum(t << (4 * t) for t in range(side * side))


def stp_pack(cells) -> int:
    """Pack a list of tiles (tile at cell p) into the nibble format."""
    s = 0
    for p, t in enumerate(cells):
        s |= int(t) << (4 * p)
    return s


def stp_cells(state: int, side: int) -> list[int]:
    return [(state >> (4 * p)) & 15 for p in range(side * side)]


def stp_walk(side: int, length: int, seed: int) -> list[int]:
    """A random walk of the blank from the goal (blank on cell 0): `length` directions,
    each legal for the blank's current cell and never the reverse of the one before."""
    rng = SplitMix64(seed)
    r = c = 0
    prev = -1
    out = []
    for _ in range(length):
        legal = []
        for d, (dr, dc) in enumerate(((-1, 0), (0, -1), (0, 1), (1, 0))):
            if prev >= 0 and d == 3 - prev:
                continue
            if 0 <= r + dr < side and 0 <= c + dc < side:
                legal.append((d, dr, dc))
        d, dr, dc = legal[rng.below(len(legal))]
        r, c, prev = r + dr, c + dc, d
        out.append(d)
    return out


def stp_walk_random_length(side: int, max_len: int, seed: int) -> list[int]:
    """The labelled-state walks: one splitmix64 stream (SplitMix64(seed)) gives first the
    length 1 + (draw mod max_len), then the moves exactly as stp_walk draws them."""
    rng = SplitMix64(seed)
    length = 1 + rng.below(max_len)
    r = c = 0
    prev = -1
    out = []
    for _ in range(length):
        legal = []
        for d, (dr, dc) in enumerate(((-1, 0), (0, -1), (0, 1), (1, 0))):
            if prev >= 0 and d == 3 - prev:
                continue
            if 0 <= r + dr < side and 0 <= c + dc < side:
                legal.append((d, dr, dc))
        d, dr, dc = legal[rng.below(len(legal))]
        r, c, prev = r + dr, c + dc, d
        out.append(d)
    return out


def random_stp_states(side: int, n: int, seed: int) -> np.ndarray:
    """n uniformly random solvable sliding-tile states, packed (uint64)."""
    ncell = side * side
    keys = splitmix64_array(seed, n * ncell).reshape(n, ncell)
    perm = np.argsort(keys, axis=1, kind="stable").astype(np.int64)  # perm[:, p] = tile at p
    # parity of the permutation (blank included as tile 0) by counting inversions
    p8 = perm.astype(np.int8)
    inv = np.zeros(n, dtype=np.int64)
    for i in range(ncell):
        inv += np.count_nonzero(p8[:, i:i + 1] > p8[:, i + 1:], axis=1)
    blank = np.argmax(perm == 0, axis=1)
    taxi = blank // side + blank % side  # blank's distance to its goal cell 0
    bad = (inv & 1) != (taxi & 1)
    # swap the tiles in the first two cells that do not hold the blank
    rows = np.nonzero(bad)[0]
    first = np.where(blank[rows] == 0, 1, 0)
    second = np.where(blank[rows] <= 1, 2, 1)
    a, b = perm[rows, first].copy(), perm[rows, second].copy()
    perm[rows, first], perm[rows, second] = b, a
    shifts = (4 * np.arange(ncell, dtype=np.uint64))
    return (perm.astype(np.uint64) << shifts).sum(axis=1, dtype=np.uint64)


# ---------------------------------------------------------------------------------------
# Rubik's cube
# ---------------------------------------------------------------------------------------

def rc_goal() -> tuple[int, int]:
    w0 = sum((c * 3) << (5 * c) for c in range(8))
    w1 = sum((e * 2) << (5 * e) for e in range(12))
    return w0, w1


def rc_scramble(length: int, seed: int) -> list[int]:
    """A face-turn sequence: move m = 3*face + (quarter turns - 1), faces U R F D L B.
    No face is turned twice in a row, and two opposite faces in a row come only in the
    order lower face index first."""
    rng = SplitMix64(seed)
    prev = -1
    out = []
    for _ in range(length):
        faces = [f for f in range(6)
                 if prev < 0 or (f != prev and not (f == (prev + 3) % 6 and f < prev))]
        f = faces[rng.below(len(faces))]
        out.append(3 * f + rng.below(3))
        prev = f
    return out


def random_rc_states(n: int, seed: int) -> np.ndarray:
    """n uniformly random reachable cube states, packed as an (n, 2) uint64 array."""
    k = splitmix64_array(seed, n * 40).reshape(n, 40)
    cslot = np.argsort(k[:, :8], axis=1, kind="stable")     # cslot[:, c] = slot of corner c
    eslot = np.argsort(k[:, 8:20], axis=1, kind="stable")   # eslot[:, e] = slot of edge e
    tw = (k[:, 20:28] % np.uint64(3)).astype(np.int64)
    tw[:, 7] = (-tw[:, :7].sum(axis=1)) % 3
    fl = (k[:, 28:40] % np.uint64(2)).astype(np.int64)
    fl[:, 11] = fl[:, :11].sum(axis=1) % 2

    def parity(p):
        m = p.shape[1]
        inv = np.zeros(p.shape[0], dtype=np.int64)
        for i in range(m):
            inv += (p[:, i:i + 1] > p[:, i + 1:]).sum(axis=1)
        return inv & 1

    bad = parity(cslot) != parity(eslot)
    eslot[bad, 0], eslot[bad, 1] = eslot[bad, 1].copy(), eslot[bad, 0].copy()
    w0 = np.zeros(n, dtype=np.uint64)
    w1 = np.zeros(n, dtype=np.uint64)
    for c in range(8):
        w0 |= (cslot[:, c] * 3 + tw[:, c]).astype(np.uint64) << np.uint64(5 * c)
    for e in range(12):
        w1 |= (eslot[:, e] * 2 + fl[:, e]).astype(np.uint64) << np.uint64(5 * e)
    return np.stack([w0, w1], axis=1)


# ---------------------------------------------------------------------------------------
# network weights
# ---------------------------------------------------------------------------------------

def _uniform_array(seed: int, count: int) -> np.ndarray:
    return (splitmix64_array(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def _normal_array(seed: int, count: int) -> np.ndarray:
    """Box-Muller in float64 over pairs of counter-based uniforms."""
    m = (count + 1) // 2
    u1 = (_uniform_array(seed, 2 * m)[0::2] * (1 - 2.0 ** -53)) + 2.0 ** -53  # (0, 1]
    u2 = _uniform_array(seed, 2 * m)[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2 * math.pi * u2)
    z[1::2] = r * np.sin(2 * math.pi * u2)
    return z[:count]


def net_weights(dims, init: str, seed: int):
    """Seeded MLP weights. dims = [in, h1, ..., out].  Layer l has W[l] of shape
    (dims[l+1], dims[l]) (row-major, float32) and b[l] of shape (dims[l+1],).

    init = "uniform": W and b ~ U(-1/sqrt(fan_in), +1/sqrt(fan_in));
    init = "kaiming": W ~ N(0, 2/fan_in), b = 0.
    Layer l draws W from seed_for(seed, 2l) and b from seed_for(seed, 2l+1)."""
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        sw, sb = seed_for(seed, 2 * l), seed_for(seed, 2 * l + 1)
        if init == "uniform":
            a = 1.0 / math.sqrt(fi)
            W = a * (2.0 * _uniform_array(sw, fo * fi) - 1.0)
            b = a * (2.0 * _uniform_array(sb, fo) - 1.0)
        elif init == "kaiming":
            W = math.sqrt(2.0 / fi) * _normal_array(sw, fo * fi)
            b = np.zeros(fo)
        else:
            raise ValueError(init)
        Ws.append(W.reshape(fo, fi).astype(np.float32))
        bs.append(b.astype(np.float32))
    return Ws, bs


# The networks of the five workload configurations (one-hot width first).
NET_C0 = dict(dims=[81, 256, 256, 1], init="uniform", seed=0)
NET_C1 = dict(dims=[256, 1024, 1024, 512, 1], init="kaiming", seed=1)
NET_C2 = dict(dims=[480, 2048, 2048, 1024, 21], init="kaiming", seed=2)
NET_C3 = dict(dims=[256, 1024, 1024, 512, 81], init="kaiming", seed=3)

# instance tags (seed_for(tag, i) gives instance i's seed)
TAG_C0, TAG_C1, TAG_C2, TAG_C3, TAG_C4 = 0xC0, 0xC1, 0xC2, 0xC3, 0xC4

# 15-puzzle tile partitions for additive PDBs (tile numbers = goal cells): the 6-6-3 split used
# for the training labels, and the 7-8 split of the paper's own STP heuristic (tiles 1-7 and
# 8-15; tables of 16!/9! = 57,657,600 and 16!/8! = 518,918,400 one-byte entries).
PATTERNS_663 = ([1, 2, 3, 5, 6, 7], [4, 8, 9, 12, 13, 14], [10, 11, 15])
PATTERNS_78 = ([1, 2, 3, 4, 5, 6, 7], [8, 9, 10, 11, 12, 13, 14, 15])
