// domain.cpp -- sliding-tile puzzle and Rubik's cube moves for the search workers.
//
// The cube is kept per cubie: corner cubie c's 5-bit field is slot*3 + twist, edge cubie
// e's is slot*2 + flip.  A clockwise quarter turn of a face carries the four cubies of the
// face around a 4-cycle of slots; each cubie gains a twist (corners) or flip (edges) that
// depends on the slot it arrives in.  The cycles below are listed in travel order.
#include "domain.h"

#include <cstring>

#include "../../include/cbdfs.h"

namespace cbdfs {
namespace {

enum { URF, UFL, ULB, UBR, DFR, DLF, DBL, DRB };
enum { UR, UF, UL, UB, DR, DF, DL, DB, FR, FL, BL, BR };

struct FaceCycle {
    int corner[4], corner_twist_on_arrival[4];
    int edge[4], edge_flip_on_arrival[4];
};

// faces U R F D L B; travel order a -> b -> c -> d -> a; the twist/flip entries belong to the
// slot arrived at (same position in the list)
const FaceCycle kFaces[6] = {
    /* U */ {{URF, UFL, ULB, UBR}, {0, 0, 0, 0}, {UR, UF, UL, UB}, {0, 0, 0, 0}},
    /* R */ {{DFR, URF, UBR, DRB}, {1, 2, 1, 2}, {FR, UR, BR, DR}, {0, 0, 0, 0}},
    /* F */ {{UFL, URF, DFR, DLF}, {2, 1, 2, 1}, {FL, UF, FR, DF}, {1, 1, 1, 1}},
    /* D */ {{DFR, DRB, DBL, DLF}, {0, 0, 0, 0}, {DR, DB, DL, DF}, {0, 0, 0, 0}},
    /* L */ {{UFL, DLF, DBL, ULB}, {1, 2, 1, 2}, {UL, FL, DL, BL}, {0, 0, 0, 0}},
    /* B */ {{UBR, ULB, DBL, DRB}, {2, 1, 2, 1}, {BR, UB, BL, DB}, {1, 1, 1, 1}},
};

// per move (face*3 + quarter turns-1): destination slot and orientation delta per source slot
struct MoveTable {
    uint8_t cdst[18][8], cadd[18][8], edst[18][12], eadd[18][12];
    MoveTable() {
        for (int f = 0; f < 6; ++f) {
            // one quarter turn
            uint8_t cd[8], ca[8], ed[12], ea[12];
            for (int s = 0; s < 8; ++s) { cd[s] = s; ca[s] = 0; }
            for (int s = 0; s < 12; ++s) { ed[s] = s; ea[s] = 0; }
            const FaceCycle &F = kFaces[f];
            for (int i = 0; i < 4; ++i) {
                const int from = F.corner[i], to = F.corner[(i + 1) & 3];
                cd[from] = to;
                ca[from] = F.corner_twist_on_arrival[(i + 1) & 3];
                const int efrom = F.edge[i], eto = F.edge[(i + 1) & 3];
                ed[efrom] = eto;
                ea[efrom] = F.edge_flip_on_arrival[(i + 1) & 3];
            }
            // compose q quarter turns
            uint8_t pd[8], pa[8], qd[12], qa[12];
            for (int s = 0; s < 8; ++s) { pd[s] = s; pa[s] = 0; }
            for (int s = 0; s < 12; ++s) { qd[s] = s; qa[s] = 0; }
            for (int q = 0; q < 3; ++q) {
                for (int s = 0; s < 8; ++s) {
                    pa[s] = (pa[s] + ca[pd[s]]) % 3;
                    pd[s] = cd[pd[s]];
                }
                for (int s = 0; s < 12; ++s) {
                    qa[s] = (qa[s] + ea[qd[s]]) % 2;
                    qd[s] = ed[qd[s]];
                }
                const int m = 3 * f + q;
                memcpy(cdst[m], pd, 8);
                memcpy(cadd[m], pa, 8);
                memcpy(edst[m], qd, 12);
                memcpy(eadd[m], qa, 12);
            }
        }
    }
};
const MoveTable kMoves;

inline void rc_apply(uint64_t *w, int m) {
    uint64_t c = 0, e = 0;
    for (int k = 0; k < 8; ++k) {
        const int f = (int)((w[0] >> (5 * k)) & 31u), s = f / 3, t = f % 3;
        const int nt = (t + kMoves.cadd[m][s]) % 3;
        c |= (uint64_t)(kMoves.cdst[m][s] * 3 + nt) << (5 * k);
    }
    for (int k = 0; k < 12; ++k) {
        const int f = (int)((w[1] >> (5 * k)) & 31u), s = f >> 1, t = f & 1;
        e |= (uint64_t)(kMoves.edst[m][s] * 2 + (t ^ kMoves.eadd[m][s])) << (5 * k);
    }
    w[0] = c;
    w[1] = e;
}

}  // namespace

void rc_corner_moves(uint8_t dst[18][8], uint8_t add[18][8]) {
    memcpy(dst, kMoves.cdst, sizeof(kMoves.cdst));
    memcpy(add, kMoves.cadd, sizeof(kMoves.cadd));
}

Domain::Domain(int d) : dom(d) {
    goal[0] = goal[1] = 0;
    if (d == CBDFS_DOM_RC3) {
        side = 0;
        words = 2;
        for (int k = 0; k < 8; ++k) goal[0] |= (uint64_t)(k * 3) << (5 * k);
        for (int k = 0; k < 12; ++k) goal[1] |= (uint64_t)(k * 2) << (5 * k);
    } else {
        side = d == CBDFS_DOM_STP3 ? 3 : 4;
        words = 1;
        for (int t = 0; t < side * side; ++t) goal[0] |= (uint64_t)t << (4 * t);
    }
}

State Domain::make(const uint64_t *packed) const {
    State s;
    s.w[0] = packed[0];
    s.w[1] = words == 2 ? packed[1] : 0;
    s.blank = -1;
    if (words == 1)
        for (int p = 0; p < side * side; ++p)
            if (((s.w[0] >> (4 * p)) & 15u) == 0) s.blank = (int8_t)p;
    return s;
}

bool Domain::apply(State &s, int m) const {
    if (words == 2) {
        if (m < 0 || m >= 18) return false;
        rc_apply(s.w, m);
        return true;
    }
    if (m < 0 || m > 3) return false;
    const int b = s.blank, r = b / side, c = b % side;
    int q;
    switch (m) {
    case 0: if (r == 0) return false; q = b - side; break;
    case 1: if (c == 0) return false; q = b - 1; break;
    case 2: if (c == side - 1) return false; q = b + 1; break;
    default: if (r == side - 1) return false; q = b + side; break;
    }
    const uint64_t t = (s.w[0] >> (4 * q)) & 15u;
    s.w[0] = (s.w[0] & ~((uint64_t)15 << (4 * q))) | (t << (4 * b));
    s.blank = (int8_t)q;
    return true;
}

int Domain::children(const State &s, int last, State *out, int8_t *moves) const {
    int n = 0;
    if (words == 2) {
        const int pf = last < 0 ? -1 : last / 3;
        for (int f = 0; f < 6; ++f) {
            if (pf >= 0 && (f == pf || (f == (pf + 3) % 6 && f < pf))) continue;
            for (int q = 0; q < 3; ++q) {
                out[n] = s;
                rc_apply(out[n].w, 3 * f + q);
                moves[n++] = (int8_t)(3 * f + q);
            }
        }
        return n;
    }
    for (int m = 0; m < 4; ++m) {
        if (last >= 0 && m == 3 - last) continue;
        out[n] = s;
        if (apply(out[n], m)) moves[n++] = (int8_t)m;
    }
    return n;
}

int Domain::manhattan(uint64_t w0) const {
    int md = 0;
    for (int p = 0; p < side * side; ++p) {
        const int t = (int)((w0 >> (4 * p)) & 15u);
        if (!t) continue;
        const int dr = p / side - t / side, dc = p % side - t % side;
        md += (dr < 0 ? -dr : dr) + (dc < 0 ? -dc : dc);
    }
    return md;
}

}  // namespace cbdfs

extern "C" {

int cbdfs_apply_moves(int domain, const uint64_t *start, const int *moves, int n, uint64_t *out) {
    if (domain < 0 || domain > 2 || !start || !out || (n > 0 && !moves)) return CBDFS_EINVAL;
    cbdfs::Domain D(domain);
    cbdfs::State s = D.make(start);
    if (D.words == 1 && s.blank < 0) return CBDFS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!D.apply(s, moves[i])) return CBDFS_EINVAL;
    out[0] = s.w[0];
    if (D.words == 2) out[1] = s.w[1];
    return CBDFS_OK;
}

int cbdfs_manhattan(int domain, uint64_t state) {
    if (domain != CBDFS_DOM_STP3 && domain != CBDFS_DOM_STP4) return CBDFS_EINVAL;
    return cbdfs::Domain(domain).manhattan(state);
}

}  // extern "C"
