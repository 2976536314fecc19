/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the batched CB-DFS hot path
 * computes, written from the paper (arXiv 2507.11916) and from the textbook definitions
 * it relies on.  Only the tests, the smoke check and the bench's CPU-baseline leg may load
 * this file's library; the product library never links or calls it, and it shares no code
 * with the product.
 *
 * Contents
 *   - sliding-tile puzzle (STP): packed nibble states, blank moves with parent pruning
 *     (the paper's "path information is maintained to prevent the search from returning
 *     to the parents", Background, AIDA* distributed node assignment), Manhattan distance.
 *   - 3x3 Rubik's cube (RC): cubie-level states, 18 face turns, the canonical move
 *     pruning (no face twice in a row; opposite faces in one order only).
 *   - breadth-first search over the 8-puzzle (full) and over RC (shallow depths).
 *   - pattern databases (Background, Heuristics): an abstraction keeps the positions of
 *     a set of pattern tiles; additive costs count only moves of pattern tiles; the table
 *     holds the abstract distance, minimised over the blank position.
 *   - one cost-bounded depth-first search (CB-DFS, Background: IDA* and BTS) with an
 *     optional expansion limit (the BTS enhancement section), counting expanded and
 *     generated nodes and the smallest f above the bound.  The IDA* and BTS drivers that call
 *     it are in the Python half of the oracle.
 *
 * Conventions that the paper leaves open and this oracle fixes:
 *   - expand a node iff g + h <= bound (the proof of the theorem states f <= threshold);
 *   - a goal is recognised when its node is taken, with h(goal) = 0, so a goal whose
 *     g <= bound ends (or, in complete mode, is recorded by) the iteration;
 *   - "expanded" counts nodes that pass the bound and are not the goal; "generated"
 *     counts children of expanded nodes; the root is evaluated but not generated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ======================================================================================
 * sliding-tile puzzle
 * ==================================================================================== */

static int stp_tile(uint64_t s, int p) { return (int)((s >> (4 * p)) & 15u); }

static uint64_t stp_goal(int side) {
    uint64_t g = 0;
    for (int t = 0; t < side * side; ++t) g |= (uint64_t)t << (4 * t);
    return g;
}

int or_stp_md(uint64_t s, int side) {
    int md = 0;
    for (int p = 0; p < side * side; ++p) {
        int t = stp_tile(s, p);
        if (t == 0) continue;
        int dr = p / side - t / side, dc = p % side - t % side;
        md += (dr < 0 ? -dr : dr) + (dc < 0 ? -dc : dc);
    }
    return md;
}

static int stp_blank(uint64_t s, int side) {
    for (int p = 0; p < side * side; ++p)
        if (stp_tile(s, p) == 0) return p;
    return -1;
}

/* Move the blank in direction d (0 up, 1 left, 2 right, 3 down). Returns 1 if legal. */
int or_stp_apply(uint64_t s, int side, int d, uint64_t *out) {
    int b = stp_blank(s, side);
    int r = b / side, c = b % side;
    static const int DR[4] = {-1, 0, 0, 1}, DC[4] = {0, -1, 1, 0};
    int nr = r + DR[d], nc = c + DC[d];
    if (nr < 0 || nr >= side || nc < 0 || nc >= side) return 0;
    int q = nr * side + nc;
    uint64_t t = (s >> (4 * q)) & 15u;
    s &= ~((uint64_t)15 << (4 * q));      /* cell q becomes the blank */
    s |= t << (4 * b);                    /* its tile moves onto the old blank cell */
    *out = s;
    return 1;
}

/* Apply a direction sequence starting from the goal. Returns 0 on an illegal move. */
int or_stp_apply_walk(int side, const int *dirs, int n, uint64_t *out) {
    uint64_t s = stp_goal(side);
    for (int i = 0; i < n; ++i)
        if (!or_stp_apply(s, side, dirs[i], &s)) return 0;
    *out = s;
    return 1;
}

/* Lexicographic (Lehmer) rank of a permutation of 0..n-1. */
int64_t or_perm_rank(const int *perm, int n) {
    int64_t r = 0;
    for (int i = 0; i < n; ++i) {
        int smaller = 0;
        for (int j = i + 1; j < n; ++j)
            if (perm[j] < perm[i]) ++smaller;
        r = r * (n - i) + smaller;
    }
    return r;
}

static void perm_unrank(int64_t r, int n, int *perm) {
    int digits[16];
    for (int i = n - 1; i >= 0; --i) {
        digits[i] = (int)(r % (n - i));
        r /= (n - i);
    }
    int used[16] = {0};
    for (int i = 0; i < n; ++i) {
        int k = digits[i];
        for (int v = 0; v < n; ++v) {
            if (used[v]) continue;
            if (k-- == 0) { perm[i] = v; used[v] = 1; break; }
        }
    }
}

/* Full breadth-first search of the 8-puzzle from the goal.  dist[rank(cells)] receives the
 * optimal distance of every state (-1 if unreachable).  Returns the number reached. */
int64_t or_stp3_bfs(int8_t *dist, int *maxd) {
    const int N = 362880;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * N);
    memset(dist, -1, N);
    int cells[9];
    for (int p = 0; p < 9; ++p) cells[p] = p;
    int32_t g = (int32_t)or_perm_rank(cells, 9);
    dist[g] = 0;
    int64_t head = 0, tail = 0;
    queue[tail++] = g;
    int md = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        perm_unrank(u, 9, cells);
        uint64_t s = 0;
        for (int p = 0; p < 9; ++p) s |= (uint64_t)cells[p] << (4 * p);
        for (int d = 0; d < 4; ++d) {
            uint64_t c;
            if (!or_stp_apply(s, 3, d, &c)) continue;
            int cc[9];
            for (int p = 0; p < 9; ++p) cc[p] = stp_tile(c, p);
            int32_t v = (int32_t)or_perm_rank(cc, 9);
            if (dist[v] < 0) {
                dist[v] = (int8_t)(dist[u] + 1);
                if (dist[v] > md) md = dist[v];
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    *maxd = md;
    return tail;
}

/* ======================================================================================
 * Rubik's cube, cubie level.  Quarter turns (clockwise seen from the face) in
 * "replaced-by" form: after the turn, slot i holds the cubie that was in slot P[i], with
 * its orientation increased by O[i].  Corner slots URF UFL ULB UBR DFR DLF DBL DRB, edge
 * slots UR UF UL UB DR DF DL DB FR FL BL BR, faces U R F D L B.  Corner twist counts the
 * clockwise turns of the cubie's U/D facelet; an edge is flipped when its reference facelet
 * (U/D facelet, else F/B facelet) sits off the slot's reference face.
 * ==================================================================================== */

enum { URF, UFL, ULB, UBR, DFR, DLF, DBL, DRB };
enum { UR, UF, UL, UB, DR, DF, DL, DB, FR, FL, BL, BR };

static const int RC_CP[6][8] = {
    {UBR, URF, UFL, ULB, DFR, DLF, DBL, DRB}, /* U */
    {DFR, UFL, ULB, URF, DRB, DLF, DBL, UBR}, /* R */
    {UFL, DLF, ULB, UBR, URF, DFR, DBL, DRB}, /* F */
    {URF, UFL, ULB, UBR, DLF, DBL, DRB, DFR}, /* D */
    {URF, ULB, DBL, UBR, DFR, UFL, DLF, DRB}, /* L */
    {URF, UFL, UBR, DRB, DFR, DLF, ULB, DBL}, /* B */
};
static const int RC_CO[6][8] = {
    {0, 0, 0, 0, 0, 0, 0, 0}, {2, 0, 0, 1, 1, 0, 0, 2}, {1, 2, 0, 0, 2, 1, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0}, {0, 1, 2, 0, 0, 2, 1, 0}, {0, 0, 1, 2, 0, 0, 2, 1},
};
static const int RC_EP[6][12] = {
    {UB, UR, UF, UL, DR, DF, DL, DB, FR, FL, BL, BR}, /* U */
    {FR, UF, UL, UB, BR, DF, DL, DB, DR, FL, BL, UR}, /* R */
    {UR, FL, UL, UB, DR, FR, DL, DB, UF, DF, BL, BR}, /* F */
    {UR, UF, UL, UB, DF, DL, DB, DR, FR, FL, BL, BR}, /* D */
    {UR, UF, BL, UB, DR, DF, FL, DB, FR, UL, DL, BR}, /* L */
    {UR, UF, UL, BR, DR, DF, DL, BL, FR, FL, UB, DB}, /* B */
};
static const int RC_EO[6][12] = {
    {0}, {0}, {0, 1, 0, 0, 0, 1, 0, 0, 1, 1, 0, 0},
    {0}, {0}, {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 1, 1},
};

typedef struct { int cp[8], co[8], ep[12], eo[12]; } rc_cube;

static void rc_unpack(const uint64_t *w, rc_cube *c) {
    for (int k = 0; k < 8; ++k) {
        int f = (int)((w[0] >> (5 * k)) & 31u);
        c->cp[f / 3] = k;
        c->co[f / 3] = f % 3;
    }
    for (int k = 0; k < 12; ++k) {
        int f = (int)((w[1] >> (5 * k)) & 31u);
        c->ep[f / 2] = k;
        c->eo[f / 2] = f % 2;
    }
}

static void rc_pack(const rc_cube *c, uint64_t *w) {
    w[0] = w[1] = 0;
    for (int s = 0; s < 8; ++s) w[0] |= (uint64_t)(s * 3 + c->co[s]) << (5 * c->cp[s]);
    for (int s = 0; s < 12; ++s) w[1] |= (uint64_t)(s * 2 + c->eo[s]) << (5 * c->ep[s]);
}

static void rc_quarter(rc_cube *c, int face) {
    rc_cube n;
    for (int i = 0; i < 8; ++i) {
        n.cp[i] = c->cp[RC_CP[face][i]];
        n.co[i] = (c->co[RC_CP[face][i]] + RC_CO[face][i]) % 3;
    }
    for (int i = 0; i < 12; ++i) {
        n.ep[i] = c->ep[RC_EP[face][i]];
        n.eo[i] = (c->eo[RC_EP[face][i]] + RC_EO[face][i]) % 2;
    }
    *c = n;
}

/* move m = 3*face + (quarter turns - 1) */
void or_rc_apply(const uint64_t *in, int m, uint64_t *out) {
    rc_cube c;
    rc_unpack(in, &c);
    for (int q = 0; q <= m % 3; ++q) rc_quarter(&c, m / 3);
    rc_pack(&c, out);
}

static void rc_goal(uint64_t *w) {
    w[0] = w[1] = 0;
    for (int k = 0; k < 8; ++k) w[0] |= (uint64_t)(k * 3) << (5 * k);
    for (int k = 0; k < 12; ++k) w[1] |= (uint64_t)(k * 2) << (5 * k);
}

void or_rc_apply_seq(const int *moves, int n, uint64_t *out) {
    uint64_t w[2];
    rc_goal(w);
    for (int i = 0; i < n; ++i) or_rc_apply(w, moves[i], w);
    out[0] = w[0];
    out[1] = w[1];
}

/* Bit 0: twist sum not 0 mod 3; bit 1: flip sum odd; bit 2: corner and edge permutation
 * parities differ; bit 3: a field is out of range or two cubies share a slot. */
int or_rc_invariants(const uint64_t *w) {
    int cseen[8] = {0}, eseen[12] = {0}, bad = 0, tw = 0, fl = 0;
    int cslot[8], eslot[12];
    for (int k = 0; k < 8; ++k) {
        int f = (int)((w[0] >> (5 * k)) & 31u);
        if (f >= 24 || cseen[f / 3]++) bad |= 8;
        cslot[k] = f / 3 % 8;
        tw += f % 3;
    }
    for (int k = 0; k < 12; ++k) {
        int f = (int)((w[1] >> (5 * k)) & 31u);
        if (f >= 24 || eseen[f / 2]++) bad |= 8;
        eslot[k] = f / 2 % 12;
        fl += f % 2;
    }
    if (tw % 3) bad |= 1;
    if (fl % 2) bad |= 2;
    int pc = 0, pe = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = i + 1; j < 8; ++j) pc += cslot[i] > cslot[j];
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j) pe += eslot[i] > eslot[j];
    if ((pc & 1) != (pe & 1)) bad |= 4;
    return bad;
}

/* canonical successor rule: face f may follow face p iff f != p and not (f opposite p and
 * f < p).  p < 0 means no previous move. */
static int rc_face_ok(int p, int f) {
    if (p < 0) return 1;
    if (f == p) return 0;
    if (f == (p + 3) % 6 && f < p) return 0;
    return 1;
}

/* simple open-addressing set of 128-bit states */
typedef struct { uint64_t *k; uint8_t *used; uint64_t cap, n; } set128;
static uint64_t h128(uint64_t a, uint64_t b) {
    uint64_t z = a * 0x9E3779B97F4A7C15ull ^ (b + 0x632BE59BD9B4E019ull) * 0xBF58476D1CE4E5B9ull;
    return z ^ (z >> 31);
}
static int set_insert(set128 *s, const uint64_t *w) {
    uint64_t i = h128(w[0], w[1]) & (s->cap - 1);
    while (s->used[i]) {
        if (s->k[2 * i] == w[0] && s->k[2 * i + 1] == w[1]) return 0;
        i = (i + 1) & (s->cap - 1);
    }
    s->used[i] = 1;
    s->k[2 * i] = w[0];
    s->k[2 * i + 1] = w[1];
    s->n++;
    return 1;
}

/* Breadth-first search over RC to maxdepth (<= 5).  distinct[d] = number of states first
 * reached at depth d (all 18 moves); tree[d] = number of canonical move sequences of
 * length d. */
int or_rc_bfs_counts(int maxdepth, int64_t *distinct, int64_t *tree) {
    if (maxdepth > 5) return -1;
    set128 seen;
    seen.cap = 1u << 24;
    seen.k = (uint64_t *)calloc(2 * seen.cap, sizeof(uint64_t));
    seen.used = (uint8_t *)calloc(seen.cap, 1);
    seen.n = 0;
    uint64_t *level = (uint64_t *)malloc(2 * sizeof(uint64_t) * 1);
    int64_t nlevel = 1;
    rc_goal(level);
    set_insert(&seen, level);
    distinct[0] = 1;
    for (int d = 1; d <= maxdepth; ++d) {
        uint64_t *next = (uint64_t *)malloc(2 * sizeof(uint64_t) * (size_t)nlevel * 18);
        int64_t nn = 0;
        for (int64_t i = 0; i < nlevel; ++i)
            for (int m = 0; m < 18; ++m) {
                uint64_t c[2];
                or_rc_apply(&level[2 * i], m, c);
                if (set_insert(&seen, c)) {
                    next[2 * nn] = c[0];
                    next[2 * nn + 1] = c[1];
                    ++nn;
                }
            }
        free(level);
        level = next;
        nlevel = nn;
        distinct[d] = nn;
    }
    free(level);
    free(seen.k);
    free(seen.used);
    /* canonical sequence counts by dynamic programming over the last face */
    int64_t byface[6];
    for (int f = 0; f < 6; ++f) byface[f] = 3;
    tree[0] = 1;
    if (maxdepth >= 1) tree[1] = 18;
    for (int d = 2; d <= maxdepth; ++d) {
        int64_t nb[6] = {0};
        for (int p = 0; p < 6; ++p)
            for (int f = 0; f < 6; ++f)
                if (rc_face_ok(p, f)) nb[f] += 3 * byface[p];
        int64_t tot = 0;
        for (int f = 0; f < 6; ++f) { byface[f] = nb[f]; tot += nb[f]; }
        tree[d] = tot;
    }
    return 0;
}

/* ======================================================================================
 * pattern databases over the sliding-tile puzzle
 * ==================================================================================== */

/* number of k-permutations of n: n! / (n-k)! */
int64_t or_npk(int n, int k) {
    int64_t r = 1;
    for (int i = 0; i < k; ++i) r *= (n - i);
    return r;
}

/* Lexicographic rank of the position vector pos[0..k-1] (distinct cells in 0..n-1)
 * among all k-permutations of n cells. */
int64_t or_pdb_rank(const int *pos, int k, int n) {
    int64_t r = 0;
    for (int i = 0; i < k; ++i) {
        int d = pos[i];
        for (int j = 0; j < i; ++j)
            if (pos[j] < pos[i]) --d;
        r += d * or_npk(n - 1 - i, k - 1 - i);
    }
    return r;
}

static void pdb_unrank(int64_t r, int k, int n, int *pos) {
    int used[16] = {0};
    for (int i = 0; i < k; ++i) {
        int64_t w = or_npk(n - 1 - i, k - 1 - i);
        int d = (int)(r / w);
        r %= w;
        for (int v = 0; v < n; ++v) {
            if (used[v]) continue;
            if (d-- == 0) { pos[i] = v; used[v] = 1; break; }
        }
    }
}

typedef struct { int32_t *a; int64_t n, cap; } ivec;
static void ivec_push(ivec *v, int32_t x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? v->cap * 2 : 1024;
        v->a = (int32_t *)realloc(v->a, sizeof(int32_t) * v->cap);
    }
    v->a[v->n++] = x;
}

/* Build the additive pattern database for the pattern tiles[0..k-1] on a side x side
 * puzzle.  Abstract states are (positions of the pattern tiles, blank cell); a blank move
 * that displaces a pattern tile costs 1, any other blank move costs 0.  A breadth-first
 * search by cost levels runs from the goal placement (tile t on cell t, blank on cell 0);
 * within a level the zero-cost moves are closed first.  table[rank(pos)] receives the
 * least distance over all blank cells; 255 marks a placement never reached.
 * Returns the number of abstract (placement, blank) states reached, or -1. */
int64_t or_pdb_build(int side, const int *tiles, int k, uint8_t *table) {
    const int n = side * side;
    const int64_t P = or_npk(n, k);
    const int64_t S = P * n;                       /* (rank, blank) index space */
    uint8_t *dist = (uint8_t *)malloc((size_t)S);
    if (!dist) return -1;
    memset(dist, 255, (size_t)S);
    int pos[16];
    for (int i = 0; i < k; ++i) pos[i] = tiles[i];
    int64_t start = or_pdb_rank(pos, k, n) * n + 0;
    dist[start] = 0;
    ivec cur = {0}, nxt = {0};
    ivec_push(&cur, (int32_t)start);
    int64_t reached = 1;
    static const int DR[4] = {-1, 0, 0, 1}, DC[4] = {0, -1, 1, 0};
    for (int d = 0; cur.n > 0; ++d) {
        for (int64_t qi = 0; qi < cur.n; ++qi) {     /* cur grows while zero-cost moves land */
            int64_t u = cur.a[qi];
            if (dist[u] != d) continue;                 /* stale entry */
            int64_t r = u / n;
            int b = (int)(u % n);
            pdb_unrank(r, k, n, pos);
            for (int m = 0; m < 4; ++m) {
                int nr = b / side + DR[m], nc = b % side + DC[m];
                if (nr < 0 || nr >= side || nc < 0 || nc >= side) continue;
                int c = nr * side + nc;
                int who = -1;
                for (int i = 0; i < k; ++i)
                    if (pos[i] == c) who = i;
                int64_t v;
                int cost;
                if (who < 0) {
                    v = r * n + c;
                    cost = 0;
                } else {
                    pos[who] = b;
                    v = or_pdb_rank(pos, k, n) * n + c;
                    pos[who] = c;
                    cost = 1;
                }
                int nd = d + cost;
                if (dist[v] == 255) ++reached;
                if (dist[v] == 255 || dist[v] > nd) {
                    dist[v] = (uint8_t)nd;
                    if (cost == 0) ivec_push(&cur, (int32_t)v);
                    else ivec_push(&nxt, (int32_t)v);
                }
            }
        }
        ivec t = cur;
        cur = nxt;
        nxt = t;
        nxt.n = 0;
    }
    free(cur.a);
    free(nxt.a);
    for (int64_t r = 0; r < P; ++r) {
        uint8_t best = 255;
        for (int b = 0; b < n; ++b)
            if (dist[r * n + b] < best) best = dist[r * n + b];
        table[r] = best;
    }
    free(dist);
    return reached;
}

/* The part of a pattern database within distance maxd of the goal, found by the same
 * cost-level search as or_pdb_build but stopped after level maxd and kept in a hash set, so
 * that it can check tables far too large to build here.  Writes every placement whose
 * least distance over blank cells is <= maxd (rank, value) into out_rank/out_val, sorted
 * by rank; returns how many, or -1 if more than cap (rank, blank) states were reached. */
typedef struct { int64_t *a; int64_t n, cap; } lvec;
static void lvec_push(lvec *v, int64_t x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? v->cap * 2 : 1024;
        v->a = (int64_t *)realloc(v->a, sizeof(int64_t) * v->cap);
    }
    v->a[v->n++] = x;
}

typedef struct { uint64_t *key; uint8_t *val; uint64_t mask; int64_t used; } hset;
static uint8_t *hset_slot(hset *h, uint64_t key, int *fresh) {
    uint64_t i = (key * 0x9E3779B97F4A7C15ull) >> 20 & h->mask;
    while (h->key[i] && h->key[i] != key + 1) i = (i + 1) & h->mask;
    *fresh = h->key[i] == 0;
    if (*fresh) { h->key[i] = key + 1; h->val[i] = 255; h->used++; }
    return &h->val[i];
}

static int cmp_pair(const void *x, const void *y) {
    const int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

int64_t or_pdb_ball(int side, const int *tiles, int k, int maxd, int64_t cap, int64_t *out_rank,
                    uint8_t *out_val) {
    const int n = side * side;
    uint64_t size = 1;
    while (size < (uint64_t)cap * 2) size <<= 1;
    hset h = {(uint64_t *)calloc(size, 8), (uint8_t *)malloc(size), size - 1, 0};
    if (!h.key || !h.val) return -1;
    int pos[16], fresh;
    for (int i = 0; i < k; ++i) pos[i] = tiles[i];
    const int64_t start = or_pdb_rank(pos, k, n) * n + 0;
    *hset_slot(&h, (uint64_t)start, &fresh) = 0;
    lvec cur = {0}, nxt = {0};
    lvec_push(&cur, start);
    static const int DR[4] = {-1, 0, 0, 1}, DC[4] = {0, -1, 1, 0};
    int64_t result = 0;
    for (int d = 0; d <= maxd && cur.n > 0 && result >= 0; ++d) {
        for (int64_t qi = 0; qi < cur.n; ++qi) {
            const int64_t u = cur.a[qi];
            if (*hset_slot(&h, (uint64_t)u, &fresh) != d) continue;  /* stale entry */
            const int64_t r = u / n;
            const int b = (int)(u % n);
            pdb_unrank(r, k, n, pos);
            for (int m = 0; m < 4; ++m) {
                int nr = b / side + DR[m], nc = b % side + DC[m];
                if (nr < 0 || nr >= side || nc < 0 || nc >= side) continue;
                int c = nr * side + nc, who = -1;
                for (int i = 0; i < k; ++i)
                    if (pos[i] == c) who = i;
                int64_t v;
                int cost;
                if (who < 0) {
                    v = r * n + c;
                    cost = 0;
                } else {
                    pos[who] = b;
                    v = or_pdb_rank(pos, k, n) * n + c;
                    pos[who] = c;
                    cost = 1;
                }
                const int nd = d + cost;
                if (nd > maxd) continue;
                uint8_t *dv = hset_slot(&h, (uint64_t)v, &fresh);
                if (h.used > cap) { result = -1; break; }
                if (*dv > nd) {
                    *dv = (uint8_t)nd;
                    lvec_push(cost == 0 ? &cur : &nxt, v);
                }
            }
            if (result < 0) break;
        }
        lvec t = cur;
        cur = nxt;
        nxt = t;
        nxt.n = 0;
    }
    if (result == 0) {
        /* least value over blank cells per placement: sort (rank, value) pairs */
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(h.used ? h.used : 1));
        int64_t m = 0;
        for (uint64_t i = 0; i <= h.mask; ++i)
            if (h.key[i]) {
                pairs[2 * m] = (int64_t)(h.key[i] - 1) / n;
                pairs[2 * m + 1] = h.val[i];
                ++m;
            }
        qsort(pairs, (size_t)m, 2 * sizeof(int64_t), cmp_pair);
        for (int64_t i = 0; i < m; ++i) {
            if (result > 0 && out_rank[result - 1] == pairs[2 * i]) {
                if (pairs[2 * i + 1] < out_val[result - 1]) out_val[result - 1] = (uint8_t)pairs[2 * i + 1];
                continue;
            }
            out_rank[result] = pairs[2 * i];
            out_val[result] = (uint8_t)pairs[2 * i + 1];
            ++result;
        }
        free(pairs);
    }
    free(cur.a);
    free(nxt.a);
    free(h.key);
    free(h.val);
    return result;
}

/* Additive PDB value of an STP state: sum over patterns of table[rank(pattern positions)]. */
int or_pdb_h(uint64_t s, int side, int npat, const int *k, const int *tiles,
             const uint8_t *const *tables) {
    int n = side * side, where[16];
    for (int p = 0; p < n; ++p) where[stp_tile(s, p)] = p;
    int h = 0, off = 0;
    for (int q = 0; q < npat; ++q) {
        int pos[16];
        for (int i = 0; i < k[q]; ++i) pos[i] = where[tiles[off + i]];
        h += tables[q][or_pdb_rank(pos, k[q], n)];
        off += k[q];
    }
    return h;
}

/* ======================================================================================
 * the cube's 8-corner pattern database (Experimental Setup: the 8-corner PDB is the cube's
 * h_PDB).  Index of a corner configuration: p_c = the slot of corner cubie c, t_c its twist
 * (packed word 0, field c = 3 p_c + t_c);
 *   index = rank(p) * 3^7 + sum_{c<7} t_c 3^c,  rank(p) = sum_i (p_i - #{j<i: p_j<p_i}) (7-i)!
 * ==================================================================================== */

int64_t or_rc_corner_index(const uint64_t *w) {
    int p[8], t[8];
    for (int c = 0; c < 8; ++c) {
        const int f = (int)((w[0] >> (5 * c)) & 31u);
        p[c] = f / 3;
        t[c] = f % 3;
    }
    int64_t rank = 0, fact = 5040; /* 7! */
    for (int i = 0; i < 8; ++i) {
        int less = 0;
        for (int j = 0; j < i; ++j) less += p[j] < p[i];
        rank += (int64_t)(p[i] - less) * fact;
        if (i < 7) fact /= (7 - i);
    }
    int64_t tw = 0, pw = 1;
    for (int c = 0; c < 7; ++c) {
        tw += t[c] * pw;
        pw *= 3;
    }
    return rank * 2187 + tw;
}

/* corner configuration <-> index; c_slot[c] / c_tw[c]: slot and twist of corner cubie c */
static void corner_unindex(int64_t idx, int *c_slot, int *c_tw) {
    int64_t r = idx / 2187, tr = idx % 2187, fact = 5040;
    int used[8] = {0}, sum = 0;
    for (int i = 0; i < 8; ++i) {
        int d = (int)(r / fact);
        r %= fact;
        if (i < 7) fact /= (7 - i);
        int s = 0;
        for (;; ++s)
            if (!used[s] && d-- == 0) break;
        used[s] = 1;
        c_slot[i] = s;
    }
    for (int c = 0; c < 7; ++c) {
        c_tw[c] = (int)(tr % 3);
        tr /= 3;
        sum += c_tw[c];
    }
    c_tw[7] = (3 - sum % 3) % 3;
}

/* The full 8-corner table by breadth-first search from the solved corners (a queue of
 * indices; each configuration is expanded once).  A face turn moves the cubie at slot
 * RC_CP[f][i] to slot i, adding RC_CO[f][i] to its twist (one quarter; q quarters in a row).
 * table: 88,179,840 bytes.  Returns the largest distance, or -1 if memory runs out. */
int or_rc_corner_pdb(uint8_t *table) {
    const int64_t E = (int64_t)40320 * 2187;
    memset(table, 255, (size_t)E);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    if (!queue) return -1;
    int inv[6][8]; /* the slot a quarter turn of face f sends slot s to */
    for (int f = 0; f < 6; ++f)
        for (int i = 0; i < 8; ++i) inv[f][RC_CP[f][i]] = i;
    int64_t head = 0, tail = 0;
    table[0] = 0;
    queue[tail++] = 0;
    int maxd = 0;
    while (head < tail) {
        const int64_t u = queue[head++];
        const int du = table[u];
        int slot[8], tw[8];
        corner_unindex(u, slot, tw);
        for (int f = 0; f < 6; ++f) {
            int ns[8], nt[8];
            memcpy(ns, slot, sizeof ns);
            memcpy(nt, tw, sizeof nt);
            for (int q = 0; q < 3; ++q) {
                for (int c = 0; c < 8; ++c) {
                    const int to = inv[f][ns[c]];
                    nt[c] = (nt[c] + RC_CO[f][to]) % 3;
                    ns[c] = to;
                }
                uint64_t w[2] = {0, 0};
                for (int c = 0; c < 8; ++c) w[0] |= (uint64_t)(ns[c] * 3 + nt[c]) << (5 * c);
                const int64_t v = or_rc_corner_index(w);
                if (table[v] == 255) {
                    table[v] = (uint8_t)(du + 1);
                    if (du + 1 > maxd) maxd = du + 1;
                    queue[tail++] = (int32_t)v;
                }
            }
        }
    }
    free(queue);
    return maxd;
}

/* Every corner configuration within maxd face turns of the solved one, by breadth-first
 * search over cube states (the corners of a turn's result depend only on the corners).
 * Writes (index, distance) pairs sorted by index; returns their number, or -1 past `cap`. */
int64_t or_rc_corner_ball(int maxd, int64_t cap, int64_t *out_index, uint8_t *out_val) {
    uint64_t size = 1;
    while (size < (uint64_t)cap * 2) size <<= 1;
    hset h = {(uint64_t *)calloc(size, 8), (uint8_t *)malloc(size), size - 1, 0};
    lvec cur = {0}, nxt = {0};
    if (!h.key || !h.val) return -1;
    uint64_t g[2];
    rc_goal(g);
    int fresh;
    *hset_slot(&h, (uint64_t)or_rc_corner_index(g), &fresh) = 0;
    lvec_push(&cur, (int64_t)g[0]);  /* the corner word is the whole BFS state */
    int64_t result = 0;
    for (int d = 0; d < maxd && cur.n > 0 && result >= 0; ++d) {
        for (int64_t qi = 0; qi < cur.n && result >= 0; ++qi) {
            uint64_t w[2] = {(uint64_t)cur.a[qi], g[1]}, o[2];
            for (int m = 0; m < 18; ++m) {
                or_rc_apply(w, m, o);
                uint8_t *dv = hset_slot(&h, (uint64_t)or_rc_corner_index(o), &fresh);
                if (h.used > cap) { result = -1; break; }
                if (fresh) {
                    *dv = (uint8_t)(d + 1);
                    lvec_push(&nxt, (int64_t)o[0]);
                }
            }
        }
        lvec t = cur;
        cur = nxt;
        nxt = t;
        nxt.n = 0;
    }
    if (result == 0) {
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(h.used ? h.used : 1));
        for (uint64_t i = 0; i <= h.mask; ++i)
            if (h.key[i]) {
                pairs[2 * result] = (int64_t)(h.key[i] - 1);
                pairs[2 * result + 1] = h.val[i];
                ++result;
            }
        qsort(pairs, (size_t)result, 2 * sizeof(int64_t), cmp_pair);
        for (int64_t i = 0; i < result; ++i) {
            out_index[i] = pairs[2 * i];
            out_val[i] = (uint8_t)pairs[2 * i + 1];
        }
        free(pairs);
    }
    free(cur.a);
    free(nxt.a);
    free(h.key);
    free(h.val);
    return result;
}

/* ======================================================================================
 * one cost-bounded depth-first search
 * ==================================================================================== */

enum { OR_DOM_STP3 = 0, OR_DOM_STP4 = 1, OR_DOM_RC3 = 2 };
enum { OR_H_ZERO = 0, OR_H_MD = 1, OR_H_PDB = 2, OR_H_CALLBACK = 3 };

typedef int (*or_heur_cb)(const uint64_t *state, void *user);

typedef struct {
    int domain, hkind;
    int npat;                     /* PDB: number of patterns */
    const int *pat_k, *pat_tiles; /* PDB: sizes, concatenated tile lists */
    const uint8_t *const *tables; /* PDB: one table per pattern */
    or_heur_cb cb;
    void *user;
} or_heur;

typedef struct {
    int64_t expanded, generated;  /* this search's counts */
    int64_t minf;                 /* least f above the bound among evaluated nodes (-1: none) */
    int found;                    /* a goal with g <= bound was taken */
    int cost;                     /* its g (least over goals in complete mode) */
    int cut;                      /* the expansion limit stopped the search */
    int path_len;
    int path[256];                /* moves from the start to the goal found first/least */
} or_result;

typedef struct {
    const or_heur *h;
    int bound, complete, side;
    int64_t limit;
    or_result *res;
    int path[256];
    int stop;
} dfs_ctx;

static int dom_words(int dom) { return dom == OR_DOM_RC3 ? 2 : 1; }

static int is_goal(int dom, const uint64_t *s) {
    if (dom == OR_DOM_RC3) {
        uint64_t g[2];
        rc_goal(g);
        return s[0] == g[0] && s[1] == g[1];
    }
    return s[0] == stp_goal(dom == OR_DOM_STP3 ? 3 : 4);
}

static int eval_h(const or_heur *h, const uint64_t *s) {
    int side = h->domain == OR_DOM_STP3 ? 3 : 4;
    if (is_goal(h->domain, s)) return 0;
    switch (h->hkind) {
    case OR_H_MD: return or_stp_md(s[0], side);
    case OR_H_PDB: return or_pdb_h(s[0], side, h->npat, h->pat_k, h->pat_tiles, h->tables);
    case OR_H_CALLBACK: return h->cb(s, h->user);
    default: return 0;
    }
}

/* Children of s given the previous move (-1 at the root): STP directions 0..3 except the
 * reverse of the last one; RC moves 0..17 on faces allowed by the canonical rule. */
static int children(int dom, const uint64_t *s, int last, uint64_t *out, int *moves) {
    int nc = 0;
    if (dom == OR_DOM_RC3) {
        for (int m = 0; m < 18; ++m) {
            if (!rc_face_ok(last < 0 ? -1 : last / 3, m / 3)) continue;
            or_rc_apply(s, m, &out[2 * nc]);
            moves[nc++] = m;
        }
    } else {
        int side = dom == OR_DOM_STP3 ? 3 : 4;
        for (int d = 0; d < 4; ++d) {
            if (last >= 0 && d == 3 - last) continue;
            if (or_stp_apply(s[0], side, d, &out[nc])) moves[nc++] = d;
        }
    }
    return nc;
}

static void dfs(dfs_ctx *c, const uint64_t *s, int g, int last, int hval, int depth) {
    int w = dom_words(c->h->domain);
    int f = g + hval;
    if (f > c->bound) {
        if (c->res->minf < 0 || f < c->res->minf) c->res->minf = f;
        return;
    }
    if (is_goal(c->h->domain, s)) {
        if (!c->res->found || g < c->res->cost) {
            c->res->cost = g;
            c->res->path_len = depth;
            memcpy(c->res->path, c->path, sizeof(int) * depth);
        }
        c->res->found = 1;
        if (!c->complete) c->stop = 1;
        return;
    }
    if (c->limit >= 0 && c->res->expanded >= c->limit) {
        c->res->cut = 1;
        c->stop = 1;
        return;
    }
    c->res->expanded++;
    uint64_t kids[2 * 18];
    int moves[18];
    int nk = children(c->h->domain, s, last, kids, moves);
    c->res->generated += nk;
    for (int i = 0; i < nk && !c->stop; ++i) {
        if (depth < 256) c->path[depth] = moves[i];
        dfs(c, &kids[w * i], g + 1, moves[i], eval_h(c->h, &kids[w * i]), depth + 1);
    }
}

/* One CB-DFS from `start` with threshold `bound`.  limit < 0: no expansion limit.
 * complete != 0: keep searching after a goal and report the least goal cost.
 * Heuristic described by `kind` etc.  Returns 0. */
int or_cbdfs(int domain, const uint64_t *start, int bound, int64_t limit, int complete,
             int hkind, int npat, const int *pat_k, const int *pat_tiles,
             const uint8_t *const *tables, or_heur_cb cb, void *user, or_result *out) {
    or_heur h = {domain, hkind, npat, pat_k, pat_tiles, tables, cb, user};
    memset(out, 0, sizeof(*out));
    out->minf = -1;
    out->cost = -1;
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    c.h = &h;
    c.bound = bound;
    c.complete = complete;
    c.limit = limit;
    c.res = out;
    dfs(&c, start, 0, -1, eval_h(&h, start), 0);
    return 0;
}

/* h of a single state under the given heuristic (the goal gets 0). */
int or_heuristic(int domain, const uint64_t *s, int hkind, int npat, const int *pat_k,
                 const int *pat_tiles, const uint8_t *const *tables) {
    or_heur h = {domain, hkind, npat, pat_k, pat_tiles, tables, 0, 0};
    return eval_h(&h, s);
}

int or_result_size(void) { return (int)sizeof(or_result); }

/* ======================================================================================
 * one cost-bounded depth-first search with a real-valued heuristic
 * (section "Regression-Based Neural Heuristics": a regression network gives real h; IDA*'s
 * thresholds then move by small steps).  f = g + h in double; the bound is a double; the
 * least f above the bound is the next threshold.  Same tree rules as `dfs` above.
 * ==================================================================================== */

typedef double (*or_heur_real_cb)(const uint64_t *state, void *user);

typedef struct {
    int64_t expanded, generated;
    double minf;                  /* least f above the bound (-1: none) */
    int found, cost, cut, path_len;
    int path[256];
} or_result_real;

typedef struct {
    int domain;
    or_heur_real_cb cb;
    void *user;
    double bound;
    int complete;
    int64_t limit;
    or_result_real *res;
    int path[256];
    int stop;
} dfs_real_ctx;

static double eval_h_real(const dfs_real_ctx *c, const uint64_t *s) {
    if (is_goal(c->domain, s)) return 0.0;
    return c->cb(s, c->user);
}

static void dfs_real(dfs_real_ctx *c, const uint64_t *s, int g, int last, double hval, int depth) {
    int w = dom_words(c->domain);
    double f = (double)g + hval;
    if (f > c->bound) {
        if (c->res->minf < 0 || f < c->res->minf) c->res->minf = f;
        return;
    }
    if (is_goal(c->domain, s)) {
        if (!c->res->found || g < c->res->cost) {
            c->res->cost = g;
            c->res->path_len = depth;
            memcpy(c->res->path, c->path, sizeof(int) * depth);
        }
        c->res->found = 1;
        if (!c->complete) c->stop = 1;
        return;
    }
    if (c->limit >= 0 && c->res->expanded >= c->limit) {
        c->res->cut = 1;
        c->stop = 1;
        return;
    }
    c->res->expanded++;
    uint64_t kids[2 * 18];
    int moves[18];
    int nk = children(c->domain, s, last, kids, moves);
    c->res->generated += nk;
    for (int i = 0; i < nk && !c->stop; ++i) {
        if (depth < 256) c->path[depth] = moves[i];
        dfs_real(c, &kids[w * i], g + 1, moves[i], eval_h_real(c, &kids[w * i]), depth + 1);
    }
}

/* One CB-DFS with a real threshold; h from `cb` (the goal gets 0). */
int or_cbdfs_real(int domain, const uint64_t *start, double bound, int64_t limit, int complete,
                  or_heur_real_cb cb, void *user, or_result_real *out) {
    memset(out, 0, sizeof(*out));
    out->minf = -1;
    out->cost = -1;
    dfs_real_ctx c;
    memset(&c, 0, sizeof(c));
    c.domain = domain;
    c.cb = cb;
    c.user = user;
    c.bound = bound;
    c.complete = complete;
    c.limit = limit;
    c.res = out;
    dfs_real(&c, start, 0, -1, eval_h_real(&c, start), 0);
    return 0;
}

int or_result_real_size(void) { return (int)sizeof(or_result_real); }
