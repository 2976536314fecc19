// domain.h -- host-side domain code of the product: packed sliding-tile and cube states,
// their moves and move pruning, the goal test and Manhattan distance.  The search workers
// (Algorithm 3's env.GetActions / env.ApplyAction) run on these.
#pragma once
#include <stdint.h>

namespace cbdfs {

// A search state as the workers keep it.  STP: w[0] packed, `blank` cached.  RC: w[0..1].
struct State {
    uint64_t w[2];
    int8_t blank;
};

struct Domain {
    int dom;    // cbdfs_domain
    int side;   // STP side (0 for RC)
    int words;  // packed words per state
    uint64_t goal[2];

    explicit Domain(int d);
    bool is_goal(const State &s) const { return s.w[0] == goal[0] && (words == 1 || s.w[1] == goal[1]); }
    State make(const uint64_t *packed) const;
    // Children of s given the move that produced s (-1 at the root): STP blank moves except
    // the reverse of the last one; RC turns on faces the canonical order allows.  Writes up
    // to 18 states and their moves; returns the count.
    int children(const State &s, int last, State *out, int8_t *moves) const;
    // Apply one move; false if it is illegal.
    bool apply(State &s, int move) const;
    int manhattan(uint64_t w0) const;
};

// The cube's corner moves: for move m and a cubie on slot s, its new slot dst[m][s] and the
// twist add[m][s] it gains (mod 3).
void rc_corner_moves(uint8_t dst[18][8], uint8_t add[18][8]);

}  // namespace cbdfs
