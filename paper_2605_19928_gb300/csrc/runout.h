// All-in run-outs evaluated in one step (runout.cu).
//
// A run-out is a chance node below a decision whose subtree holds only chance and showdown
// nodes: both players are all in and the remaining board cards are dealt.  Its value for hand
// h of player i is the sum over its boards of the showdown values (Stage 4), each carrying the
// probability of its cards; every board of a run-out has the same payoff scale u (chips in x
// probability x 1/Z), so the sum is
//     v_i(h) = u sum_o E[h][o] q(o),
// q the opponent's reach at the run-out's top node and E[h][o] the number of the run-out's
// boards on which h beats o less the number on which it loses, over the boards that share no
// card with h or o (0 if h and o share a card).  E depends on the board at the top node only,
// so it is built once per distinct run-out board.
#pragma once

#include <cstdint>

#include "pcfr_internal.h"

namespace pcfr {

struct RunoutItem {   // one run-out top node
  int32_t node;
  int32_t table;      // its table
  float u;            // payoff scale of its showdowns, FP32
  int32_t pad;
};

struct RunoutTable {  // E of one run-out board, stored [o][hstride] as unsigned with a bias
  int64_t offset;     // byte offset in the table pool (256-byte aligned)
  int32_t wide;       // 0: uint8 entries, E + 128 (at most 127 boards); 1: uint16, E + 32768
  int32_t n_boards;
  int32_t board0;     // its first entry in the board list
  int32_t pad;
};

struct RunoutGroup {  // up to kRunoutGroup top nodes of one table, evaluated by one block
  int32_t table;
  int32_t item0;      // its first item (items sorted by table)
  int32_t count;
  int32_t pad;
};
constexpr int kRunoutGroup = 8;

struct RunoutBoard {  // one showdown board of a run-out table
  uint64_t cards;     // the board's public cards
  int32_t table;      // its showdown board table (rank tie-group starts per hand)
  int32_t pad;
};

// E of every table from the hands' tie-group starts on each showdown board (gs: [board
// table][n_hands] int32, higher = stronger, equal = tie).  One launch.
int launch_runout_build(const RunoutTable* tables, int n_tables, const RunoutBoard* boards, const int32_t* gs,
                        const uint64_t* hand_mask, int n_hands, int hstride, unsigned char* pool, void* stream);

// Values of the players in player_mask (1, 2 or 3) at every run-out top node of game 0, from
// the opponent's reach (use_bar: the average-strategy reach, into cfv_br), FP32 values.  The
// groups8 use uint8 tables, groups16 uint16 ones; items are the top nodes, sorted by table.
// One launch per non-empty group list.
int launch_runout_values(const GameDev* games, const RunoutItem* items, const RunoutGroup* groups8, int n8,
                         const RunoutGroup* groups16, int n16, const RunoutTable* tables, const unsigned char* pool,
                         int n_hands, int player_mask, int use_bar, void* stream);

}  // namespace pcfr
