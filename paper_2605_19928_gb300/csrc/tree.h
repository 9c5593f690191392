// Host-side construction of one subgame: the public tree in level order and the per-hand
// tables the kernels read (card masks, rank-sorted showdown order, per-card hand lists).
#pragma once
#include <string>
#include <vector>

#include "pcfr.h"
#include "pcfr_internal.h"
#include "runout.h"

namespace pcfr {

struct HostGame {
  int game = 0, deck = 0, hand_size = 0, n_streets = 0;
  // public tree, level order (children of a node are consecutive)
  std::vector<NodeDev> nodes;
  std::vector<double> contrib;        // [n_nodes][2]
  std::vector<double> payoff;         // [n_nodes] terminal payoff times chance probability
  std::vector<int32_t> level_start;   // [n_levels + 1]
  int n_rows = 0;
  int row_begin[3] = {0, 0, 0};
  std::vector<int32_t> terminals;     // fold and showdown node ids
  std::vector<int32_t> leaves;        // depth-limit leaf node ids
  // node whose reach equals this node's up to zeroing hands that hold a dealt card: the
  // top chance node of an all-in run-out for the run-out's inner chance nodes and
  // showdowns (nobody acts below it), the node itself otherwise
  std::vector<int32_t> reach_src;
  // hands
  int n_hands = 0, hstride = 0;
  std::vector<uint8_t> hand_cards;    // [n_hands][2]
  std::vector<uint64_t> hand_mask;    // [n_hands]
  std::vector<double> range[2];       // normalised
  double Z = 0.0;
  // showdown boards
  int n_boards = 0, cl_len = 0;
  std::vector<int32_t> sd_perm, sd_gs, sd_ge, cl_hand, cl_off, cl_lo, cl_hi;
};

// Validates `spec` and fills `out`; returns CFR_OK or CFR_EINVAL with a message in `err`.
int build_game(const cfr_game_spec& spec, HostGame& out, std::string& err);

// The terminal kernel's per-board uint16 tables (layout: TermTab in pcfr_internal.h).
std::vector<uint16_t> pack_term_tables(const HostGame& g);

// Decision nodes of player 0 then player 1; begin[p] .. begin[p + 1] are player p's.
std::vector<int32_t> decision_nodes(const HostGame& g, int begin[3]);

// Decision node owning each regret row.
std::vector<int32_t> row_nodes(const HostGame& g);

// Program of the one-warp-per-32-hands schedule: the inner (decision and chance) nodes in
// depth-first pre-order, children in their natural order; terminal nodes are handled by
// their parents.  Walked forwards it is a top-down order in which a stack of reach values
// pops each node's reach and pushes its inner children's (child 0 on top); walked backwards
// it is a bottom-up order in which a stack of values pushes each node's value and pops its
// inner children's in the order 0, 1, ...  `depth` receives the deepest either stack gets,
// `max_actions` the most actions at a decision node, `ok` whether the tree suits the
// schedule (its root is inner and chance nodes have no terminal children).
std::vector<int32_t> dfs_program(const HostGame& g, int* depth, int* max_actions, bool* ok);

// Loads of node n in a pass of the stream schedule for player p (StreamArray << kArrShift |
// element offset, hstride S): bottom-up, the values of its terminal children and, at p's
// decision nodes, R of each action (then the Predictive CFR+ prediction M with pred), S of
// each action and p's reach; top-down, R (and M) of each action at p's decision nodes.
std::vector<uint32_t> node_loads(const HostGame& g, int n, int p, bool backward, uint32_t S, bool pred);

// The program as the stream kernel reads it: one ProgOp per node in pre-order.
std::vector<ProgOp> program_ops(const HostGame& g, const std::vector<int32_t>& pre);

// Load tables of the stream schedule, four passes: the bottom-up pass of player 0 and of
// player 1 and the top-down pass of player 0 and of player 1 (node_loads).  `units` receives each pass's
// loads in the order the pass uses them (StreamArray << kArrShift | element offset), unit_off[q] /
// unit_count[q] where pass q's begin and how many; the result holds each pass's chunks --
// runs of consecutive nodes whose loads fit `half` units -- as (first node position, first
// unit) pairs followed by (program length, unit count), chunk_off[q] (in pairs) and
// chunk_count[q] where pass q's begin and how many.
std::vector<int32_t> stream_tables(const HostGame& g, const std::vector<int32_t>& pre, int half, bool pred,
                                   std::vector<uint32_t>& units, int unit_off[4], int unit_count[4],
                                   int chunk_off[4], int chunk_count[4]);

// All-in run-outs of one game evaluated by win-minus-loss tables (runout.h): a run-out's top
// is a chance node below a decision whose subtree holds only chance and showdown nodes, all of
// them with one payoff; tops whose subtrees show down on the same boards share a table.
struct RunoutPlan {
  std::vector<char> top, inside;  // per node: tops a run-out / lies below a top
  std::vector<RunoutItem> items8, items16;
  std::vector<RunoutTable> tables;
  std::vector<RunoutBoard> boards;
  size_t pool_bytes = 0;
};

void plan_runouts(const HostGame& g, RunoutPlan& r);

}  // namespace pcfr
