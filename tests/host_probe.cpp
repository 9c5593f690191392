// A C shim over the library's host-side tree construction (paper_2605_19928_gb300/csrc/tree.cpp)
// for CPU tests: the tests compile it with g++ next to tree.cpp and read the public tree,
// the stream schedule's program and load tables, and the run-out reach sources that the
// kernels are given.  Nothing here computes; it copies HostGame fields out.
#include <cstring>
#include <string>
#include <vector>

#include "tree.h"

using pcfr::HostGame;

namespace {
struct Probe {
  HostGame g;
  std::vector<int32_t> prog;
  int depth = 0, max_actions = 0;
  bool ok = false;
};
thread_local std::string last_error;
}  // namespace

extern "C" {

// Builds one subgame; NULL on a rejected spec (probe_error() says why).
void* probe_create(const cfr_game_spec* spec) {
  Probe* p = new Probe();
  if (pcfr::build_game(*spec, p->g, last_error) != 0) {
    delete p;
    return nullptr;
  }
  p->prog = pcfr::dfs_program(p->g, &p->depth, &p->max_actions, &p->ok);
  return p;
}

void probe_destroy(void* h) { delete static_cast<Probe*>(h); }

const char* probe_error(void) { return last_error.c_str(); }

// sizes: n_nodes, n_hands, hstride, n_rows, program length, stack depth, max actions, ok
void probe_sizes(void* h, int32_t out[8]) {
  const Probe& p = *static_cast<Probe*>(h);
  out[0] = (int32_t)p.g.nodes.size();
  out[1] = p.g.n_hands;
  out[2] = p.g.hstride;
  out[3] = p.g.n_rows;
  out[4] = (int32_t)p.prog.size();
  out[5] = p.depth;
  out[6] = p.max_actions;
  out[7] = p.ok ? 1 : 0;
}

// per node (level order): parent, first_kid, n_kids, type, player, deal, row, reach_src;
// contrib [n][2]
void probe_nodes(void* h, int32_t* out8, double* contrib) {
  const Probe& p = *static_cast<Probe*>(h);
  for (size_t n = 0; n < p.g.nodes.size(); ++n) {
    const pcfr::NodeDev& nd = p.g.nodes[n];
    int32_t* o = out8 + 8 * n;
    o[0] = nd.parent;
    o[1] = nd.first_kid;
    o[2] = nd.n_kids;
    o[3] = nd.type;
    o[4] = nd.player;
    o[5] = nd.deal;
    o[6] = nd.row;
    o[7] = p.g.reach_src[n];
    contrib[2 * n] = p.g.contrib[2 * n];
    contrib[2 * n + 1] = p.g.contrib[2 * n + 1];
  }
}

void probe_program(void* h, int32_t* out) {
  const Probe& p = *static_cast<Probe*>(h);
  std::memcpy(out, p.prog.data(), p.prog.size() * sizeof(int32_t));
}

// The load tables for ring halves of `half` units: returns the unit count (units copied if
// cap allows) and fills unit_off/unit_count/chunk_off/chunk_count [4]; chunks (pairs,
// n_chunk_ints entries) copied if chunk_cap allows.
int probe_tables(void* h, int half, int pred, uint32_t* units, int cap, int32_t meta[16], int32_t* chunks,
                 int chunk_cap, int32_t* n_chunk_ints) {
  const Probe& p = *static_cast<Probe*>(h);
  std::vector<uint32_t> u;
  const std::vector<int32_t> ch =
      pcfr::stream_tables(p.g, p.prog, half, pred != 0, u, &meta[0], &meta[4], &meta[8], &meta[12]);
  if ((int)u.size() <= cap) std::memcpy(units, u.data(), u.size() * sizeof(uint32_t));
  if ((int)ch.size() <= chunk_cap) std::memcpy(chunks, ch.data(), ch.size() * sizeof(int32_t));
  *n_chunk_ints = (int32_t)ch.size();
  return (int)u.size();
}

// the stream program as the kernel reads it: per node (pre-order) node_off, row_off,
// code, first_kid
void probe_program_ops(void* h, int32_t* out4) {
  const Probe& p = *static_cast<Probe*>(h);
  const std::vector<pcfr::ProgOp> ops = pcfr::program_ops(p.g, p.prog);
  for (size_t k = 0; k < ops.size(); ++k) {
    out4[4 * k] = ops[k].node_off;
    out4[4 * k + 1] = ops[k].row_off;
    out4[4 * k + 2] = (int32_t)ops[k].code;
    out4[4 * k + 3] = ops[k].first_kid;
  }
}

// per node: the terminal payoff times the chance probability the kernels multiply by
void probe_payoff(void* h, double* out) {
  const Probe& p = *static_cast<Probe*>(h);
  for (size_t n = 0; n < p.g.payoff.size(); ++n) out[n] = p.g.payoff[n];
}

// the deal normaliser Z (sum of r0 r1 over the pairs of hands sharing no card)
double probe_Z(void* h) { return static_cast<Probe*>(h)->g.Z; }

// game, deck, hand_size, n_boards
void probe_game(void* h, int32_t out[4]) {
  const Probe& p = *static_cast<Probe*>(h);
  out[0] = p.g.game;
  out[1] = p.g.deck;
  out[2] = p.g.hand_size;
  out[3] = p.g.n_boards;
}

// public cards at every node (bit c = card c)
void probe_boards(void* h, uint64_t* out) {
  const Probe& p = *static_cast<Probe*>(h);
  for (size_t n = 0; n < p.g.nodes.size(); ++n) out[n] = p.g.nodes[n].board;
}

// The terminal kernel's packed tables (one block per showdown board): offsets of the
// sections (clh, cards, cloff, fold_len, perm, gs, ge, lo, hi, len) and the blocks, copied
// if cap allows; returns the number of uint16 entries.
int probe_term_tables(void* h, int32_t tt_out[10], uint16_t* out, int cap) {
  const Probe& p = *static_cast<Probe*>(h);
  const pcfr::TermTab tt(p.g.n_hands, p.g.hand_size, p.g.deck);
  const int32_t v[10] = {tt.clh, tt.cards, tt.cloff, tt.fold_len, tt.perm, tt.gs, tt.ge, tt.lo, tt.hi, tt.len};
  std::memcpy(tt_out, v, sizeof(v));
  const std::vector<uint16_t> t = pcfr::pack_term_tables(p.g);
  if ((int)t.size() <= cap) std::memcpy(out, t.data(), t.size() * sizeof(uint16_t));
  return (int)t.size();
}

// The all-in run-outs evaluated by tables (plan_runouts): sizes = (tops with uint8 tables,
// tops with uint16 tables, tables, boards), *pool = table bytes.  With non-null outputs: per
// node the top and inside flags; per top (uint8 tables first) node, table and u; per table
// wide, board count, first board and byte offset; per board its cards and board table.
void probe_runouts(void* h, int32_t sizes[4], int64_t* pool, int8_t* top, int8_t* inside, int32_t* items,
                   float* u, int64_t* tables, uint64_t* board_cards, int32_t* board_tab) {
  const Probe& p = *static_cast<Probe*>(h);
  pcfr::RunoutPlan r;
  pcfr::plan_runouts(p.g, r);
  sizes[0] = (int32_t)r.items8.size();
  sizes[1] = (int32_t)r.items16.size();
  sizes[2] = (int32_t)r.tables.size();
  sizes[3] = (int32_t)r.boards.size();
  *pool = (int64_t)r.pool_bytes;
  if (!top) return;
  for (size_t n = 0; n < r.top.size(); ++n) {
    top[n] = r.top[n];
    inside[n] = r.inside[n];
  }
  std::vector<pcfr::RunoutItem> all = r.items8;
  all.insert(all.end(), r.items16.begin(), r.items16.end());
  for (size_t k = 0; k < all.size(); ++k) {
    items[2 * k] = all[k].node;
    items[2 * k + 1] = all[k].table;
    u[k] = all[k].u;
  }
  for (size_t k = 0; k < r.tables.size(); ++k) {
    tables[4 * k] = r.tables[k].wide;
    tables[4 * k + 1] = r.tables[k].n_boards;
    tables[4 * k + 2] = r.tables[k].board0;
    tables[4 * k + 3] = r.tables[k].offset;
  }
  for (size_t k = 0; k < r.boards.size(); ++k) {
    board_cards[k] = r.boards[k].cards;
    board_tab[k] = r.boards[k].table;
  }
}

}  // extern "C"
