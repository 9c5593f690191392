// Host-side subgame construction (see tree.h).
//
// Betting rules (Section 5, "Game": heads-up poker with a fixed action abstraction,
// Section 2 "Abstraction"): player 0 acts first on every street; facing a bet the actions
// are fold, call and raises, otherwise check and bets; "max raises" counts the opening bet.
// Limit games (Kuhn, Leduc) raise by a fixed amount per street.  Hold'em subgames raise by
// pot fractions: a fraction x facing a call of d raises by d + x * (pot + d), amounts that
// reach the stack become all-in, duplicates are dropped and raises are ordered by size.
#include "tree.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>

namespace pcfr {
namespace {

struct Pending {
  uint8_t type;
  uint8_t player;  // decision: to act; fold: folder
  int parent;
  int paction;
  int level;
  double c[2];
  int street;
  int raises;
  bool checked;    // the first player checked on this street
  int nboard;
  int board[5];
  int deal;
  double chance;   // probability of the public cards dealt on the path (given both hands)
};

struct Rules {
  int game;
  int deck;
  int n_streets;
  double cap;            // hold'em: all-in contribution
  double limit_bet[2];   // limit games: raise amount per street
  std::vector<double> sizes;
  int max_raises;
};

uint64_t board_bits(const Pending& s) {
  uint64_t b = 0;
  for (int k = 0; k < s.nboard; ++k) b |= 1ull << s.board[k];
  return b;
}

// The betting on s.street is over: deal the next card or show down.
Pending street_over(const Rules& R, const Pending& s) {
  Pending e = s;
  e.type = s.street + 1 >= R.n_streets ? kShowdown : kChance;
  e.deal = kNoCard;
  return e;
}

void decision_children(const Rules& R, const Pending& s, std::vector<Pending>& kids) {
  const int p = s.player, q = 1 - p;
  const bool facing = s.c[q] > s.c[p];
  Pending base = s;
  base.deal = kNoCard;
  if (facing) {
    Pending f = base;
    f.type = kFold;
    f.player = (uint8_t)p;
    kids.push_back(f);
    Pending call = base;
    call.c[p] = s.c[q];
    kids.push_back(street_over(R, call));
  } else if (p == 1 || s.checked) {
    kids.push_back(street_over(R, base));
  } else {
    Pending chk = base;
    chk.type = kDecision;
    chk.player = (uint8_t)q;
    chk.checked = true;
    kids.push_back(chk);
  }
  if (s.raises >= R.max_raises) return;
  std::vector<double> to;
  if (R.game == CFR_GAME_HOLDEM) {
    if (!(s.c[q] < R.cap && s.c[p] < R.cap)) return;
    const double d = s.c[q] - s.c[p], pot = s.c[0] + s.c[1];
    for (double x : R.sizes) {
      double t = R.cap;
      if (x > 0.0) t = std::min(s.c[p] + (d + x * (pot + d)), R.cap);
      if (t > s.c[q] && std::find(to.begin(), to.end(), t) == to.end()) to.push_back(t);
    }
    std::sort(to.begin(), to.end());
  } else {
    to.push_back(s.c[q] + R.limit_bet[s.street]);
  }
  for (double t : to) {
    Pending r = base;
    r.type = kDecision;
    r.player = (uint8_t)q;
    r.c[p] = t;
    r.raises = s.raises + 1;
    kids.push_back(r);
  }
}

void chance_children(const Rules& R, const Pending& s, std::vector<Pending>& kids) {
  const uint64_t on = board_bits(s);
  const bool all_in = R.game == CFR_GAME_HOLDEM && std::max(s.c[0], s.c[1]) >= R.cap;
  for (int card = 0; card < R.deck; ++card) {
    if ((on >> card) & 1ull) continue;
    Pending k = s;
    k.board[k.nboard++] = card;
    k.street = s.street + 1;
    k.raises = 0;
    k.checked = false;
    if (all_in) {
      k = street_over(R, k);  // nobody can bet: run the cards out
    } else {
      k.type = kDecision;
      k.player = 0;
    }
    k.deal = card;
    kids.push_back(k);
  }
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

}  // namespace

int build_game(const cfr_game_spec& spec, HostGame& g, std::string& err) {
  g = HostGame();
  g.game = spec.game;
  Rules R{};
  R.game = spec.game;
  R.max_raises = spec.max_raises;
  Pending root{};
  root.type = kDecision;
  root.player = 0;
  root.parent = -1;
  root.deal = kNoCard;
  root.chance = 1.0;
  std::vector<int> board0;

  if (spec.game == CFR_GAME_KUHN || spec.game == CFR_GAME_LEDUC) {
    const bool kuhn = spec.game == CFR_GAME_KUHN;
    g.deck = kuhn ? 3 : 6;
    g.hand_size = 1;
    g.n_streets = kuhn ? 1 : 2;
    R.limit_bet[0] = kuhn ? 1.0 : 2.0;
    R.limit_bet[1] = 4.0;
    R.max_raises = kuhn ? 1 : 2;
    root.c[0] = root.c[1] = 1.0;  // antes
    g.n_hands = g.deck;
    if (spec.n_hands != 0 && spec.n_hands != g.deck) {
      err = "Kuhn and Leduc deal one card per player from their own deck";
      return CFR_EINVAL;
    }
    for (int c = 0; c < g.deck; ++c) {
      g.hand_cards.push_back((uint8_t)c);
      g.hand_cards.push_back(kNoCard);
      g.hand_mask.push_back(1ull << c);
    }
  } else if (spec.game == CFR_GAME_HOLDEM) {
    g.deck = 52;
    g.hand_size = 2;
    if (spec.n_board < 3 || spec.n_board > 5) {
      err = "hold'em subgames start on the flop (3 board cards), the turn (4) or the river (5)";
      return CFR_EINVAL;
    }
    if (!spec.board) {
      err = "board is NULL";
      return CFR_EINVAL;
    }
    g.n_streets = 6 - spec.n_board;  // river 1, turn 2, flop 3
    uint64_t bm = 0;
    for (int k = 0; k < spec.n_board; ++k) {
      const int c = spec.board[k];
      if (c < 0 || c >= 52 || ((bm >> c) & 1ull)) {
        err = "board cards must be distinct ids in 0..51";
        return CFR_EINVAL;
      }
      bm |= 1ull << c;
      board0.push_back(c);
      root.board[root.nboard++] = c;
    }
    if (!(spec.pot > 0.0) || !std::isfinite(spec.pot) || !finite_nonneg(spec.stack)) {
      err = "pot must be positive and stack non-negative";
      return CFR_EINVAL;
    }
    if (spec.max_raises < 0 || spec.n_bet_sizes < 0 || spec.n_bet_sizes > kMaxActions - 2 ||
        (spec.n_bet_sizes > 0 && !spec.bet_sizes)) {
      err = "bad bet-size list or raise cap";
      return CFR_EINVAL;
    }
    for (int k = 0; k < spec.n_bet_sizes; ++k) {
      if (!std::isfinite(spec.bet_sizes[k])) {
        err = "bet sizes must be finite";
        return CFR_EINVAL;
      }
      R.sizes.push_back(spec.bet_sizes[k]);
    }
    R.cap = spec.pot / 2.0 + spec.stack;
    root.c[0] = root.c[1] = spec.pot / 2.0;
    if (spec.hands) {
      if (spec.n_hands <= 0) {
        err = "n_hands must be positive";
        return CFR_EINVAL;
      }
      g.n_hands = spec.n_hands;
      std::vector<uint64_t> seen;
      for (int h = 0; h < spec.n_hands; ++h) {
        const int a = spec.hands[2 * h], b = spec.hands[2 * h + 1];
        if (a >= 52 || b >= 52 || a == b || ((bm >> a) & 1ull) || ((bm >> b) & 1ull)) {
          err = "hand " + std::to_string(h) + " has an invalid card or a card on the board";
          return CFR_EINVAL;
        }
        const uint64_t m = (1ull << a) | (1ull << b);
        seen.push_back(m);
        g.hand_cards.push_back((uint8_t)a);
        g.hand_cards.push_back((uint8_t)b);
        g.hand_mask.push_back(m);
      }
      std::sort(seen.begin(), seen.end());
      if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
        err = "duplicate hands";
        return CFR_EINVAL;
      }
    } else {
      for (int a = 0; a < 52; ++a)
        for (int b = a + 1; b < 52; ++b) {
          if (((bm >> a) & 1ull) || ((bm >> b) & 1ull)) continue;
          g.hand_cards.push_back((uint8_t)a);
          g.hand_cards.push_back((uint8_t)b);
          g.hand_mask.push_back((1ull << a) | (1ull << b));
        }
      g.n_hands = (int)g.hand_mask.size();
    }
    const int want_rows = spec.n_board == 5 ? 1 : spec.n_board == 4 ? 52 : 52 * 52;
    if (spec.depth_limit != 0 && (spec.depth_limit != 1 || spec.n_board == 5)) {
      err = "depth_limit 1 applies to flop and turn subgames only";
      return CFR_EINVAL;
    }
    if (spec.n_exact_leaves < 0 || (spec.n_exact_leaves > 0 && (spec.depth_limit != 1 || !spec.exact_leaves))) {
      err = "exact_leaves applies to depth-limited subgames (depth_limit 1) and needs its list";
      return CFR_EINVAL;
    }
    if (!spec.strength || spec.n_strength_rows != want_rows) {
      err = "strength must have 1 row (river), 52 rows (turn) or 52 x 52 rows (flop)";
      return CFR_EINVAL;
    }
  } else {
    err = "unknown game";
    return CFR_EINVAL;
  }
  R.deck = g.deck;
  R.n_streets = g.n_streets;
  const int H = g.n_hands;
  g.hstride = (H + 31) / 32 * 32;

  // ranges: non-negative, finite, normalised to sum 1
  for (int p = 0; p < 2; ++p) {
    g.range[p].assign(H, 1.0 / H);
    if (spec.range[p]) {
      double s = 0.0;
      for (int h = 0; h < H; ++h) {
        const double x = spec.range[p][h];
        if (!finite_nonneg(x)) {
          err = "ranges must be finite and non-negative";
          return CFR_EINVAL;
        }
        s += x;
      }
      if (!(s > 0.0)) {
        err = "a range sums to zero";
        return CFR_EINVAL;
      }
      for (int h = 0; h < H; ++h) g.range[p][h] = spec.range[p][h] / s;
    }
  }
  // Z = sum of r0(a) r1(b) over the pairs of hands sharing no card, in O(H): for each a,
  // player 1's mass minus the mass of the hands holding one of a's cards (inclusion-
  // exclusion; a two-card hand holding both of a's cards is a itself, hands are distinct)
  std::vector<double> card_mass((size_t)g.deck, 0.0);
  double total1 = 0.0;
  for (int b = 0; b < H; ++b) {
    total1 += g.range[1][b];
    for (int t = 0; t < g.hand_size; ++t) card_mass[g.hand_cards[2 * (size_t)b + t]] += g.range[1][b];
  }
  double Z = 0.0;
  for (int a = 0; a < H; ++a) {
    double m = total1;
    for (int t = 0; t < g.hand_size; ++t) m -= card_mass[g.hand_cards[2 * (size_t)a + t]];
    if (g.hand_size == 2) m += g.range[1][a];
    Z += g.range[0][a] * std::max(m, 0.0);
  }
  if (!(Z > 0.0)) {
    err = "no pair of hands can be dealt with positive probability";
    return CFR_EINVAL;
  }
  g.Z = Z;

  // leaves the caller wants solved exactly, by their index among the leaf positions in the
  // order they are met below (breadth first, as cfr_leaf_info lists a tree with no exact
  // leaves: expanding a leaf adds only river subtrees, which hold no leaf positions)
  std::vector<int32_t> exact;
  if (spec.game == CFR_GAME_HOLDEM && spec.n_exact_leaves > 0) {
    exact.assign(spec.exact_leaves, spec.exact_leaves + spec.n_exact_leaves);
    std::sort(exact.begin(), exact.end());
    if (exact.front() < 0 || std::adjacent_find(exact.begin(), exact.end()) != exact.end()) {
      err = "exact_leaves must be distinct leaf indices";
      return CFR_EINVAL;
    }
  }
  int leaf_seq = 0;

  // ---- public tree, breadth first: ids are level order, children consecutive
  std::deque<Pending> queue;
  queue.push_back(root);
  std::vector<Pending> kids;
  while (!queue.empty()) {
    Pending s = queue.front();
    queue.pop_front();
    const int id = (int)g.nodes.size();
    NodeDev nd{};
    nd.parent = s.parent;
    nd.first_kid = -1;
    nd.row = -1;
    nd.type = s.type;
    nd.player = s.player;
    nd.deal = (uint8_t)(s.deal < 0 ? kNoCard : s.deal);
    nd.paction = (uint8_t)(s.paction < 0 ? 0 : s.paction);
    if (s.level > 255) {
      err = "tree deeper than 255 levels";
      return CFR_EINVAL;
    }
    nd.level = (uint8_t)s.level;
    nd.board = board_bits(s);
    kids.clear();
    // depth limit: the chance node that deals the river card ends the tree when a player has
    // chips behind; the leaf network values it
    const bool all_in = std::max(s.c[0], s.c[1]) >= R.cap;
    if (s.type == kChance && spec.depth_limit && spec.game == CFR_GAME_HOLDEM && s.nboard == 4 && !all_in) {
      if (!std::binary_search(exact.begin(), exact.end(), leaf_seq++)) {  // else: exact river subtrees
        s.type = kLeaf;
        nd.type = kLeaf;
      }
    }
    if (s.type == kDecision) decision_children(R, s, kids);
    else if (s.type == kChance) chance_children(R, s, kids);
    // Terminal payoffs carry the probability of the public cards dealt on their path, so
    // the values the kernels compute are counterfactual values with chance inside the
    // counterfactual reach (Eq. cfv).  A chance node's value is then the plain sum of its
    // children over the cards the hand does not hold.
    const double per_card = 1.0 / (double)(g.deck - s.nboard - 2 * g.hand_size);
    double pay = 0.0;
    if (s.type == kFold) pay = s.c[s.player] * s.chance;
    if (s.type == kShowdown) pay = s.c[0] * s.chance;
    if (s.type == kLeaf) pay = (s.c[0] + s.c[1]) * s.chance * per_card;  // pot x P(river card)
    nd.arow = -1;
    nd.aplayer = kNoCard;
    if (s.type == kChance)
      for (Pending& kp : kids) kp.chance = s.chance * per_card;
    if (s.type == kShowdown) {
      // showdown strength row (numbered into tables below): 0 for boards fixed at the root,
      // else the dealt cards (Leduc: the public card; turn: the river card; flop: turn x 52 +
      // river)
      if (spec.game == CFR_GAME_LEDUC) nd.row = s.board[0];
      else if (spec.game == CFR_GAME_HOLDEM && g.n_streets == 2) nd.row = s.board[4];
      else if (spec.game == CFR_GAME_HOLDEM && g.n_streets == 3) nd.row = s.board[3] * 52 + s.board[4];
      else nd.row = 0;
    }
    if (s.type == kDecision ? kids.size() > (size_t)kMaxActions : kids.size() > (size_t)kMaxDeck) {
      err = "too many actions at one node";
      return CFR_EINVAL;
    }
    nd.n_kids = (uint8_t)kids.size();
    if (!kids.empty()) nd.first_kid = id + 1 + (int)queue.size();
    for (size_t k = 0; k < kids.size(); ++k) {
      kids[k].parent = id;
      kids[k].paction = (int)k;
      kids[k].level = s.level + 1;
      queue.push_back(kids[k]);
    }
    g.nodes.push_back(nd);
    g.contrib.push_back(s.c[0]);
    g.contrib.push_back(s.c[1]);
    g.payoff.push_back(pay);
    if (g.nodes.size() > (size_t)(1 << 24)) {
      err = "tree too large";
      return CFR_EINVAL;
    }
  }
  const int N = (int)g.nodes.size();
  int levels = g.nodes.back().level + 1;
  g.level_start.assign(levels + 1, 0);
  for (int n = 0; n < N; ++n) g.level_start[g.nodes[n].level + 1] = n + 1;
  for (int l = 1; l <= levels; ++l) g.level_start[l] = std::max(g.level_start[l], g.level_start[l - 1]);
  // rows: player 0's decision nodes first, then player 1's
  int row = 0;
  for (int p = 0; p < 2; ++p) {
    g.row_begin[p] = row;
    for (int n = 0; n < N; ++n)
      if (g.nodes[n].type == kDecision && g.nodes[n].player == p) {
        g.nodes[n].row = row;
        row += g.nodes[n].n_kids;
      }
  }
  g.row_begin[2] = row;
  g.n_rows = row;
  for (int n = 1; n < N; ++n) {
    const NodeDev& par = g.nodes[g.nodes[n].parent];
    if (par.type == kDecision) {
      g.nodes[n].arow = par.row + g.nodes[n].paction;
      g.nodes[n].aplayer = par.player;
    }
  }
  if (!exact.empty() && exact.back() >= leaf_seq) {
    err = "exact_leaves names leaf " + std::to_string(exact.back()) + " of " + std::to_string(leaf_seq);
    return CFR_EINVAL;
  }
  for (int n = 0; n < N; ++n) {
    if (g.nodes[n].type == kFold || g.nodes[n].type == kShowdown) g.terminals.push_back(n);
    if (g.nodes[n].type == kLeaf) g.leaves.push_back(n);
  }
  // reach sources (level order: a parent's source is known before its children's)
  g.reach_src.resize(N);
  for (int n = 0; n < N; ++n) {
    const NodeDev& nd = g.nodes[n];
    const bool below_chance = nd.parent >= 0 && g.nodes[nd.parent].type == kChance;
    const bool passes = nd.type == kChance || nd.type == kShowdown || nd.type == kFold;
    g.reach_src[n] = below_chance && passes ? g.reach_src[nd.parent] : n;
  }

  // ---- showdown tables, one per board the tree shows down on (table 0 also serves the
  // fold terminals, which only read its card lists)
  std::vector<int> keys;
  for (const NodeDev& nd : g.nodes)
    if (nd.type == kShowdown) keys.push_back(nd.row);
  if (keys.empty()) keys.push_back(0);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  for (NodeDev& nd : g.nodes)
    if (nd.type == kShowdown) nd.row = (int)(std::lower_bound(keys.begin(), keys.end(), nd.row) - keys.begin());
  std::vector<std::vector<int>> strengths(keys.size(), std::vector<int>(H));  // [board table][hand]
  for (size_t b = 0; b < keys.size(); ++b)
    for (int h = 0; h < H; ++h) {
      if (spec.game == CFR_GAME_KUHN) strengths[b][h] = h;
      else if (spec.game == CFR_GAME_LEDUC) strengths[b][h] = (h / 2 == keys[b] / 2) ? 10 + h / 2 : h / 2;
      else strengths[b][h] = spec.strength[(size_t)keys[b] * H + h];
    }
  const int B = (int)strengths.size();
  const int k = g.hand_size;
  g.n_boards = B;
  g.cl_len = k * H;
  g.sd_perm.resize((size_t)B * H);
  g.sd_gs.resize((size_t)B * H);
  g.sd_ge.resize((size_t)B * H);
  g.cl_hand.resize((size_t)B * g.cl_len);
  g.cl_off.resize((size_t)B * (g.deck + 1));
  g.cl_lo.assign((size_t)B * H * 2, 0);
  g.cl_hi.assign((size_t)B * H * 2, 0);
  std::vector<int> order(H), pos(H);
  for (int b = 0; b < B; ++b) {
    const std::vector<int>& s = strengths[b];
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return s[x] < s[y]; });
    int32_t* perm = &g.sd_perm[(size_t)b * H];
    int32_t* gs = &g.sd_gs[(size_t)b * H];
    int32_t* ge = &g.sd_ge[(size_t)b * H];
    for (int j = 0; j < H; ++j) {
      perm[j] = order[j];
      pos[order[j]] = j;
    }
    for (int j = 0; j < H;) {
      int e = j;
      while (e < H && s[order[e]] == s[order[j]]) ++e;
      for (int t = j; t < e; ++t) {
        gs[order[t]] = j;
        ge[order[t]] = e;
      }
      j = e;
    }
    // per-card lists of hands in sorted order
    int32_t* off = &g.cl_off[(size_t)b * (g.deck + 1)];
    int32_t* lst = &g.cl_hand[(size_t)b * g.cl_len];
    std::vector<int> count(g.deck, 0);
    for (int h = 0; h < H; ++h)
      for (int t = 0; t < k; ++t) count[g.hand_cards[2 * h + t]]++;
    off[0] = 0;
    for (int c = 0; c < g.deck; ++c) off[c + 1] = off[c] + count[c];
    std::vector<int> fill(off, off + g.deck);
    for (int j = 0; j < H; ++j) {
      const int h = order[j];
      for (int t = 0; t < k; ++t) lst[fill[g.hand_cards[2 * h + t]]++] = h;
    }
    int32_t* lo = &g.cl_lo[(size_t)b * H * 2];
    int32_t* hi = &g.cl_hi[(size_t)b * H * 2];
    // for the hands holding card c (its list, in increasing sorted position, so their tie
    // groups' bounds never decrease): the first entry at or after gs and at or after ge,
    // found by two pointers walking the list once
    for (int c = 0; c < g.deck; ++c) {
      const int a = off[c], z = off[c + 1];
      int x = a, y = a;
      for (int j = a; j < z; ++j) {
        const int h = lst[j];
        while (x < z && pos[lst[x]] < gs[h]) ++x;
        if (y < x) y = x;
        while (y < z && pos[lst[y]] < ge[h]) ++y;
        const int t = g.hand_cards[2 * (size_t)h] == c ? 0 : 1;
        lo[2 * h + t] = x;
        hi[2 * h + t] = y;
      }
    }
  }
  return CFR_OK;
}

std::vector<uint16_t> pack_term_tables(const HostGame& g) {
  const int H = g.n_hands, k = g.hand_size, D = g.deck;
  const TermTab tt(H, k, D);
  std::vector<uint16_t> out((size_t)g.n_boards * tt.len, 0);
  for (int b = 0; b < g.n_boards; ++b) {
    uint16_t* t = &out[(size_t)b * tt.len];
    for (int j = 0; j < k * H; ++j) t[tt.clh + j] = (uint16_t)g.cl_hand[(size_t)b * g.cl_len + j];
    for (int h = 0; h < H; ++h)
      t[tt.cards + h] = (uint16_t)(g.hand_cards[2 * h] | (g.hand_cards[2 * h + 1] << 8));
    for (int c = 0; c <= D; ++c) t[tt.cloff + c] = (uint16_t)g.cl_off[(size_t)b * (D + 1) + c];
    for (int h = 0; h < H; ++h) {
      t[tt.perm + h] = (uint16_t)g.sd_perm[(size_t)b * H + h];
      t[tt.gs + h] = (uint16_t)g.sd_gs[(size_t)b * H + h];
      t[tt.ge + h] = (uint16_t)g.sd_ge[(size_t)b * H + h];
      for (int s = 0; s < 2; ++s) {
        t[tt.lo + 2 * h + s] = (uint16_t)g.cl_lo[((size_t)b * H + h) * 2 + s];
        t[tt.hi + 2 * h + s] = (uint16_t)g.cl_hi[((size_t)b * H + h) * 2 + s];
      }
    }
  }
  return out;
}

std::vector<int32_t> decision_nodes(const HostGame& g, int begin[3]) {
  std::vector<int32_t> out;
  for (int p = 0; p < 2; ++p) {
    begin[p] = (int)out.size();
    for (size_t n = 0; n < g.nodes.size(); ++n)
      if (g.nodes[n].type == kDecision && g.nodes[n].player == p) out.push_back((int32_t)n);
  }
  begin[2] = (int)out.size();
  return out;
}

std::vector<int32_t> row_nodes(const HostGame& g) {
  std::vector<int32_t> out((size_t)g.n_rows, -1);
  for (size_t n = 0; n < g.nodes.size(); ++n)
    if (g.nodes[n].type == kDecision)
      for (int a = 0; a < g.nodes[n].n_kids; ++a) out[(size_t)g.nodes[n].row + a] = (int32_t)n;
  return out;
}

static bool is_terminal(const NodeDev& nd) { return is_end(nd.type); }

std::vector<int32_t> dfs_program(const HostGame& g, int* depth, int* max_actions, bool* ok) {
  std::vector<int32_t> pre;  // inner nodes only
  std::vector<int32_t> todo{0};
  bool fine = !is_terminal(g.nodes[0]);
  while (!todo.empty()) {
    const int n = todo.back();
    todo.pop_back();
    const NodeDev& nd = g.nodes[(size_t)n];
    if (is_terminal(nd)) continue;
    pre.push_back(n);
    for (int a = nd.n_kids - 1; a >= 0; --a) {  // child 0 first
      const NodeDev& kid = g.nodes[(size_t)(nd.first_kid + a)];
      // a chance node's children are all terminal (after an all-in) or all inner
      if (nd.type == kChance && is_terminal(kid) != is_terminal(g.nodes[(size_t)nd.first_kid])) fine = false;
      todo.push_back(nd.first_kid + a);
    }
  }
  auto inner_kids = [&](int n) {
    const NodeDev& nd = g.nodes[(size_t)n];
    int c = 0;
    for (int a = 0; a < nd.n_kids; ++a) c += !is_terminal(g.nodes[(size_t)(nd.first_kid + a)]);
    return c;
  };
  int sp = 1, most = 1, amax = 0;
  for (int n : pre) {  // top-down: pop the node's reach, push its inner children's
    sp += inner_kids(n) - 1;
    most = std::max(most, sp);
    if (g.nodes[(size_t)n].type == kDecision) amax = std::max(amax, (int)g.nodes[(size_t)n].n_kids);
  }
  sp = 0;
  for (size_t k = pre.size(); k-- > 0;) {  // bottom-up: pop the inner children's values, push the node's
    sp += 1 - inner_kids(pre[k]);
    most = std::max(most, sp);
  }
  *depth = most;
  *max_actions = amax;
  *ok = fine;
  return pre;
}

std::vector<ProgOp> program_ops(const HostGame& g, const std::vector<int32_t>& pre) {
  std::vector<ProgOp> out;
  out.reserve(pre.size());
  for (int n : pre) {
    const NodeDev& nd = g.nodes[(size_t)n];
    uint32_t tmask = 0;  // chance nodes: bit 0 when all children are terminal
    for (int a = 0; a < nd.n_kids && a < (nd.type == kChance ? 1 : 8); ++a)
      if (is_terminal(g.nodes[(size_t)(nd.first_kid + a)])) tmask |= 1u << a;
    ProgOp op;
    op.node_off = n * g.hstride;
    op.row_off = nd.type == kDecision ? nd.row * g.hstride : 0;
    op.code = (uint32_t)(nd.type & 3u) | (uint32_t)(nd.player & 1u) << 2 | (uint32_t)(nd.n_kids & 63u) << 3 |
              (uint32_t)nd.deal << 9 | tmask << 17;
    op.first_kid = nd.first_kid;
    out.push_back(op);
  }
  return out;
}

std::vector<int32_t> stream_tables(const HostGame& g, const std::vector<int32_t>& pre, int half, bool pred,
                                   std::vector<uint32_t>& units, int unit_off[4], int unit_count[4],
                                   int chunk_off[4], int chunk_count[4]) {
  std::vector<int32_t> chunks;
  units.clear();
  const int N = (int)pre.size();
  const uint32_t S = (uint32_t)g.hstride;
  for (int q = 0; q < 4; ++q) {
    const int p = q & 1;
    const bool backward = q < 2;
    unit_off[q] = (int)units.size();
    chunk_off[q] = (int)chunks.size() / 2;
    int used = 0;
    for (int k = 0; k < N; ++k) {
      const int n = pre[(size_t)(backward ? N - 1 - k : k)];
      const std::vector<uint32_t> mine = node_loads(g, n, p, backward, S, pred);
      if (k == 0 || used + (int)mine.size() > half) {
        chunks.push_back(k);
        chunks.push_back((int)units.size() - unit_off[q]);
        used = 0;
      }
      used += (int)mine.size();
      units.insert(units.end(), mine.begin(), mine.end());
    }
    unit_count[q] = (int)units.size() - unit_off[q];
    chunk_count[q] = (int)chunks.size() / 2 - chunk_off[q];
    chunks.push_back(N);
    chunks.push_back(unit_count[q]);
  }
  return chunks;
}

std::vector<uint32_t> node_loads(const HostGame& g, int n, int p, bool backward, uint32_t S, bool pred) {
  std::vector<uint32_t> mine;
  const NodeDev& nd = g.nodes[(size_t)n];
  if (backward)  // values of the terminal children, in child order
    for (int a = 0; a < nd.n_kids; ++a)
      if (is_terminal(g.nodes[(size_t)(nd.first_kid + a)]))
        mine.push_back(kArrCfv << kArrShift | (uint32_t)(nd.first_kid + a) * S);
  if (nd.type == kDecision && nd.player == p) {
    for (int a = 0; a < nd.n_kids; ++a) mine.push_back(kArrR << kArrShift | (uint32_t)(nd.row + a) * S);
    if (pred)
      for (int a = 0; a < nd.n_kids; ++a) mine.push_back(kArrM << kArrShift | (uint32_t)(nd.row + a) * S);
    if (backward) {
      for (int a = 0; a < nd.n_kids; ++a) mine.push_back(kArrS << kArrShift | (uint32_t)(nd.row + a) * S);
      mine.push_back(kArrReach << kArrShift | (uint32_t)n * S);
    }
  }
  return mine;
}

void plan_runouts(const HostGame& h, RunoutPlan& r) {
  const int N = (int)h.nodes.size();
  std::vector<char> pure(N, 0);  // a showdown, or a chance node with only such nodes below
  for (int n = N - 1; n >= 0; --n) {  // children come after their parent (level order)
    const NodeDev& nd = h.nodes[(size_t)n];
    if (nd.type == kShowdown) {
      pure[n] = 1;
    } else if (nd.type == kChance && nd.n_kids > 0) {
      bool all = true;
      for (int k = 0; k < nd.n_kids; ++k) all = all && pure[nd.first_kid + k];
      pure[n] = all;
    }
  }
  std::vector<int> top_of(N, -1);  // the candidate top above a node inside a run-out
  std::vector<char> cand(N, 0);
  for (int n = 1; n < N; ++n) {
    const int par = h.nodes[(size_t)n].parent;
    if (cand[par] || top_of[par] >= 0) top_of[n] = cand[par] ? par : top_of[par];
    else if (pure[n] && h.nodes[(size_t)n].type == kChance && h.nodes[(size_t)par].type != kChance) cand[n] = 1;
  }
  std::vector<std::vector<int>> shows(N);
  for (int n = 0; n < N; ++n)
    if (top_of[n] >= 0 && h.nodes[(size_t)n].type == kShowdown) shows[top_of[n]].push_back(n);
  std::vector<char> take(N, 0);
  std::vector<std::vector<std::pair<uint64_t, int>>> sigs;  // each table's boards (cards, board table)
  const double kappa = 1.0 / h.Z;
  for (int n = 0; n < N; ++n) {
    if (!cand[n] || shows[n].empty()) continue;
    const double pay = h.payoff[(size_t)shows[n][0]];
    bool same = true;
    for (int sd : shows[n]) same = same && h.payoff[(size_t)sd] == pay;
    if (!same) continue;  // evaluated board by board
    std::vector<std::pair<uint64_t, int>> sig;
    for (int sd : shows[n]) sig.push_back({h.nodes[(size_t)sd].board, h.nodes[(size_t)sd].row});
    std::sort(sig.begin(), sig.end());
    int tid = (int)(std::find(sigs.begin(), sigs.end(), sig) - sigs.begin());
    if (tid == (int)sigs.size()) {
      RunoutTable tb{};
      tb.wide = sig.size() > 127 ? 1 : 0;
      tb.n_boards = (int)sig.size();
      tb.board0 = (int)r.boards.size();
      tb.offset = (int64_t)r.pool_bytes;
      r.pool_bytes += ((size_t)h.n_hands * h.hstride * (tb.wide ? 2 : 1) + 255) / 256 * 256;
      for (const auto& b : sig) r.boards.push_back({b.first, b.second, 0});
      r.tables.push_back(tb);
      sigs.push_back(sig);
    }
    const RunoutItem it{n, tid, (float)(pay * kappa), 0};
    (r.tables[(size_t)tid].wide ? r.items16 : r.items8).push_back(it);
    take[n] = 1;
  }
  r.top = take;
  r.inside.assign(N, 0);
  for (int n = 0; n < N; ++n) r.inside[n] = top_of[n] >= 0 && take[top_of[n]];
}

}  // namespace pcfr
