/*
 * cfr_oracle.c -- plain, slow, FP64 reference CFR that walks every history.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant with the CUDA path; the two meet only
 * through the seeded input arrays.
 *
 * What it computes (paper: "Real-Time Parallel Counterfactual Regret Minimization"):
 *   - counterfactual values, Section 3, Eq. (cfv): v_i(sigma, I) =
 *     sum_{h in I} pi_{-i}(h) sum_z pi(h, z) u_i(z), by recursion over every history
 *     (every private deal x every public action path), no vectorisation, no prefix sums,
 *     no card-blocker formula;
 *   - instantaneous regret, Section 3 (r^t_i(I,a) = v_i(sigma_{I->a}, I) - v_i(sigma, I)),
 *     accumulated per history as pi_{-i} * pi_c * (u(h.a) - u(h));
 *   - regret matching, Section 3, Eq. (rm), uniform when no regret is positive;
 *   - the Stage 7 update (Section 4.4) for vanilla CFR, CFR+ and DCFR (Section 2, CFR
 *     algorithms), with the average strategy weighted by the player's own reach
 *     (Section 4.2, Stage 1);
 *   - a best response against the average strategy, by per-infoset maximisation over the
 *     same enumeration, and the exploitability (BR_0 + BR_1) / 2 in chips; its per-node
 *     values are counterfactual values like those of the walk (chance probabilities inside
 *     the counterfactual reach).
 *
 * Readings of points the paper leaves open:
 *   - the subgame starts with a chance deal of private hands with probability
 *     r_0(h_0) r_1(h_1) / Z over non-conflicting pairs; r_i(h_i) counts as player i's own
 *     reach, r_{-i}(h_{-i}) / Z as the opponent-and-chance part;
 *   - payoffs: a fold loses the folder's whole contribution, a showdown wins the loser's
 *     contribution, equal strengths split (payoff 0);
 *   - updates alternate: player 0 is updated first, then player 1 with player 0's new
 *     strategy; both use the same iteration number t (1-based);
 *   - DCFR at iteration t: R <- R + r, then R is multiplied by t^a/(t^a+1) where positive and
 *     by t^b/(t^b+1) elsewhere; S <- S * (t/(t+1))^g + pi_i * sigma;
 *   - CFR+: R <- max(R + r, 0), S <- S + t * pi_i * sigma;
 *   - Predictive CFR+ (evaluated beside DCFR in Section 5): R <- max(R + r, 0), the
 *     prediction M <- r, the strategy is regret matching of R + M, S <- S + t^2 pi_i sigma;
 *   - hold'em subgames start on the flop, turn or river; with a depth limit the tree ends
 *     where the river card is to come (a leaf), unless a player is all-in;
 *   - a bet of fraction x facing a call of d raises by d + x * (pot + d); sizes reaching the
 *     stack become all-in and duplicate sizes are dropped; "max raises" counts the opening
 *     bet; player 0 acts first on every street.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { G_HOLDEM = 0, G_KUHN = 1, G_LEDUC = 2 };
enum { T_DEC = 0, T_FOLD = 1, T_SHOW = 2, T_CHANCE = 3, T_LEAF = 4 };
enum { V_CFR = 0, V_CFRPLUS = 1, V_DCFR = 2, V_PCFRPLUS = 3 };

typedef struct {
  int type;        /* T_DEC, T_FOLD, T_SHOW, T_CHANCE, T_LEAF */
  int player;      /* acting player (decision) or folding player (fold) */
  int parent;      /* -1 at the root */
  int paction;     /* index of this node among its parent's children */
  int street;
  int nkids;
  int* kids;
  double c[2];     /* chips each player has put in, including the starting pot share */
  int nboard;
  int board[5];    /* public cards at this node */
  int deal;        /* card dealt by a chance parent, else -1 */
  int row;         /* decision nodes: first regret row */
  double* leafy;   /* depth-limit leaves: network outputs [ncards][2][nh] (set from outside) */
} Node;

typedef struct Oracle {
  int game, deck, hsize, nstreets;
  int nh;
  int* cards;            /* [nh][hsize] */
  uint64_t* hmask;       /* card set of each hand */
  double* r[2];          /* normalised ranges */
  int* strength;         /* hold'em: [nstr][nh] */
  int nstr;
  double pot, stack, cap;
  int nsizes;
  double sizes[16];
  int max_raises;
  int variant;
  double alpha, beta, gamma;
  int alternating;
  int nthreads;
  int depth_limit;       /* 1: a river chance node with chips behind is a leaf */
  int* exact_flags;      /* [n_exact_flags]: leaf position k (in the order the builder meets
                            them, depth first) is solved exactly instead (depth_limit 1) */
  int n_exact_flags;
  int leaf_seq;          /* leaf positions met so far while building */

  Node* nodes;
  int nn, ncap;
  int nrows;
  double *R, *S, *sig, *prof, *rinst;
  double* M;             /* Predictive CFR+: the prediction (last instantaneous regret) */
  double* cfv[2];        /* [nn][nh], counterfactual values of the last traversal of player i */
  unsigned char* compat; /* [nh][nh] 1 if the two hands share no card */
  double Z;
  int t;                 /* iterations completed */
} Oracle;

static char g_err[256];
const char* ocfr_error(void) { return g_err; }

/* ------------------------------------------------------------------ game rules */

static double street_bet_limit(const Oracle* o, int street) {
  if (o->game == G_KUHN) return 1.0;
  if (o->game == G_LEDUC) return street == 0 ? 2.0 : 4.0;
  return 0.0;
}

static int new_node(Oracle* o, int type, int player, int parent, int paction, int street,
                    const double c[2], int nboard, const int* board, int deal) {
  if (o->nn == o->ncap) {
    o->ncap = o->ncap ? 2 * o->ncap : 256;
    o->nodes = (Node*)realloc(o->nodes, sizeof(Node) * (size_t)o->ncap);
  }
  Node* n = &o->nodes[o->nn];
  memset(n, 0, sizeof(*n));
  n->type = type;
  n->player = player;
  n->parent = parent;
  n->paction = paction;
  n->street = street;
  n->c[0] = c[0];
  n->c[1] = c[1];
  n->nboard = nboard;
  for (int k = 0; k < nboard; ++k) n->board[k] = board[k];
  n->deal = deal;
  n->row = -1;
  return o->nn++;
}

static int build_decision(Oracle* o, int parent, int paction, int street, const double c[2], int nboard,
                          const int* board, int deal, int player, int nraises, int first_checked);

/* The betting on `street` is over with contributions c: deal the next card or show down. */
static int build_street_end(Oracle* o, int parent, int paction, int street, const double c[2], int nboard,
                            const int* board, int deal) {
  if (street + 1 >= o->nstreets)
    return new_node(o, T_SHOW, -1, parent, paction, street, c, nboard, board, deal);
  /* the depth limit ends the tree where the river card is to come, unless nobody can bet */
  if (o->depth_limit && o->game == G_HOLDEM && street + 2 == o->nstreets && !(c[0] >= o->cap || c[1] >= o->cap)) {
    int seq = o->leaf_seq++;
    if (!(seq < o->n_exact_flags && o->exact_flags[seq]))  /* else: the exact river card chance node */
      return new_node(o, T_LEAF, -1, parent, paction, street, c, nboard, board, deal);
  }
  int id = new_node(o, T_CHANCE, -1, parent, paction, street, c, nboard, board, deal);
  int live[64], nlive = 0;
  for (int card = 0; card < o->deck; ++card) {
    int on = 0;
    for (int k = 0; k < nboard; ++k) on |= board[k] == card;
    if (!on) live[nlive++] = card;
  }
  int* kids = (int*)malloc(sizeof(int) * (size_t)nlive);
  for (int k = 0; k < nlive; ++k) {
    int nb[5];
    for (int j = 0; j < nboard; ++j) nb[j] = board[j];
    nb[nboard] = live[k];
    int all_in = (o->game == G_HOLDEM) && (c[0] >= o->cap || c[1] >= o->cap);
    int kid;
    if (all_in)  /* nobody can bet any more: run the cards out */
      kid = build_street_end(o, id, k, street + 1, c, nboard + 1, nb, live[k]);
    else
      kid = build_decision(o, id, k, street + 1, c, nboard + 1, nb, live[k], 0, 0, 0);
    kids[k] = kid;
  }
  o->nodes[id].kids = kids;
  o->nodes[id].nkids = nlive;
  return id;
}

static int build_decision(Oracle* o, int parent, int paction, int street, const double c[2], int nboard,
                          const int* board, int deal, int p, int nraises, int first_checked) {
  int id = new_node(o, T_DEC, p, parent, paction, street, c, nboard, board, deal);
  int q = 1 - p;
  int facing = c[q] > c[p];
  /* action list: [fold], check/call, then raises in increasing size */
  double targets[20];
  int ntargets = 0;
  int can_raise = nraises < o->max_raises;
  if (o->game == G_HOLDEM) can_raise = can_raise && c[q] < o->cap && c[p] < o->cap;
  if (can_raise) {
    if (o->game == G_HOLDEM) {
      double d = c[q] - c[p];
      double potnow = c[0] + c[1];
      for (int k = 0; k < o->nsizes; ++k) {
        double target;
        if (o->sizes[k] <= 0.0) {
          target = o->cap;
        } else {
          double add = d + o->sizes[k] * (potnow + d);
          target = c[p] + add;
          if (target >= o->cap) target = o->cap;
        }
        int dup = 0;
        for (int j = 0; j < ntargets; ++j) dup |= targets[j] == target;
        if (!dup && target > c[q]) targets[ntargets++] = target;
      }
      /* increasing order (insertion sort; at most a handful) */
      for (int i = 1; i < ntargets; ++i)
        for (int j = i; j > 0 && targets[j - 1] > targets[j]; --j) {
          double tmp = targets[j];
          targets[j] = targets[j - 1];
          targets[j - 1] = tmp;
        }
    } else {
      targets[ntargets++] = c[q] + street_bet_limit(o, street);
    }
  }
  int nk = (facing ? 2 : 1) + ntargets;
  int* kids = (int*)malloc(sizeof(int) * (size_t)nk);
  int k = 0;
  if (facing) {
    kids[k] = new_node(o, T_FOLD, p, id, k, street, c, nboard, board, -1);
    ++k;
    double cc[2] = {c[0], c[1]};
    cc[p] = c[q];
    kids[k] = build_street_end(o, id, k, street, cc, nboard, board, -1);
    ++k;
  } else {
    if (first_checked || p == 1) {
      /* the second player checks behind: the street is over */
      kids[k] = build_street_end(o, id, k, street, c, nboard, board, -1);
    } else {
      kids[k] = build_decision(o, id, k, street, c, nboard, board, -1, q, nraises, 1);
    }
    ++k;
  }
  for (int j = 0; j < ntargets; ++j) {
    double cc[2] = {c[0], c[1]};
    cc[p] = targets[j];
    kids[k] = build_decision(o, id, k, street, cc, nboard, board, -1, q, nraises + 1, first_checked);
    ++k;
  }
  /* build_* calls may have moved o->nodes */
  o->nodes[id].kids = kids;
  o->nodes[id].nkids = nk;
  return id;
}

/* Showdown strength of hand h at a showdown node (higher wins, equal splits). */
static int strength_at(const Oracle* o, const Node* n, int h) {
  if (o->game == G_KUHN) return o->cards[h];
  if (o->game == G_LEDUC) {
    int rank = o->cards[h] / 2, brank = n->board[0] / 2;
    return rank == brank ? 10 + rank : rank;
  }
  /* row of the completed board: 0 (river), the river card (turn), turn x 52 + river (flop) */
  int row = o->nstr == 1 ? 0 : o->nstr == 52 ? n->board[4] : n->board[3] * 52 + n->board[4];
  return o->strength[(size_t)row * (size_t)o->nh + (size_t)h];
}

static double utility(const Oracle* o, const Node* n, int i, int hi, int ho) {
  if (n->type == T_FOLD) return n->player == i ? -n->c[i] : n->c[1 - i];
  int si = strength_at(o, n, hi), so = strength_at(o, n, ho);
  if (si > so) return n->c[1 - i];
  if (si < so) return -n->c[i];
  return 0.0;
}

static int hand_has(const Oracle* o, int h, int card) { return (int)((o->hmask[h] >> card) & 1u); }

/* Depth-limit leaf (Section 3): the river card is dealt by chance, 1/K each of the K cards
 * left given both hands, and the network's value per unit pot of player i's hand on the
 * completed board stands for the rest of the game: u_i = sum_r (1/K) pot y_i^r(h_i). */
static double leaf_utility(const Oracle* o, const Node* n, int i, int hi, int ho) {
  if (!n->leafy) return 0.0;
  uint64_t dead = o->hmask[hi] | o->hmask[ho];
  uint64_t on = 0;
  for (int k = 0; k < n->nboard; ++k) on |= 1ull << n->board[k];
  double K = (double)(o->deck - n->nboard - 2 * o->hsize), pot = n->c[0] + n->c[1], u = 0.0;
  for (int card = 0, r = 0; card < o->deck; ++card) {
    if ((on >> card) & 1u) continue;
    if (!((dead >> card) & 1u)) u += n->leafy[((size_t)r * 2 + (size_t)i) * o->nh + (size_t)hi];
    ++r;
  }
  return u * pot / K;
}

/* ------------------------------------------------------------------ creation */

Oracle* ocfr_create(int game, int nboard, const int* board, int nh, const int* cards, const double* r0,
                    const double* r1, const int* strength, int nstr, double pot, double stack, int nsizes,
                    const double* sizes, int max_raises, int variant, double alpha, double beta, double gamma,
                    int alternating, int nthreads, int depth_limit, const int* exact_flags, int n_exact_flags) {
  g_err[0] = 0;
  if (nh <= 0 || !cards || !r0 || !r1) {
    snprintf(g_err, sizeof g_err, "empty hand list or range");
    return NULL;
  }
  Oracle* o = (Oracle*)calloc(1, sizeof(Oracle));
  o->game = game;
  o->nh = nh;
  o->variant = variant;
  o->alpha = alpha;
  o->beta = beta;
  o->gamma = gamma;
  o->alternating = alternating;
  o->nthreads = nthreads < 1 ? 1 : nthreads;
  o->max_raises = max_raises;
  o->depth_limit = depth_limit;
  if (n_exact_flags > 0 && exact_flags) {
    o->exact_flags = (int*)malloc(sizeof(int) * (size_t)n_exact_flags);
    memcpy(o->exact_flags, exact_flags, sizeof(int) * (size_t)n_exact_flags);
    o->n_exact_flags = n_exact_flags;
  }
  int start_board[5] = {0};
  int nb0 = 0;
  if (game == G_KUHN) {
    o->deck = 3; o->hsize = 1; o->nstreets = 1; o->pot = 2.0;
  } else if (game == G_LEDUC) {
    o->deck = 6; o->hsize = 1; o->nstreets = 2; o->pot = 2.0;
  } else {
    o->deck = 52; o->hsize = 2;
    if (nboard == 5) o->nstreets = 1;
    else if (nboard == 4) o->nstreets = 2;
    else if (nboard == 3) o->nstreets = 3;
    else { snprintf(g_err, sizeof g_err, "hold'em subgames start on the flop, turn or river"); free(o->exact_flags); free(o); return NULL; }
    nb0 = nboard;
    for (int k = 0; k < nboard; ++k) start_board[k] = board[k];
    o->pot = pot;
    o->stack = stack;
    o->cap = pot / 2.0 + stack;
    o->nsizes = nsizes;
    for (int k = 0; k < nsizes && k < 16; ++k) o->sizes[k] = sizes[k];
    o->strength = (int*)malloc(sizeof(int) * (size_t)nstr * (size_t)nh);
    memcpy(o->strength, strength, sizeof(int) * (size_t)nstr * (size_t)nh);
    o->nstr = nstr;
    if (!((nboard == 5 && nstr == 1) || (nboard == 4 && nstr == 52) || (nboard == 3 && nstr == 52 * 52))) {
      snprintf(g_err, sizeof g_err, "strength rows do not match the board");
      free(o->strength);
      free(o->exact_flags);
      free(o);
      return NULL;
    }
  }
  o->cards = (int*)malloc(sizeof(int) * (size_t)nh * (size_t)o->hsize);
  o->hmask = (uint64_t*)calloc((size_t)nh, sizeof(uint64_t));
  uint64_t bmask = 0;
  for (int k = 0; k < nb0; ++k) bmask |= 1ull << start_board[k];
  for (int h = 0; h < nh; ++h) {
    for (int k = 0; k < o->hsize; ++k) {
      int cd = cards[h * o->hsize + k];
      o->cards[h * o->hsize + k] = cd;
      if (cd < 0 || cd >= o->deck || ((o->hmask[h] >> cd) & 1u) || ((bmask >> cd) & 1u)) {
        snprintf(g_err, sizeof g_err, "hand %d has an invalid or repeated card", h);
        return NULL;
      }
      o->hmask[h] |= 1ull << cd;
    }
  }
  /* normalise the ranges: each sums to one over the hand list */
  for (int p = 0; p < 2; ++p) {
    const double* src = p ? r1 : r0;
    double s = 0.0;
    for (int h = 0; h < nh; ++h) s += src[h];
    o->r[p] = (double*)malloc(sizeof(double) * (size_t)nh);
    for (int h = 0; h < nh; ++h) o->r[p][h] = src[h] / s;
  }
  o->compat = (unsigned char*)malloc((size_t)nh * (size_t)nh);
  double Z = 0.0;
  for (int a = 0; a < nh; ++a)
    for (int b = 0; b < nh; ++b) {
      int ok = (o->hmask[a] & o->hmask[b]) == 0;
      o->compat[(size_t)a * nh + b] = (unsigned char)ok;
      if (ok) Z += o->r[0][a] * o->r[1][b];
    }
  o->Z = Z;
  if (!(Z > 0.0)) {
    snprintf(g_err, sizeof g_err, "no pair of hands can be dealt with positive probability");
    return NULL;
  }
  double c0[2] = {o->pot / 2.0, o->pot / 2.0};
  build_decision(o, -1, 0, 0, c0, nb0, start_board, -1, 0, 0, 0);
  int rows = 0;
  for (int n = 0; n < o->nn; ++n)
    if (o->nodes[n].type == T_DEC) {
      o->nodes[n].row = rows;
      rows += o->nodes[n].nkids;
    }
  o->nrows = rows;
  size_t cells = (size_t)rows * (size_t)nh;
  o->R = (double*)calloc(cells, sizeof(double));
  o->S = (double*)calloc(cells, sizeof(double));
  o->sig = (double*)calloc(cells, sizeof(double));
  o->prof = (double*)calloc(cells, sizeof(double));
  o->rinst = (double*)calloc(cells, sizeof(double));
  o->M = (double*)calloc(cells, sizeof(double));
  o->cfv[0] = (double*)calloc((size_t)o->nn * nh, sizeof(double));
  o->cfv[1] = (double*)calloc((size_t)o->nn * nh, sizeof(double));
  return o;
}

void ocfr_destroy(Oracle* o) {
  if (!o) return;
  for (int n = 0; n < o->nn; ++n) {
    free(o->nodes[n].kids);
    free(o->nodes[n].leafy);
  }
  free(o->nodes);
  free(o->cards); free(o->hmask); free(o->r[0]); free(o->r[1]); free(o->strength);
  free(o->R); free(o->S); free(o->sig); free(o->prof); free(o->rinst); free(o->M);
  free(o->cfv[0]); free(o->cfv[1]); free(o->compat); free(o->exact_flags);
  free(o);
}

/* ------------------------------------------------------------------ regret matching, Eq. (rm) */

/* Regret matching (Eq. rm) of R; Predictive CFR+ matches R + M, the regrets plus the
 * prediction of the next instantaneous regret. */
static void regret_match(const Oracle* o, const double* R, double* out) {
  const int pred = o->variant == V_PCFRPLUS;
  for (int n = 0; n < o->nn; ++n) {
    const Node* nd = &o->nodes[n];
    if (nd->type != T_DEC) continue;
    for (int h = 0; h < o->nh; ++h) {
      double pos = 0.0;
      for (int a = 0; a < nd->nkids; ++a) {
        size_t cell = (size_t)(nd->row + a) * o->nh + h;
        double x = R[cell] + (pred ? o->M[cell] : 0.0);
        if (x > 0.0) pos += x;
      }
      for (int a = 0; a < nd->nkids; ++a) {
        size_t cell = (size_t)(nd->row + a) * o->nh + h;
        double x = R[cell] + (pred ? o->M[cell] : 0.0);
        out[cell] = pos > 0.0 ? (x > 0.0 ? x : 0.0) / pos : 1.0 / nd->nkids;
      }
    }
  }
}

/* average strategy S / sum S, uniform where nothing was accumulated */
static void average_strategy(const Oracle* o, double* out) {
  for (int n = 0; n < o->nn; ++n) {
    const Node* nd = &o->nodes[n];
    if (nd->type != T_DEC) continue;
    for (int h = 0; h < o->nh; ++h) {
      double s = 0.0;
      for (int a = 0; a < nd->nkids; ++a) s += o->S[(size_t)(nd->row + a) * o->nh + h];
      for (int a = 0; a < nd->nkids; ++a)
        out[(size_t)(nd->row + a) * o->nh + h] =
            s > 0.0 ? o->S[(size_t)(nd->row + a) * o->nh + h] / s : 1.0 / nd->nkids;
    }
  }
}

/* ------------------------------------------------------------------ the history walk */

typedef struct {
  const Oracle* o;
  const double* strat; /* strategy profile used for both players */
  int i;               /* traversing (updating) player */
  int accumulate;      /* add regrets into rinst */
  int h_begin, h_end;  /* range of player i's hands handled by this worker */
} Walk;

/* Expected utility u_i of the history (node, hands) under the profile; adds
 * pi_{-i} pi_c (u(h.a) - u(h)) to player i's instantaneous regrets and pi_{-i} pi_c u(h)
 * to the counterfactual values (Eq. cfv). */
static double walk(const Walk* w, int node, const int hands[2], double pi0, double pi1, double pc) {
  const Oracle* o = w->o;
  const Node* n = &o->nodes[node];
  int i = w->i;
  double pio = i == 0 ? pi1 : pi0;
  double u;
  if (n->type == T_FOLD || n->type == T_SHOW) {
    u = utility(o, n, i, hands[i], hands[1 - i]);
  } else if (n->type == T_LEAF) {
    u = leaf_utility(o, n, i, hands[i], hands[1 - i]);
  } else if (n->type == T_CHANCE) {
    uint64_t dead = o->hmask[hands[0]] | o->hmask[hands[1]];
    for (int k = 0; k < n->nboard; ++k) dead |= 1ull << n->board[k];
    int K = 0;
    for (int card = 0; card < o->deck; ++card) K += !((dead >> card) & 1u);
    u = 0.0;
    for (int k = 0; k < n->nkids; ++k) {
      int kid = n->kids[k];
      int card = o->nodes[kid].deal;
      if ((dead >> card) & 1u) continue;
      u += walk(w, kid, hands, pi0, pi1, pc / K) / K;
    }
  } else {
    int p = n->player;
    double ua[20];
    u = 0.0;
    for (int a = 0; a < n->nkids; ++a) {
      double s = w->strat[(size_t)(n->row + a) * o->nh + hands[p]];
      ua[a] = walk(w, n->kids[a], hands, p == 0 ? pi0 * s : pi0, p == 1 ? pi1 * s : pi1, pc);
      u += s * ua[a];
    }
    if (p == i && w->accumulate) {
      double cf = pio * pc;
      for (int a = 0; a < n->nkids; ++a) o->rinst[(size_t)(n->row + a) * o->nh + hands[i]] += cf * (ua[a] - u);
    }
  }
  o->cfv[i][(size_t)node * o->nh + hands[i]] += pio * pc * u;
  return u;
}

static void* walk_worker(void* arg) {
  const Walk* w = (const Walk*)arg;
  const Oracle* o = w->o;
  int i = w->i;
  for (int hi = w->h_begin; hi < w->h_end; ++hi) {
    for (int ho = 0; ho < o->nh; ++ho) {
      int h0 = i == 0 ? hi : ho, h1 = i == 0 ? ho : hi;
      if (!o->compat[(size_t)h0 * o->nh + h1]) continue;
      int hands[2] = {h0, h1};
      walk(w, 0, hands, o->r[0][h0], o->r[1][h1], 1.0 / o->Z);
    }
  }
  return NULL;
}

/* Walk every deal for traversing player i; work is split over player i's hands, so each
 * worker writes disjoint columns and the result does not depend on the thread count. */
static void traverse(Oracle* o, const double* strat, int i, int accumulate) {
  memset(o->cfv[i], 0, sizeof(double) * (size_t)o->nn * o->nh);
  if (accumulate) memset(o->rinst, 0, sizeof(double) * (size_t)o->nrows * o->nh);
  int nt = o->nthreads > o->nh ? o->nh : o->nthreads;
  Walk ws[256];
  pthread_t th[256];
  if (nt > 256) nt = 256;
  for (int k = 0; k < nt; ++k) {
    ws[k].o = o;
    ws[k].strat = strat;
    ws[k].i = i;
    ws[k].accumulate = accumulate;
    ws[k].h_begin = (int)((long)o->nh * k / nt);
    ws[k].h_end = (int)((long)o->nh * (k + 1) / nt);
  }
  if (nt == 1) {
    walk_worker(&ws[0]);
  } else {
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, walk_worker, &ws[k]);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  }
}

/* ------------------------------------------------------------------ Stage 7 update */

/* Own-reach walk: adds weight * pi_i(I) * sigma(I, a) to S (Section 4.2, Stage 1). */
static void own_reach(Oracle* o, int node, int i, int h, double reach, double weight) {
  const Node* n = &o->nodes[node];
  if (n->type == T_DEC) {
    for (int a = 0; a < n->nkids; ++a) {
      size_t cell = (size_t)(n->row + a) * o->nh + h;
      double s = n->player == i ? o->sig[cell] : 1.0;
      if (n->player == i) o->S[cell] += weight * reach * s;
      own_reach(o, n->kids[a], i, h, reach * s, weight);
    }
  } else if (n->type == T_CHANCE) {
    for (int k = 0; k < n->nkids; ++k) {
      int kid = n->kids[k];
      if (hand_has(o, h, o->nodes[kid].deal)) continue;
      own_reach(o, kid, i, h, reach, weight);
    }
  }
}

static void update_player(Oracle* o, int i, int t) {
  double dpos = 1.0, dneg = 1.0, dS = 1.0, wS = 1.0;
  if (o->variant == V_DCFR) {
    double ta = pow((double)t, o->alpha), tb = pow((double)t, o->beta);
    dpos = ta / (ta + 1.0);
    dneg = tb / (tb + 1.0);
    dS = pow((double)t / (double)(t + 1), o->gamma);
  } else if (o->variant == V_CFRPLUS) {
    wS = (double)t;
  } else if (o->variant == V_PCFRPLUS) {
    wS = (double)t * (double)t;  /* quadratic averaging */
  }
  for (int n = 0; n < o->nn; ++n) {
    const Node* nd = &o->nodes[n];
    if (nd->type != T_DEC || nd->player != i) continue;
    for (int a = 0; a < nd->nkids; ++a)
      for (int h = 0; h < o->nh; ++h) {
        size_t cell = (size_t)(nd->row + a) * o->nh + h;
        double x = o->R[cell] + o->rinst[cell];
        if (o->variant == V_DCFR) x *= x > 0.0 ? dpos : dneg;
        if ((o->variant == V_CFRPLUS || o->variant == V_PCFRPLUS) && x < 0.0) x = 0.0;
        o->R[cell] = x;
        if (o->variant == V_PCFRPLUS) o->M[cell] = o->rinst[cell];  /* predict the next regret */
        o->S[cell] *= dS;
      }
  }
  for (int h = 0; h < o->nh; ++h) own_reach(o, 0, i, h, o->r[i][h], wS);
}

/* Player i's update at iteration t: regret matching of the current R of both players,
 * player i's traversal, player i's update.  The iteration count is not advanced. */
void ocfr_update_player(Oracle* o, int i, int t) {
  regret_match(o, o->R, o->sig);
  traverse(o, o->sig, i, 1);
  update_player(o, i, t);
}

/* Both players' updates at iteration t from one strategy (simultaneous updates). */
void ocfr_update_both(Oracle* o, int t) {
  regret_match(o, o->R, o->sig);
  double* saved = (double*)malloc(sizeof(double) * (size_t)o->nrows * o->nh);
  traverse(o, o->sig, 0, 1);
  memcpy(saved, o->rinst, sizeof(double) * (size_t)o->nrows * o->nh);
  traverse(o, o->sig, 1, 1);
  /* player 1's regrets are in rinst; apply them, then player 0's */
  update_player(o, 1, t);
  memcpy(o->rinst, saved, sizeof(double) * (size_t)o->nrows * o->nh);
  update_player(o, 0, t);
  free(saved);
}

/* One iteration (both players), Section 4.1 pipeline order: profile, values, update. */
void ocfr_iterate(Oracle* o, int n_iters) {
  for (int it = 0; it < n_iters; ++it) {
    int t = o->t + 1;
    if (o->alternating) {
      ocfr_update_player(o, 0, t);
      ocfr_update_player(o, 1, t);
    } else {
      ocfr_update_both(o, t);
    }
    o->t = t;
  }
}

/* Overwrite one decision node's cumulative regrets and average-strategy sums ([nkids][nh]
 * each), so that a test can start an update from another implementation's state. */
int ocfr_set_node_state(Oracle* o, int node, const double* R, const double* S) {
  if (node < 0 || node >= o->nn || o->nodes[node].type != T_DEC) return -1;
  const Node* nd = &o->nodes[node];
  size_t off = (size_t)nd->row * o->nh, len = (size_t)nd->nkids * o->nh;
  memcpy(o->R + off, R, sizeof(double) * len);
  memcpy(o->S + off, S, sizeof(double) * len);
  return 0;
}

void ocfr_set_iterations(Oracle* o, int t) { o->t = t; }

/* Overwrite a decision node's Predictive CFR+ prediction ([nkids][nh]). */
int ocfr_set_node_pred(Oracle* o, int node, const double* M) {
  if (node < 0 || node >= o->nn || o->nodes[node].type != T_DEC) return -1;
  const Node* nd = &o->nodes[node];
  memcpy(o->M + (size_t)nd->row * o->nh, M, sizeof(double) * (size_t)nd->nkids * o->nh);
  return 0;
}

/* ------------------------------------------------------------------ profiles and best response */

/* kind 0: current strategy (regret matching of R); kind 1: average strategy. */
void ocfr_load_profile(Oracle* o, int kind) {
  if (kind == 0) regret_match(o, o->R, o->prof);
  else average_strategy(o, o->prof);
}

/* Overwrite one decision node's rows of the loaded profile: vals is [nkids][nh]. */
int ocfr_set_profile_node(Oracle* o, int node, const double* vals) {
  if (node < 0 || node >= o->nn || o->nodes[node].type != T_DEC) return -1;
  const Node* nd = &o->nodes[node];
  memcpy(o->prof + (size_t)nd->row * o->nh, vals, sizeof(double) * (size_t)nd->nkids * o->nh);
  return 0;
}

/* Expected utility of each player under the loaded profile (walks every history).
 * Also leaves that profile's counterfactual values in cfv[0], cfv[1]. */
void ocfr_profile_value(Oracle* o, double out[2]) {
  for (int i = 0; i < 2; ++i) {
    traverse(o, o->prof, i, 0);
    double v = 0.0;
    for (int h = 0; h < o->nh; ++h) v += o->r[i][h] * o->cfv[i][h]; /* root is node 0 */
    out[i] = v;
  }
}

typedef struct {
  const Oracle* o;
  const double* q; /* opponent reach [nn][nh] */
  int i;
  double* out;     /* [nn][nh] best-response counterfactual values */
  int h_begin, h_end;
} BRWork;

static double br_rec(const BRWork* w, int node, int h) {
  const Oracle* o = w->o;
  const Node* n = &o->nodes[node];
  int i = w->i;
  double v = 0.0;
  if (n->type == T_FOLD || n->type == T_SHOW || n->type == T_LEAF) {
    const unsigned char* cm = o->compat + (size_t)h * o->nh;
    const double* q = w->q + (size_t)node * o->nh;
    for (int ho = 0; ho < o->nh; ++ho)
      if (cm[ho] && q[ho] != 0.0)
        v += q[ho] * (n->type == T_LEAF ? leaf_utility(o, n, i, h, ho) : utility(o, n, i, h, ho));
    v /= o->Z;
  } else if (n->type == T_CHANCE) {
    /* the card probability is inside the opponent-and-chance reach q below this node */
    for (int k = 0; k < n->nkids; ++k) {
      int kid = n->kids[k];
      if (hand_has(o, h, o->nodes[kid].deal)) continue;
      v += br_rec(w, kid, h);
    }
  } else if (n->player == i) {
    v = -INFINITY;
    for (int a = 0; a < n->nkids; ++a) {
      double x = br_rec(w, n->kids[a], h);
      if (x > v) v = x;
    }
  } else {
    for (int a = 0; a < n->nkids; ++a) v += br_rec(w, n->kids[a], h);
  }
  w->out[(size_t)node * o->nh + h] = v;
  return v;
}

static void* br_worker(void* arg) {
  const BRWork* w = (const BRWork*)arg;
  for (int h = w->h_begin; h < w->h_end; ++h) br_rec(w, 0, h);
  return NULL;
}

/* Counterfactual reach of every (node, opponent hand) under the loaded profile: the
 * opponent's range and action probabilities times the probability of the public cards dealt
 * on the path (1/K per card, K the cards left given both hands), as in Eq. (cfv); cards
 * dealt on the path remove the hands that hold them. */
static void opponent_reach(const Oracle* o, int opp, double* q) {
  for (int h = 0; h < o->nh; ++h) q[h] = o->r[opp][h];
  for (int n = 0; n < o->nn; ++n) {  /* parents are created before children */
    const Node* nd = &o->nodes[n];
    if (nd->type == T_DEC) {
      for (int a = 0; a < nd->nkids; ++a)
        for (int h = 0; h < o->nh; ++h)
          q[(size_t)nd->kids[a] * o->nh + h] =
              q[(size_t)n * o->nh + h] * (nd->player == opp ? o->prof[(size_t)(nd->row + a) * o->nh + h] : 1.0);
    } else if (nd->type == T_CHANCE) {
      double K = (double)(o->deck - nd->nboard - 2 * o->hsize);
      for (int k = 0; k < nd->nkids; ++k) {
        int kid = nd->kids[k];
        for (int h = 0; h < o->nh; ++h)
          q[(size_t)kid * o->nh + h] = hand_has(o, h, o->nodes[kid].deal) ? 0.0 : q[(size_t)n * o->nh + h] / K;
      }
    }
  }
}

/* Best-response value of player i against the loaded profile of the opponent:
 * BR_i = sum_h r_i(h) v*_i(root, h).  root_out (optional) receives v*_i(root, .);
 * all_out (optional) receives v*_i for every node, [nn][nh]. */
double ocfr_best_response(Oracle* o, int i, double* root_out, double* all_out) {
  size_t cells = (size_t)o->nn * o->nh;
  double* q = (double*)malloc(sizeof(double) * cells);
  double* v = (double*)calloc(cells, sizeof(double));
  /* a child may precede its parent only if created earlier; the builder creates a node
   * before its children, so one pass in id order propagates reach top-down */
  opponent_reach(o, 1 - i, q);
  int nt = o->nthreads > o->nh ? o->nh : o->nthreads;
  if (nt > 256) nt = 256;
  BRWork ws[256];
  pthread_t th[256];
  for (int k = 0; k < nt; ++k) {
    ws[k].o = o; ws[k].q = q; ws[k].i = i; ws[k].out = v;
    ws[k].h_begin = (int)((long)o->nh * k / nt);
    ws[k].h_end = (int)((long)o->nh * (k + 1) / nt);
  }
  if (nt == 1) br_worker(&ws[0]);
  else {
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, br_worker, &ws[k]);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  }
  double br = 0.0;
  for (int h = 0; h < o->nh; ++h) br += o->r[i][h] * v[h];
  if (root_out) memcpy(root_out, v, sizeof(double) * (size_t)o->nh);
  if (all_out) memcpy(all_out, v, sizeof(double) * cells);
  free(q);
  free(v);
  return br;
}

/* Exploitability of the average strategy in chips: (BR_0 + BR_1) / 2. */
double ocfr_exploitability(Oracle* o, double br_out[2]) {
  ocfr_load_profile(o, 1);
  double b0 = ocfr_best_response(o, 0, NULL, NULL);
  double b1 = ocfr_best_response(o, 1, NULL, NULL);
  if (br_out) { br_out[0] = b0; br_out[1] = b1; }
  return 0.5 * (b0 + b1);
}

/* ------------------------------------------------------------------ depth-limit leaves */

/* Player p's own reach at `node` for every hand: p's range times p's action probabilities
 * on the path (kind 0: current strategy, regret matching of R; kind 1: average strategy),
 * zero for hands holding a card dealt on the path. */
int ocfr_node_reach(Oracle* o, int kind, int p, int node, double* out) {
  if (node < 0 || node >= o->nn) return -1;
  double* prof = (double*)malloc(sizeof(double) * (size_t)o->nrows * o->nh);
  if (kind == 0) regret_match(o, o->R, prof);
  else average_strategy(o, prof);
  for (int h = 0; h < o->nh; ++h) out[h] = o->r[p][h];
  int path[256], len = 0;
  for (int n = node; n > 0 && len < 256; n = o->nodes[n].parent) path[len++] = n;
  for (int k = len - 1; k >= 0; --k) {
    const Node* child = &o->nodes[path[k]];
    const Node* par = &o->nodes[child->parent];
    for (int h = 0; h < o->nh; ++h) {
      if (par->type == T_DEC && par->player == p) out[h] *= prof[(size_t)(par->row + child->paction) * o->nh + h];
      if (child->deal >= 0 && hand_has(o, h, child->deal)) out[h] = 0.0;
    }
  }
  free(prof);
  return 0;
}

/* Network outputs at a leaf: y [K][2][nh], one block per river card not on the leaf's board
 * (ascending), per player the value per unit pot of each hand. */
int ocfr_set_leaf_values(Oracle* o, int node, const double* y) {
  if (node < 0 || node >= o->nn || o->nodes[node].type != T_LEAF) return -1;
  Node* n = &o->nodes[node];
  const size_t K = (size_t)(o->deck - n->nboard);
  if (!n->leafy) n->leafy = (double*)malloc(sizeof(double) * K * 2 * (size_t)o->nh);
  memcpy(n->leafy, y, sizeof(double) * K * 2 * (size_t)o->nh);
  return 0;
}

/* ------------------------------------------------------------------ accessors */

int ocfr_n_nodes(const Oracle* o) { return o->nn; }
int ocfr_n_hands(const Oracle* o) { return o->nh; }
int ocfr_n_rows(const Oracle* o) { return o->nrows; }
int ocfr_iters(const Oracle* o) { return o->t; }
double ocfr_Z(const Oracle* o) { return o->Z; }

/* out[0..8] = type, player, parent, paction, nkids, street, deal, nboard, row; c[0..1] */
void ocfr_node(const Oracle* o, int node, int* out, double* c) {
  const Node* n = &o->nodes[node];
  out[0] = n->type; out[1] = n->player; out[2] = n->parent; out[3] = n->paction;
  out[4] = n->nkids; out[5] = n->street; out[6] = n->deal; out[7] = n->nboard; out[8] = n->row;
  c[0] = n->c[0];
  c[1] = n->c[1];
}

int ocfr_child(const Oracle* o, int node, int k) { return o->nodes[node].kids[k]; }

/* what: 0 cumulative regret R, 1 average-strategy sum S, 2 current strategy (regret
 * matching of R), 3 loaded profile.  out is [nkids][nh]. */
int ocfr_get_node(Oracle* o, int what, int node, double* out) {
  if (node < 0 || node >= o->nn || o->nodes[node].type != T_DEC) return -1;
  const Node* nd = &o->nodes[node];
  size_t off = (size_t)nd->row * o->nh, len = (size_t)nd->nkids * o->nh;
  if (what == 0) memcpy(out, o->R + off, sizeof(double) * len);
  else if (what == 1) memcpy(out, o->S + off, sizeof(double) * len);
  else if (what == 4) memcpy(out, o->M + off, sizeof(double) * len);
  else if (what == 2) {
    regret_match(o, o->R, o->sig);
    memcpy(out, o->sig + off, sizeof(double) * len);
  } else memcpy(out, o->prof + off, sizeof(double) * len);
  return 0;
}

/* counterfactual values v_i(node, .) from the last traversal of player i */
void ocfr_get_cfv(const Oracle* o, int i, int node, double* out) {
  memcpy(out, o->cfv[i] + (size_t)node * o->nh, sizeof(double) * (size_t)o->nh);
}

/* Run only player i's traversal under the current strategy (no update) and report the
 * counterfactual values it produces; used to pin values against brute force. */
void ocfr_values_current(Oracle* o, int i) {
  regret_match(o, o->R, o->sig);
  traverse(o, o->sig, i, 0);
}
