/*
 * pcfr.h -- C ABI of the GB300 Parallel CFR library (libpcfr.so).
 *
 * One CFR iteration over a public poker tree whose nodes hold per-private-hand range and
 * value vectors, after "Real-Time Parallel Counterfactual Regret Minimization"
 * (arxiv 2605.19928).  The iteration follows the paper's seven-stage pipeline (Section 4.1,
 * Table 1): regret matching (Section 3, Eq. rm), forward reach (Section 4.2, Stages 1-2),
 * blocker-corrected opponent reach at fold terminals (Stage 3), rank-sorted showdown values
 * (Stage 4), depth-limit leaves (Stage 5: exact chance nodes, or the BF16 leaf network on
 * the tensor cores), backward counterfactual values (Section 4.4, Stage 6, Eq. backward)
 * and the regret / average-strategy update (Stage 7) for vanilla CFR, CFR+, DCFR (Section
 * 2) and Predictive CFR+ (Section 5).  Exploitability uses a best-response pass.  One
 * handle holds one subgame or a batch of them (batched serving).
 *
 * Conventions
 *   - Every function returns CFR_OK (0) or a negative CFR_E* code; cfr_last_error()
 *     returns a thread-local message describing the last failure on the calling thread.
 *   - All pointers in this header are HOST pointers unless stated otherwise.  Input arrays
 *     are copied during create; the caller keeps ownership of everything it passes.
 *     Output buffers are caller-owned host memory.
 *   - Device memory is owned by the library.  It comes from the allocator installed with
 *     cfr_set_allocator(), else from cudaMalloc.
 *   - Work is enqueued on the CUDA stream given at create (NULL = the legacy default
 *     stream).  cfr_iterate() is asynchronous; calls that return data synchronise.
 *   - There is no CPU fallback: without a CUDA device of compute capability 10.3 the
 *     create call fails with CFR_ECUDA.
 *   - A tree handle must not be used from two threads at once.
 */
#ifndef PCFR_H
#define PCFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CFR_OK 0
#define CFR_EINVAL (-1)   /* bad argument or game description */
#define CFR_ENOMEM (-2)   /* host or device allocation failed */
#define CFR_ECUDA (-3)    /* CUDA error or no suitable device */
#define CFR_ETIMEOUT (-4) /* a bounded device-side wait gave up (reported by synchronising calls) */
#define CFR_ESTATE (-5)   /* call not valid in the handle's current state */

enum { CFR_GAME_HOLDEM = 0, CFR_GAME_KUHN = 1, CFR_GAME_LEDUC = 2 };
enum { CFR_VARIANT_CFR = 0, CFR_VARIANT_CFRPLUS = 1, CFR_VARIANT_DCFR = 2, CFR_VARIANT_PCFRPLUS = 3 };
enum { CFR_NODE_DECISION = 0, CFR_NODE_FOLD = 1, CFR_NODE_SHOWDOWN = 2, CFR_NODE_CHANCE = 3, CFR_NODE_LEAF = 4 };
enum {
  CFR_READ_REGRET = 0,
  CFR_READ_AVG_SUM = 1,
  CFR_READ_CFV = 2,
  CFR_READ_BR_CFV = 3,
  CFR_READ_PREDICTION = 4,
  CFR_READ_AVG_REACH = 5
};

/*
 * One subgame (Section 5, "Game": heads-up poker solved to the end of a betting round).
 *   game        CFR_GAME_HOLDEM: a hold'em flop (n_board 3: flop betting, a chance node
 *               over the turn card, turn betting, a chance node over the river card, river
 *               betting), turn (n_board 4: from the turn betting on) or river (n_board 5)
 *               subgame;
 *               CFR_GAME_KUHN / CFR_GAME_LEDUC: the full games (board, hands, strength,
 *               pot, stack and bet sizes are ignored; range may be NULL for uniform).
 *   board       [n_board] card ids 0..51 (card = 4 * rank + suit), distinct.
 *   hands       [n_hands][2] private two-card hands, none touching the board, no
 *               duplicates; both players share this list.  NULL = every hand not blocked
 *               by the board, in lexicographic (c1 < c2) order.
 *   range[p]    [n_hands] player p's reach at the root, >= 0, not all zero; normalised
 *               internally to sum 1.  NULL = uniform.
 *   strength    showdown strength, higher wins, equal splits: [1][n_hands] for a river
 *               subgame, [52][n_hands] for a turn subgame (row = river card) and
 *               [52 * 52][n_hands] for a flop subgame (row = turn card * 52 + river card);
 *               rows of impossible boards are ignored.
 *   pot, stack  chips in the pot (each player has put in pot / 2) and behind each player.
 *   bet_sizes   [n_bet_sizes] bet sizes as pot fractions; a size <= 0 means all-in.  A size
 *               x facing a call of d raises by d + x * (pot + d); sizes reaching the stack
 *               become all-in; duplicates are dropped.
 *   max_raises  bets plus raises allowed per street (the opening bet counts).
 *   depth_limit 0: solve to the end of the game (exact).  1 (flop and turn subgames): the
 *               tree stops at the river card (Section 3, depth-limited solving): every
 *               chance node that deals the river card with chips behind becomes a
 *               CFR_NODE_LEAF whose values the leaf network gives (cfr_set_leaf_net); the
 *               flop's turn card stays a chance node and all-in run-outs stay exact.
 *   exact_leaves [n_exact_leaves] (depth_limit 1 only; may be NULL with 0): leaves to solve
 *               exactly instead, so that one handle mixes network leaves and exact river
 *               subtrees (the fallback of a leaf whose network values were judged wrong).
 *               A leaf is named by its index in the order cfr_leaf_info lists the leaves
 *               of the same subgame built with no exact leaves (the tree's breadth-first
 *               order: by the length of the action path from the root, then by the path in
 *               lexicographic order); each named position becomes the river-card chance
 *               node with its exact river subtrees.  Indices must be distinct and name
 *               leaves (CFR_EINVAL otherwise).
 */
typedef struct cfr_game_spec {
  int game;
  int n_board;
  const int32_t* board;
  int n_hands;
  const uint8_t* hands;
  const float* range[2];
  const int32_t* strength;
  int n_strength_rows;
  double pot;
  double stack;
  int n_bet_sizes;
  const double* bet_sizes;
  int max_raises;
  int depth_limit;
  const int32_t* exact_leaves;
  int n_exact_leaves;
} cfr_game_spec;

/*
 * Solver options.  variant: CFR_VARIANT_*.  DCFR uses alpha, beta, gamma (Section 2, "CFR
 * algorithms"; the paper's default is DCFR): at iteration t, R <- R + r then positive
 * regrets are scaled by t^alpha/(t^alpha+1) and the rest by t^beta/(t^beta+1);
 * S <- S * (t/(t+1))^gamma + pi_i * sigma.  CFR+: R <- max(R + r, 0), S <- S + t pi_i sigma.
 * Predictive CFR+ (the paper's second variant, Section 5, after Farina et al.): R <-
 * max(R + r, 0), the prediction M <- r (the instantaneous regret just seen), the strategy
 * is regret matching of R + M, S <- S + t^2 pi_i sigma.
 * alternating != 0 updates player 0 then player 1 (with player 0's new strategy) each
 * iteration; 0 updates both from the same strategy.
 * chunk_hands: hands per CUDA block in the per-hand passes (0 = automatic; otherwise a
 * power of two from 1 to 32).
 * precision: CFR_PRECISION_PAIRS (default) carries reach, strategies and counterfactual
 * values as double-float pairs of FP32 (about 44 significant bits, computed on the FP32
 * pipe); CFR_PRECISION_SINGLE carries them in plain FP32.  Cumulative regrets R and
 * average-strategy sums S are FP64 in both.
 * schedule: how the update launch (Stages 1, 6 and 7 of one player) is laid out; results
 * are the same bits either way.  CFR_SCHEDULE_LEVEL: one CUDA block per chunk_hands hands
 * walks the tree level by level (lowest latency for one subgame).  CFR_SCHEDULE_STREAM: one
 * warp per 32 hands walks a depth-first program of its tree with no block barriers and no
 * inner-node state in DRAM (highest throughput for batches; needs at most 8 actions per
 * decision node; warp_hands sets 32 or 64 hands per warp).  CFR_SCHEDULE_WIDE: every pass (update, initial strategy, average, best
 * response) is one launch per tree level over all of that level's (node, hand) pairs, one
 * thread each (for one tree too large for a block to stage in shared memory: exact turns
 * and flops; one subgame per handle, at most 8 actions per decision node).
 * CFR_SCHEDULE_RESIDENT: cfr_iterate runs all its iterations in one cooperative launch;
 * each block keeps one chunk of hands of both players (regrets, strategy sums, strategy,
 * reach) in shared memory for the whole launch, and a grid barrier separates an iteration's
 * phases (the terminal values of a player, then its update), so no phase is a launch of its
 * own (lowest latency for one small subgame).  Every chunk must have a block of its own at
 * one block per SM (chunk_hands = 0 takes the smallest of 8, 16 and 32 hands that allows
 * it) and the tree must have no depth-limit leaves: CFR_EINVAL otherwise.  The other passes
 * (initial strategy, average, best response) use the level schedule's kernels.  A grid
 * barrier that waits too long gives up (about a second): cfr_sync then returns
 * CFR_ETIMEOUT and the handle's state is undefined.
 * CFR_SCHEDULE_AUTO (0) picks STREAM when the handle has at least 1216 such warps (8 per
 * SM) and every tree allows it, WIDE for one subgame too large to stage, else LEVEL.
 * term_nodes: fold and showdown nodes per CUDA block of the terminal launch (nodes of one
 * board; 0 = automatic: one while the nodes do not fill the GPU eight times over, up to
 * eight when they do; otherwise 1 to 8).  Results are the same bits for every value.
 * warp_hands: hands per warp of the stream schedule's update launch: 32 (one per lane), 64
 * (two per lane: the walk's control work is shared by two hands; needs every subgame's
 * hand rows padded to a multiple of 64, i.e. the hand count rounded up to 32 is a multiple
 * of 64, CFR_EINVAL otherwise), or 0 = automatic (32; cfr_autotune tries both).  Other
 * schedules ignore it.  Results are the same bits either way.
 * runout_tables: 1 evaluates every all-in run-out -- a chance node below a decision whose
 * subtree holds only chance and showdown nodes (nobody acts again) -- in one step instead of
 * board by board (Stage 4 summed over the run-out's boards).  The value of hand h of player
 * i at the run-out's top node is then u sum_o E[h][o] q(o): q the opponent's reach there, u
 * the showdowns' payoff scale (chips in times the probability of the cards dealt, times
 * 1/Z; the same at every board of a run-out) and E[h][o] the number of the run-out's boards
 * on which h beats o less the number on which it loses, counting the boards that share no
 * card with h or o (0 if h and o share a card).  E is built once per distinct run-out board
 * at create (int8 when a run-out has at most 127 boards, else int16, [o][h]).  The nodes
 * below the top node are then not evaluated: their values and reach stay unset, and
 * cfr_read_values returns what their arrays hold.  Needs the wide schedule, FP32 values and
 * two-card hands; CFR_EINVAL otherwise.  0 (default) evaluates every showdown node.
 */
enum { CFR_PRECISION_PAIRS = 0, CFR_PRECISION_SINGLE = 1 };
enum {
  CFR_SCHEDULE_AUTO = 0,
  CFR_SCHEDULE_LEVEL = 1,
  CFR_SCHEDULE_STREAM = 2,
  CFR_SCHEDULE_WIDE = 3,
  CFR_SCHEDULE_RESIDENT = 4
};
typedef struct cfr_solver_opts {
  int variant;
  double alpha;
  double beta;
  double gamma;
  int alternating;
  int chunk_hands;
  int precision;
  int schedule;
  int term_nodes;
  int warp_hands;
  int runout_tables;
} cfr_solver_opts;

typedef struct cfr_tree cfr_tree;

/* Device allocator hook used for all later allocations (NULL, NULL = cudaMalloc/cudaFree).
 * alloc(bytes, stream, ctx) returns a device pointer or NULL; free(ptr, ctx) releases it. */
typedef void* (*cfr_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cfr_free_fn)(void* ptr, void* ctx);
int cfr_set_allocator(cfr_alloc_fn alloc, cfr_free_fn free_fn, void* ctx);

/* Build the public tree and per-hand tables of one subgame on the host, upload them and
 * initialise the solver (R = S = 0, uniform strategy).  stream: a cudaStream_t or NULL.
 * On success *out receives a handle owned by the caller (release with cfr_tree_destroy). */
int cfr_tree_create(const cfr_game_spec* spec, const cfr_solver_opts* opts, void* stream, cfr_tree** out);

/* Same for n_games independent subgames solved together; every call below then acts on
 * all of them at once, and `game` arguments select one subgame (0 .. n_games-1). */
int cfr_batch_create(const cfr_game_spec* specs, int n_games, const cfr_solver_opts* opts, void* stream,
                     cfr_tree** out);

/* Run n_iters CFR iterations (Section 4.1 pipeline, both players), asynchronously on the
 * handle's stream, in place.  The first call records a CUDA graph of one iteration and
 * later calls replay it (the resident schedule instead runs all n_iters iterations in one
 * cooperative launch). */
int cfr_iterate(cfr_tree* tree, int n_iters);

/* Strategy at a decision node: the current one (regret matching of R, Eq. rm) or, with
 * average != 0, the average strategy S / sum S (uniform where sum S = 0).  out is a host
 * buffer of [n_actions][n_hands] floats; out_len is its length in floats.  Synchronises. */
int cfr_strategy(cfr_tree* tree, int game, int node, int average, float* out, size_t out_len);

/* Exploitability of the average strategy of every subgame: expl[g] = (BR_0 + BR_1) / 2 in
 * chips, where BR_i is player i's best-response value against the other player's average
 * strategy (root reductions in FP64).  expl: [n_games]; br: [n_games][2] or NULL.  The
 * first pass on a handle launches its kernels directly; the second records them as a CUDA
 * graph, which later passes replay (same kernels, same results).  Synchronises. */
int cfr_exploitability(cfr_tree* tree, double* expl, double* br);

/* The same pass, enqueued without waiting; cfr_exploitability_result() waits for the most
 * recent pass and returns its values (arguments as for cfr_exploitability). */
int cfr_exploitability_async(cfr_tree* tree);
int cfr_exploitability_result(cfr_tree* tree, double* expl, double* br);

/* The cfr_exploitability pass without any allocation (the paper has no counterpart: it is
 * an interface for callers that may not allocate, e.g. a serving loop under a fixed
 * device-memory budget).  Launches the passes directly on the handle's stream (no graph)
 * and keeps the FP64 root reduction's scratch in one static device array of the library
 * (148 KiB per device), so at most 1024 games and 8192 hand chunks per player per handle
 * (a chunk is chunk_hands hands, 8 by default); larger handles get CFR_EINVAL.  expl:
 * [n_games]; br: [n_games][2], both required, host memory.  The first call on each device
 * does a one-time setup (resolves the array's address, loads the reduction kernel): make
 * it before any stream capture begins.  All calls on one device share the array, so calls
 * must not overlap: two calls in flight at once (other threads or other streams) race.
 * The device the handle was created on must be the current device (CFR_EINVAL otherwise).
 * The handle's own best-response pass still reduces its root values into the handle's
 * buffers; this call adds one more reduction of the same values into the static array and
 * reads the result from there.  Synchronises. */
int cfr_exploitability_noalloc(cfr_tree* tree, double* expl, double* br);

/* Start the solve again: R = S = 0, iteration count 0, uniform strategy, initial reach
 * (asynchronous, on the handle's stream). */
int cfr_reset(cfr_tree* tree);

/* Autotuner of the launch tiling (batched serving): builds the subgames under each
 * candidate layout -- the level schedule with 4, 8, 16 and 32 hands per block, the stream
 * schedule (32 and 64 hands per warp), the wide schedule (one subgame), the resident
 * schedule (where it applies), then 1, 2, 4 or 8 terminal nodes per block for the fastest
 * unless that is the resident schedule -- times `iters` iterations of each after two warm-up
 * iterations (CUDA events on `stream`, depth-limit leaves evaluated with an all-zero
 * network), and writes the fastest options to *best (opts with schedule, chunk_hands and
 * term_nodes set; term_nodes stays 0 when the automatic count was fastest) and its mean
 * device time per iteration to *ms_per_iter (may be NULL).
 * Every candidate gives the same results bit for bit, so only time decides.  opts'
 * runout_tables applies to the wide candidate only (the others run with 0); the run-out
 * tables change the summation order of the run-out values, so a wide candidate with them
 * agrees with the others to FP32 rounding instead of bit for bit.  Handles are created and
 * destroyed one at a time (device memory of one handle at most).  Errors as for
 * cfr_batch_create; CFR_EINVAL when iters < 1.  Synchronises. */
int cfr_autotune(const cfr_game_spec* specs, int n_games, const cfr_solver_opts* opts, void* stream, int iters,
                 cfr_solver_opts* best, double* ms_per_iter);

/* The schedule the handle uses (CFR_SCHEDULE_LEVEL, CFR_SCHEDULE_STREAM,
 * CFR_SCHEDULE_WIDE or CFR_SCHEDULE_RESIDENT), or a negative status. */
int cfr_schedule(const cfr_tree* tree);

/* Sizes of one subgame and the number of iterations done.  Any out pointer may be NULL. */
int cfr_tree_info(const cfr_tree* tree, int game, int* n_nodes, int* n_hands, int* iters_done);

/* One node of a subgame's public tree.  Nodes are numbered level by level from the root
 * (0); children of a node are consecutive and ordered [fold], check/call, raises by size,
 * or by dealt card for chance nodes.  Any out pointer may be NULL; contrib receives the
 * chips each player has put in at that node. */
int cfr_node_info(const cfr_tree* tree, int game, int node, int* type, int* player, int* n_actions, int* parent,
                  int* action_in_parent, int* deal_card, double* contrib);

/* Read solver state into a host buffer of doubles (synchronises):
 *   CFR_READ_REGRET, CFR_READ_AVG_SUM, CFR_READ_PREDICTION: a decision node's cumulative
 *     regrets R, average-strategy sums S or Predictive CFR+ prediction M,
 *     [n_actions][n_hands] (player is ignored);
 *   CFR_READ_CFV: player's counterfactual values at `node` from that player's last
 *     traversal, [n_hands];
 *   CFR_READ_BR_CFV: player's best-response values at `node` from the last exploitability
 *     call, [n_hands];
 *   CFR_READ_AVG_REACH: player's own reach at `node` under the average strategy (root range
 *     times the player's average action probabilities on the path, zero for hands holding a
 *     dealt card) from the last exploitability call, [n_hands]. */
int cfr_read_values(cfr_tree* tree, int game, int what, int player, int node, double* out, size_t out_len);

/* Overwrite a decision node's cumulative regrets (CFR_READ_REGRET), average-strategy sums
 * (CFR_READ_AVG_SUM) or Predictive CFR+ prediction (CFR_READ_PREDICTION) from a host buffer
 * of [n_actions][n_hands] doubles (synchronises).
 * For tests and for evaluating a strategy found elsewhere: after writing R the current
 * strategy (regret matching, Eq. rm) and both players' reach are recomputed at once; the
 * average strategy follows S at the next exploitability or cfr_strategy call. */
int cfr_write_values(cfr_tree* tree, int game, int what, int node, const double* in, size_t in_len);

/* Block until all work queued on the handle's stream has finished.  Reports CFR_ETIMEOUT if
 * a bounded device-side wait of the handle's kernels gave up (the flag stays set: release
 * the handle). */
int cfr_sync(cfr_tree* tree);

/* Testing aid for the device-side timeout path (the paper has no counterpart; the bounded
 * waits are this library's safety net, not part of the method).  Sets how many times the
 * terminal kernel's first bulk-copy wait of each block polls its barrier before giving up
 * on the current device: polls < 0 restores the default (2^20); 0 gives up before the copy
 * can land.  A block that gives up still waits, with the default limit, for its own copies
 * to land, then sets the handle's device flag and returns without computing its values,
 * so the next synchronising call on the handle reports CFR_ETIMEOUT and the CUDA context
 * stays usable.  The same limit applies to the first grid barrier of each resident-schedule
 * launch (CFR_SCHEDULE_RESIDENT): with 0 every block but the last to arrive gives up, sets
 * the flag, and the others see it at their next barrier and leave.  Call it while none of
 * the library's kernels are in flight (e.g. after cfr_sync); it applies to every handle on
 * the device until it is called again. */
int cfr_debug_first_wait_polls(long polls);

/* Per-stage device time, after the paper's per-stage breakdown (Section 5, Table 3).
 * Runs n_iters iterations (advancing the solve exactly like cfr_iterate) launch by launch
 * instead of as a graph, with CUDA events around every stage, then one exploitability
 * pass the same way.  ms[k] receives the mean device time of one occurrence of stage k
 * (one launch; a sequence of launches for the leaf stage and under CFR_SCHEDULE_WIDE) and
 * launches[k] (may be NULL) the number of occurrences timed; both have CFR_N_STAGES
 * entries.
 *   CFR_STAGE_TERMINAL    fold and showdown values of one player (Stages 2-4)
 *   CFR_STAGE_UPDATE      backward values, regret and average update, new strategy and
 *                         forward reach of one player (Stages 6-7, then 1-2)
 *   CFR_STAGE_AVG_REACH   average strategy and its forward reach, both players
 *   CFR_STAGE_BR_TERMINAL terminal values against the average strategy, both players
 *   CFR_STAGE_BR          best-response backward pass and FP64 root reduction, both players
 *   CFR_STAGE_LEAF        depth-limit leaves (Stage 5): network inputs, the four dense layers
 *                         and the leaf values (one launch sequence per player update, and
 *                         one for both players in the exploitability pass)
 * Synchronises. */
enum {
  CFR_STAGE_TERMINAL = 0,
  CFR_STAGE_UPDATE = 1,
  CFR_STAGE_AVG_REACH = 2,
  CFR_STAGE_BR_TERMINAL = 3,
  CFR_STAGE_BR = 4,
  CFR_STAGE_LEAF = 5,
  CFR_N_STAGES = 6
};
int cfr_stage_times(cfr_tree* tree, int n_iters, double* ms, int64_t* launches);

/* Counters of the handle (any out pointer may be NULL): kernels launched so far (graph
 * replays count every kernel they contain), device bytes allocated, and bytes copied host
 * to device when the handle was created. */
int cfr_counters(const cfr_tree* tree, int64_t* kernel_launches, int64_t* device_bytes, int64_t* h2d_bytes);

/* The depth-limit leaf network (Section 3, depth-limited solving; evaluated in one batch per
 * player update, Stage 5, Section 4.3) of a handle whose trees have CFR_NODE_LEAF nodes.
 * Four dense layers, BF16 weights W[k] row-major [out][in] and FP32 biases b[k]:
 *   layer 1: 2752 -> 512, GELU     layer 2: 512 -> 512, GELU
 *   layer 3: 512 -> 512, GELU      layer 4: 512 -> 2688
 * Input (per leaf and river card r): both players' reach at the leaf over the 1326 two-card
 * slots (slot of cards a < b: b (b - 1) / 2 + a), each normalised to sum 1 over the hands
 * not holding r; a one-hot of the five board cards (offset 2652); pot / (pot + 2 stack) and
 * stack / (pot + 2 stack) at the leaf (offsets 2704, 2705); zeros up to 2752.  Output:
 * player 0's then player 1's value per unit pot over the slots (offsets 0 and 1326).  The
 * value of hand h of player i at leaf n is pot(n) P(r) kappa sum over r not in h of
 * output_i,r(h) times the opponent reach over hands sharing no card with h or r.  Host
 * buffers, copied (synchronises).  Must be set before cfr_iterate on such a handle.  When
 * all subgames of the handle share one hand list, the library stores layer 1's range
 * columns and layer 4's rows permuted to that list's order (the network is the same
 * function; its kernels then read and write hand-ordered rows); the rows
 * cfr_read_leaf_rows returns are in slot order either way. */
int cfr_set_leaf_net(cfr_tree* tree, const uint16_t* const W[4], const float* const b[4]);

/* Evaluate the leaf network once on the current state (the reach the next player update
 * would see; average != 0: under the average strategy, as the exploitability pass does)
 * and store both players' leaf values (CFR_READ_CFV, or CFR_READ_BR_CFV with average), so
 * that one evaluation can be inspected with cfr_read_leaf_rows.  Synchronises. */
int cfr_eval_leaves(cfr_tree* tree, int average);

/* Depth-limit leaves of a handle: *n_leaves their count (any out pointer may be NULL); for
 * leaf 0 .. n_leaves-1 (leaf < 0: count only) its game, node and first network row.  A
 * leaf's 48 rows follow the river cards not on its board in ascending order. */
int cfr_leaf_info(const cfr_tree* tree, int leaf, int* n_leaves, int* game, int* node, int* row0);

/* Read network rows of the last leaf evaluation into a host buffer (synchronises):
 * what 0 = inputs (n_rows x 2752 BF16 as uint16), 1 = outputs (n_rows x 2688 FP32), in
 * the slot layout cfr_set_leaf_net describes. */
int cfr_read_leaf_rows(cfr_tree* tree, int what, int row0, int n_rows, void* out);

/* One dense layer of the depth-limit leaf network (Section 3, depth-limited solving; the
 * paper's Stage 5 evaluates the network on the GPU, Section 4.3), on the tensor cores:
 * C = act(A B^T + bias).  All pointers are device memory: A [M][K] and B [N][K] BF16
 * row-major (16-byte aligned), bias [N] FP32 or NULL, C [M][N] BF16 (out_f32 = 0) or FP32.
 * act = 1 applies GELU (0.5 x (1 + erf(x / sqrt 2))), 0 none.  N must be a multiple of 128
 * and K of 64 (CFR_EINVAL otherwise).  Asynchronous on `stream` (a cudaStream_t or NULL);
 * *err (a device int) is set to 1 if a bounded device-side wait gave up. */
int cfr_gemm_bf16(const void* A, const void* B, const float* bias, void* C, int M, int N, int K, int act,
                  int out_f32, int* err, void* stream);

/* Release the handle and its device memory (NULL is ignored). */
void cfr_tree_destroy(cfr_tree* tree);

/* Thread-local description of the last error ("" if none). */
const char* cfr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PCFR_H */
