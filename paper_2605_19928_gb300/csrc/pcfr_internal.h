// Internal layout shared by the host tree builder, the C ABI and the CUDA kernels.
//
// HBM layout (per subgame; every per-hand row is padded to `hstride` elements, a multiple
// of 32, so each row starts at least 128-byte aligned).  V is the value type: a pair of
// FP32 (hi, lo) in the default precision, or one FP32.
//   R, S         FP64 [n_rows][hstride]       cumulative regret / average-strategy sums
//   sigma        V    [n_rows][hstride]       current strategy (regret matching of R)
//   sigbar       V    [n_rows][hstride]       average strategy (exploitability pass)
//   reach        V    [2][n_nodes][hstride]   reach of each player under sigma
//   reach_bar    V    [2][n_nodes][hstride]   reach under the average strategy
//   cfv, cfv_br  V    [2][n_nodes][hstride]   counterfactual values (last traversal / BR)
// A decision node with A actions owns rows [row, row + A); player 0's rows come first.
//
// Terminal tables, one block of uint16 per showdown board (TermTab gives the offsets), all
// indices below 2^15 because a player has at most 1326 hands:
//   clh    [k * H]   per-card lists of hands, each list in rank-sorted order, concatenated
//   cards  [H]       card ids of each hand, c1 | c2 << 8 (c2 = 255 for one-card hands)
//   cloff  [deck+1]  start of each card's list in clh
//   perm   [H]       hand at each rank-sorted position
//   gs, ge [H]       first / one-past-last sorted position of each hand's tie group
//   lo, hi [2 * H]   per (hand, card) the clh index of the first entry at or after gs / ge
// Fold nodes need only the first three (board 0); the block is padded to 16 bytes so that
// the terminal kernel can stage it with one bulk (TMA) copy.
#pragma once
#include <cstddef>
#include <cstdint>

#ifndef __CUDACC__  // host-only translation units share the small helpers below
#define __host__
#define __device__
#endif

namespace pcfr {

enum NodeType : uint8_t { kDecision = 0, kFold = 1, kShowdown = 2, kChance = 3, kLeaf = 4 };
// Fold, showdown and depth-limit leaf nodes: their values come from outside the per-hand
// tree passes (terminal and leaf launches).
__host__ __device__ inline bool is_end(int type) { return type == kFold || type == kShowdown || type == kLeaf; }

constexpr int kMaxActions = 16;
constexpr int kMaxDeck = 52;
constexpr uint8_t kNoCard = 255;
constexpr int kPrecisionPairs = 0;   // values as double-float FP32 pairs
constexpr int kPrecisionSingle = 1;  // values as FP32
constexpr int kDiscountCapacity = 1 << 11;  // iterations a new handle's discount table covers
                                            // (doubled on demand)
// Passes of the per-hand kernel (and of the wide schedule).
enum HandMode { kModeInit = 0, kModeUpdate = 1, kModeAvg = 2, kModeBR = 3 };

constexpr int kScheduleLevel = 1;   // per-hand passes: one block per chunk of hands, level by level
constexpr int kScheduleStream = 2;  // update pass: one warp per 32 hands walks a depth-first program
constexpr int kScheduleWide = 3;    // one large tree: every pass is a launch per level over all of
                                    // that level's (node, hand) pairs
constexpr int kStreamMaxActions = 8;  // actions at a decision node the stream schedule holds in registers
constexpr int kStreamHalfMin = 12;   // 8-byte units per lane in each half of a warp's prefetch ring,
                                      // at least (or the most one node needs, 2 A + 1)
constexpr int kStreamWarps = 4;       // warps per block of the stream schedule (one game per block)

struct alignas(16) NodeDev {
  int32_t parent;     // -1 at the root
  int32_t first_kid;  // children are consecutive: [first_kid, first_kid + n_kids)
  int32_t row;        // decision: first row; showdown: board table; otherwise -1
  int32_t arow;       // row of the action that leads here (parent's row + paction), or -1
  uint8_t type;       // NodeType
  uint8_t player;     // decision: acting player; fold: folding player
  uint8_t n_kids;
  uint8_t deal;       // card dealt by the chance parent, else kNoCard
  uint8_t paction;    // index among the parent's children
  uint8_t level;
  uint8_t aplayer;    // player acting at the parent decision, else kNoCard
  uint8_t pad;
  uint64_t board;     // public cards at this node (bit c = card c)
};
static_assert(sizeof(NodeDev) == 32, "NodeDev is 32 bytes");

// One node of the stream schedule's program (pre-order), 16 bytes.  Offsets are in
// elements of a per-hand array (multiples of hstride).
struct alignas(16) ProgOp {
  int32_t node_off;   // node * hstride
  int32_t row_off;    // decision: first row * hstride; otherwise 0
  uint32_t code;      // type (2 bits) | player << 2 | n_kids << 3 (6 bits) | deal << 9 (8 bits) |
                      // terminal-children mask << 17 (bit a: child a is a fold or showdown;
                      // chance nodes: bit 0, all children are)
  int32_t first_kid;
};

// One load of the stream schedule's prefetch: array << kArrShift | element offset.
enum StreamArray : uint32_t { kArrR = 0, kArrS = 1, kArrReach = 2, kArrCfv = 3, kArrM = 4 };
constexpr uint32_t kArrShift = 29, kArrOffMask = (1u << 29) - 1u;
static_assert(sizeof(ProgOp) == 16, "ProgOp is 16 bytes");

// Offsets (in uint16) of the terminal-table sections for H hands of k cards from a deck.
struct TermTab {
  int clh, cards, cloff, fold_len, perm, gs, ge, lo, hi, len;
  __host__ __device__ static int round8(int x) { return (x + 7) / 8 * 8; }
  __host__ __device__ TermTab(int H, int k, int deck) {
    clh = 0;
    cards = k * H;
    cloff = cards + H;
    fold_len = round8(cloff + deck + 1);
    perm = fold_len;
    gs = perm + H;
    ge = gs + H;
    lo = ge + H;
    hi = lo + 2 * H;
    len = round8(hi + 2 * H);
  }
};

// Everything one subgame's kernels need: read-only tables and the solver state.
struct GameDev {
  int n_nodes, n_levels, n_hands, hstride, hand_size, n_rows, n_terminals, deck;
  int chunk, n_chunks;  // hands per block in the per-hand passes
  int smem;             // per-hand pass keeps its chunk's state in shared memory (the same
                        // for every game of a handle)
  int row_begin[3];     // player p owns rows [row_begin[p], row_begin[p + 1])
  int n_boards;
  double kappa64;              // 1 / Z, Z = sum of r0(h0) r1(h1) over hand pairs sharing no card
  const NodeDev* nodes;
  const double* payoff;        // [n_nodes] terminal payoff magnitude times the probability of
                               // the public cards dealt on the path (fold: folder's chips in,
                               // showdown: each player's chips in); 0 elsewhere
  const float* payoff_ff;      // [n_nodes][2] payoff * kappa64 as an FP32 pair (hi, lo), rounded
                               // once on the host: the terminal scale (FP32 values use hi)
  const int32_t* level_start;  // [n_levels + 1]
  const int32_t* row_node;     // [n_rows] decision node owning each row
  const int32_t* dec_nodes;    // decision nodes of player 0, then of player 1
  int dec_begin[3];            // player p's are dec_nodes[dec_begin[p] .. dec_begin[p + 1])
  const uint64_t* hand_mask;   // [n_hands]
  const void* range_v;         // [2][hstride] normalised ranges, value type V
  const double* range64;       // [2][hstride]
  const uint16_t* term_tab;    // [n_boards][TermTab.len]
  const ProgOp* prog;          // [prog_len] inner nodes in depth-first pre-order (stream schedule)
  int prog_len;
  const int32_t* chunks;       // load chunks of the stream schedule (see stream_tables)
  int chunk_off[4], chunk_count[4];
  const uint32_t* units;       // loads of the stream schedule, in the order the passes use them
  int unit_off[4], unit_count[4];
  // state
  double* R;
  double* S;
  double* M;                   // Predictive CFR+ prediction [n_rows][hstride] (else null)
  void* sigma;
  void* sigbar;
  void* reach;
  void* reach_bar;
  void* cfv;
  void* cfv_br;
  double* br_partial;          // [2][n_chunks] per-block sums of r_i(h) v*_i(root, h)
  double* br_out;              // [2]
  unsigned* br_done;           // blocks of the best-response pass that have finished
};

struct Work {
  int game;
  int unit;  // chunk index (per-hand passes) or node id (terminal pass)
};

// Per-iteration update weights for iteration t (entry t - 1): DCFR's positive / negative
// regret discounts and average discount, and the weight of the new average contribution.
struct Discount {
  double dpos, dneg, dS, wS;
};

// Kernel entry points (kernels.cu), all asynchronous on `stream`.
struct LaunchCtx {
  const GameDev* games;        // device array
  int n_games;
  const Work* chunk_work;      // device [n_chunk_work]: (game, chunk)
  int n_chunk_work;
  const Work* term_work;       // device [n_term_work]: (game, terminal node), grouped by game and
                               // board table
  int n_term_work;
  const Work* term_runs;       // device [n_term_runs]: (first entry of term_work, count), the
                               // terminal nodes one block evaluates
  int n_term_runs;
  const int32_t* term_src;     // device [n_term_work]: node whose reach rows stand for each
                               // terminal's (HostGame::reach_src)
  int* iter;                   // device: iterations completed
  unsigned* done;              // device: block arrival counter
  int* err;                    // device: nonzero after a bounded wait gave up
  const Discount* disc;        // device [iterations covered], one entry per iteration
  size_t smem_hand;            // dynamic shared memory of the per-hand kernel; 0 = every game
                               // works on the global arrays (some tree is too large to stage)
  size_t smem_term;            // dynamic shared memory of the terminal kernel
  int variant;
  int precision;               // kPrecisionPairs or kPrecisionSingle
  int pdl;                     // chain launches with programmatic dependent launch
  int schedule;                // kScheduleLevel, kScheduleStream (update launches) or kScheduleWide
  const Work* warp_work;       // device [n_warp_work]: (game, first group of 32 hands) of each
                               // block of the stream schedule, largest trees first
  int n_warp_work;
  int stream_depth;            // stack slots per lane of the stream schedule
  int stream_prog;             // nodes of the largest tree, if its program is staged in shared
                               // memory; 0 = read from global memory
  int stream_half;             // units per lane in each half of the stream prefetch ring
  int stream_units;            // load descriptors staged per block (0 when the program is not)
  int stream_hp;               // hands per lane of the stream schedule (1 or 2): a warp owns 32 * stream_hp
  // wide schedule (one game): level l's inner nodes are wide_inner[wide_inner_off[l] ..
  // wide_inner_off[l + 1]), the nodes whose reach is stored wide_fwd[wide_fwd_off[l] ..
  // wide_fwd_off[l + 1]) (all but the run-out nodes that read their source's reach)
  int wide_levels;             // number of levels
  const int* wide_inner_off;   // host [wide_levels + 1]
  const int32_t* wide_inner;   // device: inner node ids, level by level
  const int* wide_fwd_off;     // host [wide_levels + 1]
  const int32_t* wide_fwd;     // device: node ids, level by level
  int wide_stride;             // hstride of the game
  int wide_max_dec;            // decision nodes of the player who has more
  // resident schedule (cfr_iterate only; the other passes use the level schedule's kernels)
  int resident;                // cfr_iterate runs k_resident
  int resident_grid;           // blocks of the cooperative launch (>= n_chunk_work)
  size_t smem_resident;        // its dynamic shared memory: terminal region, then hand region
  unsigned resident_term;      // bytes of the terminal region
  unsigned* resident_sync;     // device [2]: barrier arrivals, blocks finished (zero between launches)
  int alternating;
};

int launch_init(const LaunchCtx& c, void* stream);
int launch_terminal(const LaunchCtx& c, int player_mask, int use_bar, void* stream);
int launch_update(const LaunchCtx& c, int player_mask, int advance, void* stream);  // either schedule
int launch_current_rows(const LaunchCtx& c, void* stream);  // sigma = RM(R), every game (read-back)
int launch_avg_reach(const LaunchCtx& c, void* stream);
int launch_br(const LaunchCtx& c, void* stream);
int launch_average_rows(const LaunchCtx& c, void* stream);
// Kernels one pass of the wide schedule launches (which: kModeInit, kModeUpdate, kModeAvg or
// kModeBR, as the per-hand kernel's modes).
int wide_launch_count(const LaunchCtx& c, int which, int player_mask, int advance);
int hand_kernel_smem_limit();
// Shared memory the per-hand kernel needs to stage one game (es = bytes per value).
size_t hand_smem_size(int n_nodes, int n_levels, int rows_max, int W, size_t es);
int configure_kernels();  // once per process, before the first launch
// Polls of the terminal kernel's first bulk-copy wait on the current device (< 0: the
// default limit); for tests of the timeout path.  Returns 0 or -1.
int set_first_wait_polls(long polls);
// Resident schedule: shared memory of its two regions for one game, the blocks of k_resident
// one SM holds with `smem` bytes (0 if none), and the cooperative launch of n_iters iterations.
size_t resident_term_size(int n_hands, int hand_size, int deck, int hstride, size_t es);
size_t resident_hand_size(int n_nodes, int n_levels, int rows_max, int W, size_t es);
int resident_blocks_per_sm(int precision, size_t smem);
int launch_resident(const LaunchCtx& c, int n_iters, void* stream);
// Dense layer of the leaf network (leafnet.cu): C[M][N] = act(A[M][K] B[N][K]^T + bias), BF16
// A and B, FP32 accumulation, C in BF16 (out_f32 = 0) or FP32; N a multiple of 128, K of 64.
// Returns 0, -1 (launch failed), -2 (bad shape or alignment), -3 (no tensor-map encoder).
int launch_gemm_bf16(const void* A, const void* B, const float* bias, void* C, int M, int N, int K, int act,
                     int out_f32, int* err, void* stream);
int configure_gemm();

// ---- depth-limit leaf network (leafnet.cu)
// Network input per (leaf, river card): both players' reach at the leaf over the 1326
// two-card slots (each normalised to sum 1 over the hands not holding the river card), a
// one-hot of the 5 board cards, then 2 pot / stack features; zero padding to kLeafIn.
// Output: each player's value per unit pot over the 1326 slots; padding to kLeafOut.
constexpr int kLeafSlots = 1326;
constexpr int kLeafFeatures = 2 * kLeafSlots + 52 + 2;  // 2706
constexpr int kLeafIn = 2752;                           // padded to a multiple of 64
constexpr int kLeafHidden = 512;
constexpr int kLeafOut = 2688;                          // 2 x 1326 padded to a multiple of 128
constexpr int kLeafCards = 48;                          // river cards after 4 board cards

struct LeafDev {      // one depth-limit leaf
  int game, node;
  int row0;           // first of its kLeafCards network rows (river cards ascending)
  float feat[2];      // pot / (pot + 2 stack), stack / (pot + 2 stack) at the leaf
};

struct LeafCtx {
  const LeafDev* leaves;   // device [n_leaves]
  int n_leaves;
  const int16_t* slot;     // per game [hstride]: slot of each hand (device, game-major)
  const int16_t* hand_at;  // per game [kLeafSlots]: hand in each slot or -1
  int hstride_max;
  void* X;                 // [rows][kLeafIn] BF16
  void* H1;                // [rows][kLeafHidden] BF16
  void* H2;
  void* H3;
  float* Y;                // [rows][kLeafOut]
  const void* W[4];        // BF16 [out][in]
  const float* b[4];
  int hand_order;          // 1: every game has the same hand list, and the network's range
                           // inputs and value outputs are laid out in that list's order
                           // (hand h at column h of each player's 1326) -- the first and last
                           // layers' weights are permuted to match -- so the leaf kernels
                           // read and write them coalesced; 0: slot order
};

// Leaf values of player i (use_bar: against the average strategy, into cfv_br) or, with
// player -1, only the network (both players' inputs and the four layers).
int launch_leaf_inputs(const LaunchCtx& c, const LeafCtx& L, int use_bar, void* stream);
int launch_leaf_net(const LaunchCtx& c, const LeafCtx& L, void* stream);
int launch_leaf_values(const LaunchCtx& c, const LeafCtx& L, int player, int use_bar, void* stream);
// Dynamic shared memory of one stream-schedule block: the staged program (prog_nodes nodes)
// and one player's load descriptors (prog_units), and per lane a prefetch ring of 2 x half
// units of hp 8-byte entries and a stack of `depth` slots of hp values (es bytes each).
inline size_t stream_smem_size(int prog_nodes, int prog_units, int half, int depth, size_t es, int hp) {
  return (size_t)prog_nodes * sizeof(ProgOp) + (size_t)prog_units * 4 +
         (size_t)kStreamWarps * 32 * hp * (2 * (size_t)half * 8 + (size_t)depth * es);
}

}  // namespace pcfr
