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
#pragma once
#include <cstdint>

namespace pcfr {

enum NodeType : uint8_t { kDecision = 0, kFold = 1, kShowdown = 2, kChance = 3 };

constexpr int kMaxActions = 16;
constexpr int kPrecisionPairs = 0;   // values as double-float FP32 pairs
constexpr int kPrecisionSingle = 1;  // values as FP32
constexpr int kMaxDeck = 52;
constexpr uint8_t kNoCard = 255;

struct alignas(16) NodeDev {
  int32_t parent;     // -1 at the root
  int32_t first_kid;  // children are consecutive: [first_kid, first_kid + n_kids)
  int32_t row;        // decision: first row; showdown: board table; otherwise -1
  float value;        // terminal payoff (as in GameDev::payoff, rounded) or chance card probability;
                      // chance: probability of one card given both private hands
  uint8_t type;       // NodeType
  uint8_t player;     // decision: acting player; fold: folding player
  uint8_t n_kids;
  uint8_t deal;       // card dealt by the chance parent, else kNoCard
  uint8_t paction;    // index among the parent's children
  uint8_t level;
  uint8_t pad[2];
  uint64_t board;     // public cards at this node (bit c = card c)
};
static_assert(sizeof(NodeDev) == 32, "NodeDev is 32 bytes");

// Everything one subgame's kernels need: read-only tables and the solver state.
struct GameDev {
  int n_nodes, n_levels, n_hands, hstride, hand_size, n_rows, n_terminals, deck;
  int chunk, n_chunks;  // hands per block in the per-hand passes
  int smem;             // per-hand pass keeps its chunk's state in shared memory
  int row_begin[3];     // player p owns rows [row_begin[p], row_begin[p + 1])
  int n_boards, cl_len;
  double kappa64;       // 1 / Z, Z = sum of r0(h0) r1(h1) over hand pairs sharing no card
  const NodeDev* nodes;
  const double* payoff;        // [n_nodes] terminal payoff magnitude times the probability of
                               // the public cards dealt on the path (fold: folder's chips in,
                               // showdown: each player's chips in); 0 elsewhere
  const int32_t* level_start;  // [n_levels + 1]
  const uint64_t* hand_mask;   // [n_hands]
  const uint8_t* hand_cards;   // [n_hands][2] (second = kNoCard for one-card hands)
  const void* range_v;         // [2][hstride] normalised ranges, value type V
  const double* range64;       // [2][hstride]
  // showdown tables for board b (offsets b * n_hands, b * cl_len, b * (deck + 1)):
  const int32_t* sd_perm;      // hand at each rank-sorted position
  const int32_t* sd_gs;        // first sorted position of each hand's tie group
  const int32_t* sd_ge;        // one past the last sorted position of the tie group
  const int32_t* cl_hand;      // per-card hand lists in sorted order, concatenated
  const int32_t* cl_off;       // [deck + 1] start of each card's list
  const int32_t* cl_lo;        // [n_hands][2] list index of the first entry at or after gs
  const int32_t* cl_hi;        // [n_hands][2] list index of the first entry at or after ge
  // state
  double* R;
  double* S;
  void* sigma;
  void* sigbar;
  void* reach;
  void* reach_bar;
  void* cfv;
  void* cfv_br;
  double* br_partial;          // [2][n_chunks] per-block sums of r_i(h) v*_i(root, h)
  double* br_out;              // [2]
};

struct Work {
  int game;
  int unit;  // chunk index (per-hand passes) or node id (terminal pass)
};

// Kernel entry points (kernels.cu), all asynchronous on `stream`.
struct LaunchCtx {
  const GameDev* games;        // device array
  int n_games;
  const Work* chunk_work;      // device [n_chunk_work]: (game, chunk)
  int n_chunk_work;
  const Work* term_work;       // device [n_term_work]: (game, terminal node)
  int n_term_work;
  int* iter;                   // device: iterations completed
  unsigned* done;              // device: block arrival counter
  size_t smem_hand;            // dynamic shared memory of the per-hand kernel
  size_t smem_term;            // dynamic shared memory of the terminal kernel
  int variant;
  int precision;               // kPrecisionPairs or kPrecisionSingle
  double alpha, beta, gamma;
};

int launch_init(const LaunchCtx& c, void* stream);
int launch_terminal(const LaunchCtx& c, int player_mask, int use_bar, void* stream);
int launch_update(const LaunchCtx& c, int player_mask, int advance, void* stream);
int launch_avg_reach(const LaunchCtx& c, void* stream);
int launch_br(const LaunchCtx& c, void* stream);
int launch_br_reduce(const LaunchCtx& c, void* stream);
int launch_average_rows(const LaunchCtx& c, void* stream);
int hand_kernel_smem_limit();
int configure_kernels();  // once per process, before the first launch

}  // namespace pcfr
