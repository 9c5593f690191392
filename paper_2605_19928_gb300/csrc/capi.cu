// C ABI of libpcfr.so (declared in include/pcfr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "pcfr.h"
#include "pcfr_internal.h"
#include "runout.h"
#include "tree.h"

using namespace pcfr;

namespace {

thread_local std::string g_last_error;
cfr_alloc_fn g_alloc = nullptr;
cfr_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(CFR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

}  // namespace

struct cfr_tree {
  std::vector<HostGame> host;
  std::vector<GameDev> dev;     // host copies of the device structs
  GameDev* d_games = nullptr;
  Work* d_chunk_work = nullptr;
  Work* d_term_work = nullptr;
  Work* d_term_runs = nullptr;
  Work* d_warp_work = nullptr;
  int32_t* d_wide_inner = nullptr;  // wide schedule: inner node ids, level by level
  int32_t* d_wide_fwd = nullptr;    // wide schedule: nodes whose reach is stored, level by level
  int32_t* d_term_src = nullptr;    // reach source of each terminal work entry
  // all-in run-outs evaluated by win-minus-loss tables (runout_tables; none: all zero)
  RunoutItem* d_ro_items = nullptr;   // top nodes, sorted by table
  RunoutGroup* d_ro_groups8 = nullptr;
  RunoutGroup* d_ro_groups16 = nullptr;
  int ro_n8 = 0, ro_n16 = 0;          // groups of tops on uint8 / uint16 tables
  RunoutTable* d_ro_tables = nullptr;
  unsigned char* d_ro_pool = nullptr;
  std::vector<int> wide_inner_off, wide_fwd_off;
  int* d_iter = nullptr;
  unsigned* d_done = nullptr;
  unsigned* d_res_sync = nullptr;   // resident schedule: barrier and exit counters
  int* d_err = nullptr;
  Discount* d_disc = nullptr;
  int disc_capacity = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t iter_graph = nullptr;
  cudaGraphExec_t expl_graph = nullptr;
  bool expl_once = false;       // one exploitability pass has run without a graph
  double* d_br_all = nullptr;   // [n_games][2] best-response values, contiguous (one read-back)
  cfr_solver_opts opts{};
  LaunchCtx ctx{};
  int iters_done = 0;
  int64_t state_gen = 0;        // bumped whenever R or S may change
  int64_t avg_gen = -1;         // state_gen for which sigbar holds k_average_rows' output
  int64_t cur_gen = -1;         // state_gen for which sigma holds RM(R) (stream schedule)
  LeafCtx leaf{};               // depth-limit leaves and their network (none: n_leaves = 0)
  std::vector<LeafDev> leaf_host;
  std::vector<int> leaf_col;    // network column of each card-pair slot (hand order, or the slot)
  bool leaf_net_set = false;
  int64_t launches = 0;         // kernels launched (graph replays included)
  int64_t device_bytes = 0;
  int64_t h2d_bytes = 0;
  int launches_per_iteration = 0;
  int device = -1;              // the device current when the handle was created
  std::vector<std::pair<void*, bool>> blocks;  // (pointer, from hook)
  void* stream_arg = nullptr;

  void* alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    void* p = nullptr;
    bool hook = g_alloc != nullptr;
    if (hook) {
      p = g_alloc(bytes, stream_arg, g_alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) {
      blocks.push_back({p, hook});
      device_bytes += (int64_t)bytes;
    }
    return p;
  }
  ~cfr_tree() {
    if (iter_graph) cudaGraphExecDestroy(iter_graph);
    if (expl_graph) cudaGraphExecDestroy(expl_graph);
    cudaStreamSynchronize(stream);
    for (auto& b : blocks) {
      if (b.second) {
        if (g_free) g_free(b.first, g_alloc_ctx);
      } else {
        cudaFree(b.first);
      }
    }
    if (capture) cudaStreamDestroy(capture);
  }
};

namespace {

template <typename T>
int upload(cfr_tree* t, const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return CFR_OK;
  void* p = t->alloc(v.size() * sizeof(T));
  if (!p) return fail(CFR_ENOMEM, "device allocation failed");
  CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, t->stream));
  t->h2d_bytes += (int64_t)(v.size() * sizeof(T));
  *out = (T*)p;
  return CFR_OK;
}

// Terminal values of the players in player_mask (Stages 2-4): the fold and showdown launch,
// then the all-in run-outs evaluated by their tables (runout_tables).
int launch_terminals(const cfr_tree* t, int player_mask, int use_bar, cudaStream_t s) {
  if (launch_terminal(t->ctx, player_mask, use_bar, s)) return -1;
  if (t->ro_n8 + t->ro_n16 == 0) return 0;
  const HostGame& h = t->host[0];
  return launch_runout_values(t->ctx.games, t->d_ro_items, t->d_ro_groups8, t->ro_n8, t->d_ro_groups16, t->ro_n16,
                              t->d_ro_tables, t->d_ro_pool, h.n_hands, player_mask, use_bar, s);
}

// Kernels one terminal stage launches.
int terminal_launches(const cfr_tree* t) {
  return (t->ctx.n_term_work > 0 ? 1 : 0) + (t->ro_n8 > 0 ? 1 : 0) + (t->ro_n16 > 0 ? 1 : 0);
}

// One device block for every subgame's tables and state: the tables are staged on the host
// and sent with one copy, the state after them zeroed with one memset, and each buffer's
// pointer field is set once the block exists (a handle of many subgames makes a handful of
// allocations instead of a couple of dozen per subgame).  Buffers start 256-byte aligned.
struct Packer {
  using Setter = std::function<void(unsigned char*)>;  // sets one typed pointer field
  std::vector<unsigned char> stage;                    // host bytes of the tables
  size_t zero_bytes = 0;                               // bytes of zeroed state after the tables
  std::vector<std::pair<size_t, Setter>> tabs;         // (offset in the tables, field to set)
  std::vector<std::pair<size_t, Setter>> state;        // (offset in the state, field to set)
  static size_t round(size_t b) { return (b + 255) / 256 * 256; }
  template <typename F>
  static Setter setter(F** where) {
    return [where](unsigned char* p) { *where = reinterpret_cast<F*>(p); };
  }
  template <typename T, typename F>
  void table(const std::vector<T>& v, F** where) {
    *where = nullptr;
    if (v.empty()) return;
    const size_t off = stage.size(), bytes = v.size() * sizeof(T);
    stage.resize(off + round(bytes), 0);
    memcpy(stage.data() + off, v.data(), bytes);
    tabs.push_back({off, setter(where)});
  }
  template <typename F>
  void zeroed(size_t bytes, F** where) {
    state.push_back({zero_bytes, setter(where)});
    zero_bytes += round(std::max<size_t>(bytes, 1));
  }
  // allocate, copy, zero and set the fields
  int commit(cfr_tree* t) {
    const size_t total = stage.size() + zero_bytes;
    if (total == 0) return CFR_OK;
    unsigned char* block = static_cast<unsigned char*>(t->alloc(total));
    if (!block) return fail(CFR_ENOMEM, "device allocation failed");
    if (!stage.empty()) {
      CK(cudaMemcpyAsync(block, stage.data(), stage.size(), cudaMemcpyHostToDevice, t->stream));
      t->h2d_bytes += (int64_t)stage.size();
    }
    if (zero_bytes) CK(cudaMemsetAsync(block + stage.size(), 0, zero_bytes, t->stream));
    for (auto& f : tabs) f.second(block + f.first);
    for (auto& f : state) f.second(block + stage.size() + f.first);
    return CFR_OK;
  }
};

// Runs f(g) for every game g of a handle on up to one thread per host core: the host-side
// construction of one subgame (tree, tables, programs) reads only its own spec and writes
// only its own slot, so the result does not depend on the thread count.  Handles of a few
// games run on the calling thread.
template <typename F>
void parallel_games(int n_games, F f) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = n_games < 8 ? 1 : std::min(std::min(n_games, hw), 64);
  if (nt <= 1) {
    for (int g = 0; g < n_games; ++g) f(g);
    return;
  }
  std::atomic<int> next{0};
  auto work = [&] {
    for (int g = next.fetch_add(1); g < n_games; g = next.fetch_add(1)) f(g);
  };
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  for (int k = 1; k < nt; ++k) pool.emplace_back(work);
  work();
  for (std::thread& th : pool) th.join();
}

template <typename T>
int zeros(cfr_tree* t, size_t n, T** out) {
  void* p = t->alloc(std::max<size_t>(n, 1) * sizeof(T));
  if (!p) return fail(CFR_ENOMEM, "device allocation failed");
  CK(cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), t->stream));
  *out = (T*)p;
  return CFR_OK;
}

// Shared memory the per-hand kernel needs to stage one game with W hands per block.
size_t hand_smem(const HostGame& g, int W, size_t es) {
  const int rows_max = std::max(g.row_begin[1] - g.row_begin[0], g.row_begin[2] - g.row_begin[1]);
  return hand_smem_size((int)g.nodes.size(), (int)g.level_start.size() - 1, rows_max, W, es);
}

// Update weights of iterations 1 .. capacity (Stage 7; CFR+ and DCFR from Section 2):
// DCFR multiplies positive regrets by t^a / (t^a + 1), the others by t^b / (t^b + 1) and
// the average by (t / (t + 1))^g; CFR+ weighs the new average contribution by t.
// The first `capacity` entries of a variant's discount table.  Entry k depends only on the
// options and k, so the entries are computed once per process for each set of options (three
// pow calls per DCFR entry) and cut to the length asked for.
std::vector<Discount> discount_table(const cfr_solver_opts& o, int capacity) {
  static std::mutex mu;
  static std::vector<std::pair<std::array<double, 4>, std::vector<Discount>>> cache;
  const std::array<double, 4> key{(double)o.variant, o.alpha, o.beta, o.gamma};
  std::lock_guard<std::mutex> lock(mu);
  std::vector<Discount>* d = nullptr;
  for (auto& e : cache)
    if (e.first == key) d = &e.second;
  if (!d) {
    cache.push_back({key, {}});
    d = &cache.back().second;
  }
  for (int k = (int)d->size(); k < capacity; ++k) {
    const double t = (double)(k + 1);
    Discount x{1.0, 1.0, 1.0, 1.0};
    if (o.variant == CFR_VARIANT_DCFR) {
      const double ta = std::pow(t, o.alpha), tb = std::pow(t, o.beta);
      x.dpos = ta / (ta + 1.0);
      x.dneg = tb / (tb + 1.0);
      x.dS = std::pow(t / (t + 1.0), o.gamma);
    } else if (o.variant == CFR_VARIANT_CFRPLUS) {
      x.wS = t;
    } else if (o.variant == CFR_VARIANT_PCFRPLUS) {
      x.wS = t * t;  // quadratic averaging
    }
    d->push_back(x);
  }
  return std::vector<Discount>(d->begin(), d->begin() + capacity);
}

// Host copy of a per-hand vector in the value type: one float, or a (hi, lo) float pair.
std::vector<float> to_value_type(const std::vector<double>& x, int precision) {
  std::vector<float> out;
  if (precision == kPrecisionSingle) {
    for (double v : x) out.push_back((float)v);
  } else {
    for (double v : x) {
      const float hi = (float)v;
      out.push_back(hi);
      out.push_back((float)(v - (double)hi));
    }
  }
  return out;
}

int check_device() {  // two attribute queries: cudaGetDeviceProperties takes milliseconds
  int dev = 0, major = 0, minor = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
  e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (major != 10 || minor != 3)
    return fail(CFR_ECUDA, "libpcfr needs a compute capability 10.3 (GB300) device, found " +
                               std::to_string(major) + "." + std::to_string(minor));
  return CFR_OK;
}

int leaf_launches(const cfr_tree* t, int player_mask);
int pass_launches(const cfr_tree* t, int which, int player_mask, int advance);

// Depth-limit leaves of every game: their network rows, features and slot maps, and the
// network's activation and weight buffers (the weights arrive with cfr_set_leaf_net).
int setup_leaves(cfr_tree* t, const cfr_game_spec* specs, int n_games) {
  LeafCtx& L = t->leaf;
  L = LeafCtx{};
  int hmax = 0;
  for (int g = 0; g < n_games; ++g) {
    hmax = std::max(hmax, t->host[g].hstride);
    const HostGame& h = t->host[g];
    const double cap = specs[g].pot / 2.0 + specs[g].stack;
    for (int n : h.leaves) {
      LeafDev lf{};
      lf.game = g;
      lf.node = n;
      lf.row0 = (int)t->leaf_host.size() * kLeafCards;
      const double pot = h.contrib[2 * (size_t)n] + h.contrib[2 * (size_t)n + 1];
      const double behind = cap - h.contrib[2 * (size_t)n];
      lf.feat[0] = (float)(pot / (pot + 2.0 * behind));
      lf.feat[1] = (float)(behind / (pot + 2.0 * behind));
      t->leaf_host.push_back(lf);
    }
  }
  if (t->leaf_host.empty()) return CFR_OK;
  L.n_leaves = (int)t->leaf_host.size();
  L.hstride_max = hmax;
  // one hand list for all games: inputs and outputs in hand order (column of slot s)
  bool same = t->host[0].hand_size == 2;
  for (int g = 1; g < n_games && same; ++g) same = t->host[g].hand_cards == t->host[0].hand_cards;
  L.hand_order = same ? 1 : 0;
  t->leaf_col.assign(kLeafSlots, -1);
  if (same) {
    const HostGame& h0 = t->host[0];
    std::vector<char> used(kLeafSlots, 0);
    for (int k = 0; k < h0.n_hands; ++k) {
      int a = h0.hand_cards[2 * (size_t)k], b = h0.hand_cards[2 * (size_t)k + 1];
      if (a > b) std::swap(a, b);
      const int sl = b * (b - 1) / 2 + a;
      t->leaf_col[sl] = k;
      used[sl] = 1;
    }
    int next = h0.n_hands;
    for (int sl = 0; sl < kLeafSlots; ++sl)
      if (!used[sl]) t->leaf_col[sl] = next++;
  } else {
    for (int sl = 0; sl < kLeafSlots; ++sl) t->leaf_col[sl] = sl;
  }
  std::vector<int16_t> slot((size_t)n_games * hmax, 0), hand_at((size_t)n_games * kLeafSlots, -1);
  for (int g = 0; g < n_games; ++g) {
    const HostGame& h = t->host[g];
    if (h.hand_size != 2) continue;
    for (int k = 0; k < h.n_hands; ++k) {
      int a = h.hand_cards[2 * (size_t)k], b = h.hand_cards[2 * (size_t)k + 1];
      if (a > b) std::swap(a, b);
      const int sl = b * (b - 1) / 2 + a;
      slot[(size_t)g * hmax + k] = (int16_t)sl;
      hand_at[(size_t)g * kLeafSlots + sl] = (int16_t)k;
    }
  }
  const size_t rows = (size_t)L.n_leaves * kLeafCards;
  LeafDev* ld;
  int16_t *sd, *hd;
  int rc;
  if ((rc = upload(t, t->leaf_host, &ld)) || (rc = upload(t, slot, &sd)) || (rc = upload(t, hand_at, &hd))) return rc;
  L.leaves = ld;
  L.slot = sd;
  L.hand_at = hd;
  uint16_t *x, *h1, *h2, *h3;
  float* y;
  if ((rc = zeros(t, rows * kLeafIn, &x)) || (rc = zeros(t, rows * kLeafHidden, &h1)) ||
      (rc = zeros(t, rows * kLeafHidden, &h2)) || (rc = zeros(t, rows * kLeafHidden, &h3)) ||
      (rc = zeros(t, rows * kLeafOut, &y)))
    return rc;
  L.X = x; L.H1 = h1; L.H2 = h2; L.H3 = h3; L.Y = y;
  const size_t wn[4] = {(size_t)kLeafHidden * kLeafIn, (size_t)kLeafHidden * kLeafHidden,
                        (size_t)kLeafHidden * kLeafHidden, (size_t)kLeafOut * kLeafHidden};
  const size_t bn[4] = {(size_t)kLeafHidden, (size_t)kLeafHidden, (size_t)kLeafHidden, (size_t)kLeafOut};
  for (int k = 0; k < 4; ++k) {
    uint16_t* w;
    float* b;
    if ((rc = zeros(t, wn[k], &w)) || (rc = zeros(t, bn[k], &b))) return rc;
    L.W[k] = w;
    L.b[k] = b;
  }
  static const int gemm_ok = configure_gemm();
  if (gemm_ok != 0) return fail(CFR_ECUDA, "GEMM kernel attribute setup failed");
  return CFR_OK;
}

int create_impl(const cfr_game_spec* specs, int n_games, const cfr_solver_opts* opts, void* stream,
                cfr_tree** out) {
  if (!out) return fail(CFR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!specs || n_games <= 0) return fail(CFR_EINVAL, "no game given");
  cfr_solver_opts o{CFR_VARIANT_DCFR, 1.5, 0.0, 2.0, 1, 0, CFR_PRECISION_PAIRS, CFR_SCHEDULE_AUTO};
  if (opts) o = *opts;
  if (o.variant < 0 || o.variant > 3) return fail(CFR_EINVAL, "unknown CFR variant");
  if (o.precision != CFR_PRECISION_PAIRS && o.precision != CFR_PRECISION_SINGLE)
    return fail(CFR_EINVAL, "unknown precision");
  const size_t es = o.precision == CFR_PRECISION_SINGLE ? 4 : 8;
  if (o.chunk_hands < 0 || o.chunk_hands > 32 || (o.chunk_hands & (o.chunk_hands - 1)))
    return fail(CFR_EINVAL, "chunk_hands must be 0 or a power of two up to 32");
  if (o.term_nodes < 0 || o.term_nodes > 8) return fail(CFR_EINVAL, "term_nodes must be 0 to 8");
  if (o.warp_hands != 0 && o.warp_hands != 32 && o.warp_hands != 64)
    return fail(CFR_EINVAL, "warp_hands must be 0, 32 or 64");
  if (o.schedule < CFR_SCHEDULE_AUTO || o.schedule > CFR_SCHEDULE_RESIDENT) return fail(CFR_EINVAL, "unknown schedule");
  if (o.runout_tables != 0 && o.runout_tables != 1) return fail(CFR_EINVAL, "runout_tables must be 0 or 1");
  if (o.runout_tables && (o.precision != CFR_PRECISION_SINGLE || n_games != 1))
    return fail(CFR_EINVAL, "runout_tables needs one subgame with FP32 values (precision = single)");
  int rc = check_device();
  if (rc != CFR_OK) return rc;
  static int configured = configure_kernels();
  if (configured != 0) return fail(CFR_ECUDA, "kernel attribute setup failed");

  cfr_tree* t = new cfr_tree();
  t->opts = o;
  if (cudaGetDevice(&t->device) != cudaSuccess) {
    delete t;
    return fail(CFR_ECUDA, "cudaGetDevice failed");
  }
  t->stream = (cudaStream_t)stream;
  t->stream_arg = stream;
  t->host.resize(n_games);
  {
    std::vector<int> rcs(n_games, CFR_OK);
    std::vector<std::string> errs(n_games);
    parallel_games(n_games, [&](int g) { rcs[g] = build_game(specs[g], t->host[g], errs[g]); });
    for (int g = 0; g < n_games; ++g)  // the first rejected game, as a serial build reports it
      if (rcs[g] != CFR_OK) {
        delete t;
        return fail(rcs[g], "game " + std::to_string(g) + ": " + errs[g]);
      }
  }
  // Block shape: W hands per block (8 by default).  The per-hand pass stages each chunk's
  // tree and state in shared memory when every game of the handle fits in 96 KB (two blocks
  // per SM); otherwise all games work on the global arrays, which stay in L2 for trees of
  // this size.
  // The resident schedule gives every chunk a block of its own, one block per SM: its default
  // chunk is the smallest of 8, 16 and 32 hands with which the handle's chunks fit the SMs.
  const bool resident = o.schedule == CFR_SCHEDULE_RESIDENT;
  int n_sms = 0;
  if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess || n_sms < 1) {
    delete t;
    return fail(CFR_ECUDA, "cudaDeviceGetAttribute failed");
  }
  auto chunks_of = [&](int W) {
    long n = 0;
    for (int g = 0; g < n_games; ++g) n += (t->host[g].n_hands + W - 1) / W;
    return n;
  };
  int res_W = 8;
  while (resident && !o.chunk_hands && res_W < 32 && chunks_of(res_W) > n_sms) res_W *= 2;
  size_t smem_hand = 0, smem_term = 0;
  std::vector<int> chunk(n_games);
  std::vector<int> use_smem(n_games);
  bool all_fit = true;
  for (int g = 0; g < n_games; ++g) {
    const int W = o.chunk_hands ? o.chunk_hands : res_W;
    chunk[g] = W;
    all_fit = all_fit && hand_smem(t->host[g], W, es) <= 96 * 1024;
  }
  for (int g = 0; g < n_games; ++g) {
    const HostGame& h = t->host[g];
    use_smem[g] = all_fit;
    if (all_fit) smem_hand = std::max(smem_hand, hand_smem(h, chunk[g], es));
    const TermTab tt(h.n_hands, h.hand_size, h.deck);
    smem_term = std::max(smem_term, (size_t)tt.len * 2 + 2 * (size_t)h.hstride * es +
                                        (size_t)(h.hand_size * h.n_hands + 1 + h.n_hands + 1) * 8);
  }

  // Update schedule: one warp per 32 hands when the handle has enough of them to fill the
  // GPU (8 warps per SM) and every tree fits the warp's registers and stack.
  std::vector<std::vector<int32_t>> programs(n_games);
  std::vector<std::array<int, 4>> prog_meta(n_games);  // depth, max actions, fits, max loads of a node
  parallel_games(n_games, [&](int g) {
    int depth = 0, amax = 0, loads = 0;
    bool fits = false;
    programs[g] = dfs_program(t->host[g], &depth, &amax, &fits);
    for (int n : programs[g])
      for (int p = 0; p < 2; ++p)
        loads = std::max(loads, (int)node_loads(t->host[g], n, p, true, (uint32_t)t->host[g].hstride,
                                                o.variant == CFR_VARIANT_PCFRPLUS).size());
    prog_meta[g] = {depth, amax, fits ? 1 : 0, loads};
  });
  int stream_depth = 1, stream_warps = 0, actions_max = 0;
  bool stream_ok = true;
  for (int g = 0; g < n_games; ++g) {
    stream_ok = stream_ok && prog_meta[g][2];
    stream_depth = std::max(stream_depth, prog_meta[g][0]);
    actions_max = std::max(actions_max, prog_meta[g][1]);
    stream_ok = stream_ok && prog_meta[g][1] <= kStreamMaxActions;
    stream_warps += (t->host[g].n_hands + 31) / 32;
  }
  // the program of the largest tree is staged in shared memory when it takes at most 64 KB
  int max_prog = 0, max_loads = 0;
  for (int g = 0; g < n_games; ++g) {
    max_prog = std::max(max_prog, (int)programs[g].size());
    max_loads = std::max(max_loads, prog_meta[g][3]);
  }
  const int stream_prog = max_prog * (int)sizeof(ProgOp) <= 64 * 1024 ? max_prog : 0;
  const int stream_half = std::max(kStreamHalfMin, max_loads);
  // load tables of every game (units per player: both passes), and their largest size
  std::vector<std::vector<uint32_t>> unit_lists(n_games);
  std::vector<std::vector<int32_t>> chunk_lists(n_games);
  std::vector<std::array<int, 16>> table_meta(n_games);
  int stream_units_max = 0;
  parallel_games(n_games, [&](int g) {
    std::array<int, 16>& m = table_meta[g];
    chunk_lists[g] = stream_tables(t->host[g], programs[g], stream_half, o.variant == CFR_VARIANT_PCFRPLUS,
                                   unit_lists[g], &m[0], &m[4], &m[8], &m[12]);
  });
  for (int g = 0; g < n_games; ++g) {
    const std::array<int, 16>& m = table_meta[g];
    for (int p = 0; p < 2; ++p) stream_units_max = std::max(stream_units_max, m[4 + p] + m[4 + 2 + p]);
    const size_t span = std::max(t->host[g].nodes.size(), (size_t)t->host[g].n_rows) * (size_t)t->host[g].hstride;
    stream_ok = stream_ok && span < (1u << kArrShift);
  }
  stream_units_max = (stream_units_max + 3) / 4 * 4;  // keeps the ring 16-byte aligned
  const int stream_units = stream_prog ? stream_units_max : 0;
  // hands per lane: one (32 per warp) unless the options ask for 64 per warp.  Two per lane
  // share the walk's control work but double the ring and stack, which halves the warps an
  // SM holds; on the 256-subgame batch that made the update slower (0.41 vs 0.27 ms), so
  // only the autotuner tries it.
  bool rows64 = true;
  for (int g = 0; g < n_games; ++g) rows64 = rows64 && t->host[g].hstride % 64 == 0;
  auto smem_fits = [&](int hp) {
    return stream_smem_size(stream_prog, stream_units, stream_half, stream_depth, es, hp) <= 200 * 1024;
  };
  const int stream_hp = o.warp_hands == 64 ? 2 : 1;
  if (stream_hp == 2 && !rows64) {
    delete t;
    return fail(CFR_EINVAL, "warp_hands = 64 needs every subgame's hand rows padded to a multiple of 64");
  }
  stream_ok = stream_ok && smem_fits(stream_hp);
  int schedule = kScheduleLevel;
  if (o.schedule == CFR_SCHEDULE_STREAM) {
    if (!stream_ok) {
      delete t;
      return fail(CFR_EINVAL, "the stream schedule needs at most " + std::to_string(kStreamMaxActions) +
                                  " actions per decision node and a stack that fits shared memory");
    }
    schedule = kScheduleStream;
  } else if (o.schedule == CFR_SCHEDULE_AUTO && stream_ok && stream_warps >= 8 * 152) {
    schedule = kScheduleStream;
  }
  // Wide schedule: one subgame whose tree a block cannot stage (the per-hand pass would walk
  // it from global memory a few nodes at a time).
  const bool wide_ok = n_games == 1 && actions_max <= kStreamMaxActions;
  if (o.schedule == CFR_SCHEDULE_WIDE) {
    if (!wide_ok) {
      delete t;
      return fail(CFR_EINVAL, "the wide schedule takes one subgame with at most " +
                                  std::to_string(kStreamMaxActions) + " actions per decision node");
    }
    schedule = kScheduleWide;
  } else if (o.schedule == CFR_SCHEDULE_AUTO && schedule == kScheduleLevel && wide_ok && !all_fit) {
    schedule = kScheduleWide;
  }
  RunoutPlan ro;
  if (o.runout_tables) {
    if (schedule != kScheduleWide || t->host[0].hand_size != 2) {
      delete t;
      return fail(CFR_EINVAL, "runout_tables needs the wide schedule and two-card hands");
    }
    plan_runouts(t->host[0], ro);
    if (ro.pool_bytes > ((size_t)8 << 30) || ro.tables.size() > 65535) {
      delete t;
      return fail(CFR_EINVAL, "the run-out tables would take more than 8 GB (or number more than 65535)");
    }
  }
  // Resident schedule: one block per SM holds a chunk's state of both players beside a terminal
  // node's board table, and every chunk has a block.
  size_t res_term = 0, res_hand = 0;
  if (resident) {
    for (int g = 0; g < n_games; ++g) {
      const HostGame& h = t->host[g];
      const int rows_max = std::max(h.row_begin[1] - h.row_begin[0], h.row_begin[2] - h.row_begin[1]);
      res_term = std::max(res_term, resident_term_size(h.n_hands, h.hand_size, h.deck, h.hstride, es));
      res_hand = std::max(res_hand, resident_hand_size((int)h.nodes.size(), (int)h.level_start.size() - 1, rows_max,
                                                       chunk[g], es));
    }
    const int per_sm = res_term + res_hand <= 200 * 1024 ? resident_blocks_per_sm(o.precision, res_term + res_hand) : 0;
    if (per_sm < 1 || chunks_of(chunk[0]) > (long)per_sm * n_sms) {
      delete t;
      return fail(CFR_EINVAL, "the resident schedule needs every chunk of hands resident at once (" +
                                  std::to_string(chunks_of(chunk[0])) + " chunks, " + std::to_string(per_sm * n_sms) +
                                  " blocks fit)");
    }
  }
  if (schedule == kScheduleWide) {  // per level: the inner nodes, and the nodes whose reach is stored
    const HostGame& h = t->host[0];
    const int L = (int)h.level_start.size() - 1;
    t->wide_inner_off.assign(1, 0);
    t->wide_fwd_off.assign(1, 0);
    std::vector<int32_t> inner, fwd;
    for (int l = 0; l < L; ++l) {
      for (int n = h.level_start[l]; n < h.level_start[l + 1]; ++n) {
        const bool tabled = !ro.top.empty() && (ro.top[(size_t)n] || ro.inside[(size_t)n]);
        if (!is_end(h.nodes[(size_t)n].type) && !tabled) inner.push_back(n);
        if (h.reach_src[(size_t)n] == n) fwd.push_back(n);
      }
      t->wide_inner_off.push_back((int)inner.size());
      t->wide_fwd_off.push_back((int)fwd.size());
    }
    if ((rc = upload(t, inner, &t->d_wide_inner)) || (rc = upload(t, fwd, &t->d_wide_fwd))) {
      delete t;
      return rc;
    }
  }

  std::vector<Work> chunk_work, term_work, warp_work;
  // each game's device tables, prepared on the host in parallel, then packed in game order
  struct Prepared {
    std::vector<double> r64;
    std::vector<float> rv, pay32;
    std::vector<uint16_t> tab;
    std::vector<int32_t> rown, decn;
    std::vector<ProgOp> ops;
    int dec_begin[3];
  };
  std::vector<Prepared> prep(n_games);
  parallel_games(n_games, [&](int g) {
    const HostGame& h = t->host[g];
    Prepared& q = prep[g];
    const size_t S = (size_t)h.hstride;
    q.r64.assign(2 * S, 0.0);
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < h.n_hands; ++k) q.r64[p * S + k] = h.range[p][k];
    q.rv = to_value_type(q.r64, o.precision);
    q.tab = pack_term_tables(h);
    q.rown = row_nodes(h);
    q.decn = decision_nodes(h, q.dec_begin);
    const double kappa = 1.0 / h.Z;
    q.pay32.resize(2 * h.payoff.size());  // (hi, lo) of payoff * kappa per node
    for (size_t n = 0; n < h.payoff.size(); ++n) {
      const double x = h.payoff[n] * kappa;
      q.pay32[2 * n] = (float)x;
      q.pay32[2 * n + 1] = (float)(x - (double)q.pay32[2 * n]);
    }
    q.ops = program_ops(h, programs[g]);
  });
  Packer packer;
  packer.zeroed((size_t)2 * n_games * sizeof(double), &t->d_br_all);
  t->dev.resize(n_games);  // not resized again: the packer holds the addresses of its fields
  for (int g = 0; g < n_games; ++g) {
    const HostGame& h = t->host[g];
    GameDev& d = t->dev[g];
    memset(&d, 0, sizeof(d));
    const size_t N = h.nodes.size(), S = (size_t)h.hstride;
    d.n_nodes = (int)N;
    d.n_levels = (int)h.level_start.size() - 1;
    d.n_hands = h.n_hands;
    d.hstride = h.hstride;
    d.hand_size = h.hand_size;
    d.n_rows = h.n_rows;
    d.n_terminals = (int)h.terminals.size();
    d.deck = h.deck;
    d.chunk = chunk[g];
    d.n_chunks = (h.n_hands + chunk[g] - 1) / chunk[g];
    d.smem = use_smem[g];
    for (int k = 0; k < 3; ++k) d.row_begin[k] = h.row_begin[k];
    d.n_boards = h.n_boards;
    d.kappa64 = 1.0 / h.Z;
    const Prepared& q = prep[g];
    for (int k = 0; k < 3; ++k) d.dec_begin[k] = q.dec_begin[k];
    const std::vector<double>& r64 = q.r64;
    const std::vector<float>& rv = q.rv;
    const std::vector<uint16_t>& tab = q.tab;
    const std::vector<int32_t>& rown = q.rown;
    const std::vector<int32_t>& decn = q.decn;
    const std::vector<float>& pay32 = q.pay32;
    const std::vector<ProgOp>& ops = q.ops;
    for (int q = 0; q < 4; ++q) {
      d.unit_off[q] = table_meta[g][q];
      d.unit_count[q] = table_meta[g][4 + q];
      d.chunk_off[q] = table_meta[g][8 + q];
      d.chunk_count[q] = table_meta[g][12 + q];
    }
    packer.table(h.nodes, &d.nodes);
    packer.table(h.level_start, &d.level_start);
    packer.table(rown, &d.row_node);
    packer.table(h.hand_mask, &d.hand_mask);
    packer.table(rv, &d.range_v);
    packer.table(r64, &d.range64);
    packer.table(h.payoff, &d.payoff);
    packer.table(pay32, &d.payoff_ff);
    packer.table(tab, &d.term_tab);
    packer.table(decn, &d.dec_nodes);
    packer.table(ops, &d.prog);
    packer.table(chunk_lists[g], &d.chunks);
    packer.table(unit_lists[g], &d.units);
    d.prog_len = (int)programs[g].size();
    const size_t rows = (size_t)h.n_rows * S, cells = 2 * N * S;
    packer.zeroed(rows * 8, &d.R);
    packer.zeroed(rows * 8, &d.S);
    packer.zeroed(rows * es, &d.sigma);
    packer.zeroed(rows * es, &d.sigbar);
    packer.zeroed(cells * es, &d.reach);
    packer.zeroed(cells * es, &d.reach_bar);
    packer.zeroed(cells * es, &d.cfv);
    packer.zeroed(cells * es, &d.cfv_br);
    if (o.variant == CFR_VARIANT_PCFRPLUS) packer.zeroed(rows * 8, &d.M);
    packer.zeroed((size_t)2 * d.n_chunks * 8, &d.br_partial);
    packer.zeroed(4, &d.br_done);
    for (int c = 0; c < d.n_chunks; ++c) chunk_work.push_back({g, c});

    // terminals grouped by board table (fold nodes read only the board-free part of table 0)
    std::vector<int> term;
    for (int n : h.terminals)
      if (ro.inside.empty() || !ro.inside[(size_t)n]) term.push_back(n);  // run-outs: by their tables
    auto table = [&](int n) { return h.nodes[(size_t)n].type == kShowdown ? h.nodes[(size_t)n].row : 0; };
    std::stable_sort(term.begin(), term.end(), [&](int a, int b2) { return table(a) < table(b2); });
    for (int n : term) term_work.push_back({g, n});
  }
  if ((rc = packer.commit(t))) {
    delete t;
    return rc;
  }
  for (int g = 0; g < n_games; ++g) t->dev[g].br_out = t->d_br_all + 2 * g;
  if (!ro.tables.empty()) {  // the run-out tables, from each showdown board's tie groups
    const HostGame& h = t->host[0];
    // tops sorted by table, in groups of up to kRunoutGroup that share a table (one block each)
    std::vector<RunoutItem> items;
    std::vector<RunoutGroup> groups[2];
    for (const std::vector<RunoutItem>* list : {&ro.items8, &ro.items16}) {
      std::vector<RunoutItem> l = *list;
      std::stable_sort(l.begin(), l.end(), [](const RunoutItem& a, const RunoutItem& b) { return a.table < b.table; });
      for (size_t k = 0; k < l.size(); ++k) {
        std::vector<RunoutGroup>& gl = groups[ro.tables[(size_t)l[k].table].wide];
        if (k == 0 || l[k].table != l[k - 1].table || gl.back().count == kRunoutGroup)
          gl.push_back({l[k].table, (int32_t)items.size(), 0, 0});
        gl.back().count += 1;
        items.push_back(l[k]);
      }
    }
    RunoutBoard* d_boards = nullptr;
    int32_t* d_gs = nullptr;
    if ((rc = upload(t, ro.tables, &t->d_ro_tables)) || (rc = upload(t, ro.boards, &d_boards)) ||
        (rc = upload(t, h.sd_gs, &d_gs)) || (rc = upload(t, items, &t->d_ro_items)) ||
        (rc = upload(t, groups[0], &t->d_ro_groups8)) || (rc = upload(t, groups[1], &t->d_ro_groups16))) {
      delete t;
      return rc;
    }
    t->d_ro_pool = static_cast<unsigned char*>(t->alloc(ro.pool_bytes));
    if (!t->d_ro_pool) {
      delete t;
      return fail(CFR_ENOMEM, "device allocation failed");
    }
    if (launch_runout_build(t->d_ro_tables, (int)ro.tables.size(), d_boards, d_gs, t->dev[0].hand_mask, h.n_hands,
                            h.hstride, t->d_ro_pool, t->stream) != 0) {
      delete t;
      return fail(CFR_ECUDA, "run-out table launch failed");
    }
    t->ro_n8 = (int)groups[0].size();
    t->ro_n16 = (int)groups[1].size();
  }
  std::vector<int32_t> term_src(term_work.size());
  for (size_t k = 0; k < term_work.size(); ++k)
    term_src[k] = t->host[term_work[k].game].reach_src[(size_t)term_work[k].unit];
  // terminal runs: one node per block while the nodes do not fill the GPU many times over,
  // up to eight per block (same game and board table) when they do
  std::vector<Work> term_runs;
  {
    const int per = o.term_nodes ? o.term_nodes : std::max(1, std::min(8, (int)term_work.size() / (152 * 8)));
    size_t a = 0;
    while (a < term_work.size()) {
      const Work w = term_work[a];
      const NodeDev& nd = t->host[w.game].nodes[(size_t)w.unit];
      const int tb = nd.type == kShowdown ? nd.row : 0;
      int cnt = 1;
      while (cnt < per && a + cnt < term_work.size()) {
        const Work w2 = term_work[a + cnt];
        const NodeDev& n2 = t->host[w2.game].nodes[(size_t)w2.unit];
        if (w2.game != w.game || (n2.type == kShowdown ? n2.row : 0) != tb) break;
        ++cnt;
      }
      term_runs.push_back({(int)a, cnt});
      a += cnt;
    }
  }
  // stream schedule: blocks of kStreamWarps warps of one game, largest trees first so that
  // their long walks start at once and the small trees fill in behind them
  std::vector<int> by_size(n_games);
  for (int g = 0; g < n_games; ++g) by_size[g] = g;
  std::stable_sort(by_size.begin(), by_size.end(),
                   [&](int a, int b) { return t->host[a].nodes.size() > t->host[b].nodes.size(); });
  const int warp_span = 32 * stream_hp;
  for (int g : by_size)
    for (int u = 0; u < (t->host[g].n_hands + warp_span - 1) / warp_span; u += kStreamWarps) warp_work.push_back({g, u});
  if ((rc = upload(t, t->dev, &t->d_games)) || (rc = upload(t, chunk_work, &t->d_chunk_work)) ||
      (rc = upload(t, term_work, &t->d_term_work)) || (rc = upload(t, warp_work, &t->d_warp_work)) ||
      (rc = upload(t, term_src, &t->d_term_src)) ||
      (rc = upload(t, term_runs, &t->d_term_runs)) ||
      (rc = zeros(t, 1, &t->d_iter)) ||
      (rc = zeros(t, 1, &t->d_done)) || (rc = zeros(t, 1, &t->d_err)) || (rc = zeros(t, 2, &t->d_res_sync)) ||
      (rc = upload(t, discount_table(o, kDiscountCapacity), &t->d_disc))) {
    delete t;
    return rc;
  }
  LaunchCtx& c = t->ctx;
  c.games = t->d_games;
  c.n_games = n_games;
  c.chunk_work = t->d_chunk_work;
  c.n_chunk_work = (int)chunk_work.size();
  c.term_work = t->d_term_work;
  c.term_src = t->d_term_src;
  c.n_term_work = (int)term_work.size();
  c.term_runs = t->d_term_runs;
  c.n_term_runs = (int)term_runs.size();
  c.iter = t->d_iter;
  c.done = t->d_done;
  c.err = t->d_err;
  c.disc = t->d_disc;
  t->disc_capacity = kDiscountCapacity;
  c.smem_hand = smem_hand;
  c.smem_term = smem_term;
  c.variant = o.variant;
  c.precision = o.precision;
  c.pdl = 1;
  c.schedule = schedule;
  c.warp_work = t->d_warp_work;
  c.n_warp_work = (int)warp_work.size();
  c.stream_depth = stream_depth;
  c.stream_prog = stream_prog;
  c.stream_half = stream_half;
  c.stream_units = stream_units;
  c.stream_hp = stream_hp;
  c.alternating = o.alternating ? 1 : 0;
  c.resident = resident ? 1 : 0;
  c.resident_sync = t->d_res_sync;
  if (resident) {
    c.resident_term = (unsigned)res_term;
    c.smem_resident = res_term + res_hand;
    const long items = (long)term_work.size() * (o.alternating ? 1 : 2);
    c.resident_grid = (int)std::max<long>(chunk_work.size(), std::min<long>(items, n_sms));
  }
  if (schedule == kScheduleWide) {
    const HostGame& h = t->host[0];
    c.wide_levels = (int)t->wide_inner_off.size() - 1;
    c.wide_inner_off = t->wide_inner_off.data();
    c.wide_inner = t->d_wide_inner;
    c.wide_fwd_off = t->wide_fwd_off.data();
    c.wide_fwd = t->d_wide_fwd;
    c.wide_stride = h.hstride;
    int dmax = 0;
    for (int p = 0; p < 2; ++p) {
      int cnt = 0;
      for (const NodeDev& nd : h.nodes) cnt += nd.type == kDecision && nd.player == p;
      dmax = std::max(dmax, cnt);
    }
    c.wide_max_dec = dmax;
  }
  if ((rc = setup_leaves(t, specs, n_games))) {
    delete t;
    return rc;
  }
  if (resident && t->leaf.n_leaves > 0) {
    delete t;
    return fail(CFR_EINVAL, "the resident schedule has no leaf-network stage: depth-limited trees take another");
  }
  t->launches_per_iteration =
      (o.alternating ? pass_launches(t, kModeUpdate, 1, 0) + pass_launches(t, kModeUpdate, 2, 1)
                     : pass_launches(t, kModeUpdate, 3, 1)) +
      terminal_launches(t) * (o.alternating ? 2 : 1) +
      (o.alternating ? leaf_launches(t, 1) + leaf_launches(t, 2) : leaf_launches(t, 3));
  t->launches += pass_launches(t, kModeInit, 3, 0);
  if (launch_init(c, stream) != 0) {
    delete t;
    return fail(CFR_ECUDA, "initial strategy launch failed");
  }
  cudaError_t e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    delete t;
    return cuda_fail(e, "create");
  }
  *out = t;
  return CFR_OK;
}

// Depth-limit leaves (Stage 5): network inputs from both players' reach at the leaves, the
// four dense layers, then the leaf values of player 0, player 1 or both (mask 1, 2, 3).
// Launches 1 + 4 + (1 or 2) kernels; none without leaves.
int enqueue_leaves(cfr_tree* t, int player_mask, int use_bar, cudaStream_t s) {
  const LeafCtx& L = t->leaf;
  if (L.n_leaves == 0) return 0;
  const LaunchCtx& c = t->ctx;
  if (launch_leaf_inputs(c, L, use_bar, s) || launch_leaf_net(c, L, s)) return -1;
  for (int p = 0; p < 2; ++p)
    if (((player_mask >> p) & 1) && launch_leaf_values(c, L, p, use_bar, s)) return -1;
  return 0;
}

int leaf_launches(const cfr_tree* t, int player_mask) {
  return t->leaf.n_leaves == 0 ? 0 : 5 + (player_mask == 3 ? 2 : 1);
}

// Kernels one pass launches: one, or one per level under the wide schedule.
int pass_launches(const cfr_tree* t, int which, int player_mask, int advance) {
  if (t->ctx.schedule != kScheduleWide) return 1;
  return wide_launch_count(t->ctx, which, player_mask, advance);
}

// One iteration: alternating = terminal + update for player 0, then for player 1 (each
// preceded by the leaf network when the tree has depth-limit leaves).
int enqueue_iteration(cfr_tree* t, cudaStream_t s) {
  const LaunchCtx& c = t->ctx;
  if (t->opts.alternating) {
    if (enqueue_leaves(t, 1, 0, s) || launch_terminals(t, 1, 0, s) || launch_update(c, 1, 0, s) ||
        enqueue_leaves(t, 2, 0, s) || launch_terminals(t, 2, 0, s) || launch_update(c, 2, 1, s))
      return -1;
  } else {
    if (enqueue_leaves(t, 3, 0, s) || launch_terminals(t, 3, 0, s) || launch_update(c, 3, 1, s)) return -1;
  }
  return 0;
}

// Make sure the discount table covers iterations up to `last`; a larger table replaces the
// old one, and the recorded graphs (which hold its address) are recorded again.
int ensure_discounts(cfr_tree* t, int64_t last) {
  if (last <= t->disc_capacity) return CFR_OK;
  int64_t cap = t->disc_capacity;
  while (cap < last) cap *= 2;
  if (cap > (1 << 30)) return fail(CFR_EINVAL, "too many iterations for one solve");
  Discount* d = nullptr;
  int rc = upload(t, discount_table(t->opts, (int)cap), &d);
  if (rc) return rc;
  t->d_disc = d;
  t->ctx.disc = d;
  t->disc_capacity = (int)cap;
  if (t->iter_graph) cudaGraphExecDestroy(t->iter_graph);
  t->iter_graph = nullptr;
  return CFR_OK;
}

// Read the device error flag (synchronises): a bounded device-side wait that gave up.
int check_device_flag(cfr_tree* t) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, t->stream));
  CK(cudaStreamSynchronize(t->stream));
  if (flag) return fail(CFR_ETIMEOUT, "a bounded device-side wait gave up (bulk copy did not complete)");
  return CFR_OK;
}

int check_game(const cfr_tree* t, int game) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (game < 0 || game >= (int)t->host.size()) return fail(CFR_EINVAL, "game index out of range");
  return CFR_OK;
}

}  // namespace

extern "C" {

int cfr_set_allocator(cfr_alloc_fn alloc, cfr_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(CFR_EINVAL, "give both alloc and free, or neither");
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return CFR_OK;
}

int cfr_tree_create(const cfr_game_spec* spec, const cfr_solver_opts* opts, void* stream, cfr_tree** out) {
  return create_impl(spec, 1, opts, stream, out);
}

int cfr_batch_create(const cfr_game_spec* specs, int n_games, const cfr_solver_opts* opts, void* stream,
                     cfr_tree** out) {
  return create_impl(specs, n_games, opts, stream, out);
}

int cfr_iterate(cfr_tree* t, int n_iters) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (t->leaf.n_leaves > 0 && !t->leaf_net_set) return fail(CFR_ESTATE, "the tree has leaves: set the leaf network first");
  if (n_iters < 0) return fail(CFR_EINVAL, "n_iters < 0");
  if (n_iters == 0) return CFR_OK;
  int rc0 = ensure_discounts(t, (int64_t)t->iters_done + n_iters);
  if (rc0) return rc0;
  if (!t->iter_graph && !t->ctx.resident) {
    if (!t->capture) CK(cudaStreamCreateWithFlags(&t->capture, cudaStreamNonBlocking));
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(t->capture, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_iteration(t, t->capture);
    cudaError_t e = cudaStreamEndCapture(t->capture, &graph);
    if (rc != 0) return fail(CFR_ECUDA, "kernel launch failed during capture");
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&t->iter_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  }
  t->state_gen += 1;
  if (t->ctx.resident) {  // one cooperative launch per 2^20 iterations (its barrier count stays in 32 bits)
    for (int done = 0; done < n_iters; done += 1 << 20) {
      if (launch_resident(t->ctx, std::min(n_iters - done, 1 << 20), t->stream) != 0)
        return fail(CFR_ECUDA, "resident launch failed");
      t->launches += 1;
    }
    t->iters_done += n_iters;
    return CFR_OK;
  }
  for (int k = 0; k < n_iters; ++k) CK(cudaGraphLaunch(t->iter_graph, t->stream));
  t->iters_done += n_iters;
  t->launches += (int64_t)n_iters * t->launches_per_iteration;
  return CFR_OK;
}

int cfr_sync(cfr_tree* t) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  CK(cudaStreamSynchronize(t->stream));
  return check_device_flag(t);
}

int cfr_debug_first_wait_polls(long polls) {
  if (set_first_wait_polls(polls) != 0) return fail(CFR_ECUDA, "could not set the wait limit");
  return CFR_OK;
}

int cfr_strategy(cfr_tree* t, int game, int node, int average, float* out, size_t out_len) {
  int rc = check_game(t, game);
  if (rc) return rc;
  const HostGame& h = t->host[game];
  if (node < 0 || node >= (int)h.nodes.size() || h.nodes[node].type != kDecision)
    return fail(CFR_EINVAL, "node is not a decision node");
  const NodeDev& nd = h.nodes[node];
  const size_t need = (size_t)nd.n_kids * h.n_hands;
  if (!out || out_len < need) return fail(CFR_EINVAL, "output buffer too small");
  if (average && t->avg_gen != t->state_gen) {  // all games at once; reused until R or S change
    if (launch_average_rows(t->ctx, t->stream) != 0) return fail(CFR_ECUDA, "average launch failed");
    t->launches += 1;
    t->avg_gen = t->state_gen;
  }
  if (!average && t->ctx.schedule == kScheduleStream && t->cur_gen != t->state_gen) {
    // the stream schedule keeps no strategy rows: regret-match R for the read-back
    if (launch_current_rows(t->ctx, t->stream) != 0) return fail(CFR_ECUDA, "strategy launch failed");
    t->launches += 1;
    t->cur_gen = t->state_gen;
  }
  const size_t vf = t->opts.precision == CFR_PRECISION_SINGLE ? 1 : 2;
  std::vector<float> tmp(need * vf);
  const float* src = static_cast<const float*>(average ? t->dev[game].sigbar : t->dev[game].sigma);
  CK(cudaMemcpy2DAsync(tmp.data(), (size_t)h.n_hands * 4 * vf, src + (size_t)nd.row * h.hstride * vf,
                       (size_t)h.hstride * 4 * vf, (size_t)h.n_hands * 4 * vf, nd.n_kids, cudaMemcpyDeviceToHost,
                       t->stream));
  CK(cudaStreamSynchronize(t->stream));
  for (size_t k = 0; k < need; ++k) out[k] = vf == 1 ? tmp[k] : (float)((double)tmp[2 * k] + (double)tmp[2 * k + 1]);
  return CFR_OK;
}

int cfr_exploitability_async(cfr_tree* t) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  const LaunchCtx& c = t->ctx;
  if (!t->expl_graph && !t->expl_once) {  // a first pass runs without recording a graph
    if (launch_avg_reach(c, t->stream) || enqueue_leaves(t, 3, 1, t->stream) || launch_terminals(t, 3, 1, t->stream) ||
        launch_br(c, t->stream))
      return fail(CFR_ECUDA, "exploitability launch failed");
    t->expl_once = true;
  } else {  // later passes replay a graph recorded on the second call
    if (!t->expl_graph) {
      if (!t->capture) CK(cudaStreamCreateWithFlags(&t->capture, cudaStreamNonBlocking));
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(t->capture, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_avg_reach(c, t->capture) || enqueue_leaves(t, 3, 1, t->capture) ||
                     launch_terminals(t, 3, 1, t->capture) || launch_br(c, t->capture);
      cudaError_t e = cudaStreamEndCapture(t->capture, &graph);
      if (rc != 0) return fail(CFR_ECUDA, "kernel launch failed during capture");
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&t->expl_graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(t->expl_graph, t->stream));
  }
  t->avg_gen = -1;  // the pass rewrites sigbar with its own normalisation
  t->launches += terminal_launches(t) + pass_launches(t, kModeAvg, 3, 0) +
                 pass_launches(t, kModeBR, 3, 0) + leaf_launches(t, 3);
  return CFR_OK;
}

int cfr_exploitability_result(cfr_tree* t, double* expl, double* br) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (!expl) return fail(CFR_EINVAL, "expl is NULL");
  const int G = (int)t->host.size();
  std::vector<double> vals(2 * G);
  CK(cudaMemcpyAsync(vals.data(), t->d_br_all, 2 * G * sizeof(double), cudaMemcpyDeviceToHost, t->stream));
  CK(cudaStreamSynchronize(t->stream));
  const int frc = check_device_flag(t);
  if (frc) return frc;
  for (int g = 0; g < G; ++g) {
    expl[g] = 0.5 * (vals[2 * g] + vals[2 * g + 1]);
    if (br) {
      br[2 * g] = vals[2 * g];
      br[2 * g + 1] = vals[2 * g + 1];
    }
  }
  return CFR_OK;
}

int cfr_exploitability(cfr_tree* t, double* expl, double* br) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (!expl) return fail(CFR_EINVAL, "expl is NULL");
  const int rc = cfr_exploitability_async(t);
  return rc ? rc : cfr_exploitability_result(t, expl, br);
}

int cfr_reset(cfr_tree* t) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  for (const GameDev& d : t->dev) {
    const size_t rows = (size_t)d.n_rows * d.hstride * sizeof(double);
    CK(cudaMemsetAsync(d.R, 0, rows, t->stream));
    CK(cudaMemsetAsync(d.S, 0, rows, t->stream));
    if (d.M) CK(cudaMemsetAsync(d.M, 0, rows, t->stream));
  }
  CK(cudaMemsetAsync(t->d_iter, 0, sizeof(int), t->stream));
  t->state_gen += 1;
  if (launch_init(t->ctx, t->stream) != 0) return fail(CFR_ECUDA, "initial strategy launch failed");
  t->launches += pass_launches(t, kModeInit, 3, 0);
  t->iters_done = 0;
  return CFR_OK;
}

int cfr_schedule(const cfr_tree* t) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  return t->ctx.resident ? CFR_SCHEDULE_RESIDENT
         : t->ctx.schedule == kScheduleStream ? CFR_SCHEDULE_STREAM
         : t->ctx.schedule == kScheduleWide ? CFR_SCHEDULE_WIDE
                                            : CFR_SCHEDULE_LEVEL;
}

int cfr_tree_info(const cfr_tree* t, int game, int* n_nodes, int* n_hands, int* iters_done) {
  int rc = check_game(t, game);
  if (rc) return rc;
  if (n_nodes) *n_nodes = (int)t->host[game].nodes.size();
  if (n_hands) *n_hands = t->host[game].n_hands;
  if (iters_done) *iters_done = t->iters_done;
  return CFR_OK;
}

int cfr_node_info(const cfr_tree* t, int game, int node, int* type, int* player, int* n_actions, int* parent,
                  int* action_in_parent, int* deal_card, double* contrib) {
  int rc = check_game(t, game);
  if (rc) return rc;
  const HostGame& h = t->host[game];
  if (node < 0 || node >= (int)h.nodes.size()) return fail(CFR_EINVAL, "node index out of range");
  const NodeDev& nd = h.nodes[node];
  if (type) *type = nd.type;
  if (player) *player = (nd.type == kDecision || nd.type == kFold) ? nd.player : -1;
  if (n_actions) *n_actions = nd.n_kids;
  if (parent) *parent = nd.parent;
  if (action_in_parent) *action_in_parent = nd.parent < 0 ? -1 : nd.paction;
  if (deal_card) *deal_card = nd.deal == kNoCard ? -1 : nd.deal;
  if (contrib) {
    contrib[0] = h.contrib[2 * (size_t)node];
    contrib[1] = h.contrib[2 * (size_t)node + 1];
  }
  return CFR_OK;
}

int cfr_read_values(cfr_tree* t, int game, int what, int player, int node, double* out, size_t out_len) {
  int rc = check_game(t, game);
  if (rc) return rc;
  const HostGame& h = t->host[game];
  const GameDev& d = t->dev[game];
  if (node < 0 || node >= (int)h.nodes.size()) return fail(CFR_EINVAL, "node index out of range");
  if (!out) return fail(CFR_EINVAL, "out is NULL");
  const NodeDev& nd = h.nodes[node];
  const int H = h.n_hands;
  const size_t S = (size_t)h.hstride;
  if (what == CFR_READ_REGRET || what == CFR_READ_AVG_SUM || what == CFR_READ_PREDICTION) {
    if (nd.type != kDecision) return fail(CFR_EINVAL, "node is not a decision node");
    if (what == CFR_READ_PREDICTION && !d.M) return fail(CFR_EINVAL, "only Predictive CFR+ keeps a prediction");
    const size_t need = (size_t)nd.n_kids * H;
    if (out_len < need) return fail(CFR_EINVAL, "output buffer too small");
    const double* src = (what == CFR_READ_REGRET ? d.R : what == CFR_READ_AVG_SUM ? d.S : d.M) + (size_t)nd.row * S;
    CK(cudaMemcpy2DAsync(out, (size_t)H * 8, src, S * 8, (size_t)H * 8, nd.n_kids, cudaMemcpyDeviceToHost,
                         t->stream));
    CK(cudaStreamSynchronize(t->stream));
    return CFR_OK;
  }
  if (what == CFR_READ_CFV || what == CFR_READ_BR_CFV || what == CFR_READ_AVG_REACH) {
    if (player < 0 || player > 1) return fail(CFR_EINVAL, "player must be 0 or 1");
    if (out_len < (size_t)H) return fail(CFR_EINVAL, "output buffer too small");
    const size_t vf = t->opts.precision == CFR_PRECISION_SINGLE ? 1 : 2;
    std::vector<float> tmp((size_t)H * vf);
    const void* arr = what == CFR_READ_CFV ? d.cfv : what == CFR_READ_BR_CFV ? d.cfv_br : d.reach_bar;
    // a run-out node's reach is its source's with the hands holding a dealt card zeroed
    const int at = what == CFR_READ_AVG_REACH ? h.reach_src[(size_t)node] : node;
    const float* src = static_cast<const float*>(arr) + ((size_t)player * h.nodes.size() + at) * S * vf;
    CK(cudaMemcpyAsync(tmp.data(), src, (size_t)H * 4 * vf, cudaMemcpyDeviceToHost, t->stream));
    CK(cudaStreamSynchronize(t->stream));
    for (int k = 0; k < H; ++k) out[k] = vf == 1 ? (double)tmp[k] : (double)tmp[2 * k] + (double)tmp[2 * k + 1];
    if (at != node)
      for (int k = 0; k < H; ++k)
        if (h.hand_mask[(size_t)k] & nd.board) out[k] = 0.0;
    return CFR_OK;
  }
  return fail(CFR_EINVAL, "unknown read kind");
}

int cfr_write_values(cfr_tree* t, int game, int what, int node, const double* in, size_t in_len) {
  int rc = check_game(t, game);
  if (rc) return rc;
  const HostGame& h = t->host[game];
  const GameDev& d = t->dev[game];
  if (node < 0 || node >= (int)h.nodes.size() || h.nodes[node].type != kDecision)
    return fail(CFR_EINVAL, "node is not a decision node");
  if (what != CFR_READ_REGRET && what != CFR_READ_AVG_SUM && what != CFR_READ_PREDICTION)
    return fail(CFR_EINVAL, "what must be REGRET, AVG_SUM or PREDICTION");
  if (what == CFR_READ_PREDICTION && !d.M) return fail(CFR_EINVAL, "only Predictive CFR+ keeps a prediction");
  const NodeDev& nd = h.nodes[node];
  const size_t H = (size_t)h.n_hands, S = (size_t)h.hstride;
  if (!in || in_len < (size_t)nd.n_kids * H) return fail(CFR_EINVAL, "input buffer too small");
  double* dst = (what == CFR_READ_REGRET ? d.R : what == CFR_READ_AVG_SUM ? d.S : d.M) + (size_t)nd.row * S;
  CK(cudaMemcpy2DAsync(dst, S * 8, in, H * 8, H * 8, nd.n_kids, cudaMemcpyHostToDevice, t->stream));
  // new regrets: the current strategy and both players' reach follow them at once
  if (what != CFR_READ_AVG_SUM && launch_init(t->ctx, t->stream) != 0) return fail(CFR_ECUDA, "strategy launch failed");
  if (what != CFR_READ_AVG_SUM) t->launches += pass_launches(t, kModeInit, 3, 0);
  CK(cudaStreamSynchronize(t->stream));
  t->state_gen += 1;
  t->avg_gen = -1;
  return CFR_OK;
}

int cfr_stage_times(cfr_tree* t, int n_iters, double* ms, int64_t* launches) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (t->leaf.n_leaves > 0 && !t->leaf_net_set) return fail(CFR_ESTATE, "the tree has leaves: set the leaf network first");
  if (!ms || n_iters < 0) return fail(CFR_EINVAL, "bad arguments");
  const int drc = ensure_discounts(t, (int64_t)t->iters_done + n_iters);
  if (drc) return drc;
  const LaunchCtx& c = t->ctx;
  cudaStream_t s = t->stream;
  t->state_gen += 1;
  t->avg_gen = -1;
  std::vector<cudaEvent_t> ev;
  std::vector<int> stage_of;
  auto mark = [&](int stage) -> cudaError_t {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    ev.push_back(e);
    stage_of.push_back(stage);
    return cudaEventRecord(e, s);
  };
  int rc = 0;
  cudaError_t err = mark(-1);
  for (int it = 0; it < n_iters && !rc && err == cudaSuccess; ++it) {
    if (t->opts.alternating) {
      for (int p = 0; p < 2 && !rc && err == cudaSuccess; ++p) {
        if (t->leaf.n_leaves > 0) {
          rc = enqueue_leaves(t, 1 << p, 0, s);
          if (!rc) err = mark(CFR_STAGE_LEAF);
        }
        if (!rc && err == cudaSuccess) rc = launch_terminals(t, 1 << p, 0, s);
        if (!rc && terminal_launches(t) > 0) err = mark(CFR_STAGE_TERMINAL);
        if (!rc && err == cudaSuccess) rc = launch_update(c, 1 << p, p == 1, s);
        if (!rc && err == cudaSuccess) err = mark(CFR_STAGE_UPDATE);
      }
    } else {
      if (t->leaf.n_leaves > 0) {
        rc = enqueue_leaves(t, 3, 0, s);
        if (!rc) err = mark(CFR_STAGE_LEAF);
      }
      if (!rc && err == cudaSuccess) rc = launch_terminals(t, 3, 0, s);
      if (!rc && terminal_launches(t) > 0) err = mark(CFR_STAGE_TERMINAL);
      if (!rc && err == cudaSuccess) rc = launch_update(c, 3, 1, s);
      if (!rc && err == cudaSuccess) err = mark(CFR_STAGE_UPDATE);
    }
  }
  if (!rc && err == cudaSuccess) rc = launch_avg_reach(c, s);
  if (!rc && err == cudaSuccess) err = mark(CFR_STAGE_AVG_REACH);
  if (!rc && err == cudaSuccess && t->leaf.n_leaves > 0) {
    rc = enqueue_leaves(t, 3, 1, s);
    if (!rc) err = mark(CFR_STAGE_LEAF);
  }
  if (!rc && err == cudaSuccess) rc = launch_terminals(t, 3, 1, s);
  if (!rc && err == cudaSuccess && terminal_launches(t) > 0) err = mark(CFR_STAGE_BR_TERMINAL);
  if (!rc && err == cudaSuccess) rc = launch_br(c, s);
  if (!rc && err == cudaSuccess) err = mark(CFR_STAGE_BR);
  cudaError_t serr = cudaStreamSynchronize(s);
  double tot[CFR_N_STAGES] = {0};
  int64_t cnt[CFR_N_STAGES] = {0};
  for (size_t k = 1; k < ev.size() && serr == cudaSuccess && err == cudaSuccess && !rc; ++k) {
    float m = 0.f;
    cudaEventElapsedTime(&m, ev[k - 1], ev[k]);
    tot[stage_of[k]] += m;
    cnt[stage_of[k]] += 1;
  }
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  if (rc) return fail(CFR_ECUDA, "stage launch failed");
  if (err != cudaSuccess) return cuda_fail(err, "cudaEventRecord");
  if (serr != cudaSuccess) return cuda_fail(serr, "cudaStreamSynchronize");
  t->iters_done += n_iters;
  for (int k = 0; k < CFR_N_STAGES; ++k) {
    ms[k] = cnt[k] ? tot[k] / (double)cnt[k] : 0.0;
    if (launches) launches[k] = cnt[k];
  }
  t->launches += (int64_t)n_iters * t->launches_per_iteration + terminal_launches(t) +
                 pass_launches(t, kModeAvg, 3, 0) + pass_launches(t, kModeBR, 3, 0) + leaf_launches(t, 3);
  return CFR_OK;
}

int cfr_counters(const cfr_tree* t, int64_t* kernel_launches, int64_t* device_bytes, int64_t* h2d_bytes) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (kernel_launches) *kernel_launches = t->launches;
  if (device_bytes) *device_bytes = t->device_bytes;
  if (h2d_bytes) *h2d_bytes = t->h2d_bytes;
  return CFR_OK;
}

int cfr_set_leaf_net(cfr_tree* t, const uint16_t* const W[4], const float* const b[4]) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (t->leaf.n_leaves == 0) return fail(CFR_ESTATE, "the tree has no depth-limit leaves");
  if (!W || !b) return fail(CFR_EINVAL, "W and b are required");
  const size_t wn[4] = {(size_t)kLeafHidden * kLeafIn, (size_t)kLeafHidden * kLeafHidden,
                        (size_t)kLeafHidden * kLeafHidden, (size_t)kLeafOut * kLeafHidden};
  const size_t bn[4] = {(size_t)kLeafHidden, (size_t)kLeafHidden, (size_t)kLeafHidden, (size_t)kLeafOut};
  for (int k = 0; k < 4; ++k)
    if (!W[k] || !b[k]) return fail(CFR_EINVAL, "every layer needs weights and a bias");
  // the range inputs (columns of layer 1) and value outputs (rows of layer 4) move to the
  // handle's column order
  const std::vector<int>& col = t->leaf_col;
  std::vector<uint16_t> w0(wn[0]), w3(wn[3]);
  std::vector<float> b3(bn[3]);
  for (int r = 0; r < kLeafHidden; ++r) {
    const uint16_t* src = W[0] + (size_t)r * kLeafIn;
    uint16_t* dst = w0.data() + (size_t)r * kLeafIn;
    for (int c = 2 * kLeafSlots; c < kLeafIn; ++c) dst[c] = src[c];
    for (int p = 0; p < 2; ++p)
      for (int sl = 0; sl < kLeafSlots; ++sl) dst[p * kLeafSlots + col[sl]] = src[p * kLeafSlots + sl];
  }
  for (int r = 2 * kLeafSlots; r < kLeafOut; ++r) {
    for (int c = 0; c < kLeafHidden; ++c) w3[(size_t)r * kLeafHidden + c] = W[3][(size_t)r * kLeafHidden + c];
    b3[r] = b[3][r];
  }
  for (int p = 0; p < 2; ++p)
    for (int sl = 0; sl < kLeafSlots; ++sl) {
      const int ro = p * kLeafSlots + col[sl], ri = p * kLeafSlots + sl;
      for (int c = 0; c < kLeafHidden; ++c) w3[(size_t)ro * kLeafHidden + c] = W[3][(size_t)ri * kLeafHidden + c];
      b3[ro] = b[3][ri];
    }
  const void* wsrc[4] = {w0.data(), W[1], W[2], w3.data()};
  const float* bsrc[4] = {b[0], b[1], b[2], b3.data()};
  for (int k = 0; k < 4; ++k) {
    CK(cudaMemcpyAsync(const_cast<void*>(t->leaf.W[k]), wsrc[k], wn[k] * 2, cudaMemcpyHostToDevice, t->stream));
    CK(cudaMemcpyAsync(const_cast<float*>(t->leaf.b[k]), bsrc[k], bn[k] * 4, cudaMemcpyHostToDevice, t->stream));
  }
  CK(cudaStreamSynchronize(t->stream));
  t->leaf_net_set = true;
  return CFR_OK;
}

int cfr_eval_leaves(cfr_tree* t, int average) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (t->leaf.n_leaves == 0) return fail(CFR_ESTATE, "the tree has no depth-limit leaves");
  if (!t->leaf_net_set) return fail(CFR_ESTATE, "set the leaf network first");
  if (average) {
    if (launch_avg_reach(t->ctx, t->stream) != 0) return fail(CFR_ECUDA, "average launch failed");
    t->avg_gen = -1;
  }
  if (enqueue_leaves(t, 3, average ? 1 : 0, t->stream) != 0) return fail(CFR_ECUDA, "leaf launch failed");
  t->launches += (average ? pass_launches(t, kModeAvg, 3, 0) : 0) + leaf_launches(t, 3);
  return cfr_sync(t);
}

int cfr_leaf_info(const cfr_tree* t, int leaf, int* n_leaves, int* game, int* node, int* row0) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (n_leaves) *n_leaves = t->leaf.n_leaves;
  if (leaf < 0) return CFR_OK;
  if (leaf >= t->leaf.n_leaves) return fail(CFR_EINVAL, "leaf index out of range");
  const LeafDev& lf = t->leaf_host[(size_t)leaf];
  if (game) *game = lf.game;
  if (node) *node = lf.node;
  if (row0) *row0 = lf.row0;
  return CFR_OK;
}

int cfr_read_leaf_rows(cfr_tree* t, int what, int row0, int n_rows, void* out) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  const int rows = t->leaf.n_leaves * kLeafCards;
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > rows || (!out && n_rows)) return fail(CFR_EINVAL, "bad row range");
  if (what != 0 && what != 1) return fail(CFR_EINVAL, "what must be 0 (inputs) or 1 (outputs)");
  const size_t width = what == 0 ? kLeafIn : kLeafOut, es = what == 0 ? 2 : 4;
  std::vector<unsigned char> raw((size_t)n_rows * width * es);
  const unsigned char* src = what == 0 ? static_cast<const unsigned char*>(t->leaf.X)
                                       : reinterpret_cast<const unsigned char*>(t->leaf.Y);
  if (n_rows)
    CK(cudaMemcpyAsync(raw.data(), src + (size_t)row0 * width * es, raw.size(), cudaMemcpyDeviceToHost, t->stream));
  CK(cudaStreamSynchronize(t->stream));
  // back to slot order: the range / value block of each player moves from column col[s] to s
  unsigned char* o = static_cast<unsigned char*>(out);
  const std::vector<int>& col = t->leaf_col;
  for (int r = 0; r < n_rows; ++r) {
    const unsigned char* in_row = raw.data() + (size_t)r * width * es;
    unsigned char* out_row = o + (size_t)r * width * es;
    memcpy(out_row + 2 * kLeafSlots * es, in_row + 2 * kLeafSlots * es, (width - 2 * kLeafSlots) * es);
    for (int p = 0; p < 2; ++p)
      for (int sl = 0; sl < kLeafSlots; ++sl)
        memcpy(out_row + (size_t)(p * kLeafSlots + sl) * es, in_row + (size_t)(p * kLeafSlots + col[sl]) * es, es);
  }
  return CFR_OK;
}

int cfr_gemm_bf16(const void* A, const void* B, const float* bias, void* C, int M, int N, int K, int act,
                  int out_f32, int* err, void* stream) {
  if (!A || !B || !C || !err) return fail(CFR_EINVAL, "A, B, C and err are required");
  int rc = check_device();
  if (rc) return rc;
  static const int configured = configure_gemm();
  if (configured != 0) return fail(CFR_ECUDA, "GEMM kernel attribute setup failed");
  const int r = launch_gemm_bf16(A, B, bias, C, M, N, K, act, out_f32, err, stream);
  if (r == -2) return fail(CFR_EINVAL, "cfr_gemm_bf16: N must be a multiple of 128, K of 64, pointers 16-byte aligned");
  if (r == -3) return fail(CFR_ECUDA, "cfr_gemm_bf16: no tensor-map encoder in the driver");
  if (r != 0) return fail(CFR_ECUDA, "cfr_gemm_bf16: launch failed");
  return CFR_OK;
}

void cfr_tree_destroy(cfr_tree* t) { delete t; }

int cfr_autotune(const cfr_game_spec* specs, int n_games, const cfr_solver_opts* opts, void* stream, int iters,
                 cfr_solver_opts* best, double* ms_per_iter) {
  if (!specs || n_games < 1 || !opts || !best) return fail(CFR_EINVAL, "specs, opts and best are required");
  if (iters < 1) return fail(CFR_EINVAL, "iters must be at least 1");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // time one candidate; +inf when the layout does not apply (e.g. a tree the stream form refuses)
  auto trial = [&](const cfr_solver_opts& o, double* ms) -> int {
    *ms = INFINITY;
    cfr_tree* t = nullptr;
    int rc = create_impl(specs, n_games, &o, stream, &t);
    // the level schedule takes every valid handle: its refusal is the caller's error
    if (rc == CFR_EINVAL && o.schedule != CFR_SCHEDULE_LEVEL) return CFR_OK;
    if (rc) return rc;
    t->leaf_net_set = true;  // leaves, if any, run with the all-zero network the handle starts with
    rc = cfr_iterate(t, 2);
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaEventRecord(e0, s);
    if (!rc && e == cudaSuccess) rc = cfr_iterate(t, iters);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float m = 0.f;
    if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&m, e0, e1);
    if (!rc && e == cudaSuccess) rc = check_device_flag(t);
    delete t;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    *ms = (double)m / iters;
    return CFR_OK;
  };
  cfr_solver_opts cand = *opts, top = *opts;
  double top_ms = INFINITY, ms = 0.0;
  int rc = CFR_OK;
  cand.term_nodes = 0;
  cand.runout_tables = 0;  // the run-out tables apply to the wide candidate only
  const int chunks[4] = {4, 8, 16, 32};
  for (int k = 0; k < 4 && !rc; ++k) {  // level schedule, hands per block
    cand.schedule = CFR_SCHEDULE_LEVEL;
    cand.chunk_hands = chunks[k];
    rc = trial(cand, &ms);
    if (!rc && ms < top_ms) top_ms = ms, top = cand;
  }
  for (int sch : {CFR_SCHEDULE_STREAM, CFR_SCHEDULE_WIDE}) {
    if (rc || (sch == CFR_SCHEDULE_WIDE && n_games != 1)) continue;
    cand.schedule = sch;
    cand.chunk_hands = 0;
    cand.runout_tables = sch == CFR_SCHEDULE_WIDE ? opts->runout_tables : 0;
    for (int wh : {32, 64}) {  // stream schedule: hands per warp
      if (rc || (sch == CFR_SCHEDULE_WIDE && wh == 64)) continue;
      cand.warp_hands = sch == CFR_SCHEDULE_STREAM ? wh : 0;
      rc = trial(cand, &ms);
      if (!rc && ms < top_ms) top_ms = ms, top = cand;
    }
    cand.warp_hands = 0;
  }
  if (!rc) {  // resident schedule: whole iterations in one cooperative launch
    cand.schedule = CFR_SCHEDULE_RESIDENT;
    cand.chunk_hands = 0;
    cand.warp_hands = 0;
    cand.runout_tables = 0;
    rc = trial(cand, &ms);
    if (!rc && ms < top_ms) top_ms = ms, top = cand;
  }
  cand = top;
  for (int tn : {1, 2, 4, 8}) {  // terminal nodes per block, for the fastest layout
    if (cand.schedule == CFR_SCHEDULE_RESIDENT) break;  // one node per block item: no runs
    if (rc) break;
    cand.term_nodes = tn;
    rc = trial(cand, &ms);
    if (!rc && ms < top_ms) top_ms = ms, top = cand;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (!(top_ms < INFINITY)) return fail(CFR_EINVAL, "no layout applies to these subgames");
  *best = top;
  if (ms_per_iter) *ms_per_iter = top_ms;
  return CFR_OK;
}

const char* cfr_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Exploitability without allocation.
//
// cfr_exploitability records and instantiates a CUDA graph on its second call and keeps
// its per-block best-response sums in buffers of the handle.  Some callers cannot let a
// call allocate: a serving loop that runs under a fixed device-memory budget, or a
// real-time thread that must not wait in an allocator between two decisions (freeing
// device memory synchronises the whole device).  This variant launches
// the same passes directly on the handle's stream and replaces the final FP64 root
// reduction with a copy whose scratch (per-block sums, per-game arrival counters and
// results) lives in one statically sized device array of this file.  The call makes no
// device or host allocation; its only setup is resolving that array's address.

namespace {

constexpr int kStaticMaxChunks = 8192;  // hand chunks of one handle (blocks per player)
constexpr int kStaticMaxGames = 1024;   // games of one handle
constexpr size_t kStaticPartialBytes = (size_t)2 * kStaticMaxChunks * sizeof(double);
constexpr size_t kStaticOutBytes = (size_t)2 * kStaticMaxGames * sizeof(double);
constexpr size_t kStaticDoneBytes = (size_t)kStaticMaxGames * sizeof(unsigned);
constexpr size_t kStaticScratchBytes = kStaticPartialBytes + kStaticOutBytes + kStaticDoneBytes;  // 148 KiB

// Layout: partial [2][kStaticMaxChunks] FP64 (player-major, indexed by chunk-work item),
// out [kStaticMaxGames][2] FP64, done [kStaticMaxGames] uint32.  Only `done` has to start
// at zero: the call clears the counters of its games on its stream before the reduction,
// and the last block of each game clears its counter again after reading it.
static __device__ __align__(256) unsigned char g_expl_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// FP64 root best-response value of one chunk of hands, sum_h r_p(h) v*_p(root, h), and the
// per-game reduction by the last block of the game.  One warp per (player, chunk); the
// root is node 0 and the per-hand pass has left v* in cfv_br.
__global__ void __launch_bounds__(32) k_br_root_static(const GameDev* __restrict__ games,
                                                       const Work* __restrict__ work, int n_work, int precision,
                                                       unsigned char* __restrict__ scratch) {
  double* partial = reinterpret_cast<double*>(scratch);
  double* out = reinterpret_cast<double*>(scratch + kStaticPartialBytes);
  unsigned* done = reinterpret_cast<unsigned*>(scratch + kStaticPartialBytes + kStaticOutBytes);
  const int p = blockIdx.x >= (unsigned)n_work;
  const int item = blockIdx.x - p * n_work;
  const Work wk = work[item];
  const GameDev& G = games[wk.game];
  const int lane = threadIdx.x;
  const int h = wk.unit * G.chunk + lane;
  double x = 0.0;
  if (lane < G.chunk && h < G.n_hands) {
    const size_t at = ((size_t)p * G.n_nodes) * G.hstride + h;  // (player p, node 0, hand h)
    double v;
    if (precision == kPrecisionSingle) {
      v = (double)static_cast<const float*>(G.cfv_br)[at];
    } else {
      const float2 hl = static_cast<const float2*>(G.cfv_br)[at];
      v = (double)hl.x + (double)hl.y;
    }
    x = G.range64[(size_t)p * G.hstride + h] * v;
  }
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  __shared__ bool s_last;
  if (lane == 0) {
    partial[(size_t)p * kStaticMaxChunks + item] = x;
    __threadfence();
    s_last = atomicAdd(&done[wk.game], 1u) == (unsigned)(2 * G.n_chunks - 1);
  }
  __syncwarp();
  if (!s_last) return;
  __threadfence();
  // first chunk-work item of this game: the list is game-major, chunks in order
  int first = 0;
  for (int g = lane; g < wk.game; g += 32) first += games[g].n_chunks;
  for (int o = 16; o > 0; o >>= 1) first += __shfl_down_sync(0xffffffffu, first, o);
  first = __shfl_sync(0xffffffffu, first, 0);
  for (int q = 0; q < 2; ++q) {
    double s = 0.0;
    for (int c = lane; c < G.n_chunks; c += 32) s += __ldcg(&partial[(size_t)q * kStaticMaxChunks + first + c]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[2 * (size_t)wk.game + q] = s;
  }
  if (lane == 0) done[wk.game] = 0u;
}

// Once per device, with that device current: the address of this device's copy of the
// scratch array.  Also loads the reduction kernel, so that later calls do no setup.
int static_scratch(unsigned char** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CFR_ECUDA, "device ordinal beyond the scratch table");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_expl_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_expl_scratch)");
    cudaFuncAttributes attr;
    e = cudaFuncGetAttributes(&attr, k_br_root_static);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes(k_br_root_static)");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CFR_OK;
}

}  // namespace

extern "C" int cfr_exploitability_noalloc(cfr_tree* t, double* expl, double* br) {
  if (!t) return fail(CFR_EINVAL, "tree is NULL");
  if (!expl || !br) return fail(CFR_EINVAL, "expl and br are both required");
  const LaunchCtx& c = t->ctx;
  if (c.n_games > kStaticMaxGames)
    return fail(CFR_EINVAL, "cfr_exploitability_noalloc: the handle has " + std::to_string(c.n_games) +
                                " games; its static scratch holds at most " + std::to_string(kStaticMaxGames));
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != t->device)
    return fail(CFR_EINVAL, "cfr_exploitability_noalloc: the handle was created on device " +
                                std::to_string(t->device) + "; make it the current device (current: " +
                                std::to_string(dev) + ")");
  if (c.n_chunk_work > kStaticMaxChunks)
    return fail(CFR_EINVAL, "cfr_exploitability_noalloc: the handle has " + std::to_string(c.n_chunk_work) +
                                " hand chunks per player; its static scratch holds at most " +
                                std::to_string(kStaticMaxChunks));
  unsigned char* scratch = nullptr;
  int rc = static_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t s = t->stream;
  CK(cudaMemsetAsync(scratch + kStaticPartialBytes + kStaticOutBytes, 0, (size_t)c.n_games * sizeof(unsigned), s));
  t->avg_gen = -1;
  if (launch_avg_reach(c, s) || enqueue_leaves(t, 3, 1, s) || launch_terminals(t, 3, 1, s) || launch_br(c, s))
    return fail(CFR_ECUDA, "exploitability launch failed");
  k_br_root_static<<<2 * c.n_chunk_work, 32, 0, s>>>(c.games, c.chunk_work, c.n_chunk_work, c.precision, scratch);
  CK(cudaGetLastError());
  t->launches += terminal_launches(t) + pass_launches(t, kModeAvg, 3, 0) + pass_launches(t, kModeBR, 3, 0) +
                 leaf_launches(t, 3) + 1;
  CK(cudaMemcpyAsync(br, scratch + kStaticPartialBytes, (size_t)c.n_games * 2 * sizeof(double),
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  rc = check_device_flag(t);
  if (rc) return rc;
  for (int g = 0; g < c.n_games; ++g) expl[g] = 0.5 * (br[2 * g] + br[2 * g + 1]);
  return CFR_OK;
}
