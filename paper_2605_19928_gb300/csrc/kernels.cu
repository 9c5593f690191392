// CUDA kernels of one Parallel CFR iteration (sm_103a).
//
// The paper's seven stages (Section 4.1, Table 1) are regrouped by what couples them:
//   * every pass along the tree -- regret matching (Eq. rm), forward reach (Stage 1),
//     backward values (Stage 6, Eq. backward), the regret / average update (Stage 7) and
//     the best-response backward pass -- is independent per private hand.  k_hand gives
//     each CUDA block a chunk of hands and walks all tree levels for them, with only
//     __syncthreads() between levels; the chunk's per-node state sits in shared memory
//     when it fits, else in the global arrays (L2);
//   * terminal values need the opponent's whole reach vector: k_terminal gives each block
//     one fold or showdown node and evaluates it in O(hands) (Stages 2-4): card-blocker
//     inclusion-exclusion at folds, rank-sorted prefix sums with per-card corrections at
//     showdowns.
// One player's update is therefore two launches (terminal, then hand), recorded once in
// a CUDA graph.
//
// Precision: cumulative regrets R and average sums S are FP64 (GB300 runs FP64 at about
// 1/64 of the FP32 rate, so FP64 is kept to those updates).  Reach, strategies and values
// are either double-float pairs on the FP32 pipe (Pairs, the default: ~44-bit
// significands, so regrets that are small differences of large values keep their digits)
// or plain FP32 (Single).
#include <cuda_runtime.h>

#include <cstdio>

#include "pcfr_internal.h"

namespace pcfr {

constexpr int kHandThreads = 256;
constexpr int kTermThreads = 512;

enum HandMode { kModeInit = 0, kModeUpdate = 1, kModeAvg = 2, kModeBR = 3 };

// ------------------------------------------------------------------ double-float arithmetic
//
// A value is hi + lo with |lo| <= ulp(hi) / 2.  Sums use Knuth's TwoSum (TAOCP vol. 2,
// section 4.2.2) on both halves followed by renormalisation (Dekker 1971; the "accurate"
// addition of Hida, Li and Bailey's double-double library); products use the FMA form of
// Dekker's exact product.  The _rn intrinsics stop the compiler from contracting or
// reassociating the error terms.

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_of(float x) { return {x, 0.f}; }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ float ff_round(ff a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s1, s2, t1, t2;
  two_sum(a.hi, b.hi, s1, s2);
  two_sum(a.lo, b.lo, t1, t2);
  s2 = __fadd_rn(s2, t1);
  fast_two_sum(s1, s2, s1, s2);
  s2 = __fadd_rn(s2, t2);
  fast_two_sum(s1, s2, s1, s2);
  return {s1, s2};
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float hi, lo;
  fast_two_sum(p, e, hi, lo);
  return {hi, lo};
}
// 1 / b: the FP32 reciprocal refined by one Newton step in double-float.
__device__ __forceinline__ ff ff_recip(ff b) {
  const ff r = ff_of(__frcp_rn(b.hi));
  return ff_add(r, ff_mul(r, ff_sub(ff_of(1.f), ff_mul(b, r))));
}
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Exact float -> double by exponent rebias on the integer pipe (IEEE 754 binary32 ->
// binary64; subnormal floats, below 1.2e-38, become zero).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const uint64_t ed = e == 0xffu ? 0x7ffu : (uint64_t)(e + 896u);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ ff d2ff(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - f2d(hi))};
}
__device__ __forceinline__ double ff2d(ff a) { return f2d(a.hi) + f2d(a.lo); }

__device__ __forceinline__ ff ff_shfl_up(ff a, int o) {
  return {__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// ------------------------------------------------------------------ precision policies

struct Pairs {  // double-float values
  using V = ff;
  static __device__ __forceinline__ V zero() { return ff_of(0.f); }
  static __device__ __forceinline__ V add(V a, V b) { return ff_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return ff_sub(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return ff_mul(a, b); }
  static __device__ __forceinline__ V vmax(V a, V b) { return ff_gt(b, a) ? b : a; }
  static __device__ __forceinline__ bool positive(V a) { return a.hi > 0.f; }
  static __device__ __forceinline__ V recip(V a) { return ff_recip(a); }
  static __device__ __forceinline__ V of_double(double x) { return d2ff(x); }
  static __device__ __forceinline__ double to_double(V a) { return ff2d(a); }
  static __device__ __forceinline__ ff to_ff(V a) { return a; }
  static __device__ __forceinline__ V of_ff(ff a) { return a; }
};

struct Single {  // plain FP32 values
  using V = float;
  static __device__ __forceinline__ V zero() { return 0.f; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V vmax(V a, V b) { return fmaxf(a, b); }
  static __device__ __forceinline__ bool positive(V a) { return a > 0.f; }
  static __device__ __forceinline__ V recip(V a) { return 1.f / a; }
  static __device__ __forceinline__ V of_double(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double to_double(V a) { return f2d(a); }
  static __device__ __forceinline__ ff to_ff(V a) { return ff_of(a); }
  static __device__ __forceinline__ V of_ff(ff a) { return ff_round(a); }
};

// ------------------------------------------------------------------ block primitives (double-float)

template <int NT>
__device__ __forceinline__ ff block_sum_ff(ff x, ff* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = ff_add(x, ff_shfl_xor(x, o));
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    ff y = lane < NT / 32 ? red[lane] : ff_of(0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y = ff_add(y, ff_shfl_xor(y, o));
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  const ff t = red[32];
  __syncthreads();
  return t;
}

// Exclusive prefix sum of value_at(0 .. n-1) into out[0 .. n]; out[n] is the total.  Each
// thread owns a contiguous run; runs are combined by a warp-shuffle scan and a scan over
// the warp totals.
template <int NT, typename F>
__device__ __forceinline__ ff block_exclusive_scan(int n, F value_at, ff* out, ff* red) {
  const int per = (n + NT - 1) / NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int begin = min(tid * per, n), end = min(begin + per, n);
  ff local = ff_of(0.f);
  for (int j = begin; j < end; ++j) local = ff_add(local, value_at(j));
  ff x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const ff y = ff_shfl_up(x, o);
    if (lane >= o) x = ff_add(x, y);
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    ff wv = lane < NT / 32 ? red[lane] : ff_of(0.f);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const ff y = ff_shfl_up(wv, o);
      if (lane >= o) wv = ff_add(wv, y);
    }
    if (lane < NT / 32) red[lane] = wv;
  }
  __syncthreads();
  ff run = ff_sub(x, local);
  if (warp > 0) run = ff_add(run, red[warp - 1]);
  for (int j = begin; j < end; ++j) {
    out[j] = run;
    run = ff_add(run, value_at(j));
  }
  const ff total = red[NT / 32 - 1];
  if (tid == 0) out[n] = total;
  __syncthreads();
  return total;
}

// ------------------------------------------------------------------ terminal values (Stages 2-4)

// One block per (player, terminal node).  q is the opponent's reach at the node, kappa = 1/Z,
// and the node's payoff already carries the probability of the public cards dealt on its
// path, so every value is a counterfactual value in the sense of Eq. (cfv).
//   fold (Stage 3):   v_i(h) = u_i kappa (T - C[c1] - C[c2] + q[h]),  T = sum_o q[o],
//                     C[c] = sum_{o holds c} q[o]  (inclusion-exclusion over the two cards)
//   showdown (Stage 4): v_i(h) = c kappa (W(h) - L(h)), W / L the opponent reach of weaker /
//                     stronger hands that share no card with h, from exclusive prefix sums
//                     over the rank-sorted order minus per-card prefix sums; the tie group
//                     of h is excluded from both (a split pot pays 0).
// Sums and differences are taken in double-float in both precisions.
template <typename P>
__global__ void __launch_bounds__(kTermThreads) k_terminal(const GameDev* __restrict__ games,
                                                            const Work* __restrict__ work, int n_work,
                                                            int player_mask, int use_bar) {
  using V = typename P::V;
  int item = blockIdx.x;
  int i;
  if (player_mask == 3) {
    i = item >= n_work;
    item -= i * n_work;
  } else {
    i = player_mask == 1 ? 0 : 1;
  }
  const Work wk = work[item];
  const GameDev& G = games[wk.game];
  const int n = wk.unit;
  const NodeDev nd = G.nodes[n];
  const int H = G.n_hands;
  const size_t stride = (size_t)G.hstride;
  const V* __restrict__ q =
      static_cast<const V*>(use_bar ? G.reach_bar : G.reach) + ((size_t)(1 - i) * G.n_nodes + n) * stride;
  V* __restrict__ out = static_cast<V*>(use_bar ? G.cfv_br : G.cfv) + ((size_t)i * G.n_nodes + n) * stride;

  extern __shared__ __align__(16) unsigned char smt[];
  __shared__ ff red[33];
  ff* Psc = reinterpret_cast<ff*>(smt);                   // [H + 1]
  ff* CP = Psc + H + 1;                                   // [cl_len + 1]
  V* qs = reinterpret_cast<V*>(CP + G.cl_len + 1);        // [H]
  for (int h = threadIdx.x; h < H; h += kTermThreads) qs[h] = q[h];
  __syncthreads();

  // payoff for player i per unit of (opponent reach) x kappa, formed in FP64 once per block
  const double pay = G.payoff[n];
  const double u64 = (nd.type == kFold ? (nd.player == i ? -pay : pay) : pay) * G.kappa64;
  const ff u = d2ff(u64);
  const int b = nd.type == kShowdown ? nd.row : 0;
  const int32_t* __restrict__ clh = G.cl_hand + (size_t)b * G.cl_len;
  const int32_t* __restrict__ clo = G.cl_off + (size_t)b * (G.deck + 1);
  block_exclusive_scan<kTermThreads>(G.cl_len, [&](int j) { return P::to_ff(qs[clh[j]]); }, CP, red);
  const int k = G.hand_size;
  const uint64_t board = nd.board;

  if (nd.type == kFold) {
    ff loc = ff_of(0.f);
    for (int h = threadIdx.x; h < H; h += kTermThreads) loc = ff_add(loc, P::to_ff(qs[h]));
    const ff T = block_sum_ff<kTermThreads>(loc, red);
    for (int h = threadIdx.x; h < H; h += kTermThreads) {
      ff m = T;
      for (int s = 0; s < k; ++s) {
        const int c = G.hand_cards[2 * h + s];
        m = ff_sub(m, ff_sub(CP[clo[c + 1]], CP[clo[c]]));
      }
      if (k == 2) m = ff_add(m, P::to_ff(qs[h]));
      out[h] = (G.hand_mask[h] & board) ? P::zero() : P::of_ff(ff_mul(u, m));
    }
  } else {
    const int32_t* __restrict__ perm = G.sd_perm + (size_t)b * H;
    const int32_t* __restrict__ gs = G.sd_gs + (size_t)b * H;
    const int32_t* __restrict__ ge = G.sd_ge + (size_t)b * H;
    const int32_t* __restrict__ lo = G.cl_lo + (size_t)b * H * 2;
    const int32_t* __restrict__ hi = G.cl_hi + (size_t)b * H * 2;
    const ff T = block_exclusive_scan<kTermThreads>(H, [&](int j) { return P::to_ff(qs[perm[j]]); }, Psc, red);
    for (int h = threadIdx.x; h < H; h += kTermThreads) {
      ff Wn = Psc[gs[h]];
      ff Ln = ff_sub(T, Psc[ge[h]]);
      for (int s = 0; s < k; ++s) {
        const int c = G.hand_cards[2 * h + s];
        Wn = ff_sub(Wn, ff_sub(CP[lo[2 * h + s]], CP[clo[c]]));
        Ln = ff_sub(Ln, ff_sub(CP[clo[c + 1]], CP[hi[2 * h + s]]));
      }
      out[h] = (G.hand_mask[h] & board) ? P::zero() : P::of_ff(ff_mul(u, ff_sub(Wn, Ln)));
    }
  }
}

// ------------------------------------------------------------------ per-hand passes

struct Discount {
  double dpos, dneg, dS, wS;
};

// One column of a [rows][*] array: shared memory (row stride W, column w) or global
// memory (row stride hstride, column h).
template <typename T>
struct Col {
  T* base;
  size_t rs;
  __device__ __forceinline__ T& operator[](int row) const { return base[(size_t)row * rs]; }
};

// Per-hand tree passes for one chunk of W hands of player p (grid: (player, chunk)).
//   kModeInit:   sigma_p = RM(R_p) (Eq. rm), forward reach of p (Stage 1).
//   kModeUpdate: backward values of p (Stage 6, Eq. backward) from the terminal values,
//                regret and average update (Stage 7), new sigma_p, forward reach of p.
//   kModeAvg:    average strategy S / sum S of p, forward reach of p under it.
//   kModeBR:     best-response backward pass of p (max over p's actions), root sum.
// With G.smem set the block keeps v[n_nodes][W], reach[n_nodes][W], the strategy rows
// [rows_p][W] and (updates) the R and S rows [rows_p][W] of its hands in shared memory;
// otherwise it works on the global arrays directly.
template <int MODE, typename P>
__global__ void __launch_bounds__(kHandThreads) k_hand(const GameDev* __restrict__ games,
                                                       const Work* __restrict__ work, int n_work, int player_mask,
                                                       int advance, int* iter, unsigned* done, int variant,
                                                       double alpha, double beta, double gamma) {
  using V = typename P::V;
  int item = blockIdx.x;
  int p;
  if (player_mask == 3) {
    p = item >= n_work;
    item -= p * n_work;
  } else {
    p = player_mask == 1 ? 0 : 1;
  }
  const Work wk = work[item];
  const GameDev& G = games[wk.game];
  const int W = G.chunk;
  const int w = threadIdx.x % W;
  const int slot = threadIdx.x / W;
  const int nslots = kHandThreads / W;
  const int h = wk.unit * W + w;  // < hstride: hstride is a multiple of 32 and W divides 32
  const bool valid = h < G.n_hands;
  const int N = G.n_nodes;
  const size_t stride = (size_t)G.hstride;
  const int rb = G.row_begin[p], re = G.row_begin[p + 1];
  const int nrows = re - rb;
  const NodeDev* __restrict__ nodes = G.nodes;
  const int32_t* __restrict__ ls = G.level_start;
  const uint64_t hmask = valid ? G.hand_mask[h] : 0ull;
  const bool sm = G.smem != 0;

  // global arrays of this player, at column h
  V* gv = static_cast<V*>(MODE == kModeBR ? G.cfv_br : G.cfv) + (size_t)p * N * stride + h;
  V* grch = static_cast<V*>(MODE == kModeAvg ? G.reach_bar : G.reach) + (size_t)p * N * stride + h;
  V* gsg = static_cast<V*>(MODE == kModeAvg ? G.sigbar : G.sigma) + (size_t)rb * stride + h;
  double* gR = G.R + (size_t)rb * stride + h;
  double* gS = G.S + (size_t)rb * stride + h;

  extern __shared__ __align__(16) unsigned char smraw[];
  const bool stage_rs = sm && MODE == kModeUpdate;
  double* sR = reinterpret_cast<double*>(smraw);                          // [nrows][W]
  double* sS = sR + (stage_rs ? (size_t)nrows * W : 0);                   // [nrows][W]
  V* sv = reinterpret_cast<V*>(sS + (stage_rs ? (size_t)nrows * W : 0));  // [N][W]
  V* srch = sv + (size_t)N * W;                                           // [N][W]
  V* ssg = srch + (size_t)N * W;                                          // [nrows][W]

  const Col<V> v = sm ? Col<V>{sv + w, (size_t)W} : Col<V>{gv, stride};
  const Col<V> rch = sm ? Col<V>{srch + w, (size_t)W} : Col<V>{grch, stride};
  const Col<V> sg = sm ? Col<V>{ssg + w, (size_t)W} : Col<V>{gsg, stride};
  const Col<double> Rc = stage_rs ? Col<double>{sR + w, (size_t)W} : Col<double>{gR, stride};
  const Col<double> Sc = stage_rs ? Col<double>{sS + w, (size_t)W} : Col<double>{gS, stride};
  __shared__ Discount disc;

  if (MODE == kModeUpdate && threadIdx.x == 0) {
    const int t = *iter + 1;
    Discount d{1.0, 1.0, 1.0, 1.0};
    if (variant == 2) {
      const double ta = pow((double)t, alpha), tb = pow((double)t, beta);
      d.dpos = ta / (ta + 1.0);
      d.dneg = tb / (tb + 1.0);
      d.dS = pow((double)t / (double)(t + 1), gamma);
    } else if (variant == 1) {
      d.wS = (double)t;
    }
    disc = d;
  }

  // ---- stage what the pass starts from
  if (sm && (MODE == kModeUpdate || MODE == kModeBR)) {
    for (int n = slot; n < N; n += nslots) {
      const uint8_t ty = nodes[n].type;
      if (ty == kFold || ty == kShowdown) v[n] = gv[(size_t)n * stride];
    }
  }
  if (sm && MODE == kModeUpdate) {
    for (int n = slot; n < N; n += nslots) rch[n] = grch[(size_t)n * stride];
    for (int r = slot; r < nrows; r += nslots) {
      sg[r] = gsg[(size_t)r * stride];
      Rc[r] = gR[(size_t)r * stride];
      Sc[r] = gS[(size_t)r * stride];
    }
  }
  if (MODE == kModeInit || MODE == kModeAvg) {
    // strategy rows of player p: regret matching of R (Eq. rm), or S / sum S
    const double* src = (MODE == kModeInit ? G.R : G.S) + h;
    for (int n = slot; n < N; n += nslots) {
      const NodeDev nd = nodes[n];
      if (nd.type != kDecision || nd.player != p) continue;
      const int A = nd.n_kids;
      V tot = P::zero();
      int npos = 0, last = 0;
      for (int a = 0; a < A; ++a) {
        const double x = src[(size_t)(nd.row + a) * stride];
        const V xv = x > 0.0 ? P::of_double(x) : P::zero();
        if (x > 0.0) ++npos, last = a;
        if (sm || valid) sg[nd.row - rb + a] = xv;
        tot = P::add(tot, xv);
      }
      if (npos == 1) {  // x / x = 1 exactly, as the definition gives
        for (int a = 0; a < A; ++a)
          if (sm || valid) sg[nd.row - rb + a] = a == last ? P::of_double(1.0) : P::zero();
      } else if (P::positive(tot)) {
        const V inv = P::recip(tot);
        for (int a = 0; a < A; ++a)
          if (sm || valid) sg[nd.row - rb + a] = P::mul(sg[nd.row - rb + a], inv);
      } else {
        const V uni = P::of_double(1.0 / A);
        for (int a = 0; a < A; ++a)
          if (sm || valid) sg[nd.row - rb + a] = uni;
      }
    }
  }
  __syncthreads();

  // ---- backward pass (Stage 6) with the Stage 7 update, or the best-response pass
  if (MODE == kModeUpdate || MODE == kModeBR) {
    const Discount d = disc;
    for (int l = G.n_levels - 1; l >= 0; --l) {
      const int a0 = ls[l], cnt = ls[l + 1] - a0;
      for (int idx = slot; idx < cnt; idx += nslots) {
        const int n = a0 + idx;
        const NodeDev nd = nodes[n];
        if (nd.type == kFold || nd.type == kShowdown) continue;
        const int A = nd.n_kids, k0 = nd.first_kid;
        V val = P::zero();
        if (nd.type == kChance) {
          // children values already carry the card probabilities; cards in the hand are out
          for (int a = 0; a < A; ++a) {
            const int card = nodes[k0 + a].deal;
            if (!((hmask >> card) & 1ull)) val = P::add(val, v[k0 + a]);
          }
        } else if (nd.player != p) {
          for (int a = 0; a < A; ++a) val = P::add(val, v[k0 + a]);
        } else if (MODE == kModeBR) {
          val = v[k0];
          for (int a = 1; a < A; ++a) val = P::vmax(val, v[k0 + a]);
        } else {
          const int r0 = nd.row - rb;
          for (int a = 0; a < A; ++a) val = P::add(val, P::mul(sg[r0 + a], v[k0 + a]));
          const V own = rch[n];
          V pos = P::zero();
          int npos = 0, last = 0;
          for (int a = 0; a < A; ++a) {
            const V r = P::sub(v[k0 + a], val);                            // instantaneous regret
            const double contrib = P::to_double(P::mul(own, sg[r0 + a]));  // pi_i(I) sigma(I, a)
            double x = Rc[r0 + a] + P::to_double(r);
            if (variant == 2) x *= x > 0.0 ? d.dpos : d.dneg;
            if (variant == 1 && x < 0.0) x = 0.0;
            const double s = fma(Sc[r0 + a], d.dS, d.wS * contrib);
            const V xv = x > 0.0 ? P::of_double(x) : P::zero();  // positive part of the new R
            if (x > 0.0) ++npos, last = a;
            if (sm || valid) {
              Rc[r0 + a] = x;
              Sc[r0 + a] = s;
              sg[r0 + a] = xv;
            }
            pos = P::add(pos, xv);
          }
          // regret matching of the updated R (Eq. rm); sg holds its positive part
          if (npos == 1) {  // x / x = 1 exactly, as the definition gives
            for (int a = 0; a < A; ++a)
              if (sm || valid) sg[r0 + a] = a == last ? P::of_double(1.0) : P::zero();
          } else if (P::positive(pos)) {
            const V inv = P::recip(pos);
            for (int a = 0; a < A; ++a)
              if (sm || valid) sg[r0 + a] = P::mul(sg[r0 + a], inv);
          } else {
            const V uni = P::of_double(1.0 / A);
            for (int a = 0; a < A; ++a)
              if (sm || valid) sg[r0 + a] = uni;
          }
        }
        if (sm || valid) v[n] = val;
      }
      __syncthreads();
    }
    if (sm && valid)
      for (int n = slot; n < N; n += nslots) gv[(size_t)n * stride] = v[n];
    if (MODE == kModeBR) {
      if (threadIdx.x == 0) {
        double acc = 0.0;
        const double* r64 = G.range64 + (size_t)p * stride;
        const V* root = static_cast<const V*>(G.cfv_br) + (size_t)p * N * stride;
        for (int j = 0; j < W; ++j) {
          const int hh = wk.unit * W + j;
          if (hh < G.n_hands) acc += r64[hh] * P::to_double(sm ? sv[j] : root[hh]);
        }
        G.br_partial[(size_t)p * G.n_chunks + wk.unit] = acc;
      }
      return;
    }
    if (sm && valid)
      for (int r = slot; r < nrows; r += nslots) {
        gR[(size_t)r * stride] = Rc[r];
        gS[(size_t)r * stride] = Sc[r];
      }
  }

  // ---- forward reach of player p (Stages 1-2) under the strategy in sg
  {
    if (slot == 0) {
      const V r0 = valid ? static_cast<const V*>(G.range_v)[(size_t)p * stride + h] : P::zero();
      if (sm || valid) rch[0] = r0;
    }
    __syncthreads();
    for (int l = 1; l < G.n_levels; ++l) {
      const int a0 = ls[l], cnt = ls[l + 1] - a0;
      for (int idx = slot; idx < cnt; idx += nslots) {
        const int n = a0 + idx;
        const NodeDev nd = nodes[n];
        const NodeDev par = nodes[nd.parent];
        V x = (sm || valid) ? rch[nd.parent] : P::zero();
        if (par.type == kDecision && par.player == p) x = P::mul(x, sg[par.row - rb + nd.paction]);
        if (par.type == kChance && ((hmask >> nd.deal) & 1ull)) x = P::zero();
        if (sm || valid) rch[n] = x;
      }
      __syncthreads();
    }
    if (sm && valid) {
      for (int n = slot; n < N; n += nslots) grch[(size_t)n * stride] = rch[n];
      for (int r = slot; r < nrows; r += nslots) gsg[(size_t)r * stride] = sg[r];
    }
  }

  if (MODE == kModeUpdate && advance) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(done, 1u);
      if (prev == gridDim.x - 1) {  // last block of the launch: every block has read *iter
        *done = 0u;
        *iter += 1;
        __threadfence();
      }
    }
  }
}

// FP64 sum of the per-chunk best-response partials: one block per game, fixed order.
__global__ void k_br_reduce(const GameDev* __restrict__ games) {
  const GameDev& G = games[blockIdx.x];
  if (threadIdx.x < 2) {
    const int p = threadIdx.x;
    double acc = 0.0;
    for (int c = 0; c < G.n_chunks; ++c) acc += G.br_partial[(size_t)p * G.n_chunks + c];
    G.br_out[p] = acc;
  }
}

// Average strategy S / sum S of every decision node of every game (for read-back).
template <typename P>
__global__ void k_average_rows(const GameDev* __restrict__ games, int n_games) {
  using V = typename P::V;
  for (int g = 0; g < n_games; ++g) {
    const GameDev& G = games[g];
    const size_t stride = (size_t)G.hstride;
    const int total = G.n_nodes * G.n_hands;
    V* out = static_cast<V*>(G.sigbar);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
      const int n = e / G.n_hands, h = e - n * G.n_hands;
      const NodeDev nd = G.nodes[n];
      if (nd.type != kDecision) continue;
      double tot = 0.0;
      for (int a = 0; a < nd.n_kids; ++a) tot += G.S[(size_t)(nd.row + a) * stride + h];
      for (int a = 0; a < nd.n_kids; ++a)
        out[(size_t)(nd.row + a) * stride + h] =
            P::of_double(tot > 0.0 ? G.S[(size_t)(nd.row + a) * stride + h] / tot : 1.0 / nd.n_kids);
    }
  }
}

// ------------------------------------------------------------------ launchers

static int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of %s failed: %s\n", what, cudaGetErrorString(e));
    return -1;
  }
  return 0;
}

int hand_kernel_smem_limit() { return 227 * 1024; }

template <typename P>
static cudaError_t configure_precision() {
  const int smem = hand_kernel_smem_limit() - 1024;
  cudaError_t e = cudaFuncSetAttribute(k_hand<kModeInit, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hand<kModeUpdate, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hand<kModeAvg, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hand<kModeBR, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_terminal<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

int configure_kernels() {
  cudaError_t e = configure_precision<Pairs>();
  if (e == cudaSuccess) e = configure_precision<Single>();
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: kernel attribute setup failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return 0;
}

template <int MODE, typename P>
static int launch_hand_p(const LaunchCtx& c, int player_mask, int advance, void* stream) {
  const int players = player_mask == 3 ? 2 : 1;
  k_hand<MODE, P><<<c.n_chunk_work * players, kHandThreads, c.smem_hand, (cudaStream_t)stream>>>(
      c.games, c.chunk_work, c.n_chunk_work, player_mask, advance, c.iter, c.done, c.variant, c.alpha, c.beta,
      c.gamma);
  return check_launch("k_hand");
}

template <int MODE>
static int launch_hand(const LaunchCtx& c, int player_mask, int advance, void* stream) {
  return c.precision == kPrecisionSingle ? launch_hand_p<MODE, Single>(c, player_mask, advance, stream)
                                         : launch_hand_p<MODE, Pairs>(c, player_mask, advance, stream);
}

int launch_init(const LaunchCtx& c, void* stream) { return launch_hand<kModeInit>(c, 3, 0, stream); }
int launch_update(const LaunchCtx& c, int player_mask, int advance, void* stream) {
  return launch_hand<kModeUpdate>(c, player_mask, advance, stream);
}
int launch_avg_reach(const LaunchCtx& c, void* stream) { return launch_hand<kModeAvg>(c, 3, 0, stream); }
int launch_br(const LaunchCtx& c, void* stream) { return launch_hand<kModeBR>(c, 3, 0, stream); }

int launch_terminal(const LaunchCtx& c, int player_mask, int use_bar, void* stream) {
  if (c.n_term_work == 0) return 0;
  const int players = player_mask == 3 ? 2 : 1;
  if (c.precision == kPrecisionSingle)
    k_terminal<Single><<<c.n_term_work * players, kTermThreads, c.smem_term, (cudaStream_t)stream>>>(
        c.games, c.term_work, c.n_term_work, player_mask, use_bar);
  else
    k_terminal<Pairs><<<c.n_term_work * players, kTermThreads, c.smem_term, (cudaStream_t)stream>>>(
        c.games, c.term_work, c.n_term_work, player_mask, use_bar);
  return check_launch("k_terminal");
}

int launch_br_reduce(const LaunchCtx& c, void* stream) {
  k_br_reduce<<<c.n_games, 32, 0, (cudaStream_t)stream>>>(c.games);
  return check_launch("k_br_reduce");
}

int launch_average_rows(const LaunchCtx& c, void* stream) {
  if (c.precision == kPrecisionSingle)
    k_average_rows<Single><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  else
    k_average_rows<Pairs><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  return check_launch("k_average_rows");
}

}  // namespace pcfr
