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
// a CUDA graph.  Inside k_hand the FP64 regret / average update is one fully parallel pass
// over (row, hand) items after the backward levels, so GB300's long FP64 latency is paid
// once per launch rather than once per tree level.
//
// Precision: cumulative regrets R and average sums S are FP64 (GB300 runs FP64 at about
// 1/64 of the FP32 rate, so FP64 is kept to those updates).  Reach, strategies and values
// are either double-float pairs on the FP32 pipe (Pairs, the default: ~44-bit
// significands, so regrets that are small differences of large values keep their digits)
// or plain FP32 (Single).
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>

#include "pcfr_internal.h"

namespace pcfr {

constexpr int kHandThreads = 256;
constexpr int kTermThreads = 512;


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
// Sum of two double-floats of the same sign (no cancellation possible): TwoSum of the high
// parts, low parts added in FP32, one renormalisation -- about half the operations of ff_add.
__device__ __forceinline__ ff ff_add_pos(ff a, ff b) {
  float s, e, hi, lo;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  fast_two_sum(s, e, hi, lo);
  return {hi, lo};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float hi, lo;
  fast_two_sum(p, e, hi, lo);
  return {hi, lo};
}
// Compensated accumulation (Ogita, Rump and Oishi 2005, "Accurate sum and dot product",
// Sum2 / Dot2): a running FP32 sum s, with every rounding error -- found exactly by TwoSum
// and by the FMA form of TwoProduct -- added into a separate FP32 error sum e.  The
// critical path is one FP32 addition per term, and s + e, kept as a pair, carries about
// twice the working precision.
struct acc2 {
  float s, e;
};
__device__ __forceinline__ acc2 acc_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ void acc_add(acc2& a, ff x) {
  float t, err;
  two_sum(a.s, x.hi, t, err);
  a.s = t;
  a.e = __fadd_rn(a.e, __fadd_rn(err, x.lo));
}
__device__ __forceinline__ void acc_fma(acc2& a, ff x, ff y) {  // a += x * y
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = __fmaf_rn(x.hi, y.hi, -p);
  const float cross = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  float t, err;
  two_sum(a.s, p, t, err);
  a.s = t;
  a.e = __fadd_rn(a.e, __fadd_rn(err, __fadd_rn(pe, cross)));
}
__device__ __forceinline__ void acc_merge(acc2& a, acc2 b) {
  float t, err;
  two_sum(a.s, b.s, t, err);
  a.s = t;
  a.e = __fadd_rn(a.e, __fadd_rn(err, b.e));
}
__device__ __forceinline__ ff acc_value(acc2 a) {
  float hi, lo;
  two_sum(a.s, a.e, hi, lo);
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
  static __device__ __forceinline__ V one() { return ff_of(1.f); }
  static __device__ __forceinline__ V uniform(int A) { return ff_recip(ff_of((float)A)); }  // 1 / A
  static __device__ __forceinline__ V of_double(double x) { return d2ff(x); }
  static __device__ __forceinline__ double to_double(V a) { return ff2d(a); }
  static __device__ __forceinline__ ff to_ff(V a) { return a; }
  static __device__ __forceinline__ V of_ff(ff a) { return a; }
  using Acc = acc2;
  static __device__ __forceinline__ Acc acc0() { return acc_zero(); }
  static __device__ __forceinline__ void acc(Acc& a, V x) { acc_add(a, x); }
  static __device__ __forceinline__ void acc_mul(Acc& a, V x, V y) { acc_fma(a, x, y); }
  static __device__ __forceinline__ V value(Acc a) { return acc_value(a); }
};

struct Single {  // plain FP32 values
  using V = float;
  static __device__ __forceinline__ V zero() { return 0.f; }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ V vmax(V a, V b) { return fmaxf(a, b); }
  static __device__ __forceinline__ bool positive(V a) { return a > 0.f; }
  // correctly rounded reciprocal: the same bits as 1 / a in IEEE division
  static __device__ __forceinline__ V recip(V a) { return __frcp_rn(a); }
  static __device__ __forceinline__ V one() { return 1.f; }
  static __device__ __forceinline__ V uniform(int A) { return __frcp_rn((float)A); }
  static __device__ __forceinline__ V of_double(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double to_double(V a) { return f2d(a); }
  static __device__ __forceinline__ ff to_ff(V a) { return ff_of(a); }
  static __device__ __forceinline__ V of_ff(ff a) { return ff_round(a); }
  using Acc = float;
  static __device__ __forceinline__ Acc acc0() { return 0.f; }
  static __device__ __forceinline__ void acc(Acc& a, V x) { a = __fadd_rn(a, x); }
  static __device__ __forceinline__ void acc_mul(Acc& a, V x, V y) { a = fmaf(x, y, a); }
  static __device__ __forceinline__ V value(Acc a) { return a; }
};

// ------------------------------------------------------------------ block primitives (double-float)

__device__ __forceinline__ acc2 acc_shfl_up(acc2 a, int o) {
  return {__shfl_up_sync(0xffffffffu, a.s, o), __shfl_up_sync(0xffffffffu, a.e, o)};
}

// Exclusive prefix sum of the non-negative values value_at(0 .. n-1) into out[0 .. n]
// (out[n] = total) by one group of GT consecutive threads (gtid = rank in the group; every
// thread of the block must call it, so that the block barriers inside line up).  Each
// thread owns a contiguous run; runs are combined by a warp-shuffle scan and a scan over the
// group's warp totals in red[GT / 32].  Sums are compensated (acc2).
template <int GT, typename F>
__device__ __forceinline__ ff group_exclusive_scan(int n, F value_at, ff* out, acc2* red, int gtid) {
  const int per = (n + GT - 1) / GT;
  const int lane = gtid & 31, warp = gtid >> 5;
  const int begin = min(gtid * per, n), end = min(begin + per, n);
  acc2 local = acc_zero();
  for (int j = begin; j < end; ++j) acc_add(local, value_at(j));
  acc2 x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const acc2 y = acc_shfl_up(x, o);
    if (lane >= o) acc_merge(x, y);
  }
  acc2 run = acc_shfl_up(x, 1);
  if (lane == 0) run = acc_zero();
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    acc2 wv = lane < GT / 32 ? red[lane] : acc_zero();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const acc2 y = acc_shfl_up(wv, o);
      if (lane >= o) acc_merge(wv, y);
    }
    if (lane < GT / 32) red[lane] = wv;
  }
  __syncthreads();
  if (warp > 0) acc_merge(run, red[warp - 1]);
  for (int j = begin; j < end; ++j) {  // value read before out[j] is written: out may be the input
    const ff v = value_at(j);
    out[j] = acc_value(run);
    acc_add(run, v);
  }
  const ff total = acc_value(red[GT / 32 - 1]);
  if (gtid == 0) out[n] = total;
  __syncthreads();
  return total;
}

// The same exclusive prefix sum in plain FP32 (values of the single-precision path; the
// error of a prefix stays within a few dozen ulps of the total).
template <int GT, typename F>
__device__ __forceinline__ float group_exclusive_scan_f32(int n, F value_at, float* out, float* red, int gtid) {
  const int per = (n + GT - 1) / GT;
  const int lane = gtid & 31, warp = gtid >> 5;
  const int begin = min(gtid * per, n), end = min(begin + per, n);
  float local = 0.f;
  for (int j = begin; j < end; ++j) local = __fadd_rn(local, value_at(j));
  float x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = __fadd_rn(x, y);
  }
  float run = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) run = 0.f;
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    float wv = lane < GT / 32 ? red[lane] : 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, wv, o);
      if (lane >= o) wv = __fadd_rn(wv, y);
    }
    if (lane < GT / 32) red[lane] = wv;
  }
  __syncthreads();
  if (warp > 0) run = __fadd_rn(run, red[warp - 1]);
  for (int j = begin; j < end; ++j) {  // value read before out[j] is written: out may be the input
    const float v = value_at(j);
    out[j] = run;
    run = __fadd_rn(run, v);
  }
  const float total = red[GT / 32 - 1];
  if (gtid == 0) out[n] = total;
  __syncthreads();
  return total;
}

// ------------------------------------------------------------------ bulk copies (TMA) into shared memory

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make the barrier's initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// One-dimensional bulk copy global -> shared; both addresses and the size are multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Asynchronous element copies global -> shared (cp.async): every copy of a block is in
// flight at once instead of one load-then-store round trip per loop iteration.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Programmatic dependent launch.  Every kernel first stages what launches two or more steps
// back produced, then waits for its immediate predecessor (griddepcontrol.wait returns once
// that grid has completed and its writes are visible), and only then lets its own dependent
// start.  So whenever a kernel is running, everything but its immediate predecessor has
// completed, which is what makes the early staging safe.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bounded wait for phase `parity` of the barrier: false if it did not complete within
// `limit` polls.
constexpr long kWaitLimit = 1l << 20;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long limit = kWaitLimit) {
  for (long k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Polls the terminal kernel's first bulk-copy wait of each block makes before it gives up:
// kWaitLimit, unless a test lowers it to exercise the timeout path (with 0 the block gives
// up before its copies can land, drains them with the full limit, sets the error flag and
// returns).  Every other wait keeps kWaitLimit.
__device__ long g_first_wait_polls = kWaitLimit;

// ------------------------------------------------------------------ terminal values (Stages 2-4)

// Whether hand h (its cards from the staged table: c1 | c2 << 8) holds a card of `board`.
__device__ __forceinline__ bool holds_board_card(const uint16_t* cards, int h, int k, uint64_t board) {
  const unsigned cw = cards[h];
  return (((board >> (cw & 0xffu)) | (k == 2 ? board >> (cw >> 8) : 0ull)) & 1ull) != 0;
}

// Values of player i at one fold or showdown node n (Stages 2-4), the opponent's reach q
// at n already in shared memory.  kappa = 1/Z, and the node's payoff already carries the
// probability of the public cards dealt on its path, so every value is a counterfactual
// value in the sense of Eq. (cfv).
//   fold (Stage 3):   v_i(h) = u_i kappa (T - C[c1] - C[c2] + q[h]),  T = sum_o q[o],
//                     C[c] = sum_{o holds c} q[o]  (inclusion-exclusion over the two cards)
//   showdown (Stage 4): v_i(h) = c kappa (W(h) - L(h)), W / L the opponent reach of weaker /
//                     stronger hands that share no card with h, from exclusive prefix sums
//                     over the rank-sorted order minus per-card prefix sums; the tie group
//                     of h is excluded from both (a split pot pays 0).
// Sums and differences are double-float with FP32-pair values, plain FP32 with FP32
// values.  Every thread of the block calls it (it holds block barriers).
template <typename P>
__device__ __forceinline__ void terminal_values(const GameDev& G, const NodeDev& nd, int i, ff u,
                                                const TermTab& tt, const uint16_t* tab,
                                                const typename P::V* __restrict__ qs, ff* CP, ff* Psc,
                                                typename P::V* __restrict__ out) {
  using V = typename P::V;
  __shared__ acc2 red[2][kTermThreads / 64];
  const float uf = u.hi;  // FP32 values: the scale rounded once to FP32
  const int H = G.n_hands, k = G.hand_size;
  const bool show = nd.type == kShowdown;
  const uint64_t board = nd.board;
  const uint16_t* clh = tab + tt.clh;
  const uint16_t* cards = tab + tt.cards;
  const uint16_t* cloff = tab + tt.cloff;
  const uint16_t* perm = tab + tt.perm;
  if constexpr (std::is_same<P, Single>::value) {
    if (!show) {
      // fold (FP32 values): no prefix sums needed.  T: warp 0 keeps 32 lane-strided partial
      // sums of q and combines them by a fixed xor tree (lane 0's result); C[c]: one thread
      // per card sums card c's list in list order.  Few warps work and the others wait at
      // one barrier, which the other blocks on the SM fill.
      __shared__ float Cs[kMaxDeck];
      __shared__ float Tsh;
      const int lane = threadIdx.x & 31;
      if (threadIdx.x < 32) {
        float t = 0.f;
#pragma unroll 8
        for (int h = lane; h < H; h += 32) t = __fadd_rn(t, qs[h]);
        for (int o = 16; o > 0; o >>= 1) t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) Tsh = t;
      } else if (threadIdx.x - 32 < G.deck) {
        const int c = threadIdx.x - 32;
        float x = 0.f;
#pragma unroll 4
        for (int j = cloff[c]; j < cloff[c + 1]; ++j) x = __fadd_rn(x, qs[clh[j]]);
        Cs[c] = x;
      }
      __syncthreads();
      const float T = Tsh;
      for (int h = threadIdx.x; h < H; h += kTermThreads) {
        const unsigned cw = cards[h];
        const unsigned c1 = cw & 0xffu, c2 = cw >> 8;
        float m = __fsub_rn(T, Cs[c1]);
        bool blocked = (board >> c1) & 1ull;
        if (k == 2) {
          m = __fadd_rn(__fsub_rn(m, Cs[c2]), qs[h]);
          blocked = blocked || ((board >> c2) & 1ull);
        }
        out[h] = blocked ? 0.f : __fmul_rn(uf, m);
      }
      __syncthreads();  // Cs and Tsh are reused by the next node
      return;
    }
    // FP32 values: the same scans and differences in plain FP32 (a value's error stays
    // within about 1e-6 of the largest value at the node)
    __shared__ float redf[2][kTermThreads / 32];
    __shared__ float cps[kMaxDeck], cpe[kMaxDeck];  // prefix at the start / end of each card's list
    float* CPf = reinterpret_cast<float*>(CP);  // [k H + 1]
    float* Pf = CPf + (k * H + 1);             // [H + 1]
    {  // the reach in rank order and along the card lists, gathered once into the scans'
       // output arrays (lanes on consecutive entries), then scanned in place, each thread
       // over a contiguous run: the same sums as scanning the gathers directly, with half
       // the random shared-memory reads.  Two-card hands' card lists hold 2 H entries, so 11
       // warps scan them and 5 the H rank-ordered entries (about 7 per thread on both sides).
      for (int j = threadIdx.x; j < H; j += kTermThreads) Pf[j] = qs[show ? perm[j] : j];
      for (int j = threadIdx.x; j < k * H; j += kTermThreads) CPf[j] = qs[clh[j]];
      __syncthreads();
      constexpr int gp = 5 * 32;
      if (threadIdx.x < gp)
        group_exclusive_scan_f32<gp>(H, [&](int j) { return Pf[j]; }, Pf, redf[0], threadIdx.x);
      else
        group_exclusive_scan_f32<kTermThreads - gp>(k * H, [&](int j) { return CPf[j]; }, CPf, redf[1],
                                                     threadIdx.x - gp);
    }
    for (int c = threadIdx.x; c < G.deck; c += kTermThreads) {
      cps[c] = CPf[cloff[c]];
      cpe[c] = CPf[cloff[c + 1]];
    }
    __syncthreads();
    const float T = Pf[H];
    if (!show) {
      for (int h = threadIdx.x; h < H; h += kTermThreads) {
        const unsigned cw = cards[h];
        const unsigned c1 = cw & 0xffu, c2 = cw >> 8;
        float m = __fsub_rn(T, __fsub_rn(CPf[cloff[c1 + 1]], CPf[cloff[c1]]));
        bool blocked = (board >> c1) & 1ull;
        if (k == 2) {
          m = __fsub_rn(m, __fsub_rn(CPf[cloff[c2 + 1]], CPf[cloff[c2]]));
          m = __fadd_rn(m, qs[h]);
          blocked = blocked || ((board >> c2) & 1ull);
        }
        out[h] = blocked ? 0.f : __fmul_rn(uf, m);
      }
    } else {
      const uint16_t* gs = tab + tt.gs;
      const uint16_t* ge = tab + tt.ge;
      const uint16_t* lo = tab + tt.lo;
      const uint16_t* hi = tab + tt.hi;
      if (k == 2) {  // the same differences, card 1 then card 2, in straight-line code
        for (int h = threadIdx.x; h < H; h += kTermThreads) {
          const unsigned cw = cards[h];
          const unsigned c1 = cw & 0xffu, c2 = cw >> 8;
          float Wn = Pf[gs[h]];
          float Ln = __fsub_rn(T, Pf[ge[h]]);
          Wn = __fsub_rn(Wn, __fsub_rn(CPf[lo[2 * h]], cps[c1]));
          Ln = __fsub_rn(Ln, __fsub_rn(cpe[c1], CPf[hi[2 * h]]));
          Wn = __fsub_rn(Wn, __fsub_rn(CPf[lo[2 * h + 1]], cps[c2]));
          Ln = __fsub_rn(Ln, __fsub_rn(cpe[c2], CPf[hi[2 * h + 1]]));
          const bool blocked = ((board >> c1) | (board >> c2)) & 1ull;
          out[h] = blocked ? 0.f : __fmul_rn(uf, __fsub_rn(Wn, Ln));
        }
      } else {  // one-card hands (Kuhn, Leduc)
        for (int h = threadIdx.x; h < H; h += kTermThreads) {
          const unsigned c = cards[h] & 0xffu;
          const float Wn = __fsub_rn(Pf[gs[h]], __fsub_rn(CPf[lo[2 * h]], cps[c]));
          const float Ln = __fsub_rn(__fsub_rn(T, Pf[ge[h]]), __fsub_rn(cpe[c], CPf[hi[2 * h]]));
          out[h] = ((board >> c) & 1ull) ? 0.f : __fmul_rn(uf, __fsub_rn(Wn, Ln));
        }
      }
    }
    return;
  }
  // Two scans at once, one per half of the block: the first half takes the reach in
  // rank-sorted order (showdown) or in hand order (fold, for the total T), the second half
  // the reach along the per-card hand lists.
  {  // each scan's values gathered once into its output array, then scanned in place
    for (int j = threadIdx.x; j < H; j += kTermThreads) Psc[j] = P::to_ff(qs[show ? perm[j] : j]);
    for (int j = threadIdx.x; j < k * H; j += kTermThreads) CP[j] = P::to_ff(qs[clh[j]]);
    __syncthreads();
    constexpr int half = kTermThreads / 2;
    const bool first = threadIdx.x < half;
    const int gtid = first ? threadIdx.x : threadIdx.x - half;
    if (first)
      group_exclusive_scan<half>(H, [&](int j) { return Psc[j]; }, Psc, red[0], gtid);
    else
      group_exclusive_scan<half>(k * H, [&](int j) { return CP[j]; }, CP, red[1], gtid);
  }
  const ff T = Psc[H];

  if (!show) {
    for (int h = threadIdx.x; h < H; h += kTermThreads) {
      const unsigned cw = cards[h];
      const unsigned c1 = cw & 0xffu, c2 = cw >> 8;
      ff m = ff_sub(T, ff_sub(CP[cloff[c1 + 1]], CP[cloff[c1]]));
      bool blocked = (board >> c1) & 1ull;
      if (k == 2) {
        m = ff_sub(m, ff_sub(CP[cloff[c2 + 1]], CP[cloff[c2]]));
        m = ff_add(m, P::to_ff(qs[h]));
        blocked = blocked || ((board >> c2) & 1ull);
      }
      out[h] = blocked ? P::zero() : P::of_ff(ff_mul(u, m));
    }
  } else {
    const uint16_t* gs = tab + tt.gs;
    const uint16_t* ge = tab + tt.ge;
    const uint16_t* lo = tab + tt.lo;
    const uint16_t* hi = tab + tt.hi;
    for (int h = threadIdx.x; h < H; h += kTermThreads) {
      const unsigned cw = cards[h];
      ff Wn = Psc[gs[h]];
      ff Ln = ff_sub(T, Psc[ge[h]]);
      bool blocked = false;
      for (int s = 0; s < k; ++s) {
        const unsigned c = s == 0 ? (cw & 0xffu) : (cw >> 8);
        Wn = ff_sub(Wn, ff_sub(CP[lo[2 * h + s]], CP[cloff[c]]));
        Ln = ff_sub(Ln, ff_sub(CP[cloff[c + 1]], CP[hi[2 * h + s]]));
        blocked = blocked || ((board >> c) & 1ull);
      }
      out[h] = blocked ? P::zero() : P::of_ff(ff_mul(u, ff_sub(Wn, Ln)));
    }
  }
}

// Terminal values (Stages 2-4).  One block per (player, run): a run is up to eight fold or
// showdown nodes of one game that read the same board table, which is staged once by a
// bulk (TMA) copy; the opponent reach rows of the run's nodes arrive by bulk copies into
// two alternating buffers, each node's row landing while the node before it computes.  A
// showdown below an all-in run-out reads the run-out's reach row (src) and zeroes the hands
// holding a dealt card itself (nobody acts below the run-out, so that is its reach).
// Every wait is bounded: on a timeout the block sets *err, lets its copies drain and leaves.
// RUNS = false is the one-node form (latency: all registers it wants); RUNS = true fits four
// blocks per SM for handles whose terminal nodes fill the GPU many times over.
template <typename P, bool RUNS>
__global__ void __launch_bounds__(kTermThreads, RUNS ? 4 : 1) k_terminal(const GameDev* __restrict__ games,
                                                            const Work* __restrict__ work,
                                                            const int32_t* __restrict__ src,
                                                            const Work* __restrict__ runs, int n_runs,
                                                            int player_mask, int use_bar, int* err) {
  using V = typename P::V;
  int item = blockIdx.x;
  int i;
  if (player_mask == 3) {
    i = item >= n_runs;
    item -= i * n_runs;
  } else {
    i = player_mask == 1 ? 0 : 1;
  }
  const Work run = runs[item];  // (first entry of `work`, count)
  const int first = run.game, count = RUNS ? run.unit : 1;
  const GameDev& G = games[work[first].game];
  const int H = G.n_hands, k = G.hand_size;
  const size_t stride = (size_t)G.hstride;
  const TermTab tt(H, k, G.deck);
  bool show_any = false;
  int b = 0;
  for (int j = 0; j < count; ++j) {
    const NodeDev nd = G.nodes[work[first + j].unit];
    if (nd.type == kShowdown) show_any = true, b = nd.row;
  }
  const unsigned tab_bytes = (unsigned)(show_any ? tt.len : tt.fold_len) * 2u;
  const unsigned q_bytes = (unsigned)(stride * sizeof(V));
  const V* qsrc = static_cast<const V*>(use_bar ? G.reach_bar : G.reach) + (size_t)(1 - i) * G.n_nodes * stride;
  V* dst = static_cast<V*>(use_bar ? G.cfv_br : G.cfv) + (size_t)i * G.n_nodes * stride;

  extern __shared__ __align__(128) unsigned char smt[];
  __shared__ __align__(8) uint64_t bar[2];
  uint16_t* tab = reinterpret_cast<uint16_t*>(smt);                                // [tt.len]
  V* qbuf = reinterpret_cast<V*>(smt + (size_t)tt.len * 2);                         // [2][hstride]
  ff* CP = reinterpret_cast<ff*>(smt + (size_t)tt.len * 2 + 2 * (size_t)q_bytes);   // [k H + 1]
  ff* Psc = CP + (k * H + 1);                                                       // [H + 1]

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the board tables are static: copy them before waiting
    mbar_arrive_expect_tx(&bar[0], tab_bytes + q_bytes);
    bulk_copy_g2s(tab, G.term_tab + (size_t)b * tt.len, tab_bytes, &bar[0]);
  }
  pdl_wait();  // the reach rows come from the launch just before this one
  pdl_trigger();
  if (threadIdx.x == 0) {
    bulk_copy_g2s(qbuf, qsrc + (size_t)src[first] * stride, q_bytes, &bar[0]);
    if (RUNS && count > 1) {
      mbar_arrive_expect_tx(&bar[1], q_bytes);
      bulk_copy_g2s(qbuf + stride, qsrc + (size_t)src[first + 1] * stride, q_bytes, &bar[1]);
    }
  }
  for (int j = 0; j < count; ++j) {
    const int n = work[first + j].unit;
    const NodeDev nd = G.nodes[n];
    // payoff for player i per unit of (opponent reach) x kappa: the FP64 product as a pair of
    // FP32 rounded once on the host (FP32 values use its high part): no FP64 work per thread
    const bool neg = nd.type == kFold && nd.player == i;
    const ff u = {neg ? -G.payoff_ff[2 * n] : G.payoff_ff[2 * n], neg ? -G.payoff_ff[2 * n + 1] : G.payoff_ff[2 * n + 1]};
    const bool ok = threadIdx.x >= 32 ||  // one warp polls
                    mbar_wait_bounded(&bar[j & 1], (j >> 1) & 1, j == 0 ? g_first_wait_polls : kWaitLimit);
    if (__syncthreads_or(!ok)) {  // a copy did not land: report, let the copies drain, leave
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait_bounded(&bar[j & 1], (j >> 1) & 1);
        if (j + 1 < count) mbar_wait_bounded(&bar[(j + 1) & 1], ((j + 1) >> 1) & 1);
      }
      __syncthreads();
      return;
    }
    if (src[first + j] != n) {  // below an all-in run-out: the run-out's reach, without the
      V* qb = qbuf + (size_t)(j & 1) * stride;  // hands holding a card dealt on the way
      for (int h = threadIdx.x; h < H; h += blockDim.x)
        if (holds_board_card(tab + tt.cards, h, k, nd.board)) qb[h] = P::zero();
      __syncthreads();
    }
    terminal_values<P>(G, nd, i, u, tt, tab, qbuf + (size_t)(j & 1) * stride, CP, Psc, dst + (size_t)n * stride);
    if (!RUNS) break;
    __syncthreads();  // buffer j & 1 and the scan arrays are free again
    if (threadIdx.x == 0 && j + 2 < count) {
      mbar_arrive_expect_tx(&bar[j & 1], q_bytes);
      bulk_copy_g2s(qbuf + (size_t)(j & 1) * stride, qsrc + (size_t)src[first + j + 2] * stride, q_bytes,
                    &bar[j & 1]);
    }
  }
}

// ------------------------------------------------------------------ per-hand passes

// One column of a [rows][*] array: shared memory (row stride W, column w) or global
// memory (row stride hstride, column h).
template <typename T>
struct Col {
  T* base;
  size_t rs;
  __device__ __forceinline__ T& operator[](int row) const { return base[(size_t)row * rs]; }
};

__host__ __device__ inline size_t round16(size_t x) { return (x + 15) / 16 * 16; }

// Shared memory of the per-hand kernel for one game (must match the layout in k_hand):
// nodes, level offsets, row -> node map, decision-node list (fewer entries than rows), R and
// S rows, then values, reach and strategy.
__host__ __device__ inline size_t hand_smem_bytes(int n_nodes, int n_levels, int rows_max, int W, size_t es) {
  return round16((size_t)n_nodes * sizeof(NodeDev)) + round16((size_t)(n_levels + 1) * 4) +
         2 * round16((size_t)rows_max * 4) + 2 * round16((size_t)rows_max * W * 8) +
         (size_t)(2 * n_nodes + rows_max) * W * es;
}

// The per-hand passes of one chunk of W hands of player p, on whichever arrays hold the
// chunk's columns (shared memory, or the global arrays at column h).  Each node and each row
// is computed by one thread in a fixed order, so the result does not depend on how many
// threads share the work (slot / nslots): the level and resident schedules give the same bits.
template <typename P>
struct HandView {
  const NodeDev* nodes;
  const int* ls;      // level offsets [L + 1]
  const int* rown;    // node of each row of p
  const int* decs;    // decision nodes of p
  int L, ndec, nrows, rb, p;
  int slot, nslots;   // this thread's slot and the block's slot count
  bool valid;         // a real hand (h < n_hands)
  bool wr;            // this lane may write its column of the working arrays
  uint64_t hmask;     // cards of the hand
  Col<typename P::V> v, rch, sg;
  Col<double> Rc, Sc;
};

// Value of one inner node from its children's stored values (Stage 6, Eq. backward);
// MODE = kModeBR takes the max over p's actions (best response).
template <int MODE, typename P>
__device__ __forceinline__ typename P::V node_value(const HandView<P>& hv, const NodeDev& nd) {
  using V = typename P::V;
  const int A = nd.n_kids, k0 = nd.first_kid;
  if (MODE == kModeBR && nd.type == kDecision && nd.player == hv.p) {
    V val = hv.v[k0];
    for (int a = 1; a < A; ++a) val = P::vmax(val, hv.v[k0 + a]);
    return val;
  }
  typename P::Acc acc = P::acc0();
  if (nd.type == kChance) {
    // children values already carry the card probabilities; cards in the hand are out
    for (int a = 0; a < A; ++a)
      if (!((hv.hmask >> hv.nodes[k0 + a].deal) & 1ull)) P::acc(acc, hv.v[k0 + a]);
  } else if (nd.player != hv.p) {
#pragma unroll 4  // the children's loads go out together; the sum keeps its order
    for (int a = 0; a < A; ++a) P::acc(acc, hv.v[k0 + a]);
  } else {
    const int r0 = nd.row - hv.rb;
#pragma unroll 4
    for (int a = 0; a < A; ++a) P::acc_mul(acc, hv.sg[r0 + a], hv.v[k0 + a]);
  }
  return P::value(acc);
}

// Backward values (Stage 6, Eq. backward), level by level from the leaves.
template <int MODE, typename P>
__device__ __forceinline__ void hand_backward(const HandView<P>& hv) {
  for (int l = hv.L - 1; l >= 0; --l) {
    const int a0 = hv.ls[l], cnt = hv.ls[l + 1] - a0;
    for (int idx = hv.slot; idx < cnt; idx += hv.nslots) {
      const int n = a0 + idx;
      const NodeDev nd = hv.nodes[n];
      if (is_end(nd.type)) continue;
      const typename P::V val = node_value<MODE, P>(hv, nd);
      if (hv.wr) hv.v[n] = val;
    }
    __syncthreads();
  }
}

// Positive parts of the strategy source into sg, one (row, hand) item per thread:
//   update: the Stage 7 update of R and S (new rows to Rout / Sout where out_ok, the
//           prediction to M where the hand is real), then the positive part of the new R;
//   init: the positive part of R (+ M);  average: S.
// (sign tests of FP64 values read the sign bit on the integer pipe: x > 0 exactly when the
// bits, as a signed integer, are positive)
template <int MODE, typename P>
__device__ __forceinline__ void hand_rows(const HandView<P>& hv, const Discount& d, int variant, Col<double> Rout,
                                          Col<double> Sout, bool out_ok, Col<double> M) {
  using V = typename P::V;
  for (int r = hv.slot; r < hv.nrows; r += hv.nslots) {
    double x;
    if (MODE == kModeUpdate) {
      const int n = hv.rown[r];
      const NodeDev nd = hv.nodes[n];
      const V rr = P::sub(hv.v[nd.first_kid + (hv.rb + r - nd.row)], hv.v[n]);  // instantaneous regret
      const double contrib = P::to_double(P::mul(hv.rch[n], hv.sg[r]));      // pi_i(I) sigma(I, a)
      const double rd = P::to_double(rr);
      x = hv.Rc[r] + rd;
      if (variant == 2) x *= __double_as_longlong(x) > 0 ? d.dpos : d.dneg;
      if ((variant == 1 || variant == 3) && __double_as_longlong(x) < 0) x = 0.0;  // CFR+, Predictive CFR+
      const double sn = fma(hv.Sc[r], d.dS, (variant == 1 || variant == 3) ? d.wS * contrib : contrib);
      if (out_ok) {
        Rout[r] = x;
        Sout[r] = sn;
      }
      if (variant == 3 && hv.valid) M[r] = rd;  // the prediction of the next regret
      if (variant == 3) x += rd;                // Predictive CFR+ matches R + M
    } else {
      x = MODE == kModeInit ? hv.Rc[r] : hv.Sc[r];
      if (MODE == kModeInit && M.base) x += hv.valid ? M[r] : 0.0;
    }
    if (hv.wr) hv.sg[r] = __double_as_longlong(x) > 0 ? P::of_double(x) : P::zero();
  }
  __syncthreads();
}

// Regret matching (Eq. rm) / normalisation of the average, per decision node of p.
template <typename P>
__device__ __forceinline__ void hand_rm(const HandView<P>& hv) {
  using V = typename P::V;
  for (int k = hv.slot; k < hv.ndec; k += hv.nslots) {
    const NodeDev nd = hv.nodes[hv.decs[k]];
    const int A = nd.n_kids, r0 = nd.row - hv.rb;
    V tot = P::zero();
    int npos = 0, last = 0;
    for (int a = 0; a < A; ++a) {
      const V x = hv.sg[r0 + a];
      if (P::positive(x)) ++npos, last = a;
      tot = P::add(tot, x);
    }
    if (!hv.wr) continue;
    if (npos == 1) {  // x / x = 1 exactly, as the definition gives
      for (int a = 0; a < A; ++a) hv.sg[r0 + a] = a == last ? P::one() : P::zero();
    } else if (npos > 1) {
      const V inv = P::recip(tot);
      for (int a = 0; a < A; ++a) hv.sg[r0 + a] = P::mul(hv.sg[r0 + a], inv);
    } else {
      const V uni = P::uniform(A);
      for (int a = 0; a < A; ++a) hv.sg[r0 + a] = uni;
    }
  }
  __syncthreads();
}

// Forward reach of player p (Stages 1-2) under the strategy in sg, from the root reach `root`.
template <typename P>
__device__ __forceinline__ void hand_forward(const HandView<P>& hv, typename P::V root) {
  using V = typename P::V;
  if (hv.slot == 0 && hv.wr) hv.rch[0] = root;
  __syncthreads();
  for (int l = 1; l < hv.L; ++l) {
    const int a0 = hv.ls[l], cnt = hv.ls[l + 1] - a0;
    for (int idx = hv.slot; idx < cnt; idx += hv.nslots) {
      const int n = a0 + idx;
      const NodeDev nd = hv.nodes[n];
      V x = hv.wr ? hv.rch[nd.parent] : P::zero();
      if (nd.aplayer == hv.p) x = P::mul(x, hv.sg[nd.arow - hv.rb]);
      if (nd.deal != kNoCard && ((hv.hmask >> nd.deal) & 1ull)) x = P::zero();
      if (hv.wr) hv.rch[n] = x;
    }
    __syncthreads();
  }
}

// Per-hand tree passes for one chunk of W hands of player p (grid: (player, chunk)).
//   kModeInit:   sigma_p = RM(R_p) (Eq. rm), forward reach of p (Stage 1).
//   kModeUpdate: backward values of p (Stage 6, Eq. backward) from the terminal values,
//                regret and average update (Stage 7), new sigma_p, forward reach of p.
//   kModeAvg:    average strategy S / sum S of p, forward reach of p under it.
//   kModeBR:     best-response backward pass of p (max over p's actions) and the FP64
//                root sum r_p(h) v*_p(root, h), reduced by the last block of each game.
// With G.smem set the block stages the tree and its hands' state in shared memory;
// otherwise it works on the global arrays directly (trees too large to stage).
template <int MODE, typename P, bool SM>
__global__ void __launch_bounds__(kHandThreads, 1) k_hand(const GameDev* __restrict__ games,
                                                       const Work* __restrict__ work, int n_work, int player_mask,
                                                       int advance, int* iter, unsigned* done,
                                                       const Discount* __restrict__ disc_tab, int variant) {
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
  const int tid = threadIdx.x;
  const int w = tid % W;
  const int slot = tid / W;
  const int nslots = kHandThreads / W;
  const int h = wk.unit * W + w;  // < hstride: hstride is a multiple of 32 and W divides 32
  const bool valid = h < G.n_hands;
  const int N = G.n_nodes, L = G.n_levels;
  const size_t stride = (size_t)G.hstride;
  const int rb = G.row_begin[p], re = G.row_begin[p + 1];
  const int nrows = re - rb;
  const int rows_max = max(G.row_begin[1] - G.row_begin[0], G.row_begin[2] - G.row_begin[1]);
  const uint64_t hmask = valid ? G.hand_mask[h] : 0ull;
  constexpr bool sm = SM;       // the launch stages every game in shared memory
  const bool wr = sm || valid;  // this lane may write its column of the working arrays

  // global arrays of this player, at column h
  V* gv = static_cast<V*>(MODE == kModeBR ? G.cfv_br : G.cfv) + (size_t)p * N * stride + h;
  V* grch = static_cast<V*>(MODE == kModeAvg ? G.reach_bar : G.reach) + (size_t)p * N * stride + h;
  V* gsg = static_cast<V*>(MODE == kModeAvg ? G.sigbar : G.sigma) + (size_t)rb * stride + h;
  double* gR = G.R + (size_t)rb * stride + h;
  double* gS = G.S + (size_t)rb * stride + h;

  // shared layout (see hand_smem_bytes)
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* cur = smraw;
  NodeDev* snodes = reinterpret_cast<NodeDev*>(cur);
  cur += round16((size_t)N * sizeof(NodeDev));
  int* sls = reinterpret_cast<int*>(cur);
  cur += round16((size_t)(L + 1) * 4);
  int* srow = reinterpret_cast<int*>(cur);
  cur += round16((size_t)rows_max * 4);
  int* sdec = reinterpret_cast<int*>(cur);
  cur += round16((size_t)rows_max * 4);
  double* sR = reinterpret_cast<double*>(cur);
  cur += round16((size_t)rows_max * W * 8);
  double* sS = reinterpret_cast<double*>(cur);
  cur += round16((size_t)rows_max * W * 8);
  V* sv = reinterpret_cast<V*>(cur);
  V* srch = sv + (size_t)N * W;
  V* ssg = srch + (size_t)N * W;

  const NodeDev* nodes = sm ? snodes : G.nodes;
  const int* ls = sm ? sls : G.level_start;
  const int* rown = sm ? srow : G.row_node + rb;
  const int db = G.dec_begin[p], ndec = G.dec_begin[p + 1] - db;
  const int* decs = sm ? sdec : G.dec_nodes + db;
  const Col<V> v = sm ? Col<V>{sv + w, (size_t)W} : Col<V>{gv, stride};
  const Col<V> rch = sm ? Col<V>{srch + w, (size_t)W} : Col<V>{grch, stride};
  const Col<V> sg = sm ? Col<V>{ssg + w, (size_t)W} : Col<V>{gsg, stride};
  const Col<double> Rc = sm ? Col<double>{sR + w, (size_t)W} : Col<double>{gR, stride};
  const Col<double> Sc = sm ? Col<double>{sS + w, (size_t)W} : Col<double>{gS, stride};
  __shared__ Discount disc;
  __shared__ int s_last;
  __shared__ double red64[kHandThreads];

  // ---- stage: every load is independent of the others, so they are all in flight at once
  if (MODE == kModeUpdate && tid == 0) disc = disc_tab[*iter];
  if constexpr (SM) {
    constexpr int VB = (int)sizeof(V);
    const int4* gn = reinterpret_cast<const int4*>(G.nodes);
    int4* sn = reinterpret_cast<int4*>(snodes);
    for (int k = tid; k < 2 * N; k += kHandThreads) cp_async<16>(sn + k, gn + k);
    for (int k = tid; k <= L; k += kHandThreads) cp_async<4>(sls + k, G.level_start + k);
    for (int k = tid; k < nrows; k += kHandThreads) cp_async<4>(srow + k, G.row_node + rb + k);
    for (int k = tid; k < ndec; k += kHandThreads) cp_async<4>(sdec + k, G.dec_nodes + db + k);
    if (MODE == kModeUpdate) {
      for (int n = slot; n < N; n += nslots) cp_async<VB>(&rch[n], grch + (size_t)n * stride);
      for (int r = slot; r < nrows; r += nslots) {
        cp_async<VB>(&sg[r], gsg + (size_t)r * stride);
        cp_async<8>(&Rc[r], gR + (size_t)r * stride);
        cp_async<8>(&Sc[r], gS + (size_t)r * stride);
      }
    }
    if (MODE == kModeInit)
      for (int r = slot; r < nrows; r += nslots) cp_async<8>(&Rc[r], gR + (size_t)r * stride);
    if (MODE == kModeAvg)
      for (int r = slot; r < nrows; r += nslots) cp_async<8>(&Sc[r], gS + (size_t)r * stride);
  }
  pdl_wait();  // terminal values come from the launch just before this one
  pdl_trigger();
  if constexpr (SM) {
    constexpr int VB = (int)sizeof(V);
    if (MODE == kModeUpdate || MODE == kModeBR)
      for (int n = slot; n < N; n += nslots) cp_async<VB>(&v[n], gv + (size_t)n * stride);
    cp_async_wait_all();
  }
  __syncthreads();

  const HandView<P> hv{nodes, ls, rown, decs, L, ndec, nrows, rb, p, slot, nslots, valid, wr, hmask, v, rch, sg, Rc, Sc};

  // ---- backward pass (Stage 6), level by level from the leaves
  if (MODE == kModeUpdate || MODE == kModeBR) {
    hand_backward<MODE, P>(hv);
    if (sm && valid)
      for (int n = slot; n < N; n += nslots) gv[(size_t)n * stride] = v[n];
  }

  // ---- best response: FP64 root sum of this chunk, then the last block of the game
  //      reduces all chunks of both players in a fixed order
  if (MODE == kModeBR) {
    if (tid < W) {  // slot 0: one lane per hand of the chunk, all in warp 0
      double x = valid ? G.range64[(size_t)p * stride + h] * P::to_double(v[0]) : 0.0;
      const unsigned mask = W == 32 ? 0xffffffffu : (1u << W) - 1u;
      for (int o = W / 2; o > 0; o >>= 1) x += __shfl_down_sync(mask, x, o, W);
      if (tid == 0) G.br_partial[(size_t)p * G.n_chunks + wk.unit] = x;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      s_last = atomicAdd(G.br_done, 1u) == (unsigned)(2 * G.n_chunks - 1);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (int q = 0; q < 2; ++q) {
        double x = 0.0;
        for (int c = tid; c < G.n_chunks; c += kHandThreads) x += G.br_partial[(size_t)q * G.n_chunks + c];
        red64[tid] = x;
        __syncthreads();
        for (int o = kHandThreads / 2; o > 0; o >>= 1) {
          if (tid < o) red64[tid] += red64[tid + o];
          __syncthreads();
        }
        if (tid == 0) G.br_out[q] = red64[0];
        __syncthreads();
      }
      if (tid == 0) *G.br_done = 0u;
    }
    return;
  }

  // ---- positive parts of the strategy source (the update writes R and S to the global rows)
  hand_rows<MODE, P>(hv, disc, variant, Col<double>{gR, stride}, Col<double>{gS, stride}, valid,
                     Col<double>{G.M ? G.M + (size_t)rb * stride + h : nullptr, stride});
  // ---- regret matching (Eq. rm) / normalisation of the average, per decision node of p
  hand_rm<P>(hv);
  // ---- forward reach of player p (Stages 1-2) under the strategy in sg
  hand_forward<P>(hv, valid ? static_cast<const V*>(G.range_v)[(size_t)p * stride + h] : P::zero());
  if (sm && valid) {
    for (int n = slot; n < N; n += nslots) grch[(size_t)n * stride] = rch[n];
    for (int r = slot; r < nrows; r += nslots) gsg[(size_t)r * stride] = sg[r];
  }

  if (MODE == kModeUpdate && advance) {
    __syncthreads();
    if (tid == 0) {
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


// ------------------------------------------------------------------ resident schedule
//
// The latency form of whole iterations, for handles whose hand chunks all fit the GPU at
// once (a single subgame): one cooperative launch runs n iterations.  Block b owns hand chunk
// b of both players and keeps its R, S, strategy and reach rows in shared memory for the whole
// launch, beside the board table of the terminal nodes it evaluates.  An iteration's phases --
// the terminal values of player i (Stages 2-4), then i's update (Stages 6, 7 and 1) -- each
// read what the whole grid wrote in the phase before, so a grid barrier separates them.  What
// crosses blocks (terminal values, reach rows) goes through global memory and is read past L1
// (ld.global.cg), since another block of the same launch wrote it.  The arithmetic is that of
// k_terminal and k_hand, and the global state left at the end is theirs: the level and
// resident schedules give the same bits.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <typename V>
__device__ __forceinline__ V ld_cg(const V* p);
template <>
__device__ __forceinline__ float ld_cg<float>(const float* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ ff ld_cg<ff>(const ff* p) {
  const float2 x = __ldcg(reinterpret_cast<const float2*>(p));
  return {x.x, x.y};
}

// Bounded grid barrier: after a block barrier, one thread counts the block's arrival with a
// release reduction (the block's writes of the phase, ordered before it by the block barrier,
// are visible to whoever acquires the count) and polls with acquire loads until `target`
// arrivals (a multiple of the grid size) have been counted; the block barrier after it orders
// the other threads' reads after that acquire.  Those reads of other blocks' data go past L1
// (ld.global.cg), so no stale line is read.  False when the wait gave up, after `limit` polls
// or because another block gave up: the error flag is then set and the caller leaves.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* err, long limit) {
  __shared__ int s_ok;
  __syncthreads();  // the block's writes of this phase are done
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    int ok = 1;
    for (long k = 0; ld_acquire_u32(count) < target; ++k)
      if (k >= limit || ld_relaxed_s32(err) != 0) {
        ok = 0;
        break;
      }
    if (!ok) atomicExch(err, 1);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__host__ __device__ inline size_t resident_term_bytes(int H, int k, int deck, int hstride, size_t es) {
  return (size_t)TermTab(H, k, deck).len * 2 + (size_t)hstride * es + (size_t)(k * H + 1 + H + 1) * 8;
}

// Shared memory of the resident kernel's hand region for one game (must match k_resident):
// nodes, level offsets, per player the row -> node map and decision-node list, R, S, then the
// values (one player at a time), and per player the reach and strategy.
__host__ __device__ inline size_t resident_hand_bytes(int n_nodes, int n_levels, int rows_max, int W, size_t es) {
  return round16((size_t)n_nodes * sizeof(NodeDev)) + round16((size_t)(n_levels + 1) * 4) +
         4 * round16((size_t)rows_max * 4) + 4 * round16((size_t)rows_max * W * 8) +
         round16((size_t)n_nodes * W * es) + 2 * round16((size_t)n_nodes * W * es) +
         2 * round16((size_t)rows_max * W * es);
}

// One terminal node of player i (Stages 2-4) in the resident kernel: the board table stays in
// shared memory while the nodes the block evaluates read the same one (tab_game / tab_b name
// it); the opponent's reach row is read past L1.  Ends with a block barrier.
template <typename P>
__device__ __forceinline__ void resident_terminal(const GameDev* __restrict__ games, Work e, int src, int i,
                                                  unsigned char* smr, int& tab_game, int& tab_b) {
  using V = typename P::V;
  const GameDev& G = games[e.game];
  const int n = e.unit;
  const NodeDev nd = G.nodes[n];
  const TermTab tt(G.n_hands, G.hand_size, G.deck);
  const size_t stride = (size_t)G.hstride;
  uint16_t* tab = reinterpret_cast<uint16_t*>(smr);
  V* qs = reinterpret_cast<V*>(smr + (size_t)tt.len * 2);
  ff* CP = reinterpret_cast<ff*>(smr + (size_t)tt.len * 2 + stride * sizeof(V));
  ff* Psc = CP + (G.hand_size * G.n_hands + 1);
  // a fold reads table 0, as in k_terminal (each table orders its per-card hand lists by its
  // own board's ranks, so another table's lists would sum the same reach in another order)
  const int b = nd.type == kShowdown ? nd.row : 0;
  if (tab_game != e.game || tab_b != b) {  // len is a multiple of 8 entries: 16-byte pieces
    const uint4* src4 = reinterpret_cast<const uint4*>(G.term_tab + (size_t)b * tt.len);
    for (int k = threadIdx.x; k < tt.len / 8; k += blockDim.x) reinterpret_cast<uint4*>(tab)[k] = __ldg(src4 + k);
    tab_game = e.game;
    tab_b = b;
  }
  {  // the row is a multiple of 128 bytes (hstride is a multiple of 32)
    const uint4* q4 = reinterpret_cast<const uint4*>(static_cast<const V*>(G.reach) +
                                                     ((size_t)(1 - i) * G.n_nodes + src) * stride);
    for (int k = threadIdx.x; k < (int)(stride * sizeof(V) / 16); k += blockDim.x)
      reinterpret_cast<uint4*>(qs)[k] = __ldcg(q4 + k);
  }
  __syncthreads();
  if (src != n) {  // below an all-in run-out: zero the hands holding a card dealt on the way
    for (int h = threadIdx.x; h < G.n_hands; h += blockDim.x)
      if (holds_board_card(tab + tt.cards, h, G.hand_size, nd.board)) qs[h] = P::zero();
    __syncthreads();
  }
  const bool neg = nd.type == kFold && nd.player == i;
  const ff u = {neg ? -G.payoff_ff[2 * n] : G.payoff_ff[2 * n], neg ? -G.payoff_ff[2 * n + 1] : G.payoff_ff[2 * n + 1]};
  terminal_values<P>(G, nd, i, u, tt, tab, qs, CP, Psc,
                     static_cast<V*>(G.cfv) + ((size_t)i * G.n_nodes + n) * stride);
  __syncthreads();  // the row buffer and the scan arrays are free again
}

// n_iters iterations (alternating: terminal and update of player 0, then of player 1;
// otherwise both players' terminals, then both updates).  Launched cooperatively, every block
// resident: grid >= n_chunk_work.  sync[0] counts barrier arrivals, sync[1] blocks that have
// finished; the last block to finish resets both and advances *iter by n_iters.
template <typename P>
__global__ void __launch_bounds__(kTermThreads, 1) k_resident(
    const GameDev* __restrict__ games, const Work* __restrict__ chunk_work, int n_chunk_work,
    const Work* __restrict__ term_work, const int32_t* __restrict__ term_src, int n_term_work, int alternating,
    int n_iters, int* iter, const Discount* __restrict__ disc_tab, int variant, unsigned* sync, int* err,
    unsigned term_bytes) {
  using V = typename P::V;
  constexpr size_t es = sizeof(V);
  extern __shared__ __align__(16) unsigned char smr[];
  const int tid = threadIdx.x;
  const bool owner = (int)blockIdx.x < n_chunk_work;
  const Work wk = owner ? chunk_work[blockIdx.x] : Work{0, 0};
  const GameDev& G = games[wk.game];
  const int W = G.chunk, w = tid % W, slot = tid / W, nslots = kTermThreads / W;
  const int h = wk.unit * W + w;  // < hstride
  const bool valid = owner && h < G.n_hands;
  const int N = G.n_nodes, L = G.n_levels;
  const size_t stride = (size_t)G.hstride;
  const int rows_max = max(G.row_begin[1] - G.row_begin[0], G.row_begin[2] - G.row_begin[1]);
  const uint64_t hmask = valid ? G.hand_mask[h] : 0ull;

  // hand region (see resident_hand_bytes), after the terminal region
  unsigned char* cur = smr + term_bytes;
  NodeDev* snodes = reinterpret_cast<NodeDev*>(cur);
  cur += round16((size_t)N * sizeof(NodeDev));
  int* sls = reinterpret_cast<int*>(cur);
  cur += round16((size_t)(L + 1) * 4);
  const size_t ri = round16((size_t)rows_max * 4), rd8 = round16((size_t)rows_max * W * 8);
  int* srow[2] = {reinterpret_cast<int*>(cur), reinterpret_cast<int*>(cur + ri)};
  cur += 2 * ri;
  int* sdec[2] = {reinterpret_cast<int*>(cur), reinterpret_cast<int*>(cur + ri)};
  cur += 2 * ri;
  double* sR[2] = {reinterpret_cast<double*>(cur), reinterpret_cast<double*>(cur + rd8)};
  cur += 2 * rd8;
  double* sS[2] = {reinterpret_cast<double*>(cur), reinterpret_cast<double*>(cur + rd8)};
  cur += 2 * rd8;
  const size_t nv = round16((size_t)N * W * es), rv = round16((size_t)rows_max * W * es);
  V* sv = reinterpret_cast<V*>(cur);
  cur += nv;
  V* srch[2] = {reinterpret_cast<V*>(cur), reinterpret_cast<V*>(cur + nv)};
  cur += 2 * nv;
  V* ssg[2] = {reinterpret_cast<V*>(cur), reinterpret_cast<V*>(cur + rv)};

  // ---- stage the tree and the chunk's state of both players (written by earlier launches)
  if (owner) {
    const int4* gn = reinterpret_cast<const int4*>(G.nodes);
    for (int k = tid; k < 2 * N; k += kTermThreads) reinterpret_cast<int4*>(snodes)[k] = __ldg(gn + k);
    for (int k = tid; k <= L; k += kTermThreads) sls[k] = G.level_start[k];
    for (int p = 0; p < 2; ++p) {
      const int rb = G.row_begin[p], nrows = G.row_begin[p + 1] - rb;
      const int db = G.dec_begin[p], ndec = G.dec_begin[p + 1] - db;
      for (int k = tid; k < nrows; k += kTermThreads) srow[p][k] = G.row_node[rb + k];
      for (int k = tid; k < ndec; k += kTermThreads) sdec[p][k] = G.dec_nodes[db + k];
      for (int r = slot; r < nrows; r += nslots) {
        const size_t g = (size_t)(rb + r) * stride + h;
        sR[p][r * W + w] = G.R[g];
        sS[p][r * W + w] = G.S[g];
        ssg[p][r * W + w] = static_cast<const V*>(G.sigma)[g];
      }
      const V* grch = static_cast<const V*>(G.reach) + (size_t)p * N * stride + h;
      for (int n = slot; n < N; n += nslots) srch[p][n * W + w] = grch[(size_t)n * stride];
    }
  }
  __syncthreads();

  const int it0 = *iter;  // written only by the last block to finish
  const int steps = alternating ? 2 : 1;
  unsigned nbar = 0;
  bool ok = true;
  int tab_game = -1, tab_b = -1;
  for (int it = 0; it < n_iters && ok; ++it) {
    const Discount d = disc_tab[it0 + it];
    for (int step = 0; step < steps && ok; ++step) {
      const int pm = alternating ? 1 << step : 3;
      const int p0 = pm == 2 ? 1 : 0, np = pm == 3 ? 2 : 1;
      // ---- terminal values of the player(s) of this step (Stages 2-4)
      for (int item = blockIdx.x; item < np * n_term_work; item += gridDim.x) {
        const int e = item % n_term_work;
        resident_terminal<P>(games, term_work[e], term_src[e], p0 + item / n_term_work, smr, tab_game, tab_b);
      }
      ++nbar;
      ok = grid_barrier(&sync[0], nbar * gridDim.x, err, nbar == 1 ? g_first_wait_polls : kWaitLimit);
      if (!ok) break;
      // ---- the update of the chunk's hands (Stages 6, 7, then 1 with the new strategy)
      if (owner) {
        for (int p = p0; p < p0 + np; ++p) {
          const int rb = G.row_begin[p], nrows = G.row_begin[p + 1] - rb;
          const int ndec = G.dec_begin[p + 1] - G.dec_begin[p];
          V* gv = static_cast<V*>(G.cfv) + (size_t)p * N * stride + h;
          V* grch = static_cast<V*>(G.reach) + (size_t)p * N * stride + h;
          const Col<V> v{sv + w, (size_t)W};
          for (int n = slot; n < N; n += nslots) v[n] = ld_cg(gv + (size_t)n * stride);
          __syncthreads();
          const HandView<P> hv{snodes, sls, srow[p], sdec[p], L, ndec, nrows, rb, p, slot, nslots, valid, true, hmask,
                               v, Col<V>{srch[p] + w, (size_t)W}, Col<V>{ssg[p] + w, (size_t)W},
                               Col<double>{sR[p] + w, (size_t)W}, Col<double>{sS[p] + w, (size_t)W}};
          hand_backward<kModeUpdate, P>(hv);
          if (valid)
            for (int n = slot; n < N; n += nslots) gv[(size_t)n * stride] = v[n];
          hand_rows<kModeUpdate, P>(hv, d, variant, hv.Rc, hv.Sc, true,
                                    Col<double>{G.M ? G.M + (size_t)rb * stride + h : nullptr, stride});
          hand_rm<P>(hv);
          hand_forward<P>(hv, valid ? static_cast<const V*>(G.range_v)[(size_t)p * stride + h] : P::zero());
          if (valid)  // the opponent's terminal values read these rows
            for (int n = slot; n < N; n += nslots) grch[(size_t)n * stride] = hv.rch[n];
        }
      }
      ++nbar;
      ok = grid_barrier(&sync[0], nbar * gridDim.x, err, kWaitLimit);
    }
  }

  // ---- the chunk's R, S and strategy rows back to global memory
  if (ok && valid) {
    for (int p = 0; p < 2; ++p) {
      const int rb = G.row_begin[p], nrows = G.row_begin[p + 1] - rb;
      for (int r = slot; r < nrows; r += nslots) {
        const size_t g = (size_t)(rb + r) * stride + h;
        G.R[g] = sR[p][r * W + w];
        G.S[g] = sS[p][r * W + w];
        static_cast<V*>(G.sigma)[g] = ssg[p][r * W + w];
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&sync[1], 1u) == gridDim.x - 1) {  // every other block has left its waits
      sync[0] = 0u;
      sync[1] = 0u;
      *iter += n_iters;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------ stream schedule
//
// The throughput form of the update launch (Stages 6, 7 and then 1 of one player), for
// handles whose hands fill the GPU many times over (batches of subgames).  One warp owns 32
// consecutive hands of one subgame and walks the subgame's depth-first program alone: no
// block barriers, every access to an R, S, reach or value row is one coalesced 32-lane
// segment, and the only per-node state kept is a stack per lane in shared memory.
//   1. bottom-up over the program in reverse: values of Eq. (backward) from the terminal
//      values, and at each of the player's decision nodes the regrets and the Stage 7
//      update of R and S with sigma = RM(R) (Eq. rm) and the player's reach there (stored
//      by the previous update of this player, or by the initial pass);
//   2. top-down over the program with the new strategy RM(R'): the player's reach at its
//      decision nodes (for its next update) and at the terminals (for the opponent's next
//      terminal launch).
// Strategies and the values of inner nodes never go to DRAM.  Every address a pass reads
// is fixed by the program, so each pass is cut into chunks (stream_tables) that are loaded
// into a per-lane ring in shared memory with cp.async one chunk ahead of the computation.
// The arithmetic (regret matching, child order of every sum, the update) is that of k_hand,
// so both schedules give the same bits.


// Regret matching of one node's A rows (Eq. rm), as k_hand computes it: positive parts in
// the value type, their sum in action order, exactly 1 for a lone positive action.
template <typename P>
__device__ __forceinline__ void regret_match(const double (&Rv)[kStreamMaxActions], int A,
                                             typename P::V (&sg)[kStreamMaxActions]) {
  using V = typename P::V;
  V tot = P::zero();
  int npos = 0, last = 0;
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a) {
    if (a < A) {
      const V x = __double_as_longlong(Rv[a]) > 0 ? P::of_double(Rv[a]) : P::zero();
      sg[a] = x;
      if (P::positive(x)) ++npos, last = a;
      tot = P::add(tot, x);
    }
  }
  if (npos == 1) {
#pragma unroll
    for (int a = 0; a < kStreamMaxActions; ++a) sg[a] = a == last ? P::one() : P::zero();
  } else if (npos > 1) {
    const V inv = P::recip(tot);
#pragma unroll
    for (int a = 0; a < kStreamMaxActions; ++a)
      if (a < A) sg[a] = P::mul(sg[a], inv);
  } else {
    const V uni = P::uniform(A);
#pragma unroll
    for (int a = 0; a < kStreamMaxActions; ++a) sg[a] = uni;
  }
}

// regret_match with a compile-time action count (same arithmetic, no per-action guards), with
// the three cases selected per lane instead of branched on: the hands of a warp often fall
// in different cases, and a branch would run all three paths for them.
template <typename P, int NA>
__device__ __forceinline__ void regret_match_n(const double (&Rv)[NA], typename P::V (&sg)[NA]) {
  using V = typename P::V;
  V tot = P::zero();
  int npos = 0, last = 0;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const V x = __double_as_longlong(Rv[a]) > 0 ? P::of_double(Rv[a]) : P::zero();
    sg[a] = x;
    if (P::positive(x)) ++npos, last = a;
    tot = P::add(tot, x);
  }
  const V inv = P::recip(tot);  // unused (and possibly not finite) unless npos > 1
  const V uni = P::uniform(NA);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const V many = P::mul(sg[a], inv);
    sg[a] = npos > 1 ? many : npos == 1 ? (a == last ? P::one() : P::zero()) : uni;
  }
}

__device__ __forceinline__ void load_rows(const double* __restrict__ base, size_t stride, int A,
                                          double (&out)[kStreamMaxActions]) {
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a) out[a] = a < A ? base[(size_t)a * stride] : 0.0;
}

// A program node, decoded.
struct Op {
  int node_off, row_off, type, player, A, deal, tmask, first_kid;
};
__device__ __forceinline__ Op decode(const ProgOp& o) {
  return {o.node_off,
          o.row_off,
          (int)(o.code & 3u),
          (int)((o.code >> 2) & 1u),
          (int)((o.code >> 3) & 63u),
          (int)((o.code >> 9) & 0xffu),
          (int)((o.code >> 17) & 0xffu),
          o.first_kid};
}

// One lane's view of its subgame for the stream passes.  A warp owns 32 * HP consecutive
// hands; lane l holds hands l, l + 32, ..., l + 32 (HP - 1) of them (HP = 1 or 2), so the
// walk's control work (program decode, branches, stack and ring bookkeeping, load issue)
// is shared by HP hands per lane and each lane has HP independent arithmetic chains.
template <typename P, int HP>
struct StreamLane {
  using V = typename P::V;
  const GameDev& G;
  const ProgOp* prog;     // the program (shared memory when staged)
  const uint32_t* units;  // this player's loads, bottom-up pass then top-down pass
  int p;
  bool valid[HP];         // hand l + 32 k exists
  uint64_t hmask[HP];
  size_t stride;
  double* R;        // column of the lane's first hand of R (hand k: + 32 k)
  double* S;
  double* M;        // the same of the Predictive CFR+ prediction (null otherwise)
  V* reach;         // column of the lane's first hand in player p's reach plane
  V* cfv;           // the same in player p's value plane
  uint64_t* ring;   // this lane's entry of the prefetch ring: unit u of half k at
                    // ring[(k * half + u) * 32 * HP], its hand k at + 32 k
  int half;         // units in each half of the ring
  V* st;            // this lane's stack: slot s, hand k at st[(s * HP + k) * 32]
};

// Issue loads [u0, u1) of a pass into ring half `half` (one commit group).  A unit is the
// warp's segment of 32 * HP consecutive elements of one row (256 * HP bytes of FP64 or pair
// values, 128 * HP of FP32 ones), landing at slot u - u0 of the ring half.  The warp's lanes
// split the units into 16-byte pieces (16 * HP per FP64 unit), so that one copy instruction
// moves pieces of several units.
template <typename P, int HP>
__device__ __forceinline__ void stream_issue(const StreamLane<P, HP>& L, const uint32_t* units, int u0, int u1,
                                             int half) {
  using V = typename P::V;
  constexpr int kPieces = 16 * HP;  // 16-byte pieces of one unit
  const int lane = threadIdx.x & 31;
  unsigned char* ring = reinterpret_cast<unsigned char*>(L.ring - lane + (size_t)half * L.half * 32 * HP);
  const int pieces = (u1 - u0) * kPieces;
  for (int k = lane; k < pieces; k += 32) {
    const int u = u0 + k / kPieces, part = k % kPieces;
    const uint32_t d = units[u];
    const uint32_t arr = d >> kArrShift, off = d & kArrOffMask;
    // the row's segment starts at the warp's first hand: the lane's column pointer minus its lane
    const void* src;
    if (arr == kArrR)
      src = L.R - lane + off + 2 * part;
    else if (arr == kArrS)
      src = L.S - lane + off + 2 * part;
    else if (arr == kArrM)
      src = L.M - lane + off + 2 * part;
    else if (part * 16 >= 32 * HP * (int)sizeof(V))  // FP32 rows fill half a slot
      continue;
    else
      src = reinterpret_cast<const unsigned char*>((arr == kArrReach ? L.reach : L.cfv) - lane + off) + part * 16;
    cp_async<16>(ring + (size_t)(u - u0) * 256 * HP + (size_t)part * 16, src);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This lane's value of its hand k in a ring unit (slot: the lane's entry of the unit):
// 8-byte values sit at entry lane + 32 k, FP32 values packed at float lane + 32 k.
template <typename P, int HP>
__device__ __forceinline__ typename P::V ring_value(const uint64_t* slot, int k) {
  using V = typename P::V;
  if constexpr (sizeof(V) == 4) {
    const int lane = threadIdx.x & 31;
    return reinterpret_cast<const V*>(slot - lane)[lane + 32 * k];
  } else {
    return *reinterpret_cast<const V*>(slot + 32 * k);
  }
}

// Bottom-up work at one of the player's decision nodes with NA actions (Stages 6-7), for
// each of the lane's HP hands: the children's values (ring or stack), regret matching of R
// (R + M for Predictive CFR+), the node value, and the new R, S (and M) rows.  NA is a
// compile-time constant so that the actions' FP64 update chains are straight-line code the
// compiler can interleave.
template <typename P, int NA, int HP>
__device__ __forceinline__ void decision_back(const StreamLane<P, HP>& L, const Op& nd, const uint64_t* ring, int& u,
                                              int& sp, const Discount& d, int variant, typename P::V (&val)[HP]) {
  using V = typename P::V;
  constexpr int U = 32 * HP;  // ring entries per unit
  V* st = L.st;
  V c[NA][HP];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    if ((nd.tmask >> a) & 1) {
#pragma unroll
      for (int k = 0; k < HP; ++k) c[a][k] = ring_value<P, HP>(ring + (size_t)u * U, k);
      ++u;
    } else {
      --sp;
#pragma unroll
      for (int k = 0; k < HP; ++k) c[a][k] = st[(sp * HP + k) * 32];
    }
  }
  const bool pred = L.M != nullptr;  // Predictive CFR+: R, M, S, reach
  const double* Rr = reinterpret_cast<const double*>(ring + (size_t)u * U);
  const double* Mr = reinterpret_cast<const double*>(ring + (size_t)(u + NA) * U);
  const double* Sr = reinterpret_cast<const double*>(ring + (size_t)(u + (pred ? 2 : 1) * NA) * U);
  const uint64_t* pislot = ring + (size_t)(u + (pred ? 3 : 2) * NA) * U;
  u += (pred ? 3 : 2) * NA + 1;
#pragma unroll
  for (int k = 0; k < HP; ++k) {
    const V pi = ring_value<P, HP>(pislot, k);
    double Rv[NA];
    V sg[NA];
    {
      double Rm[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) Rv[a] = Rm[a] = Rr[(size_t)a * U + 32 * k];
      if (pred) {  // Predictive CFR+ matches R + M (no FP64 add for the other variants)
#pragma unroll
        for (int a = 0; a < NA; ++a) Rm[a] = Rv[a] + Mr[(size_t)a * U + 32 * k];
      }
      regret_match_n<P, NA>(Rm, sg);
    }
    typename P::Acc acc = P::acc0();
#pragma unroll
    for (int a = 0; a < NA; ++a) P::acc_mul(acc, sg[a], c[a][k]);
    val[k] = P::value(acc);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const V rr = P::sub(c[a][k], val[k]);                    // instantaneous regret
      const double contrib = P::to_double(P::mul(pi, sg[a]));  // pi_i(I) sigma(I, a)
      const double rd = P::to_double(rr);
      double x = Rv[a] + rd;
      if (variant == 2) x *= __double_as_longlong(x) > 0 ? d.dpos : d.dneg;
      if ((variant == 1 || variant == 3) && __double_as_longlong(x) < 0) x = 0.0;
      const double sn =
          fma(Sr[(size_t)a * U + 32 * k], d.dS, (variant == 1 || variant == 3) ? d.wS * contrib : contrib);
      if (L.valid[k]) {
        const size_t at = (size_t)nd.row_off + (size_t)a * L.stride + 32 * k;
        L.R[at] = x;
        L.S[at] = sn;
        if (pred) L.M[at] = rd;
      }
    }
  }
}

// Top-down work at one of the player's decision nodes with NA actions: the reach x there is
// recorded, sigma = RM(R) (of R + M for Predictive CFR+) is formed from the ring, and each
// child's reach x sigma(a) goes to the terminal's row or onto the stack (child 0 on top).  NA
// is a compile-time constant, as in decision_back.
template <typename P, int NA, int HP>
__device__ __forceinline__ void decision_fwd(const StreamLane<P, HP>& L, const Op& nd, const uint64_t* ring, int& u,
                                             int& sp, const typename P::V (&x)[HP]) {
  using V = typename P::V;
  constexpr int U = 32 * HP;
  V* st = L.st;
  const bool pred = L.M != nullptr;  // Predictive CFR+: R then M
  const double* Rr = reinterpret_cast<const double*>(ring + (size_t)u * U);
  const double* Mr = reinterpret_cast<const double*>(ring + (size_t)(u + NA) * U);
  u += (pred ? 2 : 1) * NA;
  V sg[NA][HP];
#pragma unroll
  for (int k = 0; k < HP; ++k) {
    if (L.valid[k]) L.reach[(size_t)nd.node_off + 32 * k] = x[k];
    double Rv[NA];
    V s1[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) Rv[a] = Rr[(size_t)a * U + 32 * k];
    if (pred) {  // Predictive CFR+ matches R + M
#pragma unroll
      for (int a = 0; a < NA; ++a) Rv[a] += Mr[(size_t)a * U + 32 * k];
    }
    regret_match_n<P, NA>(Rv, s1);
#pragma unroll
    for (int a = 0; a < NA; ++a) sg[a][k] = s1[a];
  }
#pragma unroll
  for (int a = NA - 1; a >= 0; --a) {
    if ((nd.tmask >> a) & 1) {
#pragma unroll
      for (int k = 0; k < HP; ++k)
        if (L.valid[k]) L.reach[(size_t)(nd.first_kid + a) * L.stride + 32 * k] = P::mul(x[k], sg[a][k]);
    } else {
#pragma unroll
      for (int k = 0; k < HP; ++k) st[(sp * HP + k) * 32] = P::mul(x[k], sg[a][k]);
      ++sp;
    }
  }
}

// Bottom-up pass over chunk [k0, k1) (program positions counted from its end).  A node's
// children values come from the ring (terminal children, in child order) or from the stack
// (inner children, child 0 on top).
template <typename P, int HP>
__device__ __forceinline__ void stream_backward_chunk(const StreamLane<P, HP>& L, int k0, int k1, int half, int& sp,
                                                      const Discount& d, int variant) {
  using V = typename P::V;
  constexpr int U = 32 * HP;
  const int N = L.G.prog_len;
  const uint64_t* ring = L.ring + (size_t)half * L.half * U;
  V* st = L.st;
  int u = 0;
  for (int k = k0; k < k1; ++k) {
    const Op nd = decode(L.prog[N - 1 - k]);
    const int A = nd.A;
    V val[HP];
    if (nd.type == kChance || nd.player != L.p) {
      // chance: children values carry the card probabilities (a hand holding the card gets
      // nothing from that child); opponent: the plain sum
      const bool chance = nd.type == kChance;
      const bool term_all = nd.tmask & 1;  // chance: all children terminal (after an all-in) or all inner
      typename P::Acc acc[HP];
#pragma unroll
      for (int j = 0; j < HP; ++j) acc[j] = P::acc0();
      for (int a = 0; a < A; ++a) {
        const bool term = chance ? term_all : ((nd.tmask >> a) & 1);
        const int deal = chance ? L.G.nodes[nd.first_kid + a].deal : 0;
        if (!term) --sp;
#pragma unroll
        for (int j = 0; j < HP; ++j) {
          const V x = term ? ring_value<P, HP>(ring + (size_t)u * U, j) : st[(sp * HP + j) * 32];
          if (!chance || !((L.hmask[j] >> deal) & 1ull)) P::acc(acc[j], x);
        }
        if (term) ++u;
      }
#pragma unroll
      for (int j = 0; j < HP; ++j) val[j] = P::value(acc[j]);
    } else {  // the player's decision node: its action count as a compile-time constant
      switch (A) {
        case 1: decision_back<P, 1, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 2: decision_back<P, 2, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 3: decision_back<P, 3, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 4: decision_back<P, 4, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 5: decision_back<P, 5, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 6: decision_back<P, 6, HP>(L, nd, ring, u, sp, d, variant, val); break;
        case 7: decision_back<P, 7, HP>(L, nd, ring, u, sp, d, variant, val); break;
        default: decision_back<P, kStreamMaxActions, HP>(L, nd, ring, u, sp, d, variant, val); break;
      }
    }
#pragma unroll
    for (int j = 0; j < HP; ++j) st[(sp * HP + j) * 32] = val[j];
    ++sp;
  }
}

// Top-down pass over chunk [k0, k1) with sigma = RM(R): records the reach at the player's
// decision nodes, at chance nodes and, for the terminal children, at the terminals; pushes
// the reach of the inner children (child 0 on top).
template <typename P, int HP>
__device__ __forceinline__ void stream_forward_chunk(const StreamLane<P, HP>& L, int k0, int k1, int half, int& sp) {
  using V = typename P::V;
  constexpr int U = 32 * HP;
  const uint64_t* ring = L.ring + (size_t)half * L.half * U;
  V* st = L.st;
  int u = 0;
  for (int k = k0; k < k1; ++k) {
    const Op nd = decode(L.prog[k]);
    --sp;
    V x[HP];
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      x[j] = st[(sp * HP + j) * 32];
      if (nd.deal != kNoCard && ((L.hmask[j] >> nd.deal) & 1ull)) x[j] = P::zero();
    }
    const int A = nd.A;
    if (nd.type == kDecision && nd.player == L.p) {  // its action count as a compile-time constant
      switch (A) {
        case 1: decision_fwd<P, 1, HP>(L, nd, ring, u, sp, x); break;
        case 2: decision_fwd<P, 2, HP>(L, nd, ring, u, sp, x); break;
        case 3: decision_fwd<P, 3, HP>(L, nd, ring, u, sp, x); break;
        case 4: decision_fwd<P, 4, HP>(L, nd, ring, u, sp, x); break;
        case 5: decision_fwd<P, 5, HP>(L, nd, ring, u, sp, x); break;
        case 6: decision_fwd<P, 6, HP>(L, nd, ring, u, sp, x); break;
        case 7: decision_fwd<P, 7, HP>(L, nd, ring, u, sp, x); break;
        default: decision_fwd<P, kStreamMaxActions, HP>(L, nd, ring, u, sp, x); break;
      }
    } else if (nd.type == kChance) {  // the player's reach passes through to each card
#pragma unroll
      for (int j = 0; j < HP; ++j)
        if (L.valid[j]) L.reach[(size_t)nd.node_off + 32 * j] = x[j];  // read by an all-in run-out's showdowns
      if (nd.tmask & 1) {  // terminal children: their reach, zero where the hand holds the card
        for (int a = 0; a < A; ++a) {
          const int deal = L.G.nodes[nd.first_kid + a].deal;
#pragma unroll
          for (int j = 0; j < HP; ++j)
            if (L.valid[j])
              L.reach[(size_t)(nd.first_kid + a) * L.stride + 32 * j] = ((L.hmask[j] >> deal) & 1ull) ? P::zero() : x[j];
        }
      } else {  // inner children apply their own card when they pop it
        for (int a = 0; a < A; ++a) {
#pragma unroll
          for (int j = 0; j < HP; ++j) st[(sp * HP + j) * 32] = x[j];
          ++sp;
        }
      }
    } else {  // opponent decision: the player's reach passes through
      for (int a = A - 1; a >= 0; --a) {
        if ((nd.tmask >> a) & 1) {
#pragma unroll
          for (int j = 0; j < HP; ++j)
            if (L.valid[j]) L.reach[(size_t)(nd.first_kid + a) * L.stride + 32 * j] = x[j];
        } else {
#pragma unroll
          for (int j = 0; j < HP; ++j) st[(sp * HP + j) * 32] = x[j];
          ++sp;
        }
      }
    }
  }
}

// One pass (list q of the load tables): chunk c + 1 loads while chunk c computes.
template <typename P, int HP, typename F>
__device__ __forceinline__ void stream_pass(const StreamLane<P, HP>& L, int q, const uint32_t* units, F compute) {
  const int32_t* ch = L.G.chunks + 2 * (size_t)L.G.chunk_off[q];  // (node, unit) pairs
  const int nch = L.G.chunk_count[q];
  stream_issue<P, HP>(L, units, ch[1], ch[3], 0);
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch)
      stream_issue<P, HP>(L, units, ch[2 * c + 3], ch[2 * c + 5], (c + 1) & 1);
    else
      asm volatile("cp.async.commit_group;" ::: "memory");
    cp_async_wait_group<1>();  // chunk c has landed: this lane's pieces
    __syncwarp();              // and the other lanes' (each lane reads its own column of every piece)
    compute(ch[2 * c], ch[2 * c + 2], c & 1);
  }
  cp_async_wait_group<0>();
}

// Grid: one block per (player, work item); a work item is a game and the first of the
// kStreamWarps consecutive groups of 32 * HP hands its warps own.
template <typename P, int HP>
__global__ void __launch_bounds__(kStreamWarps * 32) k_stream_update(
    const GameDev* __restrict__ games, const Work* __restrict__ work, int n_work, int player_mask, int advance,
    int* iter, unsigned* done, const Discount* __restrict__ disc_tab, int variant, int depth, int prog_nodes,
    int prog_units, int half_units) {
  using V = typename P::V;
  extern __shared__ __align__(16) unsigned char sms[];
  __shared__ Discount disc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int item = blockIdx.x;
  int p = player_mask == 2 ? 1 : 0;
  if (player_mask == 3 && item >= n_work) p = 1, item -= n_work;
  const Work wk = work[item];
  const GameDev& G = games[wk.game];
  const int unit = wk.unit + warp;
  const bool active = unit * 32 * HP < G.n_hands;
  if (threadIdx.x == 0) disc = disc_tab[*iter];
  // shared memory: the program, then per warp a prefetch ring (2 halves of half_units
  // units of 32 * HP 8-byte entries) and a stack (depth slots of HP values per lane)
  const size_t tables = (size_t)prog_nodes * sizeof(ProgOp) + (size_t)prog_units * 4;  // multiple of 16
  ProgOp* sprog = reinterpret_cast<ProgOp*>(sms);
  uint32_t* sunits = reinterpret_cast<uint32_t*>(sms + (size_t)prog_nodes * sizeof(ProgOp));
  uint64_t* ring = reinterpret_cast<uint64_t*>(sms + tables) + (size_t)warp * 2 * half_units * 32 * HP + lane;
  V* st = reinterpret_cast<V*>(sms + tables + (size_t)kStreamWarps * 2 * half_units * 32 * HP * 8) +
          (size_t)warp * depth * 32 * HP + lane;
  // this player's loads: the bottom-up pass's, then the top-down pass's
  const uint32_t* gunits_b = G.units + G.unit_off[p];
  const uint32_t* gunits_f = G.units + G.unit_off[2 + p];
  const int nb = G.unit_count[p], nf = G.unit_count[2 + p];
  if (prog_nodes > 0) {  // static: staged while the previous launch finishes
    const int4* src = reinterpret_cast<const int4*>(G.prog);
    int4* dst = reinterpret_cast<int4*>(sprog);
    for (int k = threadIdx.x; k < G.prog_len; k += blockDim.x) dst[k] = __ldg(src + k);
    for (int k = threadIdx.x; k < nb; k += blockDim.x) sunits[k] = __ldg(gunits_b + k);
    for (int k = threadIdx.x; k < nf; k += blockDim.x) sunits[nb + k] = __ldg(gunits_f + k);
  }
  pdl_wait();  // the terminal values come from the launch just before this one
  pdl_trigger();
  __syncthreads();  // disc, program
  if (active) {
    const int h = unit * 32 * HP + lane;  // hand k is h + 32 k < hstride (a multiple of 32 * HP)
    const size_t stride = (size_t)G.hstride;
    const size_t plane = (size_t)p * G.n_nodes * stride + h;
    const bool staged = prog_nodes > 0;
    StreamLane<P, HP> L{G, staged ? sprog : G.prog, staged ? sunits : gunits_b, p, {}, {}, stride,
                        G.R + h, G.S + h, G.M ? G.M + h : nullptr, static_cast<V*>(G.reach) + plane,
                        static_cast<V*>(G.cfv) + plane, ring, half_units, st};
#pragma unroll
    for (int k = 0; k < HP; ++k) {
      L.valid[k] = h + 32 * k < G.n_hands;
      L.hmask[k] = L.valid[k] ? G.hand_mask[h + 32 * k] : 0ull;
    }
    const Discount d = disc;
    int sp = 0;
    stream_pass<P, HP>(L, p, L.units, [&](int k0, int k1, int half) {
      stream_backward_chunk<P, HP>(L, k0, k1, half, sp, d, variant);
    });
#pragma unroll
    for (int k = 0; k < HP; ++k)
      if (L.valid[k]) L.cfv[32 * k] = st[k * 32];  // root value (read-back)
    __threadfence_block();  // the new R rows are read back by the warp's copies below
    __syncwarp();
#pragma unroll
    for (int k = 0; k < HP; ++k)
      st[k * 32] = L.valid[k] ? static_cast<const V*>(G.range_v)[(size_t)p * stride + h + 32 * k] : P::zero();
    sp = 1;
    stream_pass<P, HP>(L, 2 + p, staged ? sunits + nb : gunits_f,
                       [&](int k0, int k1, int half) { stream_forward_chunk<P, HP>(L, k0, k1, half, sp); });
  }

  if (advance) {
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

// sigma = RM(R) at every decision node of every game (current strategy, for read-back when
// the update launches do not store it).
template <typename P>
__global__ void k_current_rows(const GameDev* __restrict__ games, int n_games) {
  using V = typename P::V;
  for (int g = 0; g < n_games; ++g) {
    const GameDev& G = games[g];
    const size_t stride = (size_t)G.hstride;
    const int total = G.n_nodes * G.n_hands;
    V* out = static_cast<V*>(G.sigma);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
      const int n = e / G.n_hands, h = e - n * G.n_hands;
      const NodeDev nd = G.nodes[n];
      if (nd.type != kDecision || nd.n_kids > kStreamMaxActions) continue;
      double Rv[kStreamMaxActions];
      V sg[kStreamMaxActions];
      load_rows(G.R + (size_t)nd.row * stride + h, stride, nd.n_kids, Rv);
      if (G.M) {  // Predictive CFR+: regret matching of R + M
        double Mv[kStreamMaxActions];
        load_rows(G.M + (size_t)nd.row * stride + h, stride, nd.n_kids, Mv);
#pragma unroll
        for (int a = 0; a < kStreamMaxActions; ++a) Rv[a] += Mv[a];
      }
      regret_match<P>(Rv, nd.n_kids, sg);
#pragma unroll
      for (int a = 0; a < kStreamMaxActions; ++a)
        if (a < nd.n_kids) out[(size_t)(nd.row + a) * stride + h] = sg[a];
    }
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

// ------------------------------------------------------------------ wide schedule
//
// For one tree too large to stage in shared memory, each pass of the per-hand kernel
// becomes one launch per level in which every thread owns one (node, hand) pair: the hand
// index is the fastest-moving coordinate, so each warp reads and writes 32 consecutive
// entries of a row, and a level of n nodes runs n x hstride threads at once instead of
// stepping through its nodes in a few blocks.  The arithmetic per (node, hand) -- the order
// of every sum over children, regret matching, the Stage 7 update -- is the per-hand
// kernel's, so the schedules agree bit for bit.

constexpr int kWideThreads = 256;

// Bottom-up step at the inner nodes of one level (Stage 6, Eq. backward) for player p =
// blockIdx.y when both players are in the launch.  kModeUpdate: at p's decision nodes also
// the regrets, the Stage 7 update of R and S and the new strategy RM(R') (Eq. rm);
// kModeBR: the best-response value max_a v(child a) at p's decision nodes.
template <int MODE, typename P>
__global__ void __launch_bounds__(kWideThreads, 4) k_wide_back(const GameDev* __restrict__ games,
                                                            const int32_t* __restrict__ inner, int cnt,
                                                            int player_mask, const int* __restrict__ iter,
                                                            const Discount* __restrict__ disc_tab, int variant) {
  using V = typename P::V;
  pdl_wait();
  pdl_trigger();
  const GameDev& G = games[0];
  const int p = player_mask == 3 ? (int)blockIdx.y : (player_mask == 1 ? 0 : 1);
  const size_t S = (size_t)G.hstride;
  const size_t e = (size_t)blockIdx.x * kWideThreads + threadIdx.x;
  if (e >= (size_t)cnt * S) return;
  const int n = inner[e / S], h = (int)(e % S);
  if (h >= G.n_hands) return;
  const NodeDev nd = G.nodes[n];
  const size_t N = (size_t)G.n_nodes;
  V* v = static_cast<V*>(MODE == kModeBR ? G.cfv_br : G.cfv) + (size_t)p * N * S + h;
  const int A = nd.n_kids, k0 = nd.first_kid;
  V val;
  if (MODE == kModeBR && nd.type == kDecision && nd.player == p) {
    val = v[(size_t)k0 * S];
    for (int a = 1; a < A; ++a) val = P::vmax(val, v[(size_t)(k0 + a) * S]);
    v[(size_t)n * S] = val;
    return;
  }
  if (nd.type == kChance) {
    // children values already carry the card probabilities; cards in the hand are out
    const uint64_t hmask = G.hand_mask[h];
    typename P::Acc acc = P::acc0();
    for (int a = 0; a < A; ++a)
      if (!((hmask >> G.nodes[k0 + a].deal) & 1ull)) P::acc(acc, v[(size_t)(k0 + a) * S]);
    v[(size_t)n * S] = P::value(acc);
    return;
  }
  if (nd.player != p || MODE == kModeBR) {
    typename P::Acc acc = P::acc0();
    for (int a = 0; a < A; ++a) P::acc(acc, v[(size_t)(k0 + a) * S]);
    v[(size_t)n * S] = P::value(acc);
    return;
  }
  // p's decision node: value under the current strategy, then the Stage 7 update
  V* sgp = static_cast<V*>(G.sigma) + (size_t)nd.row * S + h;
  V c[kStreamMaxActions], sg[kStreamMaxActions];
  typename P::Acc acc = P::acc0();
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a)
    if (a < A) {
      c[a] = v[(size_t)(k0 + a) * S];
      sg[a] = sgp[(size_t)a * S];
      P::acc_mul(acc, sg[a], c[a]);
    }
  val = P::value(acc);
  v[(size_t)n * S] = val;
  const Discount d = disc_tab[*iter];
  const V pi = static_cast<const V*>(G.reach)[((size_t)p * N + n) * S + h];
  double* Rp = G.R + (size_t)nd.row * S + h;
  double* Sp = G.S + (size_t)nd.row * S + h;
  double* Mp = variant == 3 ? G.M + (size_t)nd.row * S + h : nullptr;
  double Rm[kStreamMaxActions];
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a) {
    Rm[a] = 0.0;
    if (a < A) {
      const V rr = P::sub(c[a], val);                          // instantaneous regret
      const double contrib = P::to_double(P::mul(pi, sg[a]));  // pi_i(I) sigma(I, a)
      const double rd = P::to_double(rr);
      double x = Rp[(size_t)a * S] + rd;
      if (variant == 2) x *= __double_as_longlong(x) > 0 ? d.dpos : d.dneg;
      if ((variant == 1 || variant == 3) && __double_as_longlong(x) < 0) x = 0.0;  // CFR+, Predictive CFR+
      const double sn = fma(Sp[(size_t)a * S], d.dS, (variant == 1 || variant == 3) ? d.wS * contrib : contrib);
      Rp[(size_t)a * S] = x;
      Sp[(size_t)a * S] = sn;
      Rm[a] = x;
      if (variant == 3) {
        Mp[(size_t)a * S] = rd;  // the prediction of the next regret
        Rm[a] = x + rd;          // Predictive CFR+ matches R + M
      }
    }
  }
  V sn[kStreamMaxActions];
  regret_match<P>(Rm, A, sn);
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a)
    if (a < A) sgp[(size_t)a * S] = sn[a];
}

// Strategy rows of player p (blockIdx.y when both): RM(R) (+ M for Predictive CFR+) into
// sigma (avg = 0), or the average S / sum S into sigbar (avg = 1), as the per-hand kernel
// computes them: positive parts in the value type, their sum in action order.
template <typename P>
__global__ void __launch_bounds__(kWideThreads) k_wide_rows(const GameDev* __restrict__ games, int player_mask,
                                                            int avg) {
  using V = typename P::V;
  pdl_wait();
  pdl_trigger();
  const GameDev& G = games[0];
  const int p = player_mask == 3 ? (int)blockIdx.y : (player_mask == 1 ? 0 : 1);
  const size_t S = (size_t)G.hstride;
  const int db = G.dec_begin[p], ndec = G.dec_begin[p + 1] - db;
  const size_t e = (size_t)blockIdx.x * kWideThreads + threadIdx.x;
  if (e >= (size_t)ndec * S) return;
  const int h = (int)(e % S);
  if (h >= G.n_hands) return;
  const NodeDev nd = G.nodes[G.dec_nodes[db + (int)(e / S)]];
  double x[kStreamMaxActions];
  load_rows((avg ? G.S : G.R) + (size_t)nd.row * S + h, S, nd.n_kids, x);
  if (!avg && G.M) {
    double m[kStreamMaxActions];
    load_rows(G.M + (size_t)nd.row * S + h, S, nd.n_kids, m);
#pragma unroll
    for (int a = 0; a < kStreamMaxActions; ++a) x[a] += m[a];
  }
  V sg[kStreamMaxActions];
  regret_match<P>(x, nd.n_kids, sg);
  V* out = static_cast<V*>(avg ? G.sigbar : G.sigma) + (size_t)nd.row * S + h;
#pragma unroll
  for (int a = 0; a < kStreamMaxActions; ++a)
    if (a < nd.n_kids) out[(size_t)a * S] = sg[a];
}

// Top-down step at the nodes of one level whose reach is stored (list[0 .. cnt)) (Stages
// 1-2): p's reach is the parent's times p's probability of the action, and zero for hands
// holding a dealt card.  Level 0 (the root) takes p's range.
template <typename P>
__global__ void __launch_bounds__(kWideThreads) k_wide_fwd(const GameDev* __restrict__ games,
                                                           const int32_t* __restrict__ list, int cnt,
                                                           int player_mask, int avg) {
  using V = typename P::V;
  pdl_wait();
  pdl_trigger();
  const GameDev& G = games[0];
  const int p = player_mask == 3 ? (int)blockIdx.y : (player_mask == 1 ? 0 : 1);
  const size_t S = (size_t)G.hstride;
  const size_t e = (size_t)blockIdx.x * kWideThreads + threadIdx.x;
  if (e >= (size_t)cnt * S) return;
  const int n = list[e / S], h = (int)(e % S);
  if (h >= G.n_hands) return;
  V* rch = static_cast<V*>(avg ? G.reach_bar : G.reach) + (size_t)p * G.n_nodes * S + h;
  if (n == 0) {
    rch[0] = static_cast<const V*>(G.range_v)[(size_t)p * S + h];
    return;
  }
  const NodeDev nd = G.nodes[n];
  V x = rch[(size_t)nd.parent * S];
  if (nd.aplayer == p) x = P::mul(x, static_cast<const V*>(avg ? G.sigbar : G.sigma)[(size_t)nd.arow * S + h]);
  if (nd.deal != kNoCard && ((G.hand_mask[h] >> nd.deal) & 1ull)) x = P::zero();
  rch[(size_t)n * S] = x;
}

// FP64 root sums of the best response, one block per player: sum_h r_p(h) v*_p(root, h),
// each thread over a fixed stride of hands, then a fixed-order tree in shared memory.
template <typename P>
__global__ void __launch_bounds__(kWideThreads) k_wide_root(const GameDev* __restrict__ games) {
  __shared__ double red[kWideThreads];
  pdl_wait();
  const GameDev& G = games[0];
  const int p = blockIdx.x;
  const size_t S = (size_t)G.hstride;
  using V = typename P::V;
  const V* v = static_cast<const V*>(G.cfv_br) + (size_t)p * G.n_nodes * S;
  double x = 0.0;
  for (int h = threadIdx.x; h < G.n_hands; h += kWideThreads) x += G.range64[(size_t)p * S + h] * P::to_double(v[h]);
  red[threadIdx.x] = x;
  __syncthreads();
  for (int o = kWideThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) G.br_out[p] = red[0];
}

__global__ void k_wide_advance(int* iter) {
  pdl_wait();
  *iter += 1;
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

size_t hand_smem_size(int n_nodes, int n_levels, int rows_max, int W, size_t es) {
  return hand_smem_bytes(n_nodes, n_levels, rows_max, W, es);
}

size_t resident_term_size(int n_hands, int hand_size, int deck, int hstride, size_t es) {
  return round16(resident_term_bytes(n_hands, hand_size, deck, hstride, es));
}
size_t resident_hand_size(int n_nodes, int n_levels, int rows_max, int W, size_t es) {
  return resident_hand_bytes(n_nodes, n_levels, rows_max, W, es);
}
int resident_blocks_per_sm(int precision, size_t smem) {
  int n = 0;
  const cudaError_t e =
      precision == kPrecisionSingle
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_resident<Single>, kTermThreads, smem)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_resident<Pairs>, kTermThreads, smem);
  return e == cudaSuccess ? n : 0;
}

// Every kernel asks for the same shared-memory carveout (the maximum), so the SMs never
// have to be reconfigured between the terminal and per-hand launches of an iteration.
template <typename K>
static cudaError_t configure_one(K kernel, int smem) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

template <typename P, bool SM>
static cudaError_t configure_hand() {
  const int smem = hand_kernel_smem_limit() - 4096;
  cudaError_t e = configure_one(k_hand<kModeInit, P, SM>, smem);
  if (e == cudaSuccess) e = configure_one(k_hand<kModeUpdate, P, SM>, smem);
  if (e == cudaSuccess) e = configure_one(k_hand<kModeAvg, P, SM>, smem);
  if (e == cudaSuccess) e = configure_one(k_hand<kModeBR, P, SM>, smem);
  return e;
}

template <typename P>
static cudaError_t configure_precision() {
  cudaError_t e = configure_hand<P, true>();
  if (e == cudaSuccess) e = configure_hand<P, false>();
  if (e == cudaSuccess) e = configure_one(k_terminal<P, false>, 200 * 1024);
  if (e == cudaSuccess) e = configure_one(k_terminal<P, true>, 200 * 1024);
  if (e == cudaSuccess) e = configure_one(k_average_rows<P>, 0);
  if (e == cudaSuccess) e = configure_one(k_stream_update<P, 1>, 200 * 1024);
  if (e == cudaSuccess) e = configure_one(k_stream_update<P, 2>, 200 * 1024);
  if (e == cudaSuccess) e = configure_one(k_current_rows<P>, 0);
  if (e == cudaSuccess) e = configure_one(k_resident<P>, 200 * 1024);
  return e;
}

int set_first_wait_polls(long polls) {
  const long v = polls < 0 ? kWaitLimit : polls;
  return cudaMemcpyToSymbol(g_first_wait_polls, &v, sizeof(v)) == cudaSuccess ? 0 : -1;
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

// Launch with programmatic stream serialisation (c.pdl) so the kernel may start while its
// predecessor finishes; kernels order their reads with pdl_wait().
template <typename... KArgs, typename... Args>
static cudaError_t launch_kernel(void (*kernel)(KArgs...), int grid, int block, size_t smem, void* stream, bool pdl,
                                 Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <int MODE, typename P>
static int launch_hand_p(const LaunchCtx& c, int player_mask, int advance, void* stream, bool pdl) {
  const int players = player_mask == 3 ? 2 : 1;
  const int grid = c.n_chunk_work * players;
  cudaError_t e;
  if (c.smem_hand > 0)
    e = launch_kernel(k_hand<MODE, P, true>, grid, kHandThreads, c.smem_hand, stream, pdl, c.games, c.chunk_work,
                      c.n_chunk_work, player_mask, advance, c.iter, c.done, c.disc, c.variant);
  else
    e = launch_kernel(k_hand<MODE, P, false>, grid, kHandThreads, 0, stream, pdl, c.games, c.chunk_work,
                      c.n_chunk_work, player_mask, advance, c.iter, c.done, c.disc, c.variant);
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of k_hand failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return check_launch("k_hand");
}

template <int MODE>
static int launch_hand(const LaunchCtx& c, int player_mask, int advance, void* stream, bool pdl) {
  return c.precision == kPrecisionSingle ? launch_hand_p<MODE, Single>(c, player_mask, advance, stream, pdl)
                                         : launch_hand_p<MODE, Pairs>(c, player_mask, advance, stream, pdl);
}

// ---- wide schedule: a pass is a sequence of per-level launches (host loop over levels)

static unsigned wide_blocks(size_t items) { return (unsigned)((items + kWideThreads - 1) / kWideThreads); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_wide(void (*kernel)(KArgs...), unsigned blocks, int players, void* stream, bool pdl,
                               Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, (unsigned)players);
  cfg.blockDim = dim3(kWideThreads);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <int MODE, typename P>
static cudaError_t wide_backward(const LaunchCtx& c, int player_mask, void* stream) {
  const int players = player_mask == 3 ? 2 : 1;
  const size_t S = (size_t)c.wide_stride;
  for (int l = c.wide_levels - 1; l >= 0; --l) {
    const int cnt = c.wide_inner_off[l + 1] - c.wide_inner_off[l];
    if (cnt == 0) continue;
    const cudaError_t e =
        launch_wide(k_wide_back<MODE, P>, wide_blocks((size_t)cnt * S), players, stream, c.pdl != 0, c.games,
                    c.wide_inner + c.wide_inner_off[l], cnt, player_mask, c.iter, c.disc, c.variant);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename P>
static cudaError_t wide_forward(const LaunchCtx& c, int player_mask, int avg, int first_level, void* stream) {
  const int players = player_mask == 3 ? 2 : 1;
  const size_t S = (size_t)c.wide_stride;
  for (int l = first_level; l < c.wide_levels; ++l) {
    const int a0 = c.wide_fwd_off[l], cnt = c.wide_fwd_off[l + 1] - a0;
    if (cnt == 0) continue;
    const cudaError_t e = launch_wide(k_wide_fwd<P>, wide_blocks((size_t)cnt * S), players, stream, c.pdl != 0,
                                      c.games, c.wide_fwd + a0, cnt, player_mask, avg);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename P>
static cudaError_t wide_rows(const LaunchCtx& c, int avg, void* stream) {
  // rows of both players: the larger player's decision-node count sizes the grid
  return launch_wide(k_wide_rows<P>, wide_blocks((size_t)c.wide_max_dec * c.wide_stride), 2, stream, c.pdl != 0,
                     c.games, 3, avg);
}

template <typename P>
static int wide_pass(const LaunchCtx& c, int which, int player_mask, int advance, void* stream) {
  cudaError_t e = cudaSuccess;
  if (which == kModeUpdate) {
    e = wide_backward<kModeUpdate, P>(c, player_mask, stream);
    if (e == cudaSuccess) e = wide_forward<P>(c, player_mask, 0, 1, stream);
    if (e == cudaSuccess && advance) e = launch_wide(k_wide_advance, 1, 1, stream, c.pdl != 0, c.iter);
  } else if (which == kModeInit || which == kModeAvg) {
    const int avg = which == kModeAvg;
    e = wide_rows<P>(c, avg, stream);
    if (e == cudaSuccess) e = wide_forward<P>(c, 3, avg, 0, stream);
  } else {  // kModeBR
    e = wide_backward<kModeBR, P>(c, 3, stream);
    if (e == cudaSuccess) e = launch_wide(k_wide_root<P>, 2, 1, stream, c.pdl != 0, c.games);
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of a wide-schedule kernel failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return check_launch("wide schedule");
}

static int launch_wide_pass(const LaunchCtx& c, int which, int player_mask, int advance, void* stream) {
  return c.precision == kPrecisionSingle ? wide_pass<Single>(c, which, player_mask, advance, stream)
                                         : wide_pass<Pairs>(c, which, player_mask, advance, stream);
}

int wide_launch_count(const LaunchCtx& c, int which, int player_mask, int advance) {
  int back = 0, fwd = 0;
  for (int l = 0; l < c.wide_levels; ++l) {
    back += c.wide_inner_off[l + 1] > c.wide_inner_off[l];
    fwd += c.wide_fwd_off[l + 1] > c.wide_fwd_off[l];
  }
  (void)player_mask;
  if (which == kModeUpdate) return back + (fwd - 1) + (advance ? 1 : 0);
  if (which == kModeInit || which == kModeAvg) return 1 + fwd;
  return back + 1;
}

int launch_init(const LaunchCtx& c, void* stream) {
  if (c.schedule == kScheduleWide) return launch_wide_pass(c, kModeInit, 3, 0, stream);
  return launch_hand<kModeInit>(c, 3, 0, stream, false);
}
template <typename P, int HP>
static int launch_stream_p(const LaunchCtx& c, int player_mask, int advance, void* stream) {
  const int players = player_mask == 3 ? 2 : 1;
  const int grid = c.n_warp_work * players;
  const size_t smem =
      stream_smem_size(c.stream_prog, c.stream_units, c.stream_half, c.stream_depth, sizeof(typename P::V), HP);
  const cudaError_t e = launch_kernel(k_stream_update<P, HP>, grid, kStreamWarps * 32, smem, stream, c.pdl != 0,
                                      c.games, c.warp_work, c.n_warp_work, player_mask, advance, c.iter, c.done,
                                      c.disc, c.variant, c.stream_depth, c.stream_prog, c.stream_units,
                                      c.stream_half);
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of k_stream_update failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return check_launch("k_stream_update");
}

int launch_update(const LaunchCtx& c, int player_mask, int advance, void* stream) {
  if (c.schedule == kScheduleWide) return launch_wide_pass(c, kModeUpdate, player_mask, advance, stream);
  if (c.schedule == kScheduleStream)
    return c.precision == kPrecisionSingle
               ? (c.stream_hp == 2 ? launch_stream_p<Single, 2>(c, player_mask, advance, stream)
                                   : launch_stream_p<Single, 1>(c, player_mask, advance, stream))
               : (c.stream_hp == 2 ? launch_stream_p<Pairs, 2>(c, player_mask, advance, stream)
                                   : launch_stream_p<Pairs, 1>(c, player_mask, advance, stream));
  return launch_hand<kModeUpdate>(c, player_mask, advance, stream, c.pdl != 0);
}

int launch_current_rows(const LaunchCtx& c, void* stream) {
  if (c.precision == kPrecisionSingle)
    k_current_rows<Single><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  else
    k_current_rows<Pairs><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  return check_launch("k_current_rows");
}
int launch_avg_reach(const LaunchCtx& c, void* stream) {
  if (c.schedule == kScheduleWide) return launch_wide_pass(c, kModeAvg, 3, 0, stream);
  return launch_hand<kModeAvg>(c, 3, 0, stream, false);
}
int launch_br(const LaunchCtx& c, void* stream) {
  if (c.schedule == kScheduleWide) return launch_wide_pass(c, kModeBR, 3, 0, stream);
  return launch_hand<kModeBR>(c, 3, 0, stream, c.pdl != 0);
}

int launch_terminal(const LaunchCtx& c, int player_mask, int use_bar, void* stream) {
  if (c.n_term_runs == 0) return 0;
  const int players = player_mask == 3 ? 2 : 1;
  const int grid = c.n_term_runs * players;
  const bool pdl = c.pdl != 0;
  cudaError_t e;
  const bool runs = c.n_term_runs < c.n_term_work;
  if (c.precision == kPrecisionSingle)
    e = runs ? launch_kernel(k_terminal<Single, true>, grid, kTermThreads, c.smem_term, stream, pdl, c.games,
                             c.term_work, c.term_src, c.term_runs, c.n_term_runs, player_mask, use_bar, c.err)
             : launch_kernel(k_terminal<Single, false>, grid, kTermThreads, c.smem_term, stream, pdl, c.games,
                             c.term_work, c.term_src, c.term_runs, c.n_term_runs, player_mask, use_bar, c.err);
  else
    e = runs ? launch_kernel(k_terminal<Pairs, true>, grid, kTermThreads, c.smem_term, stream, pdl, c.games,
                             c.term_work, c.term_src, c.term_runs, c.n_term_runs, player_mask, use_bar, c.err)
             : launch_kernel(k_terminal<Pairs, false>, grid, kTermThreads, c.smem_term, stream, pdl, c.games,
                             c.term_work, c.term_src, c.term_runs, c.n_term_runs, player_mask, use_bar, c.err);
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of k_terminal failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return check_launch("k_terminal");
}

// One cooperative launch: every block is resident at once, which the grid barriers need
// (the launch fails rather than run a grid that does not fit).
template <typename P>
static cudaError_t launch_resident_p(const LaunchCtx& c, int n_iters, void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.resident_grid);
  cfg.blockDim = dim3(kTermThreads);
  cfg.dynamicSmemBytes = c.smem_resident;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_resident<P>, c.games, c.chunk_work, c.n_chunk_work, c.term_work,
                            static_cast<const int32_t*>(c.term_src), c.n_term_work, c.alternating, n_iters, c.iter,
                            c.disc, c.variant, c.resident_sync, c.err, c.resident_term);
}

int launch_resident(const LaunchCtx& c, int n_iters, void* stream) {
  const cudaError_t e = c.precision == kPrecisionSingle ? launch_resident_p<Single>(c, n_iters, stream)
                                                        : launch_resident_p<Pairs>(c, n_iters, stream);
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of k_resident failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return check_launch("k_resident");
}

int launch_average_rows(const LaunchCtx& c, void* stream) {
  if (c.precision == kPrecisionSingle)
    k_average_rows<Single><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  else
    k_average_rows<Pairs><<<152, 256, 0, (cudaStream_t)stream>>>(c.games, c.n_games);
  return check_launch("k_average_rows");
}

}  // namespace pcfr
