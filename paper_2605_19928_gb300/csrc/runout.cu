// All-in run-outs evaluated in one step: the win-minus-loss tables E and the values
// u E q at each run-out's top node (see runout.h).
#include <cuda_runtime.h>

#include <cstdint>

#include "runout.h"

namespace pcfr {
namespace {

constexpr int kBuildThreads = 256;

// Thread (o, h) of table blockIdx.z: E[h][o] over the table's boards, stored at [o][h] with
// the table's bias (padding hands h >= n_hands hold E = 0).
__global__ void __launch_bounds__(kBuildThreads) k_runout_build(const RunoutTable* __restrict__ tables,
                                                                const RunoutBoard* __restrict__ boards,
                                                                const int32_t* __restrict__ gs,
                                                                const uint64_t* __restrict__ hand_mask, int H,
                                                                int ld, unsigned char* __restrict__ pool) {
  const RunoutTable tb = tables[blockIdx.z];
  const int o = blockIdx.y, h = blockIdx.x * kBuildThreads + threadIdx.x;
  if (h >= ld) return;
  int e = 0;
  if (h < H) {
    const uint64_t mo = hand_mask[o], mh = hand_mask[h];
    if (!(mo & mh)) {
      for (int b = 0; b < tb.n_boards; ++b) {
        const RunoutBoard bd = boards[tb.board0 + b];
        if (bd.cards & (mo | mh)) continue;  // a card of the board is in one of the hands
        const int32_t* g = gs + (size_t)bd.table * H;
        const int d = g[h] - g[o];
        e += (d > 0) - (d < 0);
      }
    }
  }
  const size_t at = (size_t)o * ld + h;
  if (tb.wide)
    reinterpret_cast<uint16_t*>(pool + tb.offset)[at] = (uint16_t)(e + 32768);
  else
    pool[tb.offset + at] = (uint8_t)(e + 128);
}

// An unsigned table entry x = E + bias as a float: x is placed in the mantissa of 2^23 (exact
// for x < 2^23), and the bias and 2^23 come off in one exact subtraction.
__device__ __forceinline__ float entry(uint32_t x, float bias) { return __uint_as_float(0x4b000000u | x) - bias; }

constexpr int kValueThreads = 128;  // 4 hands a thread: 512 hands a block

// Block (group, hand block, player): up to kRunoutGroup top nodes of one table; thread t owns
// hands 4t .. 4t + 3 of the block and, for each top g, sums E[h][o] q_g(o) over the opponent
// hands o in order (FP32), the tops' q staged in shared memory as [o][g]; each table row is
// loaded once for all the group's tops.  out = u_g times the sum.
template <typename T>
__global__ void __launch_bounds__(kValueThreads) k_runout_values(const GameDev* __restrict__ games,
                                                                 const RunoutItem* __restrict__ items,
                                                                 const RunoutGroup* __restrict__ groups,
                                                                 const RunoutTable* __restrict__ tables,
                                                                 const unsigned char* __restrict__ pool,
                                                                 int player_mask, int use_bar) {
  extern __shared__ float4 qs4[];  // [H][kRunoutGroup / 4]
  float* qs = reinterpret_cast<float*>(qs4);
  const GameDev& G = games[0];
  const RunoutGroup gr = groups[blockIdx.x];
  const int i = player_mask == 3 ? (int)blockIdx.z : (player_mask == 1 ? 0 : 1);
  const int H = G.n_hands;
  const size_t S = (size_t)G.hstride, N = (size_t)G.n_nodes;
  const float* reach = static_cast<const float*>(use_bar ? G.reach_bar : G.reach) + (size_t)(1 - i) * N * S;
  for (int x = threadIdx.x; x < kRunoutGroup * H; x += blockDim.x) {
    const int g = x / H, o = x - g * H;
    qs[o * kRunoutGroup + g] = g < gr.count ? reach[(size_t)items[gr.item0 + g].node * S + o] : 0.f;
  }
  __syncthreads();
  const int h0 = 4 * (int)(blockIdx.y * kValueThreads + threadIdx.x);
  if (h0 >= H) return;
  const RunoutTable tb = tables[gr.table];
  const T* F = reinterpret_cast<const T*>(pool + tb.offset) + h0;
  constexpr float bias = sizeof(T) == 1 ? 8388608.f + 128.f : 8388608.f + 32768.f;
  float acc[kRunoutGroup][4];
#pragma unroll
  for (int g = 0; g < kRunoutGroup; ++g)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[g][j] = 0.f;
#pragma unroll 2
  for (int o = 0; o < H; ++o) {
    float e[4];
    if constexpr (sizeof(T) == 1) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(F + (size_t)o * S));
      e[0] = entry(w & 0xffu, bias);
      e[1] = entry((w >> 8) & 0xffu, bias);
      e[2] = entry((w >> 16) & 0xffu, bias);
      e[3] = entry(w >> 24, bias);
    } else {
      const uint2 w = __ldg(reinterpret_cast<const uint2*>(F + (size_t)o * S));
      e[0] = entry(w.x & 0xffffu, bias);
      e[1] = entry(w.x >> 16, bias);
      e[2] = entry(w.y & 0xffffu, bias);
      e[3] = entry(w.y >> 16, bias);
    }
    const float4 qa = qs4[2 * o], qb = qs4[2 * o + 1];
    const float q[kRunoutGroup] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
    for (int g = 0; g < kRunoutGroup; ++g)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[g][j] = fmaf(e[j], q[g], acc[g][j]);
  }
#pragma unroll
  for (int g = 0; g < kRunoutGroup; ++g) {
    if (g >= gr.count) break;
    const RunoutItem it = items[gr.item0 + g];
    float* out = static_cast<float*>(use_bar ? G.cfv_br : G.cfv) + ((size_t)i * N + it.node) * S + h0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (h0 + j < H) out[j] = it.u * acc[g][j];
  }
}

}  // namespace

int launch_runout_build(const RunoutTable* tables, int n_tables, const RunoutBoard* boards, const int32_t* gs,
                        const uint64_t* hand_mask, int n_hands, int hstride, unsigned char* pool, void* stream) {
  if (n_tables == 0) return 0;
  const dim3 grid((unsigned)((hstride + kBuildThreads - 1) / kBuildThreads), (unsigned)n_hands, (unsigned)n_tables);
  k_runout_build<<<grid, kBuildThreads, 0, (cudaStream_t)stream>>>(tables, boards, gs, hand_mask, n_hands, hstride,
                                                                  pool);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_runout_values(const GameDev* games, const RunoutItem* items, const RunoutGroup* groups8, int n8,
                         const RunoutGroup* groups16, int n16, const RunoutTable* tables, const unsigned char* pool,
                         int n_hands, int player_mask, int use_bar, void* stream) {
  const unsigned players = player_mask == 3 ? 2u : 1u;
  const unsigned hand_blocks = (unsigned)((n_hands + 4 * kValueThreads - 1) / (4 * kValueThreads));
  const size_t smem = (size_t)n_hands * kRunoutGroup * sizeof(float);
  static_assert(kRunoutGroup == 8, "the staged reach is read as two float4 per opponent hand");
  if (n8 > 0)
    k_runout_values<uint8_t><<<dim3((unsigned)n8, hand_blocks, players), kValueThreads, smem, (cudaStream_t)stream>>>(
        games, items, groups8, tables, pool, player_mask, use_bar);
  if (n16 > 0)
    k_runout_values<uint16_t><<<dim3((unsigned)n16, hand_blocks, players), kValueThreads, smem,
                                (cudaStream_t)stream>>>(games, items, groups16, tables, pool, player_mask, use_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pcfr
