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

// Block (item, player): thread t owns hands 4t .. 4t + 3 and sums E[h][o] q(o) over the
// opponent hands o in order (FP32), q staged in shared memory; out = u times the sum.
template <typename T>
__global__ void k_runout_values(const GameDev* __restrict__ games, const RunoutItem* __restrict__ items,
                                const RunoutTable* __restrict__ tables, const unsigned char* __restrict__ pool,
                                int player_mask, int use_bar) {
  extern __shared__ float qs[];
  const GameDev& G = games[0];
  const RunoutItem it = items[blockIdx.x];
  const int i = player_mask == 3 ? (int)blockIdx.y : (player_mask == 1 ? 0 : 1);
  const int H = G.n_hands;
  const size_t S = (size_t)G.hstride, N = (size_t)G.n_nodes;
  const float* q = static_cast<const float*>(use_bar ? G.reach_bar : G.reach) + ((size_t)(1 - i) * N + it.node) * S;
  for (int o = threadIdx.x; o < H; o += blockDim.x) qs[o] = q[o];
  __syncthreads();
  const int h0 = 4 * (int)threadIdx.x;
  if (h0 >= H) return;
  const RunoutTable tb = tables[it.table];
  const T* F = reinterpret_cast<const T*>(pool + tb.offset) + h0;
  constexpr float bias = sizeof(T) == 1 ? 8388608.f + 128.f : 8388608.f + 32768.f;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
  for (int o = 0; o < H; ++o) {
    const float qo = qs[o];
    if constexpr (sizeof(T) == 1) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(F + (size_t)o * S));
      a0 = fmaf(entry(w & 0xffu, bias), qo, a0);
      a1 = fmaf(entry((w >> 8) & 0xffu, bias), qo, a1);
      a2 = fmaf(entry((w >> 16) & 0xffu, bias), qo, a2);
      a3 = fmaf(entry(w >> 24, bias), qo, a3);
    } else {
      const uint2 w = __ldg(reinterpret_cast<const uint2*>(F + (size_t)o * S));
      a0 = fmaf(entry(w.x & 0xffffu, bias), qo, a0);
      a1 = fmaf(entry(w.x >> 16, bias), qo, a1);
      a2 = fmaf(entry(w.y & 0xffffu, bias), qo, a2);
      a3 = fmaf(entry(w.y >> 16, bias), qo, a3);
    }
  }
  float* out = static_cast<float*>(use_bar ? G.cfv_br : G.cfv) + ((size_t)i * N + it.node) * S + h0;
  const float a[4] = {a0, a1, a2, a3};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (h0 + j < H) out[j] = it.u * a[j];
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

int launch_runout_values(const GameDev* games, const RunoutItem* items8, int n8, const RunoutItem* items16, int n16,
                         const RunoutTable* tables, const unsigned char* pool, int n_hands, int hstride,
                         int player_mask, int use_bar, void* stream) {
  const unsigned players = player_mask == 3 ? 2u : 1u;
  const unsigned threads = (unsigned)(((hstride + 3) / 4 + 31) / 32 * 32);
  const size_t smem = (size_t)n_hands * sizeof(float);
  if (n8 > 0)
    k_runout_values<uint8_t><<<dim3((unsigned)n8, players), threads, smem, (cudaStream_t)stream>>>(
        games, items8, tables, pool, player_mask, use_bar);
  if (n16 > 0)
    k_runout_values<uint16_t><<<dim3((unsigned)n16, players), threads, smem, (cudaStream_t)stream>>>(
        games, items16, tables, pool, player_mask, use_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pcfr
