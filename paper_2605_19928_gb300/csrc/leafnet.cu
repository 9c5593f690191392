// Dense layers of the depth-limit leaf network (Section 3, depth-limited solving; Stage 5,
// Section 4.3): C = act(A B^T + bias) with A the [M][K] BF16 activations, B the [N][K] BF16
// weights (both K-major), FP32 accumulation on the 5th-generation tensor cores.
//
// A persistent kernel, one CTA per SM, walks 128 x BN tiles of C (BN = 256, 192 or 128,
// the largest that divides N; the N tiles of one block of rows are consecutive so that the
// CTAs reading that block of A run together and share it through L2):
//   * one lane of warp 0 streams 128 x 64 tiles of A and BN x 64 tiles of B into a 4-stage
//     ring of shared memory with TMA (128-byte swizzle, the layout the MMA descriptors below
//     describe);
//   * one lane of warp 1 issues tcgen05.mma (M 128, N BN, K 16 per instruction, four per
//     64-wide stage) into one of two TMEM accumulators, commits each stage back to its
//     "empty" barrier and each finished tile to its accumulator's "full" barrier;
//   * eight warps each read half the columns of one 32-lane quarter of the finished
//     accumulator with tcgen05.ld, add the bias, apply GELU (hidden layers), store BF16 (or
//     FP32, staged in shared memory and written by bulk tensor stores) and hand the
//     accumulator back, so a tile's epilogue runs while the next tile's MMAs fill the other.
// Every mbarrier wait is bounded; a wait that gives up sets *err, the CTA stops issuing,
// waits for the copies and MMAs it has in flight and frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "pcfr_internal.h"

namespace pcfr {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 4, kBNMax = 256;
constexpr int kATile = kBM * kBK * 2;        // 16 KB: one A stage
constexpr int kBTileMax = kBNMax * kBK * 2;  // 32 KB: one B stage of the widest tile
constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter, each half the columns
constexpr int kStageBufs = 8 / kEpiWarps;    // 4 KB output staging blocks per epilogue warp (32 KB in all)
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // warp 0 TMA, warp 1 MMA, then the epilogue warps
constexpr int kTmemCols = 512;               // two accumulators of up to 256 columns
constexpr long kGemmWaitLimit = 1l << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  for (long k = 0; k < kGemmWaitLimit; ++k)
    if (bar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 64 BF16
// (128 bytes), 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1,
// layout type 2 (128-byte swizzle).  The tile starts 1024-byte aligned; the K offset within
// the 128-byte row is added to the start address (32 bytes per MMA step of K = 16).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fffu);   // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused with swizzle): 16 B
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 1024 B between 8-row groups
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = bn,
// M = kBM.
__host__ __device__ constexpr uint32_t instr_desc(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ uint16_t to_bf16(float x) {  // round to nearest even (finite inputs)
  uint32_t u = __float_as_uint(x);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Hint: bring one box of the tensor into L2 (no shared memory, no barrier; a box past the
// tensor's end is not fetched).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

// Bulk tensor store shared -> global of one box (the issuing thread's bulk async-group).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const __grid_constant__ CUtensorMap map_c, const float* __restrict__ bias, void* __restrict__ out,
                int M, int N, int K, int bn, int act, int out_f32, int* err) {
  extern __shared__ __align__(1024) unsigned char smg[];
  // 1024-byte aligned stage buffers: A stages, then B stages
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smg) + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = base;
  unsigned char* sb = base + kStages * kATile;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int failed;  // set by any role whose bounded wait gave up; the others poll it
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_nt = N / bn, n_tiles = n_nt * ((M + kBM - 1) / kBM), kb_count = K / kBK;
  const uint32_t b_bytes = (uint32_t)bn * kBK * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&acc_full[b], 1);   // one tcgen05.commit per finished tile
      bar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
    }
    bar_init(&mma_done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int m0 = (tile / n_nt) * kBM, n0 = (tile % n_nt) * bn;
        const int next = tile + (int)gridDim.x, m0_next = (next / n_nt) * kBM;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % kStages;
          // the A box a full ring ahead (into the CTA's next tile near the end) goes to L2
          // now, so that its load, issued when a stage frees up, waits on L2 rather than DRAM
          if (kb + kStages < kb_count)
            tma_prefetch_2d(&map_a, (kb + kStages) * kBK, m0);
          else if (next < n_tiles && kb + kStages - kb_count < kb_count)
            tma_prefetch_2d(&map_a, (kb + kStages - kb_count) * kBK, m0_next);
          if (!bar_wait(&empty[s], ((uint32_t)(it / kStages) & 1u) ^ 1u)) {
            failed = 1;
            break;
          }
          bar_expect_tx(&full[s], kATile + b_bytes);
          tma_load_2d(sa + s * kATile, &map_a, kb * kBK, m0, &full[s]);
          tma_load_2d(sb + s * kBTileMax, &map_b, kb * kBK, n0, &full[s]);
        }
      }
      // the copies of the last round of each stage have landed before the CTA can leave
      for (int j = it - 1; j >= 0 && j >= it - kStages; --j) bar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = instr_desc(bn);
      int it = 0, lt = 0;
      for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x, ++lt) {
        const int acc = lt & 1;
        if (!bar_wait(&acc_empty[acc], ((uint32_t)(lt >> 1) & 1u) ^ 1u)) {  // the epilogue has drained it
          failed = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * kBNMax);
        bool ok = true;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % kStages;
          if (!bar_wait(&full[s], (uint32_t)(it / kStages) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_addr(sa + s * kATile), b0 = smem_addr(sb + s * kBTileMax);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            mma_bf16(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (!ok) {
          failed = 1;
          break;
        }
        mma_commit(&acc_full[acc]);  // the tile's accumulator is complete
      }
      mma_commit(&mma_done);  // every MMA issued above has completed
      bar_wait(&mma_done, 0);
    }
    __syncwarp();
  } else {  // epilogue: warp w reads accumulator lanes (rows) 32 (w % 4) .. + 31, columns of part
            // (w - 2) / 4 of the tile
    constexpr int parts = kEpiWarps / 4;  // warps per lane quarter, each a share of the columns
    const int q = warp & 3, part = (warp - 2) >> 2;
    const int c_begin = part * (bn / parts), c_end = c_begin + bn / parts;
    // FP32 output: 32 x 32 staging blocks in the TMA store's 128-byte-swizzled layout
    // (16-byte chunk j of row r at chunk j ^ (r % 8)), each written by the warp and stored by
    // one bulk tensor copy
    unsigned char* stage = sb + kStages * kBTileMax + (size_t)(warp - 2) * kStageBufs * 4096;
    int cc = 0;  // 32-column blocks this warp has staged
    int lt = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++lt) {
      const int acc = lt & 1;
      const bool ok = bar_wait(&acc_full[acc], (uint32_t)(lt >> 1) & 1u);
      if (!__all_sync(0xffffffffu, ok) || failed) {
        if (lane == 0) failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = (tile / n_nt) * kBM, n0 = (tile % n_nt) * bn;
      const int row = m0 + q * 32 + lane;
      for (int c0 = c_begin; c0 < c_end; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBNMax + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int col = n0 + c0;
        if (out_f32) {
          unsigned char* buf = stage + (cc % kStageBufs) * 4096;
          if (cc >= kStageBufs) {  // the store that last read this block has finished reading it
            if (lane == 0) {
              if (kStageBufs == 2)
                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
              else
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
            __syncwarp();
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              y[e] = __uint_as_float(v[4 * j + e]) + (bias ? bias[col + 4 * j + e] : 0.f);
              if (act) y[e] = gelu(y[e]);
            }
            *reinterpret_cast<float4*>(buf + lane * 128 + ((j ^ (lane & 7)) << 4)) = make_float4(y[0], y[1], y[2], y[3]);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the bulk copy
          __syncwarp();
          if (lane == 0) tma_store_2d(&map_c, col, m0 + q * 32, buf);  // rows past M are clipped
          ++cc;
        } else if (row < M) {
          float y[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            y[j] = __uint_as_float(v[j]) + (bias ? bias[col + j] : 0.f);
            if (act) y[j] = gelu(y[j]);
          }
          {
            uint4* dst = reinterpret_cast<uint4*>(static_cast<uint16_t*>(out) + (size_t)row * N + col);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint32_t w[4];
#pragma unroll
              for (int e = 0; e < 4; ++e)
                w[e] = (uint32_t)to_bf16(y[8 * j + 2 * e]) | ((uint32_t)to_bf16(y[8 * j + 2 * e + 1]) << 16);
              dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&acc_empty[acc]);  // this quarter of the accumulator is free
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // every store has completed
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// Row-major [rows][cols] FP32 matrix, 32 x 32 boxes with 128-byte swizzle (the epilogue's
// bulk stores).
bool encode_out_f32(CUtensorMap* map, void* ptr, int rows, int cols) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Row-major [rows][cols] BF16 matrix, box_rows x 64 boxes with 128-byte swizzle.
bool encode(CUtensorMap* map, const void* ptr, int rows, int cols, int box_rows) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// stages of A and B, the epilogue warps' 4 KB output staging blocks, alignment slack
size_t gemm_smem_bytes() { return (size_t)kStages * (kATile + kBTileMax) + kEpiWarps * kStageBufs * 4096 + 1024; }

int configure_gemm() {
  return cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes()) ==
                 cudaSuccess
             ? 0
             : -1;
}

int launch_gemm_bf16(const void* A, const void* B, const float* bias, void* C, int M, int N, int K, int act,
                     int out_f32, int* err, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || N % 128 || K % kBK) return -2;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) return -2;
  const int bn = N % 256 == 0 ? 256 : N % 192 == 0 ? 192 : 128;  // the widest tile that divides N
  const long tiles = (long)(N / bn) * ((M + kBM - 1) / kBM);
  if (tiles > (1l << 30)) return -2;
  CUtensorMap ma, mb, mc = {};
  if (!encode(&ma, A, M, K, kBM) || !encode(&mb, B, N, K, bn)) return -3;
  if (out_f32 && !encode_out_f32(&mc, C, M, N)) return -3;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return -1;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);  // persistent: one CTA per SM
  k_gemm_bf16<<<grid, kGemmThreads, gemm_smem_bytes(), (cudaStream_t)stream>>>(ma, mb, mc, bias, C, M, N, K, bn,
                                                                               act, out_f32, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "pcfr: launch of k_gemm_bf16 failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  return 0;
}

// ------------------------------------------------------------------ leaf inputs and values
//
// Depth-limit leaves (Section 3: a network maps both players' normalised reach and the public
// state to counterfactual values; Stage 5 evaluates all leaves in one batch, Section 4.3).
// Each leaf is a river-card chance node; the network is evaluated once per river card r
// that is not on the board, on the board completed by r.  The value of hand h of player i
// at leaf n is then
//     v_i(n, h) = payoff(n) kappa  sum_{r not in h}  y_i^r(h) M_r(h)
// with payoff(n) = pot at n x P(river card) (1/44 given both hands), y_i^r(h) the network's
// value per unit pot of h, and M_r(h) the opponent reach at n over hands sharing no card
// with h or r (inclusion-exclusion as at fold nodes, with the river card removed).

namespace {

constexpr int kLeafThreads = 256;

template <typename V>
__device__ __forceinline__ float vf(const V& x);
template <>
__device__ __forceinline__ float vf<float>(const float& x) { return x; }
template <>
__device__ __forceinline__ float vf<float2>(const float2& x) { return x.x + x.y; }

__device__ __forceinline__ float block_sum(float x, float* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  float t = 0.f;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];  // fixed order
  return t;
}

// Slot of the two-card hand {a, b} (a != b): b (b - 1) / 2 + a with a < b.
__device__ __forceinline__ int pair_slot(int a, int b) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return b * (b - 1) / 2 + a;
}

// Per input column of a leaf's rows, what the column depends on: the reach of the hand it
// holds (player p = column / kLeafSlots) and that hand's two cards.
constexpr int kLeafChunks = kLeafIn / 8;                 // 16-byte chunks of a row of X (344)
constexpr int kLeafHandChunks = 2 * kLeafSlots / 8;      // chunks of player columns only (331)
constexpr int kLeafInThreads = 352;                      // one thread per chunk (11 warps)
constexpr int kLeafInWarps = kLeafInThreads / 32;
constexpr int kStageCols = (kLeafIn + kLeafInThreads - 1) / kLeafInThreads;  // columns per thread
constexpr uint16_t kNoHand = 0xffffu;                    // no hand, or one holding a board card
static_assert((2 * kLeafSlots + 52) % 8 == 0, "the two features open a 16-byte chunk");

// The k-th card not on a leaf's board (its board holds 4 cards; c stays a card regardless).
__device__ __forceinline__ int river_card(uint64_t board, int k) {
  int c = 0;
  for (int n = -1; c < 51; ++c)
    if (!((board >> c) & 1ull) && ++n == k) break;
  return c;
}

// Two floats to BF16 (round to nearest even), lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ float warp_sum_f32(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ int warp_sum_i32(int x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block (leaf, part): rows [part R, part R + R) of the leaf's kLeafCards rows of X, R =
// kLeafCards / gridDim.y, one contiguous span written in 16-byte chunks (thread j writes chunk
// j of every row).  For river card r the inputs of player p are p's reach over the hands
// holding neither a board card nor r, divided by their sum; a player with no such hand of
// positive reach gets the uniform range over them (its values are then unused).  The sum is
// the total of p's reach over the hands live on the board less the sum over the (at most 51)
// of them holding r, both in FP32 in a fixed order: the total is at most 24 roundings deep
// (8 terms a thread, 5 tree levels, 11 warps) and the held sum 7, so the difference is within
// 2e-6 of the total.  Where the difference is below 2e-3 of the total (more than 99.8 % of
// the reach on hands holding r) that bound is no longer 1e-3 of the result, and the sum is
// taken directly over the hands instead.  The rows are written without regard to r, then the columns of the
// hands holding r are cleared in each row.
template <typename V>
__global__ void __launch_bounds__(kLeafInThreads) k_leaf_inputs(const GameDev* __restrict__ games, LeafCtx L,
                                                                int use_bar) {
  __shared__ __align__(16) float qc[kLeafIn];       // reach of each column's live hand (0: none)
  __shared__ __align__(16) uint16_t cc[kLeafIn];    // its cards c1 | c2 << 8, or kNoHand
  __shared__ int16_t col_of[kLeafSlots];            // column of the hand in each slot, or -1
  __shared__ float mul[2][kLeafCards], add[2][kLeafCards];
  __shared__ int rc[kLeafCards];                    // this block's river cards, ascending
  __shared__ int slow_row[kLeafCards];              // a player of the row takes the uniform range
  __shared__ float tot_w[2][kLeafInWarps];
  __shared__ int cnt_w[3][kLeafInWarps];
  const LeafDev lf = L.leaves[blockIdx.x];
  const GameDev& G = games[lf.game];
  const NodeDev nd = G.nodes[lf.node];
  const int R = kLeafCards / gridDim.y, k0 = blockIdx.y * R;
  const int nh = G.n_hands < kLeafSlots ? G.n_hands : kLeafSlots;
  const size_t stride = (size_t)G.hstride;
  const V* reach = static_cast<const V*>(use_bar ? G.reach_bar : G.reach);
  const int16_t* hand_at = L.hand_at + (size_t)lf.game * kLeafSlots;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // stage the columns: three rounds of independent loads (slot table, hand masks, reach)
  {
    int hs[kStageCols], h[kStageCols];
    uint64_t m[kStageCols];
#pragma unroll
    for (int u = 0; u < kStageCols; ++u) {
      const int col = threadIdx.x + u * kLeafInThreads;
      const int p = col >= kLeafSlots, s = col - p * kLeafSlots;
      hs[u] = col < 2 * kLeafSlots && (p == 0 || !L.hand_order) ? hand_at[s] : -1;
    }
#pragma unroll
    for (int u = 0; u < kStageCols; ++u) {
      const int col = threadIdx.x + u * kLeafInThreads;
      const int p = col >= kLeafSlots, s = col - p * kLeafSlots;
      h[u] = col >= 2 * kLeafSlots ? -1 : L.hand_order ? (s < nh ? s : -1) : hs[u];
      m[u] = h[u] >= 0 ? G.hand_mask[h[u]] : 0ull;
      if (col < kLeafSlots) col_of[s] = (int16_t)(hs[u] < 0 ? -1 : (L.hand_order ? hs[u] : s));
    }
    float t0 = 0.f, t1 = 0.f;
    int n = 0, pos0 = 0, pos1 = 0;
#pragma unroll
    for (int u = 0; u < kStageCols; ++u) {
      const int col = threadIdx.x + u * kLeafInThreads;
      if (col >= kLeafIn) break;
      const int p = col >= kLeafSlots;
      const bool live = h[u] >= 0 && !(m[u] & nd.board);
      const float q = live ? vf(reach[((size_t)p * G.n_nodes + lf.node) * stride + h[u]]) : 0.f;
      qc[col] = q;
      cc[col] = live ? (uint16_t)((__ffsll((long long)m[u]) - 1) | ((63 - __clzll((long long)m[u])) << 8)) : kNoHand;
      if (p == 0) t0 += q, n += live, pos0 += q > 0.f;
      else t1 += q, pos1 += q > 0.f;
    }
    t0 = warp_sum_f32(t0);
    t1 = warp_sum_f32(t1);
    n = warp_sum_i32(n);
    pos0 = warp_sum_i32(pos0);
    pos1 = warp_sum_i32(pos1);
    if (lane == 0) {
      tot_w[0][warp] = t0;
      tot_w[1][warp] = t1;
      cnt_w[0][warp] = n;
      cnt_w[1][warp] = pos0;
      cnt_w[2][warp] = pos1;
    }
  }
  if ((int)threadIdx.x < R) {
    rc[threadIdx.x] = river_card(nd.board, k0 + threadIdx.x);
    slow_row[threadIdx.x] = 0;
  }
  __syncthreads();
  // per (player, river card): the sum over the hands holding r, one warp each
  for (int item = warp; item < 2 * R; item += kLeafInWarps) {
    const int p = item / R, k = item - p * R, r = rc[k];
    float c = 0.f;
    int nr = 0, posr = 0;
    for (int x = lane; x < 52; x += 32) {
      const int col = x == r ? -1 : col_of[pair_slot(r, x)];
      if (col >= 0) {
        const float q = qc[p * kLeafSlots + col];
        c += q;
        nr += cc[p * kLeafSlots + col] != kNoHand;
        posr += q > 0.f;
      }
    }
    c = warp_sum_f32(c);
    nr = warp_sum_i32(nr);
    posr = warp_sum_i32(posr);
    float tot = 0.f;
    int n = 0, pos = 0;
    for (int w = 0; w < kLeafInWarps; ++w) tot += tot_w[p][w], n += cnt_w[0][w], pos += cnt_w[1 + p][w];
    const int live = n - nr;  // hands holding neither a board card nor r
    float s = 0.f;
    if (pos - posr > 0) {
      const float d = tot - c;
      if (d > 2e-3f * tot) {
        s = d;
      } else {  // most of the reach on hands holding r: sum directly
        float a = 0.f;
        for (int j = lane; j < kLeafSlots; j += 32) {
          const uint32_t cards = cc[p * kLeafSlots + j];
          if (cards != kNoHand && (cards & 0xffu) != (uint32_t)r && (cards >> 8) != (uint32_t)r)
            a += qc[p * kLeafSlots + j];
        }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        s = a;
      }
    }
    if (lane == 0) {  // input = q mul + add
      // (finite, so that a column with no hand, q = 0, stays 0 when the sum is subnormal)
      mul[p][k] = s > 0.f ? fminf(1.f / s, 3.402823466e38f) : 0.f;
      add[p][k] = s > 0.f || live == 0 ? 0.f : 1.f / (float)live;
      if (!(s > 0.f)) slow_row[k] = 1;
    }
  }
  __syncthreads();
  uint16_t* Xb = static_cast<uint16_t*>(L.X) + (size_t)(lf.row0 + k0) * kLeafIn;
  const int j = threadIdx.x;
  if (j < kLeafChunks) {
    float q[8];
    uint32_t dead = 0, p1 = 0, board_on = 0;  // per column: no live hand; player 1; board card
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = 8 * j + e;
      q[e] = qc[col];
      dead |= (cc[col] == kNoHand ? 1u : 0u) << e;
      p1 |= (col >= kLeafSlots ? 1u : 0u) << e;
      const int c = col - 2 * kLeafSlots;
      board_on |= (c >= 0 && c < 52 && ((nd.board >> c) & 1ull) ? 1u : 0u) << e;
    }
    const int p = 8 * j >= kLeafSlots;
    const bool one_player = j < kLeafHandChunks && (8 * j + 7 < kLeafSlots || 8 * j >= kLeafSlots);
    const bool features = 8 * j == 2 * kLeafSlots + 52;
    uint4* X = reinterpret_cast<uint4*>(Xb) + j;
    for (int k = 0; k < R; ++k) {
      uint4 out;
      if (one_player && !slow_row[k]) {  // a dead column has q = 0
        const float mk = mul[p][k];
        out = make_uint4(pack_bf16x2(q[0] * mk, q[1] * mk), pack_bf16x2(q[2] * mk, q[3] * mk),
                         pack_bf16x2(q[4] * mk, q[5] * mk), pack_bf16x2(q[6] * mk, q[7] * mk));
      } else {  // the chunk straddling the players, the tail, and rows with a uniform range
        const float m0 = mul[0][k], m1 = mul[1][k], a0 = add[0][k], a1 = add[1][k];
        const int rpos = 2 * kLeafSlots + rc[k] - 8 * j;  // the river card's one-hot column
        const uint32_t ones = board_on | (rpos >= 0 && rpos < 8 ? 1u << rpos : 0u);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const bool pe = (p1 >> e) & 1u;
          v[e] = (dead >> e) & 1u ? 0.f : fmaf(q[e], pe ? m1 : m0, pe ? a1 : a0);
          if ((ones >> e) & 1u) v[e] = 1.f;
        }
        if (features) {  // both features open this chunk
          v[0] = lf.feat[0];
          v[1] = lf.feat[1];
        }
        out = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                         pack_bf16x2(v[6], v[7]));
      }
      X[(size_t)k * kLeafChunks] = out;
    }
  }
  __syncthreads();  // the rows are written; clear the columns of the hands holding each r
  for (int t = threadIdx.x; t < R * 52; t += blockDim.x) {
    const int k = t / 52, x = t - k * 52, r = rc[k];
    if (x == r) continue;
    const int col = col_of[pair_slot(r, x)];
    if (col >= 0) {
      uint16_t* row = Xb + (size_t)k * kLeafIn;
      row[col] = 0;
      row[kLeafSlots + col] = 0;
    }
  }
}

// Block (leaf, part): the leaf values of player i for part of the leaf's hands.  The
// opponent's reach is staged as a 52 x 52 table over card pairs (0 where no hand); the totals
// T and C[c] (reach of the hands holding card c: the row of c, one warp per card, fixed order)
// and T - C[r] per river card r feed the inclusion-exclusion of each (hand, river card) term.
template <typename V>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_values(const GameDev* __restrict__ games, LeafCtx L,
                                                              int i, int use_bar) {
  struct RiverCard {
    int c;     // the card
    float tc;  // T - C[c]
  };
  __shared__ float Q2[52 * 52];
  __shared__ float C[52];
  __shared__ RiverCard rt[kLeafCards];
  __shared__ float red[kLeafThreads / 32];
  const LeafDev lf = L.leaves[blockIdx.x];
  const GameDev& G = games[lf.game];
  const NodeDev nd = G.nodes[lf.node];
  const int nh = G.n_hands < kLeafSlots ? G.n_hands : kLeafSlots;
  const size_t stride = (size_t)G.hstride;
  const V* q = static_cast<const V*>(use_bar ? G.reach_bar : G.reach) + ((size_t)(1 - i) * G.n_nodes + lf.node) * stride;
  V* out = static_cast<V*>(use_bar ? G.cfv_br : G.cfv) + ((size_t)i * G.n_nodes + lf.node) * stride;
  const int16_t* slot = L.slot + (size_t)lf.game * L.hstride_max;
  for (int x = threadIdx.x; x < 52 * 52; x += blockDim.x) Q2[x] = 0.f;
  if (threadIdx.x < kLeafCards) rt[threadIdx.x].c = river_card(nd.board, threadIdx.x);
  __syncthreads();
  float t = 0.f;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    const uint64_t m = G.hand_mask[h];
    const int a = __ffsll((long long)m) - 1, b = 63 - __clzll((long long)m);
    const float x = vf(q[h]);
    Q2[a * 52 + b] = x;
    Q2[b * 52 + a] = x;
    t += x;
  }
  const float T = block_sum(t, red);  // its barriers also publish Q2
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < 52; c += kLeafThreads / 32) {
    float s = Q2[c * 52 + lane];
    if (lane < 20) s += Q2[c * 52 + 32 + lane];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[c] = s;
  }
  __syncthreads();
  if (threadIdx.x < kLeafCards) rt[threadIdx.x].tc = T - C[rt[threadIdx.x].c];
  __syncthreads();
  const float scale = (float)(G.payoff[lf.node] * G.kappa64);
  const float* Y = L.Y + (size_t)lf.row0 * kLeafOut + i * kLeafSlots;
  const int per = (nh + gridDim.y - 1) / gridDim.y, h1 = min(nh, ((int)blockIdx.y + 1) * per);
  for (int h = blockIdx.y * per + threadIdx.x; h < h1; h += blockDim.x) {
    const uint64_t hm = G.hand_mask[h];
    const int c1 = __ffsll((long long)hm) - 1, c2 = 63 - __clzll((long long)hm);
    const float* q1row = Q2 + c1 * 52;
    const float* q2row = Q2 + c2 * 52;
    const float qh = q1row[c2], C1 = C[c1], C2 = C[c2];
    const float* y = Y + (L.hand_order ? h : slot[h]);
    float acc = 0.f;
#pragma unroll 16
    for (int k = 0; k < kLeafCards; ++k) {
      const RiverCard e = rt[k];
      const float yk = __ldg(y + (size_t)k * kLeafOut);
      if (e.c == c1 || e.c == c2) continue;  // the hand holds the river card
      const float M = e.tc - (C1 - q1row[e.c]) - (C2 - q2row[e.c]) + qh;
      acc = fmaf(yk, M, acc);
    }
    const float v = ((nd.board & hm) ? 0.f : scale * acc);
    if constexpr (sizeof(V) == 4)
      out[h] = v;
    else
      out[h] = make_float2(v, 0.f);
  }
}

}  // namespace

// Blocks per leaf (a divisor of n) so that n_leaves x parts fills the GPU about `waves` times.
static int leaf_parts(int n_leaves, int n, int waves) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  int parts = 1;
  while (parts < n && (long long)n_leaves * parts < (long long)waves * sms) {
    ++parts;
    while (n % parts) ++parts;
  }
  return parts;
}

int launch_leaf_inputs(const LaunchCtx& c, const LeafCtx& L, int use_bar, void* stream) {
  if (L.n_leaves == 0) return 0;
  const dim3 grid((unsigned)L.n_leaves, (unsigned)leaf_parts(L.n_leaves, kLeafCards, 8));
  if (c.precision == kPrecisionSingle)
    k_leaf_inputs<float><<<grid, kLeafInThreads, 0, (cudaStream_t)stream>>>(c.games, L, use_bar);
  else
    k_leaf_inputs<float2><<<grid, kLeafInThreads, 0, (cudaStream_t)stream>>>(c.games, L, use_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_leaf_net(const LaunchCtx& c, const LeafCtx& L, void* stream) {
  if (L.n_leaves == 0) return 0;
  const int rows = L.n_leaves * kLeafCards;
  if (launch_gemm_bf16(L.X, L.W[0], L.b[0], L.H1, rows, kLeafHidden, kLeafIn, 1, 0, c.err, stream) ||
      launch_gemm_bf16(L.H1, L.W[1], L.b[1], L.H2, rows, kLeafHidden, kLeafHidden, 1, 0, c.err, stream) ||
      launch_gemm_bf16(L.H2, L.W[2], L.b[2], L.H3, rows, kLeafHidden, kLeafHidden, 1, 0, c.err, stream) ||
      launch_gemm_bf16(L.H3, L.W[3], L.b[3], L.Y, rows, kLeafOut, kLeafHidden, 0, 1, c.err, stream))
    return -1;
  return 0;
}

int launch_leaf_values(const LaunchCtx& c, const LeafCtx& L, int player, int use_bar, void* stream) {
  if (L.n_leaves == 0) return 0;
  // at most kLeafThreads hands per block, and enough blocks to fill the GPU about 4 times
  const int per_block = (L.hstride_max + kLeafThreads - 1) / kLeafThreads;
  int parts = leaf_parts(L.n_leaves, 16, 4);
  if (parts < per_block) parts = per_block;
  const dim3 grid((unsigned)L.n_leaves, (unsigned)parts);
  if (c.precision == kPrecisionSingle)
    k_leaf_values<float><<<grid, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, player, use_bar);
  else
    k_leaf_values<float2><<<grid, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, player, use_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pcfr
