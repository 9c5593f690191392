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

// One block per network row (leaf, river card): writes the row of X.
template <typename V>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_inputs(const GameDev* __restrict__ games, LeafCtx L,
                                                              int use_bar) {
  __shared__ float red[kLeafThreads / 32];
  const int row = blockIdx.x;
  const int li = row / kLeafCards, ri = row - li * kLeafCards;
  const LeafDev lf = L.leaves[li];
  const GameDev& G = games[lf.game];
  const NodeDev nd = G.nodes[lf.node];
  // the ri-th card not on the board
  int r = -1;
  for (int c = 0, k = 0; c < 52; ++c)
    if (!((nd.board >> c) & 1ull)) {
      if (k == ri) {
        r = c;
        break;
      }
      ++k;
    }
  const size_t stride = (size_t)G.hstride;
  const V* reach = static_cast<const V*>(use_bar ? G.reach_bar : G.reach);
  const int16_t* slot = L.slot + (size_t)lf.game * L.hstride_max;
  uint16_t* x = static_cast<uint16_t*>(L.X) + (size_t)row * kLeafIn;
  for (int k = threadIdx.x; k < kLeafIn; k += blockDim.x) x[k] = 0;
  // live hands hold neither a card of the leaf's board (the flop's turn card) nor r
  const uint64_t dead = nd.board | (1ull << r);
  float sum[2], cnt = 0.f;
  for (int p = 0; p < 2; ++p) {
    const V* q = reach + ((size_t)p * G.n_nodes + lf.node) * stride;
    float s = 0.f, n = 0.f;
    for (int h = threadIdx.x; h < G.n_hands; h += blockDim.x)
      if (!(G.hand_mask[h] & dead)) s += vf(q[h]), n += 1.f;
    sum[p] = block_sum(s, red);
    if (p == 0) cnt = block_sum(n, red);
  }
  __syncthreads();  // the zero fill is complete
  for (int p = 0; p < 2; ++p) {
    const V* q = reach + ((size_t)p * G.n_nodes + lf.node) * stride;
    // a player who never reaches the leaf: uniform over the hands (the values are then unused)
    const float inv = sum[p] > 0.f ? 1.f / sum[p] : 0.f;
    for (int h = threadIdx.x; h < G.n_hands; h += blockDim.x)
      if (!(G.hand_mask[h] & dead)) {
        const float v = sum[p] > 0.f ? vf(q[h]) * inv : 1.f / cnt;
        x[p * kLeafSlots + (L.hand_order ? h : slot[h])] = to_bf16(v);
      }
  }
  if (threadIdx.x < 52) {
    const bool on = ((nd.board >> threadIdx.x) & 1ull) || (int)threadIdx.x == r;
    if (on) x[2 * kLeafSlots + threadIdx.x] = 0x3f80;  // 1.0
  }
  if (threadIdx.x == 0) {
    x[2 * kLeafSlots + 52] = to_bf16(lf.feat[0]);
    x[2 * kLeafSlots + 53] = to_bf16(lf.feat[1]);
  }
}

// One block per leaf: the leaf values of player i.
template <typename V>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_values(const GameDev* __restrict__ games, LeafCtx L,
                                                              int i, int use_bar) {
  __shared__ float C[52];
  __shared__ float red[kLeafThreads / 32];
  const LeafDev lf = L.leaves[blockIdx.x];
  const GameDev& G = games[lf.game];
  const NodeDev nd = G.nodes[lf.node];
  const size_t stride = (size_t)G.hstride;
  const V* q = static_cast<const V*>(use_bar ? G.reach_bar : G.reach) + ((size_t)(1 - i) * G.n_nodes + lf.node) * stride;
  V* out = static_cast<V*>(use_bar ? G.cfv_br : G.cfv) + ((size_t)i * G.n_nodes + lf.node) * stride;
  const int16_t* slot = L.slot + (size_t)lf.game * L.hstride_max;
  const int16_t* hand_at = L.hand_at + (size_t)lf.game * kLeafSlots;
  // opponent totals: T and C[c] = sum over hands holding c (one warp per card, fixed order)
  float t = 0.f;
  for (int h = threadIdx.x; h < G.n_hands; h += blockDim.x) t += vf(q[h]);
  const float T = block_sum(t, red);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < 52; c += kLeafThreads / 32) {
    float s = 0.f;
    for (int h = lane; h < G.n_hands; h += 32)
      if ((G.hand_mask[h] >> c) & 1ull) s += vf(q[h]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C[c] = s;
  }
  __syncthreads();
  const float scale = (float)(G.payoff[lf.node] * G.kappa64);
  for (int h = threadIdx.x; h < G.n_hands; h += blockDim.x) {
    const uint64_t hm = G.hand_mask[h];
    int c1 = -1, c2 = -1;
    for (int c = 0; c < 52; ++c)
      if ((hm >> c) & 1ull) {
        if (c1 < 0) c1 = c;
        else c2 = c;
      }
    const float qh = vf(q[h]);
    const int s = slot[h];
    float acc = 0.f;
    for (int c = 0, ri = 0; c < 52; ++c) {
      if ((nd.board >> c) & 1ull) continue;
      const int row = lf.row0 + ri++;
      if ((hm >> c) & 1ull) continue;  // the hand holds the river card
      const int h1 = hand_at[pair_slot(c1, c)], h2 = hand_at[pair_slot(c2, c)];
      const float q1 = h1 >= 0 ? vf(q[h1]) : 0.f, q2 = h2 >= 0 ? vf(q[h2]) : 0.f;
      const float M = T - C[c] - (C[c1] - q1) - (C[c2] - q2) + qh;
      acc = fmaf(L.Y[(size_t)row * kLeafOut + i * kLeafSlots + (L.hand_order ? h : s)], M, acc);
    }
    const float v = ((nd.board & hm) ? 0.f : scale * acc);
    if constexpr (sizeof(V) == 4)
      out[h] = v;
    else
      out[h] = make_float2(v, 0.f);
  }
}

}  // namespace

int launch_leaf_inputs(const LaunchCtx& c, const LeafCtx& L, int use_bar, void* stream) {
  if (L.n_leaves == 0) return 0;
  const int rows = L.n_leaves * kLeafCards;
  if (c.precision == kPrecisionSingle)
    k_leaf_inputs<float><<<rows, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, use_bar);
  else
    k_leaf_inputs<float2><<<rows, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, use_bar);
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
  if (c.precision == kPrecisionSingle)
    k_leaf_values<float><<<L.n_leaves, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, player, use_bar);
  else
    k_leaf_values<float2><<<L.n_leaves, kLeafThreads, 0, (cudaStream_t)stream>>>(c.games, L, player, use_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pcfr
