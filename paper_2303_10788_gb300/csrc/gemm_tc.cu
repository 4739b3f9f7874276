// Tensor-core split-K GEMM of the recombination in BF16 (Sec. V-C's
// contraction over the 4^k cut index, written as C = Q_hub x R').
//
// One CTA per (128-row M tile, K split), six warps.  Warp 0 lane 0 streams A
// (the hub operand, M x K bf16, K-major) and B (R'^T, N x K bf16, K-major)
// tiles of 64 along K through an 8-stage shared-memory ring with TMA
// (cp.async.bulk.tensor, 128-byte swizzle).  Warp 1 lane 0 issues tcgen05.mma
// (kind::f16, bf16 x bf16 -> f32, M = 128, N = 16 or 32, K = 16 per
// instruction) into one of two tensor-memory accumulators, switching every 4
// K-tiles.  The signed terms of the contraction cancel heavily, so long
// tensor-core accumulations lose accuracy: warps 2-5 drain each finished
// accumulator (256 products) with tcgen05.ld into Kahan-compensated FP32
// registers while the other accumulator fills, then write the FP32 partial
// tile.  Split-K partials are summed in FP64 by the common reduction kernel.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the
// kernel records an error bit in the status word, stops issuing, waits
// (bounded) for its own copies in flight, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "kernels.cuh"

namespace ccs {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 8;
constexpr unsigned long long kWaitBudget = 2000000000ull;   // ~1 s of SM clocks

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}

// true once the phase with parity `phase` has completed; false after the budget
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const unsigned long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(s_addr(bar)), "r"(phase)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitBudget) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          s_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(s_addr(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows with the
// 128-byte swizzle; 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile) {
  const uint64_t a = s_addr(tile);
  uint64_t d = (a & 0x3FFFFull) >> 4;       // start address
  d |= (uint64_t)(16 >> 4) << 16;           // leading-dimension offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride between 8-row groups
  d |= 1ull << 46;                          // descriptor version
  d |= 2ull << 61;                          // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

constexpr int kGroup = 4;   // K-tiles per tensor-memory accumulation

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
}

__global__ void __launch_bounds__(192, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
                        int N, int k_tiles, int tiles_per_split, int mtiles, float* partials, unsigned* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = kBM * kBK * 2, b_bytes = N * kBK * 2;
  uint8_t* A_s = smem;
  uint8_t* B_s = smem + kStages * a_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(B_s + kStages * b_bytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;      // [2]: accumulator b complete
  uint64_t* acc_empty = acc_full + 2;        // [2]: accumulator b drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x % mtiles, split = blockIdx.x / mtiles;
  const int kt0 = split * tiles_per_split;
  const int kt1 = min(k_tiles, kt0 + tiles_per_split);
  const int nk = kt1 > kt0 ? kt1 - kt0 : 0;
  const int ngroups = (nk + kGroup - 1) / kGroup;
  const uint32_t tmem_cols = 2 * N <= 32 ? 32 : 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // instruction descriptor: f32 accumulate, bf16 A and B, both K-major, M = 128, N
  const uint32_t idesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  int issued = 0;   // TMA stages issued by the producer
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int s = i % kStages;
        if (i >= kStages && !mbar_wait(&empty[s], ((i / kStages) - 1) & 1)) {
          atomicOr(status, 4u);
          *abort_flag = 1;
        }
        if (*abort_flag) break;
        mbar_expect_tx(&full[s], (uint32_t)(a_bytes + b_bytes));
        tma_load_2d(A_s + s * a_bytes, &tmA, &full[s], (kt0 + i) * kBK, mt * kBM);
        tma_load_2d(B_s + s * b_bytes, &tmB, &full[s], (kt0 + i) * kBK, 0);
        issued = i + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int g = 0; g < ngroups && !*abort_flag; ++g) {
        const int b = g & 1;
        if (g >= 2 && !mbar_wait(&acc_empty[b], ((g >> 1) - 1) & 1)) {
          atomicOr(status, 4u);
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int i1 = min(nk, (g + 1) * kGroup);
        for (int i = g * kGroup; i < i1; ++i) {
          const int s = i % kStages;
          if (!mbar_wait(&full[s], (i / kStages) & 1) || *abort_flag) {
            atomicOr(status, 4u);
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t ad = smem_desc_sw128(A_s + s * a_bytes), bd = smem_desc_sw128(B_s + s * b_bytes);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)   // 16 bf16 = 32 bytes = 2 descriptor units per step
            mma_bf16(tmem + (uint32_t)(b * N), ad + 2 * kk, bd + 2 * kk, idesc,
                     (i > g * kGroup || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        mma_commit(&acc_full[b]);   // arrives when this group's MMAs have completed
      }
    }
  } else {
    // drain warps: TMEM lanes 32*(warp % 4) .. +31 = tile rows
    const int lg = warp & 3;
    float sum[32], comp[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { sum[j] = 0.f; comp[j] = 0.f; }
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      bool ok = !*abort_flag && mbar_wait(&acc_full[b], (g >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok) != 0;
      if (!ok) {
        if (lane == 0) { atomicOr(status, 4u); *abort_flag = 1; }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        if (c0 < N) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * N + c0), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {   // Kahan-compensated sum of the drained accumulators
            const float y = v[j] - comp[c0 + j];
            const float t = sum[c0 + j] + y;
            comp[c0 + j] = (t - sum[c0 + j]) - y;
            sum[c0 + j] = t;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    const int m = mt * kBM + lg * 32 + lane;
    if (m < M) {
      float* dst = partials + ((long long)split * M + m) * N;
      const bool good = !*abort_flag;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < N) dst[j] = good ? sum[j] : 0.f;
    }
  }
  __syncwarp();
  if (warp == 0 && lane == 0 && *abort_flag) {
    // let copies already issued land before the shared memory is released
    for (int i = max(0, issued - kStages); i < issued; ++i) mbar_wait(&full[i % kStages], (i / kStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, long long inner, long long rows, int box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc_supported(int M, int N, long long K) {
  return (N == 16 || N == 32) && K % kBK == 0 && K >= 1024 && M >= 1;
}

size_t gemm_tc_smem(int N) { return (size_t)kStages * (kBM * kBK * 2 + N * kBK * 2) + 1024 + 256; }

cudaError_t launch_gemm_tc(const void* A, const void* Bt, int M, int N, long long K, int splits, float* partials,
                           unsigned* status, cudaStream_t s) {
  if (!gemm_tc_supported(M, N, K)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(Bt) & 15)) return cudaErrorMisalignedAddress;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, K, M, kBM) || !make_map(&tb, Bt, K, N, N)) return cudaErrorInvalidValue;
  const int k_tiles = (int)(K / kBK);
  const int per = (k_tiles + splits - 1) / splits;
  const int mtiles = (M + kBM - 1) / kBM;
  const size_t smem = gemm_tc_smem(N);
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gemm_bf16_tc_kernel<<<mtiles * splits, 192, smem, s>>>(ta, tb, M, N, k_tiles, per, mtiles, partials, status); note_launch();
  return cudaGetLastError();
}

}  // namespace ccs
