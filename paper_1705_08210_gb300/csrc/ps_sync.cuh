// ps_sync.cuh -- shared-memory mbarriers, tensor-memory-accelerator (TMA)
// tile loads and bounded waits for the warp-specialised kernels.
//
// Every wait here is bounded: after `limit_ns` of %globaltimer time (the
// handle's wait_limit_ns, 2 s by default) the waiter raises the CTA's abort
// word and a device error flag and gives up, so a lost copy cannot hang the
// GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ps {
namespace sy {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void bar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

// One arrival plus `bytes` of expected transaction count (the TMA copies
// that complete the phase).
__device__ __forceinline__ void bar_arrive_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_test(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the barrier phase with `parity`.  Returns false
// when the CTA is aborting (abort word set by another waiter) or when this
// wait passed `limit_ns` (then it sets the abort word and *err).
__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t parity, int* abort_word,
                                         int* err, unsigned long long limit_ns) {
  if (bar_test(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 1;; ++it) {
    if (bar_test(b, parity)) return true;
    if ((it & 31) == 0) {
      if (*(volatile int*)abort_word) return false;
      if (now_ns() - t0 > limit_ns) {
        *(volatile int*)abort_word = 1;
        if (err) {
          atomicExch(err, 1);
          __threadfence_system();
        }
        return false;
      }
    }
  }
}

// Wait until the grid-wide counter *c reaches `need` (relaxed loads: the
// counter only paces the producers, it guards no data).  False when the CTA
// is aborting or `limit_ns` passed (then it sets the abort word and *err).
__device__ __forceinline__ bool counter_wait(const unsigned* c, unsigned need, int* abort_word, int* err,
                                             unsigned long long limit_ns) {
  auto load = [c]() {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    return v;
  };
  if (load() >= need) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    __nanosleep(64);
    if (load() >= need) return true;
    if (*(volatile int*)abort_word) return false;
    if (now_ns() - t0 > limit_ns) {
      *(volatile int*)abort_word = 1;
      if (err) {
        atomicExch(err, 1);
        __threadfence_system();
      }
      return false;
    }
  }
}

// 2-D tiled TMA load of the box at element coordinates (x, y) (x innermost)
// into shared memory; completion is signalled on barrier `b` as transaction
// bytes.  x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(b))
      : "memory");
}

// After an abort: keep the CTA (and its shared memory) alive for 1 ms so
// that copies (and tensor-core operations) already issued land before the
// memory is released.
__device__ __forceinline__ void drain_after_abort() {
  const unsigned long long t0 = now_ns();
  while (now_ns() - t0 < 1000000ull) {
  }
}

// ---- host: 2-D FP32 tensor maps through the driver entry point ----
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    EncodeTiledFn f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
    return f;
  }();
  return fn;
}

// 2-D byte matrix (rows of `pitch` bytes, `cols` valid bytes per row) as a
// tensor with boxes of box_cols x box_rows bytes and the 128-byte swizzle
// (the K-major tensor-core operand layout); zero fill outside.
inline bool make_map_u8_sw128(CUtensorMap* m, const void* p, int64_t cols, int64_t rows, int64_t pitch,
                              int box_cols, int box_rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Field-major FP32 matrix (element (i, q) at p[i + q ld]) as a 2-D tensor:
// x = vector index (nv, contiguous), y = field (nf rows, ld floats apart);
// box box_x vectors x box_y fields, zero fill outside the matrix.  Needs p
// 16-byte aligned and ld % 4 == 0; box_x * 4 bytes a multiple of 16.
inline bool make_map_f32(CUtensorMap* m, const float* p, int64_t nv, int64_t nf, int64_t ld, int box_x,
                         int box_y) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc || nv < 1) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)nv, (cuuint64_t)(nf > 0 ? nf : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace sy
}  // namespace ps
