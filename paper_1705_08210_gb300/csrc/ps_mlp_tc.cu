// ps_mlp_tc.cu -- the encoder's products on the 5th-generation tensor cores.
//
// Not in the paper (the encoder belongs to the learned block proposal).
// C[M x N] = A[M x K] . B[N x K]^T with A and B in BF16, both K-major (row
// i of A and row n of B hold their K values contiguously, pitch a multiple of
// 8 elements), FP32 accumulation in tensor memory, and an epilogue functor
// applied to every (row, column, value) of the tile.
//
// Kernel: one CTA per 128 x TN output tile, 6 warps.
//   warp 0      TMA producer: per K-block of 64 elements (128 bytes) one
//               128 x 128-byte box of A and one TN x 128-byte box of B, with
//               the 128-byte swizzle, into a 4-stage mbarrier ring;
//   warp 1      allocates TN tensor-memory columns and issues, per K-block,
//               four tcgen05.mma.kind::f16 (M = 128, N = TN, K = 16);
//               tcgen05.commit frees the stage, and after the last block
//               signals the accumulator;
//   warps 2..5  epilogue: each warp reads its 32-lane quadrant of the
//               accumulator with tcgen05.ld (thread = output row) and calls
//               the functor.
// Rows past M and columns past N or K are zero-filled by the TMA and never
// passed to the functor.  Every wait is bounded (the handle's wait limit);
// on a timeout the CTA raises `err`, lets issued copies and products finish,
// frees its tensor memory and returns.
#include "ps_internal.cuh"
#include "ps_sync.cuh"

#include <algorithm>
#include <mutex>

namespace ps {
namespace tc {

constexpr int TM = 128, KB = 64, KBYTES = 128, TSTAGES = 4, NTHREADS = 192;

template <int TN>
struct __align__(1024) SmemG {
  uint8_t A[TSTAGES][TM * KBYTES];
  uint8_t B[TSTAGES][TN * KBYTES];
  unsigned long long full[TSTAGES];
  unsigned long long empty[TSTAGES];
  unsigned long long done;
  uint32_t tmem_base;
  int abort;
};

// UMMA shared-memory descriptor of a K-major operand written by the TMA with
// the 128-byte swizzle: 8-row x 128-byte atoms, 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                      // leading offset (unused for swizzled K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;  // stride offset: the next 8-row atom
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// M = 128, N = TN.
template <int TN>
constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   sy::smem_addr(bar))
               : "memory");
}

// 32 lanes x 32 columns of FP32 from tensor memory: thread t gets row
// (lane base + t), columns c .. c + 31.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
}

template <int TN, class Epi>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                     int N, int K, Epi epi, int* err, unsigned long long wait_ns) {
  extern __shared__ unsigned char smem_raw[];
  SmemG<TN>& sm = *reinterpret_cast<SmemG<TN>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int nkb = (K + KB - 1) / KB;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.empty[s], 1);
    }
    sy::bar_init(&sm.done, 1);
    sm.abort = 0;
    sy::bar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sy::smem_addr(&sm.tmem_base)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer ----
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TSTAGES;
        const uint32_t ph = (kb / TSTAGES) & 1u;
        if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) break;
        sy::bar_arrive_tx(&sm.full[s], (uint32_t)(TM + TN) * KBYTES);
        sy::tma_load_2d(sm.A[s], &mapA, kb * KBYTES, m0, &sm.full[s]);
        sy::tma_load_2d(sm.B[s], &mapB, kb * KBYTES, n0, &sm.full[s]);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer ----
      constexpr uint32_t IDESC = idesc_bf16<TN>();
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TSTAGES;
        const uint32_t ph = (kb / TSTAGES) & 1u;
        if (!sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = sy::smem_addr(sm.A[s]), b0 = sy::smem_addr(sm.B[s]);
#pragma unroll
        for (int kk = 0; kk < KBYTES / 32; ++kk)  // K = 16 BF16 = 32 bytes per product
          umma_bf16(tmem, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), IDESC, (kb | kk) ? 1u : 0u);
        umma_commit(&sm.empty[s]);
      }
      if (ok) umma_commit(&sm.done);
    }
    __syncwarp();
  } else {  // ---- epilogue: warps 2..5 ----
    const int quad = warp & 3;  // the tensor-memory lane quadrant this warp may read
    int ok = 0;
    if (lane == 0) ok = sy::bar_wait(&sm.done, 0, &sm.abort, err, wait_ns) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + quad * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + (uint32_t)c0 + ((uint32_t)(quad * 32) << 16), v);
        if (row < M) {
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (n0 + c0 + c < N) epi(row, n0 + c0 + c, v[c]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // let copies and products already issued finish before the memory goes away
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TN)
                 : "memory");
}

}  // namespace tc
}  // namespace ps
