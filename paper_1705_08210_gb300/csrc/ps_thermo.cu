// ps_thermo.cu -- thermometer-coded min-product on the 5th-generation tensor
// cores (tcgen05), for quantized data.
//
// Not in the paper: with levels a, b in [0, L-1] and the thermometer code of
// ps_quant.cu, n2(i,j) = sum_q min(a_iq, a_jq) = T_i . T_j, where T is an
// nv x n_f(L-1) matrix of 0/1.  0 and 1 are exact in FP8 E4M3 and every
// partial sum is an integer below 2^24, so tcgen05.mma kind::f8f6f4 with FP32
// accumulation computes n2 exactly.  (kind::i8 does not exist on sm_103a.)
//
// Kernel structure (one CTA per SM, persistent, 6 warps), default tile
// 256 x 256 (MH = 2; MH = 1 gives 128 x 256):
//   warp 0        TMA producer: a 256 x 128-byte tile of T for rows I and a
//                 256 x 128-byte tile for rows J per stage (128-byte swizzle),
//                 3-stage ring guarded by full/empty mbarriers;
//   warp 1        TMEM owner and MMA issuer: per stage 4 K-steps x 2 halves
//                 of tcgen05.mma (M=128, N=256, K=32, the halves share the B
//                 tile) into a 512-column FP32 accumulator in TMEM;
//                 tcgen05.commit frees the stage;
//   warps 2..5    epilogue: tcgen05.ld of the finished accumulator (each warp
//                 its TMEM lane quadrant), c2 = 2 n2 / (S_i + S_j) with the
//                 integer level sums, transposed through shared memory so
//                 that each store instruction writes one contiguous row
//                 segment of the packed upper-triangular output.
// (With MH = 1 two 256-column accumulators let the epilogue of one tile
// overlap the MMAs of the next.)  Tiles: only blocks that hold some i < j
// (Section 3.1's triangle), walked in 12 x 12 super-blocks so that the CTAs
// running together share operand panels in L2; measured 2.4% faster from the
// larger tile alone and 12% more from the super-block order.
// K-synchronised producers: the CTAs that share a panel only hit each
// other's lines in L2 while they read the same K range at about the same
// time.  Over the ~54 rounds of tiles at nv = 32768 the persistent CTAs drift
// apart and the operand was re-read ~55x from DRAM (224 GB per launch for a
// 4 GB operand).  So the producers meet at a grid-wide counter every
// `sync_kb` k-blocks (cooperative launch: all CTAs are resident): a producer
// does not issue chunk m of its round-r tile before every CTA has issued all
// earlier chunks.
// Every mbarrier and counter wait is bounded (the handle's wait limit,
// ps_sync.cuh); on timeout the CTA raises `err`, lets in-flight copies drain,
// frees its TMEM and returns.
#include "ps_internal.cuh"
#include "ps_sync.cuh"

#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <vector>

namespace ps {
namespace {

constexpr int TN = 256, TKB = 128;  // tile columns, K bytes per stage
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;

// MH M=128 halves per CTA tile: MH = 1 -> 128 x 256 tile, 4 stages of 48 KB,
// two 256-column accumulators (epilogue overlaps the next tile); MH = 2 ->
// 256 x 256 tile (two MMAs share each B tile), 3 stages of 64 KB, one
// 512-column accumulator.
template <int MH>
struct TCfg {
  static constexpr int TM = 128 * MH;
  static constexpr int STAGES = MH == 1 ? 4 : 3;
  static constexpr int ACC_SETS = MH == 1 ? 2 : 1;
  static constexpr int A_BYTES = TM * TKB, B_BYTES = TN * TKB;
};

template <int MH>
struct __align__(1024) SmemTC {
  uint8_t A[TCfg<MH>::STAGES][TCfg<MH>::A_BYTES];
  uint8_t B[TCfg<MH>::STAGES][TCfg<MH>::B_BYTES];
  float xpose[4][32][33];
  unsigned long long full[TCfg<MH>::STAGES];
  unsigned long long empty[TCfg<MH>::STAGES];
  unsigned long long tfull[2];
  unsigned long long tempty[2];
  uint32_t tmem_base;
  int abort;
};

using sy::smem_addr;

// UMMA shared-memory descriptor, K-major operand written by TMA with the
// 128-byte swizzle: 8-row x 128-byte atoms, 1024 bytes apart (SBO).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(1) << 16;                    // LBO (unused for swizzled K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;  // SBO
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100)
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f8f6f4, A = B = E4M3, D = F32, both K-major,
// M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4)                 // D format F32
                           | (0u << 7) | (0u << 10)  // A, B format E4M3
                           | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM: thread t gets row (lane base + t).
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

// Tile walk: every (I, J) with I*TM < (J+1)*TN (some i < j in the tile),
// listed on the host in G x G super-blocks of (row block, column block), so
// that the CTAs running at the same time share their operand panels in L2.
constexpr int TILE_GROUP = 12;

std::vector<int2> tile_list(int TI, int TJ, int TM) {
  std::vector<int2> v;
  const int r = TN / TM;  // row blocks per column block
  for (int sj = 0; sj < TJ; sj += TILE_GROUP)
    for (int si = 0; si < TI; si += TILE_GROUP * r)
      for (int J = sj; J < std::min(TJ, sj + TILE_GROUP); ++J)
        for (int I = si; I < std::min(TI, si + TILE_GROUP * r); ++I)
          if (I < r * (J + 1)) v.push_back(make_int2(I, J));
  return v;
}

__device__ __forceinline__ int64_t pair_index(int64_t nv, int64_t i, int64_t j) {
  return i * (2 * nv - i - 1) / 2 + (j - i - 1);
}

template <int MH>
__global__ void __launch_bounds__(NTHREADS, 1)
    thermo_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                       const __grid_constant__ CUtensorMap mapB, int nkb, int nv,
                       const int2* __restrict__ tiles, int64_t ntiles, const int* __restrict__ SQ,
                       void* __restrict__ out, int out_mode, int* __restrict__ err,
                       unsigned* __restrict__ sync, int sync_kb, unsigned long long wait_ns) {
  extern __shared__ unsigned char smem_raw[];
  using CF = TCfg<MH>;
  constexpr int TM = CF::TM, TSTAGES = CF::STAGES, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES;
  SmemTC<MH>& sm = *reinterpret_cast<SmemTC<MH>*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      sy::bar_init(&sm.tfull[a], 1);
      sy::bar_init(&sm.tempty[a], 128);
    }
    sm.abort = 0;
    sy::bar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&sm.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer ----------------
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      const unsigned cpt = sync_kb > 0 ? (unsigned)((nkb + sync_kb - 1) / sync_kb) : 0u;
      int64_t r = 0;  // round: this CTA's r-th tile
      for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++r) {
        const int I = tiles[t].x, J = tiles[t].y;
        // CTAs holding a tile in this round
        const unsigned P = (unsigned)min((int64_t)gridDim.x, ntiles - r * (int64_t)gridDim.x);
        for (int kb = 0; kb < nkb; ++kb) {
          if (cpt && kb % sync_kb == 0 && (r | kb) != 0) {
            // chunks issued before chunk kb/sync_kb of round r, over all CTAs
            const unsigned need = (unsigned)r * cpt * gridDim.x + (unsigned)(kb / sync_kb) * P;
            if (!sy::counter_wait(sync, need, &sm.abort, err, wait_ns)) { ok = false; break; }
          }
          if (!sy::bar_wait(&sm.empty[stage], phase ^ 1, &sm.abort, err, wait_ns)) { ok = false; break; }
          sy::bar_arrive_tx(&sm.full[stage], A_BYTES + B_BYTES);
          sy::tma_load_2d(sm.A[stage], &mapA, kb * TKB, I * TM, &sm.full[stage]);
          sy::tma_load_2d(sm.B[stage], &mapB, kb * TKB, J * TN, &sm.full[stage]);
          if (++stage == TSTAGES) { stage = 0; phase ^= 1; }
          if (cpt && ((kb + 1) % sync_kb == 0 || kb + 1 == nkb)) atomicAdd(sync, 1u);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer ----------------
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        if (!sy::bar_wait(&sm.tempty[acc], aphase ^ 1, &sm.abort, err, wait_ns)) break;
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(acc * MH * TN);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!sy::bar_wait(&sm.full[stage], phase, &sm.abort, err, wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_addr(sm.A[stage]), b0 = smem_addr(sm.B[stage]);
#pragma unroll
          for (int kk = 0; kk < TKB / 32; ++kk)
#pragma unroll
            for (int hh = 0; hh < MH; ++hh)  // the M halves share the B tile
              umma_f8(dcol + (uint32_t)(hh * TN), umma_desc_sw128(a0 + hh * 128 * TKB + kk * 32),
                      umma_desc_sw128(b0 + kk * 32), (kb | kk) ? 1u : 0u);
          umma_commit(&sm.empty[stage]);
          if (++stage == TSTAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        umma_commit(&sm.tfull[acc]);
        if (++acc == CF::ACC_SETS) { acc = 0; aphase ^= 1; }
      }
    }
    __syncwarp();
  } else {  // ---------------- epilogue: warps 2..5 ----------------
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    float(*xp)[33] = sm.xpose[warp - 2];
    int acc = 0;
    uint32_t aphase = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int I = tiles[t].x, J = tiles[t].y;
      // warp-uniform wait: lane 0 polls, the warp follows its verdict
      int ok = 0;
      if (lane == 0) ok = sy::bar_wait(&sm.tfull[acc], aphase, &sm.abort, err, wait_ns) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      for (int hh = 0; hh < MH; ++hh) {
        const int row0 = I * TM + hh * 128 + quad * 32;
        const int my_row = row0 + lane;
        const int sq_row = my_row < nv ? SQ[my_row] : 0;
        for (int ch = 0; ch < TN / 32; ++ch) {
          float v[32];
          tmem_ld32(tmem + (uint32_t)((acc * MH + hh) * TN + ch * 32) + ((uint32_t)(quad * 32) << 16), v);
          const int col0 = J * TN + ch * 32;
          // transpose through shared memory: lane <-> column for the stores
#pragma unroll
          for (int c = 0; c < 32; ++c) xp[lane][c] = v[c];
          __syncwarp();
          const int j = col0 + lane;
          const int sq_j = j < nv ? SQ[j] : 0;
          for (int rr = 0; rr < 32; ++rr) {
            const int si = __shfl_sync(0xffffffffu, sq_row, rr);
            const int i = row0 + rr;
            if (i >= nv || j >= nv || j <= i) continue;
            const float n2 = xp[rr][lane];
            const int64_t o = pair_index(nv, i, j);
            if (out_mode == OUT2_C2_F64) {
              const double d = (double)si + (double)sq_j;
              static_cast<double*>(out)[o] = d == 0.0 ? 0.0 : (2.0 * (double)n2) / d;
            } else {
              const float d = (float)(si + sq_j);
              const float c2 = d == 0.0f ? 0.0f : __fdiv_rn(2.0f * n2, d);
              if (out_mode == OUT2_C2_U8)
                static_cast<unsigned char*>(out)[o] = c2_code(c2);
              else
                static_cast<float*>(out)[o] = c2;
            }
          }
          __syncwarp();
        }
      }
      tc_fence_before();
      sy::bar_arrive(&sm.tempty[acc]);
      if (++acc == CF::ACC_SETS) { acc = 0; aphase ^= 1; }
    }
  }
  __syncthreads();
  // let copies and MMAs already issued finish before the memory goes away
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ---- host ----
// T (rows x Kpad bytes) as a tensor with TKB x box_rows boxes, 128-byte swizzle
bool make_map(CUtensorMap* m, const uint8_t* T, int64_t Kpad, int rows, int box_rows) {
  return sy::make_map_u8_sw128(m, T, Kpad, rows, Kpad, TKB, box_rows);
}

uint64_t g_thermo_attr_devices[3] = {};

template <int MH>
cudaError_t launch_mh(ps_ctx* h, const uint8_t* T, int64_t Kpad, int nv, int nv_pad, const int* SQ,
                      void* out, int out_mode, int* err, unsigned* sync, cudaStream_t s) {
  constexpr int TM = TCfg<MH>::TM;
  if (Kpad % TKB != 0 || nv_pad % TN != 0 || nv_pad % TM != 0 || ((uintptr_t)T % 16) != 0)
    return cudaErrorInvalidValue;
  const uint64_t bit = 1ull << (h->device & 63);
  const size_t smem = sizeof(SmemTC<MH>) + 1024;
  if (!(g_thermo_attr_devices[MH] & bit)) {
    cudaError_t e = cudaFuncSetAttribute(thermo_gemm_kernel<MH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_thermo_attr_devices[MH] |= bit;
  }
  CUtensorMap mA, mB;
  if (!make_map(&mA, T, Kpad, nv_pad, TM) || !make_map(&mB, T, Kpad, nv_pad, TN))
    return cudaErrorInvalidValue;
  const int TI = nv_pad / TM, TJ = nv_pad / TN;
  const std::vector<int2> tl = tile_list(TI, TJ, TM);
  const int64_t ntiles = (int64_t)tl.size();
  int2* dtl = static_cast<int2*>(ws_get(h, WS_BLOCKS, tl.size() * sizeof(int2) + 256));
  if (!dtl) return cudaErrorMemoryAllocation;
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  cudaError_t e = cudaMemcpyAsync(dtl, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int nkb = (int)(Kpad / TKB);
  const int grid = (int)std::min<int64_t>(ntiles, h->num_sms);
  // producers meet only when there is more than one round of tiles
  const int sync_kb = (ntiles > grid && h->thermo_sync_kb > 0) ? h->thermo_sync_kb : 0;
  if (sync_kb) {
    e = cudaMemsetAsync(sync, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = sync_kb ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, thermo_gemm_kernel<MH>, mA, mB, nkb, nv, (const int2*)dtl, ntiles, SQ,
                            out, out_mode, err, sync, sync_kb, h->wait_ns);
}

}  // namespace

cudaError_t launch_thermo_gemm(ps_ctx* h, const uint8_t* T, int64_t Kpad, int nv, int nv_pad,
                               const int* SQ, void* out, int out_mode, int* err, unsigned* sync,
                               cudaStream_t s) {
  const int tm = h->thermo_tile_m ? h->thermo_tile_m : (Kpad >= 16384 ? 256 : 128);
  if (tm == 256)
    return launch_mh<2>(h, T, Kpad, nv, nv_pad, SQ, out, out_mode, err, sync, s);
  return launch_mh<1>(h, T, Kpad, nv, nv_pad, SQ, out, out_mode, err, sync, s);
}

}  // namespace ps
