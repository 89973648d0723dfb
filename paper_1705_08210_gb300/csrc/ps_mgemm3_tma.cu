// ps_mgemm3_tma.cu -- the 3-way pivot-min product of Section 3.2 fed by the
// tensor memory accelerator.
//
// Work item = (pivot j, row tile I, column tile K) with rows i < j and
// columns k > j (only the part of B_j = X_j^T (min) V that holds i < j < k),
// the cp.async kernel's (mgemm3_kernel) walk, read from a table written
// before the launch (one load per tile, fetched a tile ahead).  Per BK-field
// slice, lane 0 of warp 0 issues three TMA loads into an mbarrier-guarded
// ring: the 128-vector row panel, the 128-vector column panel, and a
// 4-vector box holding the pivot column v_j.  X_j = min(V, v_j) is never
// stored: one slice ahead of the compute each warp min-s its BK/16 field
// rows of the row panel with the pivot value in place and arrives on the
// slice's `ready` barrier; before computing a slice a warp waits there for
// the other warps' rows (a bounded mbarrier wait, not a CTA barrier), then
// runs the 2-way micro-kernel (8 x 4 outputs per lane, FP32 min + packed
// FP32 add, TwoSum fold every 64 fields) on it.
//
// Warp placement (mg::Lanes3).  A warp owns a 32 x 32 block.  The tile that
// straddles the pivot has rows i >= j (past the pivot's rectangle) and
// columns k <= j (before it); warps whose whole block lies outside skip the
// min-add loop.  Warp w = 4g + s (scheduler s) takes row block g and column
// block (g + s) mod 4, so skipping whole row blocks or column blocks frees
// every scheduler equally.
#include "ps_mgemm_impl.cuh"
#include "ps_sync.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace ps {
namespace {

using C = mg::T128W16;  // 128 x 128 tile, 16 warps, 8 x 4 outputs per lane
constexpr int NW = C::NT / 32;
constexpr int PBOX = 4;  // pivot box: 4 vectors (16 bytes) x BK fields

using Lanes3 = mg::Lanes3;

template <int BK, int STAGES>
struct __align__(128) Smem3 {
  float A[STAGES][BK][C::BM];  // row panel (min-ed with the pivot in place)
  float B[STAGES][BK][C::BN];  // column panel
  float P[STAGES][BK][PBOX];   // pivot column: v_j at [kk][j % 4]
  int pcol[STAGES];            // j % 4 of the slice's pivot (written by the producer)
  int tile_of[STAGES];         // counter schedule: work item of local item lt at [lt % STAGES], -1 = none
  int2 pitem;                  // the producer's current work item
  int p_done;                  // counter schedule: the producer has issued the end marker
  unsigned long long full[STAGES];
  unsigned long long ready[STAGES];
  unsigned long long empty[STAGES];
  int abort;
};

// BK k-steps of the micro-kernel on one prepared slice.
template <int BK, int KU>
__device__ __forceinline__ void compute_slice3(const float* As, const float* Bs, mg::AccMix<C::NJ>& acc) {
#pragma unroll KU
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + kk * C::BM);
    const float4 a1 = *reinterpret_cast<const float4*>(As + kk * C::BM + mg::Lanes3::RUN);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * C::BN);
    const float b[4] = {b0.x, b0.y, b0.z, b0.w};
    acc.step(a, b);
  }
}

// Work item {j, (I << 16) | K} -> pivot j and tile origin (row0, col0).
__device__ __forceinline__ void item3(int2 w, int& j, int& row0, int& col0) {
  j = w.x;
  row0 = (w.y >> 16) * C::BM;
  col0 = (w.y & 0xffff) * C::BN;
}

// THRESH: the thresholded search instead of the slab output: every triple
// i < j < k of the item with c3 >= tau is appended as in
// mgemm3_thresh_kernel (same values, same keys).
template <int BK, int STAGES, int KU, bool DYN, bool THRESH = false>
__global__ void __launch_bounds__(C::NT, 1)
    mgemm3_tma_kernel(const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapP,
                      int nv, int nf, const double* __restrict__ S, const float* __restrict__ n2sq,
                      const int2* __restrict__ items, int jb, float* __restrict__ out, int64_t ntiles,
                      int* err, unsigned long long* __restrict__ item_ctr, unsigned long long wait_ns,
                      ThreshArgs ta) {
  static_assert(mg::FOLD * mg::BK % BK == 0 && BK % NW == 0, "slice shape");
  constexpr int FOLD_SLICES = mg::FOLD * mg::BK / BK;
  constexpr int ROWS_PER_WARP = BK / NW;  // field rows of a slice each warp min-s with the pivot
  constexpr uint32_t SLICE_BYTES = (2u * BK * C::BM + BK * PBOX) * sizeof(float);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem3<BK, STAGES>& sm = *reinterpret_cast<Smem3<BK, STAGES>*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.ready[s], NW);
      sy::bar_init(&sm.empty[s], NW);
    }
    sm.abort = 0;
    sm.p_done = 0;
    sy::bar_init_fence();
  }
  __syncthreads();
  const int nkb = (nf + BK - 1) / BK;
  // Work schedule.  Static (DYN false): this CTA's items are blockIdx.x,
  // blockIdx.x + gridDim.x, ...  Counter (DYN true): the producer claims the
  // next item from the grid-wide counter when it loads the item's first
  // slice, after that slice's ring stage is free, and hands the item index
  // to the warps in tile_of[lt % STAGES], published by the stage's full
  // barrier; a claim past the end publishes -1 with a plain arrival (no
  // copies), which stops the warps.  Entry lt % STAGES is rewritten only
  // when item lt + STAGES is claimed, which waits for every warp to release
  // slice (lt + STAGES) nkb - STAGES >= lt nkb, so every warp has read the
  // entry of item lt by then.  The warps read nothing else the producer
  // rewrites per item: the epilogue reads its item from the global table.
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // slices of this CTA (< 2^32, checked by the launcher); unbounded with DYN
  const uint32_t n_slices = DYN ? 0xffffffffu : (uint32_t)(my_tiles * nkb);

  // producer (lane 0 of warp 0): loads slice g (waiting until its ring
  // stage is free); false on abort.  Its work item is kept in shared memory
  // (registers are the micro-kernel's).
  const bool producer = threadIdx.x == 0;
  auto issue_one = [&](uint32_t g) -> bool {
    Smem3<BK, STAGES>& sm = *reinterpret_cast<Smem3<BK, STAGES>*>(smem_raw);
    if (g >= n_slices || (DYN && sm.p_done)) return true;
    const int s = (int)(g % STAGES);
    const uint32_t ph = (g / STAGES) & 1u;
    const int kb = (int)(g % (uint32_t)nkb);
    const uint32_t r = g / (uint32_t)nkb;  // this CTA's r-th item
    if (!DYN && kb == 0) sm.pitem = items[blockIdx.x + (int64_t)r * gridDim.x];
    if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) return false;
    if (DYN && kb == 0) {
      const unsigned long long t = atomicAdd(item_ctr, 1ull);
      if (t >= (unsigned long long)ntiles) {
        sm.tile_of[r % STAGES] = -1;
        sy::bar_arrive(&sm.full[s]);  // completes the phase with no copies
        sm.p_done = 1;
        return true;
      }
      sm.tile_of[r % STAGES] = (int)t;  // published by the arrival below
      sm.pitem = items[t];
    }
    int pj, prow0, pcol0;
    item3(sm.pitem, pj, prow0, pcol0);
    sm.pcol[s] = pj & (PBOX - 1);  // published by the arrival below
    sy::bar_arrive_tx(&sm.full[s], SLICE_BYTES);
    sy::tma_load_2d(&sm.A[s][0][0], &mapV, prow0, kb * BK, &sm.full[s]);
    sy::tma_load_2d(&sm.B[s][0][0], &mapV, pcol0, kb * BK, &sm.full[s]);
    sy::tma_load_2d(&sm.P[s][0][0], &mapP, pj & ~(PBOX - 1), kb * BK, &sm.full[s]);
    return true;
  };
  if (producer)
    for (uint32_t g = 0; g + 1 < STAGES; ++g)
      if (!issue_one(g)) break;

  // X_j = min(V, v_j) on this warp's field rows of slice g's row panel,
  // then one arrival on the slice's `ready` barrier; false on abort.  (With
  // DYN, the first slice of the end marker has nothing to prepare.)
  auto prepare = [&](uint32_t g) -> bool {
    // (the shared array itself, not the captured reference: through the
    // capture the compiler would emit generic loads and stores)
    Smem3<BK, STAGES>& sm = *reinterpret_cast<Smem3<BK, STAGES>*>(smem_raw);
    const int s = (int)(g % STAGES);
    const uint32_t ph = (g / STAGES) & 1u;
    const bool landed = sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns);
    if (!__all_sync(0xffffffffu, landed)) return false;
    if (DYN && g % (uint32_t)nkb == 0 && sm.tile_of[(g / (uint32_t)nkb) % STAGES] < 0) return true;
    const int pc = sm.pcol[s];
#pragma unroll
    for (int rr = 0; rr < ROWS_PER_WARP; ++rr) {
      const int kk = warp * ROWS_PER_WARP + rr;
      const float p = sm.P[s][kk][pc];
      float4* a = reinterpret_cast<float4*>(&sm.A[s][kk][lane * 4]);
      float4 v = *a;
      v.x = fminf(v.x, p);
      v.y = fminf(v.y, p);
      v.z = fminf(v.z, p);
      v.w = fminf(v.w, p);
      *a = v;
    }
    // the TMA refill of this stage comes later through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) sy::bar_arrive(&sm.ready[s]);
    return true;
  };

  const Lanes3 L;
  // columns 0, 1 of each lane by packed adds, 2, 3 by scalar adds (more FP32
  // mins per clock than all-packed adds; identical values)
  mg::AccMix<C::NJ> acc;
  uint32_t it = 0;
  // slices are prepared one ahead of the compute, so that a warp waiting for
  // the other warps' rows of slice it waited a whole slice earlier
  bool ok = n_slices == 0 || prepare(0);
  for (int64_t lt = 0; ok; ++lt) {
    int64_t t;
    if (DYN) {
      t = sm.tile_of[lt % STAGES];  // published by the full barrier prepare() waited on
      if (t < 0) break;
    } else {
      t = blockIdx.x + lt * gridDim.x;
      if (t >= ntiles) break;
    }
    int j, row0, col0;
    item3(items[t], j, row0, col0);
    // a warp whose block has no row i < j, no column k > j, or no column
    // inside the matrix has no output here and skips the min-adds
    const bool active = row0 + L.wrow0 < j && col0 + L.wcol0 + Lanes3::BW - 1 > j && col0 + L.wcol0 < nv;
    acc.zero();
    for (int kb = 0; kb < nkb; ++kb, ++it) {
      // slice it + STAGES - 1 (its stage was released by every warp after
      // slice it - 1, which none of them needs this warp for)
      if (producer) ok = issue_one(it + STAGES - 1);
      ok = __all_sync(0xffffffffu, ok);
      if (ok && it + 1 < n_slices) ok = prepare(it + 1);
      if (!ok) break;
      const int s = (int)(it % STAGES);
      const uint32_t ph = (it / STAGES) & 1u;
      const bool prepared = sy::bar_wait(&sm.ready[s], ph, &sm.abort, err, wait_ns);
      if (!__all_sync(0xffffffffu, prepared)) { ok = false; break; }
      if (active) compute_slice3<BK, KU>(&sm.A[s][0][L.am], &sm.B[s][0][L.bn], acc);
      __syncwarp();
      if (lane == 0) sy::bar_arrive(&sm.empty[s]);
      if ((kb + 1) % FOLD_SLICES == 0) acc.fold();
    }
    if (!ok) break;
    acc.fold();
    if constexpr (THRESH) {
      mg::thresh_append3<C::NJ>(acc, L, row0, col0, j, nv, S, n2sq, ta);
      continue;
    }
    // Section 2.2 eq. (1) into pivot j's slab block (rows i < j, columns k > j)
    const int64_t w = nv - 1 - j;
    const int64_t base = mg::slab_offset(nv, jb, j);
    const float Sj = (float)S[j];
    float Skf[C::NJ];
#pragma unroll
    for (int c = 0; c < C::NJ; ++c) {
      const int k = col0 + L.col(c);
      Skf[c] = k < nv ? (float)S[k] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= j) continue;
      const float Sij = __fadd_rn((float)S[i], Sj);
      const float n2ij = n2sq[(int64_t)i * nv + j];
#pragma unroll
      for (int c = 0; c < C::NJ; ++c) {
        const int k = col0 + L.col(c);
        if (k <= j || k >= nv) continue;
        out[base + (int64_t)i * w + (k - j - 1)] =
            mg::c3_value(acc.hl(r, c), n2ij, n2sq[(int64_t)i * nv + k], n2sq[(int64_t)j * nv + k],
                         __fadd_rn(Sij, Skf[c]));
      }
    }
  }
  __syncthreads();
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
}

// ---- host side ----
template <int BK, int STAGES, int KU, bool DYN, bool THRESH = false>
struct Tma3Launch {
  static constexpr size_t smem = sizeof(Smem3<BK, STAGES>);
  static cudaError_t run(ps_ctx* h, const VF32& V, const double* S, const float* n2sq, const int2* items, int jb,
                         float* out, int64_t ntiles, int* err, unsigned long long* item_ctr, cudaStream_t st,
                         const ThreshArgs& ta = ThreshArgs{}) {
    static std::mutex mu;
    static uint64_t attr_done = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      const uint64_t bit = 1ull << (h->device & 63);
      if (!(attr_done & bit)) {
        const cudaError_t e = cudaFuncSetAttribute(mgemm3_tma_kernel<BK, STAGES, KU, DYN, THRESH>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done |= bit;
      }
    }
    CUtensorMap mapV, mapP;
    if (!sy::make_map_f32(&mapV, V.p, V.nv, V.nf, V.ld, C::BM, BK) ||
        !sy::make_map_f32(&mapP, V.p, V.nv, V.nf, V.ld, PBOX, BK))
      return cudaErrorInvalidValue;
    if (DYN) {
      const cudaError_t e = cudaMemsetAsync(item_ctr, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)h->num_sms);
    mgemm3_tma_kernel<BK, STAGES, KU, DYN, THRESH><<<grid, C::NT, smem, st>>>(mapV, mapP, V.nv, V.nf, S, n2sq, items, jb,
                                                                      out, ntiles, err, item_ctr, h->wait_ns, ta);
    return cudaGetLastError();
  }
};

// Work items of the thresholded search: block b = (I, Jt, K) of 128-vector
// tiles contributes pivots j of tile Jt with rows i < j in tile I and
// columns k > j in tile K, the range j in [jlo, jhi] (first[b] items before
// it); one CTA of 128 threads per block.
__global__ void __launch_bounds__(128) thresh_items_kernel(const int* __restrict__ blocks,
                                                           const int64_t* __restrict__ first, int nv,
                                                           int2* __restrict__ items) {
  const int b = blockIdx.x;
  const int I = blocks[3 * b], Jt = blocks[3 * b + 1], K = blocks[3 * b + 2];
  const int jlo = max(Jt * 128, I * 128 + 1), jhi = min(min(Jt * 128 + 127, nv - 1), K * 128 + 126);
  const int j = Jt * 128 + (int)threadIdx.x;
  if (j >= jlo && j <= jhi) items[first[b] + (j - jlo)] = make_int2(j, (I << 16) | K);
}

}  // namespace

cudaError_t launch_mgemm3_thresh_tma(ps_ctx* h, const VF32& V, const double* S, const float* n2sq,
                                     const int* blocks, const int* blocks_host, int64_t nblocks, const ThreshArgs& ta,
                                     int* err, cudaStream_t st) {
  if ((uintptr_t)V.p % 16 != 0 || V.ld % 4 != 0 || V.nv < 1 || V.nf < 1) return cudaErrorInvalidValue;
  // item offsets of every block (host: the block list is built there)
  const int nv = V.nv;
  std::vector<int64_t> first((size_t)nblocks + 1, 0);
  for (int64_t b = 0; b < nblocks; ++b) {
    const int I = blocks_host[3 * b], Jt = blocks_host[3 * b + 1], K = blocks_host[3 * b + 2];
    const int jlo = std::max(Jt * 128, I * 128 + 1), jhi = std::min(std::min(Jt * 128 + 127, nv - 1), K * 128 + 126);
    first[(size_t)b + 1] = first[(size_t)b] + std::max(0, jhi - jlo + 1);
  }
  const int64_t nitems = first[(size_t)nblocks];
  if (nitems == 0) return cudaSuccess;
  if (nitems >= ((int64_t)1 << 31) ||
      (double)ceil_div(nitems, h->num_sms) * (double)ceil_div(V.nf, 16) >= 4294967295.0)
    return cudaErrorInvalidValue;
  int64_t* dfirst = static_cast<int64_t*>(ws_get(h, WS_AUX0, ((size_t)nblocks + 1) * sizeof(int64_t)));
  int2* items = static_cast<int2*>(ws_get(h, WS_ITEMS, (size_t)nitems * sizeof(int2)));
  unsigned* sync = static_cast<unsigned*>(ws_get(h, WS_SYNC, 256));
  if (!dfirst || !items || !sync) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpyAsync(dfirst, first.data(), ((size_t)nblocks + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  thresh_items_kernel<<<(unsigned)nblocks, 128, 0, st>>>(blocks, dfirst, nv, items);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the host vector must outlive the asynchronous copy
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(sync + 4);
  const int bk = V.nf <= 16 ? 16 : (V.nf <= 32 ? 32 : 64);
#define PS_TMA3T_RUN(...)                                                                                      \
  (h->mgemm3_dynamic                                                                                          \
       ? Tma3Launch<__VA_ARGS__, true, true>::run(h, V, S, n2sq, items, 0, nullptr, nitems, err, ctr, st, ta)  \
       : Tma3Launch<__VA_ARGS__, false, true>::run(h, V, S, n2sq, items, 0, nullptr, nitems, err, ctr, st, ta))
  if (bk == 16) return PS_TMA3T_RUN(16, 8, 8);
  if (bk == 32) return PS_TMA3T_RUN(32, 4, 16);
  return PS_TMA3T_RUN(64, 3, 16);
#undef PS_TMA3T_RUN
}

cudaError_t launch_mgemm3_tma(ps_ctx* h, const VF32& V, const double* S, const float* n2sq, const int2* items,
                              int jb, float* out, int64_t ntiles, int* err, cudaStream_t st) {
  // TMA: 16-byte aligned base and row pitch; 128-wide tiles
  if ((uintptr_t)V.p % 16 != 0 || V.ld % 4 != 0 || V.nv < 1) return cudaErrorInvalidValue;
  // item indices in 31 bits, slices per CTA counted in 32 bits
  if (ntiles >= ((int64_t)1 << 31) ||
      (double)ceil_div(ntiles, h->num_sms) * (double)ceil_div(V.nf, 16) >= 4294967295.0)
    return cudaErrorInvalidValue;
  // slice width by n_f (a wider slice than n_f is mostly zero fill): 64
  // fields in 3 stages above 32 (2048 x 4096: 433.0 ms; 32 fields in 4
  // stages 457.2 ms, in 3 stages 450.7 ms: the per-slice pivot min, waits
  // and releases are what a wider slice saves), 16 k-steps per unrolled
  // iteration (457.8 vs 463.5 ms with 8 at 32-field slices)
  const int bk = V.nf <= 16 ? 16 : (V.nf <= 32 ? 32 : (h->mgemm_tma_bk ? h->mgemm_tma_bk : 64));
  // work items claimed from a grid-wide counter (default) or round-robin;
  // the counter is its own word of the handle's counter slot (bytes 16..23;
  // the 2-way kernel uses bytes 0..15) and is zeroed before each launch
  unsigned* sync = static_cast<unsigned*>(ws_get(h, WS_SYNC, 256));
  if (!sync) return cudaErrorMemoryAllocation;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(sync + 4);
#define PS_TMA3_RUN(...)                                                                                 \
  (h->mgemm3_dynamic ? Tma3Launch<__VA_ARGS__, true>::run(h, V, S, n2sq, items, jb, out, ntiles, err, ctr, st) \
                     : Tma3Launch<__VA_ARGS__, false>::run(h, V, S, n2sq, items, jb, out, ntiles, err, ctr, st))
  if (bk == 16) return PS_TMA3_RUN(16, 8, 8);
  if (bk == 64) return PS_TMA3_RUN(64, 3, 16);
  if (h->mgemm_tma_ku == 8) return PS_TMA3_RUN(32, 4, 8);
  if (h->mgemm_tma_stages == 3) return PS_TMA3_RUN(32, 3, 16);
  return PS_TMA3_RUN(32, 4, 16);
#undef PS_TMA3_RUN
}

}  // namespace ps
