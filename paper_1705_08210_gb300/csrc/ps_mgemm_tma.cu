// ps_mgemm_tma.cu -- the 2-way FP32 min-product (Section 3.1's mGEMM) fed by
// the tensor memory accelerator.
//
// Same tile (128 x 128 outputs, upper-triangle tiles only, banded walk),
// same micro-kernel (a lane owns 8 x 4 outputs; one FP32 min + one packed
// FP32 add per comparison; TwoSum fold every 64 fields) and same epilogue as
// the cp.async kernel of ps_mgemm_impl.cuh, but the operands arrive through
// the TMA: per BK-field slice, two 2-D tensor loads (the 128-vector row
// panel and the 128-vector column panel of V, field-major, zero-filled past
// nv and nf) into an STAGES-deep shared-memory ring guarded by full/empty
// mbarriers.  Lane 0 of warp 0 is the producer: before computing slice s it
// loads slice s + look, look <= STAGES - 1 (the walk over this CTA's tiles is one flat
// sequence of slices, so near the end of a tile it already loads the next
// tile's first slices, which then land while the warps write outputs).  A
// warp releases a slice with one arrival when it is done with it.  The 16
// warps compute no addresses and never meet at a CTA barrier.  (A separate
// producer warp would make 17 warps; the SM's register file, split across
// four schedulers, would then cap every thread at 96 registers.)
// Every wait is bounded (ps_sync.cuh); on a timeout the kernel raises the
// handle's mapped error word, lets issued copies land and returns.
#include "ps_mgemm_impl.cuh"
#include "ps_sync.cuh"

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace ps {
namespace {

using C = mg::T128W16;  // 128 x 128 tile, 16 warps of 8 x 4 outputs per lane
constexpr int NW = C::NT / 32;

template <int BK, int STAGES>
struct __align__(128) SmemT {
  float A[STAGES][BK][C::BM];  // rows: field q of the slice; 128 consecutive vectors
  float B[STAGES][BK][C::BN];
  unsigned long long full[STAGES];
  unsigned long long empty[STAGES];
  int2 tile_of[STAGES];  // (I, J) of this CTA's local tile lt at [lt % STAGES]; I = -1: no tile left
  // producer state (thread 0 only; kept here to leave registers to the
  // micro-kernel): next slice to load, schedule exhausted, its tile
  uint32_t p_next;
  int p_done, pI, pJ;
  int abort;
};

// BK k-steps of the micro-kernel on one landed slice.
template <int BK, int KU, class ACC>
__device__ __forceinline__ void compute_slice_tma(const float* As, const float* Bs, ACC& acc) {
#pragma unroll KU
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + kk * C::BM);
    const float4 a1 = *reinterpret_cast<const float4*>(As + kk * C::BM + 32);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * C::BN);
    const float b[4] = {b0.x, b0.y, b0.z, b0.w};
    acc.step(a, b);
  }
}

// EPI: epilogue of the interior tiles.  0: store_tile2 (__fdiv_rn).  1:
// store_tile2_lean (branch-free correctly rounded division, FP32 sums with
// zero-vector substitution from NarrowPrep) when the call's inputs are in
// its range, else store_tile2.  2: as 1, for n_f <= 64: no compensated fold
// (at most 64 fields per accumulator, the fold's own bound; values are the
// same bit for bit, since a single fold of 0 + lo is exact) and the rows'
// and columns' sums loaded when the tile starts.
// ADDS: the add form of the accumulators (identical values).  1 (default):
// columns 0 and 1 of each lane by one packed add.rn.f32x2, columns 2 and 3
// by scalar adds (mg::AccMix); 0: all packed; 2: all scalar.  Packed adds
// halve the add instructions, but the SM then retires fewer FP32 mins per
// clock (measured register-only: 16.7 Tcmp/s with packed adds, 19.3 with
// scalar ones, 18.8 mixed); mixed keeps the issue count below the ALU
// pipe's two cycles per min: 266.98 vs 273.66 ms at 32768 x 8192.
template <int ADDS>
using AccT = std::conditional_t<ADDS == 1, mg::AccMix<C::NJ>,
                                std::conditional_t<ADDS == 0, mg::Acc<true, C::NJ>, mg::Acc<false, C::NJ>>>;

// THRESH: the thresholded search instead of the packed output: every pair
// with c2 >= tau appended (mg::thresh_append2; values as the FP32 output).
template <int BK, int STAGES, int KU, int EPI, bool DYN, int ADDS = 1, bool THRESH = false>
__global__ void __launch_bounds__(C::NT, 1)
    mgemm2_tma_kernel(const __grid_constant__ CUtensorMap mapV, int nv, int nf,
                      const double* __restrict__ S, void* __restrict__ out, int mode, int T, int R0,
                      int R1, int G, int64_t ntiles, int* err, unsigned* __restrict__ sync, int sync_sl,
                      unsigned long long* __restrict__ tile_ctr, unsigned long long wait_ns,
                      const float* __restrict__ Sf, const unsigned* __restrict__ lean_words, int look,
                      ThreshArgs ta) {
  static_assert(!THRESH || EPI == 0, "the thresholded search has the plain epilogue");
  static_assert(mg::FOLD * mg::BK % BK == 0, "a fold boundary ends a slice");
  constexpr int FOLD_SLICES = mg::FOLD * mg::BK / BK;  // 64 fields per compensated fold
  constexpr uint32_t SLICE_BYTES = 2u * BK * C::BM * sizeof(float);
  // (cast straight from the shared array, so that the compiler keeps shared
  // loads for the operands: realigning through an integer made them generic)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemT<BK, STAGES>& sm = *reinterpret_cast<SmemT<BK, STAGES>*>(smem_raw);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.empty[s], NW);
    }
    sm.abort = 0;
    sm.p_next = 0;
    sm.p_done = 0;
    sy::bar_init_fence();
  }
  __syncthreads();
  const int nkb = (nf + BK - 1) / BK;
  // Tile schedule.  Static (tile_ctr null): this CTA's tiles are blockIdx.x,
  // blockIdx.x + gridDim.x, ...  Dynamic: the producer claims the next tile
  // of the walk from the grid-wide counter when it loads the tile's first
  // slice.  Either way the producer hands the tile's coordinates (I, J) to
  // the warps through tile_of (so no warp evaluates the walk); the tiles in
  // flight then always stay a window of about gridDim.x consecutive tiles
  // (which share their panels in L2), and a faster CTA simply takes more
  // tiles.  (Statically scheduled CTAs drift apart over the ~200 rounds at
  // nv = 32768 and re-read the panels from DRAM; making them meet fixes the
  // traffic but paces the grid at its slowest CTA.)
  constexpr bool dyn = DYN;  // (tile_ctr is used only when DYN)
  const int my_tiles = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
  // slices of this CTA (< 2^32, checked by the launcher); unbounded when dynamic
  const uint32_t n_slices = dyn ? 0xffffffffu : (uint32_t)my_tiles * (uint32_t)nkb;
  const bool producer = threadIdx.x == 0;
  // With sync_sl > 0 (static schedule only) the producers of all CTAs
  // (co-resident: cooperative launch) meet at the grid-wide counter every
  // sync_sl slices: a producer does not load chunk c of its round-r tile
  // before every CTA has loaded all earlier chunks.
  const int cpt = (!DYN && sync_sl > 0) ? (nkb + sync_sl - 1) / sync_sl : 0;  // chunks per tile
  // producer: loads its next slice (waiting until the ring stage is free);
  // false on abort
  // dynamic schedule: the producer's next claim, made one tile ahead of its
  // use so that the atomic's latency is not on the producer's (a compute
  // warp's) path; each CTA claims at most one tile past the end
  unsigned long long next_claim = 0;
  if (dyn && producer) next_claim = atomicAdd(tile_ctr, 1ull);
  auto issue_one = [&]() -> bool {
    SmemT<BK, STAGES>& sm = *reinterpret_cast<SmemT<BK, STAGES>*>(smem_raw);
    const uint32_t g = sm.p_next;
    if (sm.p_done || g >= n_slices) return true;
    const int s = (int)(g % STAGES);
    const uint32_t ph = (g / STAGES) & 1u;
    const int kb = (int)(g % (uint32_t)nkb);
    const int r = (int)(g / (uint32_t)nkb);  // this CTA's r-th tile
    int pI, pJ;
    if (!dyn && kb == 0) {
      mg::band_tile(blockIdx.x + (int64_t)r * gridDim.x, T, R0, R1, G, pI, pJ);
      sm.pI = pI;
      sm.pJ = pJ;
    }
    if (cpt && kb % sync_sl == 0 && (r | kb) != 0) {
      // CTAs holding a tile in round r, and the chunks issued before this one
      const int64_t P = min((int64_t)gridDim.x, ntiles - (int64_t)r * gridDim.x);
      const unsigned need = (unsigned)((int64_t)r * cpt * gridDim.x + (int64_t)(kb / sync_sl) * P);
      if (!sy::counter_wait(sync, need, &sm.abort, err, wait_ns)) return false;
    }
    if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) return false;
    if (dyn && kb == 0) {
      const unsigned long long t = next_claim;
      if (t < (unsigned long long)ntiles) next_claim = atomicAdd(tile_ctr, 1ull);
      if (t >= (unsigned long long)ntiles) {
        sm.tile_of[r % STAGES] = make_int2(-1, -1);
        sy::bar_arrive(&sm.full[s]);  // completes the phase with no copies: the warps see -1 and stop
        sm.p_done = 1;
        return true;
      }
      mg::band_tile((int64_t)t, T, R0, R1, G, pI, pJ);
      sm.pI = pI;
      sm.pJ = pJ;
    }
    // the tile's coordinates for the warps, published by the arrival below
    // (the stage being free means every warp has read entry r - STAGES)
    if (kb == 0) sm.tile_of[r % STAGES] = make_int2(sm.pI, sm.pJ);
    pI = sm.pI;
    pJ = sm.pJ;
    sy::bar_arrive_tx(&sm.full[s], SLICE_BYTES);
    sy::tma_load_2d(&sm.A[s][0][0], &mapV, pI * C::BM, kb * BK, &sm.full[s]);
    sy::tma_load_2d(&sm.B[s][0][0], &mapV, pJ * C::BN, kb * BK, &sm.full[s]);
    if (cpt && ((kb + 1) % sync_sl == 0 || kb + 1 == nkb)) atomicAdd(sync, 1u);
    sm.p_next = g + 1;
    return true;
  };
  if (producer)
    for (int p = 0; p < look; ++p)
      if (!issue_one()) break;

  const mg::Lanes<C> L;
  AccT<ADDS> acc;
  // lean epilogue for this call: FP32 or one-byte output and inputs inside
  // div_rn_lean's range (decided once, from NarrowPrep's words)
  const bool lean = EPI != 0 && (mode == OUT2_C2_F32 || mode == OUT2_C2_U8) && mg::lean_division_ok(lean_words);
  uint32_t it = 0;
  bool ok = true;
  for (int lt = 0; ok && (dyn || lt < my_tiles); ++lt) {
    int I = 0, J = 0;
    float Sfi[8], Sfj[C::NJ];
    acc.zero();
    for (int kb = 0; kb < nkb; ++kb, ++it) {
      if (producer) ok = issue_one();  // slice it + look
      const int s = (int)(it % STAGES);
      const uint32_t ph = (it / STAGES) & 1u;
      // every lane waits (each gets the barrier's acquire); the warp follows
      // the common verdict so that it never diverges here
      const bool mine = ok && sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns);
      if (!__all_sync(0xffffffffu, mine)) { ok = false; break; }
      if (kb == 0) {
        const int2 ij = sm.tile_of[lt % STAGES];
        I = ij.x;
        J = ij.y;
        if (I < 0) break;  // no tile left
      }
      if (EPI == 2 && kb == 0) {
        // the epilogue's sums, loaded while the tile computes
#pragma unroll
        for (int r = 0; r < 8; ++r) Sfi[r] = lean ? __ldg(Sf + min(I * C::BM + L.row(r), nv - 1)) : 0.0f;
#pragma unroll
        for (int c = 0; c < C::NJ; ++c) Sfj[c] = lean ? __ldg(Sf + min(J * C::BN + L.col(c), nv - 1)) : 0.0f;
      }
      compute_slice_tma<BK, KU>(&sm.A[s][0][L.am], &sm.B[s][0][L.bn], acc);
      __syncwarp();
      if (lane == 0) sy::bar_arrive(&sm.empty[s]);
      if (EPI != 2 && (kb + 1) % FOLD_SLICES == 0) acc.fold();
    }
    if (!ok || I < 0) break;
    if (EPI != 2) acc.fold();
    const int row0 = I * C::BM, col0 = J * C::BN;
    if (EPI != 0 && lean && col0 >= row0 + C::BM && col0 + C::BN <= nv) {
      if (EPI == 1) {
#pragma unroll
        for (int r = 0; r < 8; ++r) Sfi[r] = __ldg(Sf + row0 + L.row(r));
#pragma unroll
        for (int c = 0; c < C::NJ; ++c) Sfj[c] = __ldg(Sf + col0 + L.col(c));
      }
      // (EPI 2 never folds: hi is 0 and n2 is lo itself)
      if (mode == OUT2_C2_U8)
        mg::store_tile2_lean<C, true, true, EPI == 2>(acc, L, row0, col0, nv, Sfi, Sfj, out);
      else
        mg::store_tile2_lean<C, true, false, EPI == 2>(acc, L, row0, col0, nv, Sfi, Sfj, out);
    } else if constexpr (THRESH) {
      mg::thresh_append2<C::NJ>(acc, L, row0, col0, nv, S, ta);
    } else {
      mg::store_tile2<C, true>(acc, L, row0, col0, nv, S, out, mode);
    }
  }
  __syncthreads();
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
}

// ---- host side ----
template <int BK, int STAGES, int KU, int EPI = 0, bool DYN = false, int ADDS = 1, bool THRESH = false>
struct TmaLaunch {
  static constexpr size_t smem = sizeof(SmemT<BK, STAGES>);
  static cudaError_t run(ps_ctx* h, const VF32& V, const double* S, void* out, int mode, cudaStream_t st,
                         int T, int R0, int R1, int G, int64_t ntiles, int* err, unsigned* sync,
                         const NarrowPrep& np, const ThreshArgs& ta = ThreshArgs{}) {
    static std::mutex mu;
    static uint64_t attr_done = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      const uint64_t bit = 1ull << (h->device & 63);
      if (!(attr_done & bit)) {
        const cudaError_t e = cudaFuncSetAttribute(mgemm2_tma_kernel<BK, STAGES, KU, EPI, DYN, ADDS, THRESH>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done |= bit;
      }
    }
    CUtensorMap map;
    if (!sy::make_map_f32(&map, V.p, V.nv, V.nf, V.ld, C::BM, BK)) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)h->num_sms);
    // producers meet only when there is more than one round of tiles
    const int sync_sl = (ntiles > (int64_t)grid && h->mgemm_tma_sync > 0) ? h->mgemm_tma_sync : 0;
    // dynamic schedule: tile counter 8 bytes past the meeting counter
    unsigned long long* tile_ctr = DYN ? reinterpret_cast<unsigned long long*>(sync + 2) : nullptr;
    if (sync_sl || tile_ctr) {
      const cudaError_t e = cudaMemsetAsync(sync, 0, 16, st);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the meetings always end
    attr[0].val.cooperative = sync_sl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mgemm2_tma_kernel<BK, STAGES, KU, EPI, DYN, ADDS, THRESH>, map, (int)V.nv, (int)V.nf, S, out,
                              mode, T, R0, R1, G, ntiles, err, sync, sync_sl, tile_ctr, h->wait_ns, np.Sf, np.words,
                              h->tma_lookahead ? std::min(h->tma_lookahead, STAGES - 1) : STAGES - 1, ta);
  }
};

}  // namespace

cudaError_t launch_mgemm2_tma(ps_ctx* h, const VF32& V, const double* S, void* out, int mode, cudaStream_t st,
                              int T, int R0, int R1, int G, int64_t ntiles, int* err) {
  // TMA: 16-byte aligned base and row pitch; the tile walk assumes 128-wide tiles
  if ((uintptr_t)V.p % 16 != 0 || V.ld % 4 != 0 || V.nv < 1) return cudaErrorInvalidValue;
  // tile indices and per-CTA slice counts in 32 bits
  if (ntiles >= ((int64_t)1 << 31) ||
      (double)ceil_div(ntiles, h->num_sms) * (double)ceil_div(V.nf, 16) >= 4294967295.0)
    return cudaErrorInvalidValue;
  unsigned* sync = static_cast<unsigned*>(ws_get(h, WS_SYNC, 256));
  if (!sync) return cudaErrorMemoryAllocation;
  // the lean epilogue where the division is much of the work (n_f <= 256;
  // see mgemm2_tma_kernel's EPI), without the compensated fold up to 64
  // fields; at large n_f its registers would cost more than it saves
  const int epi = (mode == OUT2_C2_F32 || mode == OUT2_C2_U8) ? (V.nf <= 64 ? 2 : (V.nf <= 256 ? 1 : 0)) : 0;
  // k-steps per unrolled loop iteration: 16 (0 = automatic), 8 or 32
  const int ku = h->mgemm_tma_ku ? h->mgemm_tma_ku : 16;
  const int stages = h->mgemm_tma_stages;
  // slice width: 16 fields up to n_f = 32 (wider slices would be mostly zero
  // fill); for the plain epilogue (n_f > 256) 64 fields in a 3-stage ring
  // (half the waits and releases per field; 262.6 vs 266.8 ms at 32768 x
  // 8192) unless a 32-field variant is configured (add form, ring depth,
  // unroll) or the last 64-field slice would be mostly zero fill (n_f mod 64
  // in 1..32, below 2048 fields); else 32.  (Bands of 32 or 64 tile rows
  // would take 261.8 or 261.7 ms but read 93 or 118 GB from DRAM per launch
  // instead of 34 GB.)
  const bool knob32 = h->mgemm_add == 1 || h->mgemm_add == 2 || stages == 6 || ku != 16;
  const bool fill64 = V.nf >= 2048 || V.nf % 64 == 0 || V.nf % 64 > 32;
  const int bk =
      V.nf <= 32 ? 16 : (h->mgemm_tma_bk ? h->mgemm_tma_bk : (epi == 0 && !knob32 && fill64 ? 64 : 32));
  NarrowPrep np{nullptr, nullptr};
  if (epi) {
    float* Sf = static_cast<float*>(ws_get(h, WS_SUMSF, (size_t)round_up(V.nv, 64) * sizeof(float) + 256));
    if (!Sf) return cudaErrorMemoryAllocation;
    unsigned* words = reinterpret_cast<unsigned*>(Sf + round_up(V.nv, 64));
    const cudaError_t e = launch_narrow_prep(V, S, Sf, words, st);
    if (e != cudaSuccess) return e;
    np = NarrowPrep{Sf, words};
  }
  // dynamic tile schedule (the default) unless the producers are to meet,
  // which needs the static rounds; the other slice shapes are static only
  const bool dyn = h->mgemm_tma_dynamic && h->mgemm_tma_sync <= 0;
  // few fields: the kernel that overlaps each tile's epilogue with the next
  // tile's comparisons (unless a slice width is configured)
  if (epi == 2 && !h->mgemm_tma_bk && narrow_applies(h, V.nf, mode))
    return launch_mgemm2_narrow(h, V, np, out, mode, st, T, R0, R1, G, ntiles, err, sync);
#define PS_TMA_RUN(...) TmaLaunch<__VA_ARGS__>::run(h, V, S, out, mode, st, T, R0, R1, G, ntiles, err, sync, np)
  if (bk == 16) {
    // (16-field slices above n_f = 64 only when configured: the plain epilogue)
    if (epi == 2) return dyn ? PS_TMA_RUN(16, 8, 8, 2, true) : PS_TMA_RUN(16, 8, 8, 2);
    return dyn ? PS_TMA_RUN(16, 8, 8, 0, true) : PS_TMA_RUN(16, 8, 8);
  }
  if (bk == 64) return dyn ? PS_TMA_RUN(64, 3, 16, 0, true) : PS_TMA_RUN(64, 3, 16);
  if (epi == 2) return dyn ? PS_TMA_RUN(32, 4, 16, 2, true) : PS_TMA_RUN(32, 4, 16, 2);
  if (epi == 1) return dyn ? PS_TMA_RUN(32, 4, 16, 1, true) : PS_TMA_RUN(32, 4, 16, 1);
  if (stages == 6) return PS_TMA_RUN(32, 6, 16);
  // add forms other than the mixed default: packed (1) or scalar (2) adds
  if (h->mgemm_add == 1) return dyn ? PS_TMA_RUN(32, 4, 16, 0, true, 0) : PS_TMA_RUN(32, 4, 16, 0, false, 0);
  if (h->mgemm_add == 2) return dyn ? PS_TMA_RUN(32, 4, 16, 0, true, 2) : PS_TMA_RUN(32, 4, 16, 0, false, 2);
  if (ku == 8) return PS_TMA_RUN(32, 4, 8);
  if (ku == 32) return PS_TMA_RUN(32, 4, 32);
  return dyn ? PS_TMA_RUN(32, 4, 16, 0, true) : PS_TMA_RUN(32, 4, 16);
#undef PS_TMA_RUN
}

// The thresholded 2-way search (every pair with c2 >= tau) on the TMA-fed
// pipeline, over the whole upper triangle.
cudaError_t launch_mgemm2_thresh_tma(ps_ctx* h, const VF32& V, const double* S, const ThreshArgs& ta,
                                     cudaStream_t st, int* err) {
  if ((uintptr_t)V.p % 16 != 0 || V.ld % 4 != 0 || V.nv < 1 || V.nf < 1) return cudaErrorInvalidValue;
  const int T = (int)ceil_div(V.nv, C::BM);
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  if (ntiles >= ((int64_t)1 << 31) ||
      (double)ceil_div(ntiles, h->num_sms) * (double)ceil_div(V.nf, 16) >= 4294967295.0)
    return cudaErrorInvalidValue;
  unsigned* sync = static_cast<unsigned*>(ws_get(h, WS_SYNC, 256));
  if (!sync) return cudaErrorMemoryAllocation;
  const NarrowPrep np{nullptr, nullptr};
  const int G = std::max(1, h->mgemm_band);
  const bool dyn = h->mgemm_tma_dynamic && h->mgemm_tma_sync <= 0;
#define PS_TMAT_RUN(...) \
  TmaLaunch<__VA_ARGS__>::run(h, V, S, nullptr, OUT2_C2_F32, st, T, 0, T, G, ntiles, err, sync, np, ta)
  // slice widths as the packed-output kernel's
  const bool fill64 = V.nf >= 2048 || V.nf % 64 == 0 || V.nf % 64 > 32;
  if (V.nf <= 32) return dyn ? PS_TMAT_RUN(16, 8, 8, 0, true, 1, true) : PS_TMAT_RUN(16, 8, 8, 0, false, 1, true);
  if (V.nf > 256 && fill64)
    return dyn ? PS_TMAT_RUN(64, 3, 16, 0, true, 1, true) : PS_TMAT_RUN(64, 3, 16, 0, false, 1, true);
  return dyn ? PS_TMAT_RUN(32, 4, 16, 0, true, 1, true) : PS_TMAT_RUN(32, 4, 16, 0, false, 1, true);
#undef PS_TMAT_RUN
}

}  // namespace ps
