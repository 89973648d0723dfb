// ps_mgemm_narrow.cu -- the 2-way FP32 min-product (Section 3.1's mGEMM)
// for vectors of few fields (n_f <= 64), where writing the metrics costs as
// much as computing them.
//
// At n_f = 16 a pair takes 16 comparisons but also one correctly rounded
// division and one store.  The general TMA kernel computes a tile and then
// writes it, and since the 16 warps of a CTA all meet at the same slices,
// the SM alternates between a burst of FP32 mins (ALU pipe busy, store queue
// idle) and a burst of divisions and stores (the reverse).  Here a tile is
// one slice (BK >= n_f fields, zero fill past n_f is exact because
// min(0, x) = 0) and each warp writes the metrics of its previous tile while
// it computes the current one: the 32 divisions and stores of a lane's
// previous outputs are spread over the k-steps of the current tile, so the
// FP32 mins, the division arithmetic and the stores issue side by side.
//
// Pipeline: as in the general TMA kernel -- lane 0 of warp 0 is the
// producer, loads tile t + look (look < STAGES) into a ring of STAGES slices guarded by
// full / empty mbarriers, claims tiles from a grid-wide counter one tile
// ahead of their use (banded walk order), and hands each tile's (I, J) to the
// warps through a ring entry published by the stage's full barrier.  The
// producer writes ring entry s only after the stage's empty barrier showed
// that every warp released the slice that used entry s before, and a warp
// reads the entry before releasing its slice.
//
// Epilogue values are those of the other 2-way kernels bit for bit: n2 is the
// FP32 sum of the mins (at most 64 fields, no compensation needed), the
// metric 2 n2 / (S_i + S_j) with FP32 sums in which a zero sum is replaced by
// 1.0 (the pair's n2 is then 0 and so is the metric), computed as
// n2 / (S_i / 2 + S_j / 2) with div_rn_lean when the call's inputs lie in
// its range (decided once per launch from NarrowPrep's words), else as
// 2 n2 / (S_i + S_j) with __fdiv_rn.  Tiles on
// the diagonal or past the last vector are written at once, with guards;
// all others through the overlapped path.
//
// Thread -> output layout: a lane owns 8 rows x 4 columns, warp w rows
// 8w..8w+7 and lane l columns l, l + 32, l + 64, l + 96, so one store
// instruction writes 32 consecutive metrics of one row (4 or 5 32-byte
// sectors; one-byte codes 1 or 2).  The row operands are a shared-memory
// broadcast, the column operands four scalar loads per k-step.  (The general
// kernels' 64 x 16 warp blocks make each store instruction touch 8 rows x 4
// scattered columns, 16 sectors or more.)
// Every wait is bounded (ps_sync.cuh); on a timeout the kernel raises the
// handle's mapped error word, lets issued copies land and returns.
#include "ps_mgemm_impl.cuh"
#include "ps_sync.cuh"

#include <algorithm>
#include <mutex>

namespace ps {
namespace {

constexpr int BM = 128, BN = 128, NT = 512, NW = NT / 32;

template <int BK, int STAGES>
struct __align__(128) NarrowSmem {
  float A[STAGES][BK][BM];  // field q of the slice; 128 consecutive vectors
  float B[STAGES][BK][BN];
  unsigned long long full[STAGES];
  unsigned long long empty[STAGES];
  int2 tile_of[STAGES];  // (I, J) of the tile in stage s; I = -1: no tile left
  uint32_t p_next;       // producer: next tile (slice) to load
  int p_done;            // producer: the schedule is exhausted
  int abort;
};

// Thread -> output coordinates: rows row0 + ra + kr(r), columns
// col0 + cb + cs(c).
struct NLanes {
  int ra, cb;  // first row / column of this lane within the tile
  __device__ __forceinline__ NLanes() : ra(8 * (threadIdx.x >> 5)), cb(threadIdx.x & 31) {}
  static __device__ __forceinline__ constexpr int kr(int r) { return r; }
  static __device__ __forceinline__ constexpr int cs(int c) { return 32 * c; }
  __device__ __forceinline__ void load(const float* As, const float* Bs, int kk, float (&a)[8],
                                       float (&b)[4]) const {
    const float4 a0 = *reinterpret_cast<const float4*>(As + kk * BM + ra);
    const float4 a1 = *reinterpret_cast<const float4*>(As + kk * BM + ra + 4);
    a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
    a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = Bs[kk * BN + cb + 32 * c];
  }
};

// The previous tile's epilogue inputs, held while the next tile computes.
struct Prev {
  unsigned long long n2[8][2];  // FP32 pairs (columns 2p, 2p + 1)
  float Sfi[8], Sfj[4];
  int64_t off0;  // packed position of (row0 + ra, col0 + cb)
  int step0;     // nv - (row0 + ra) - 2: packed row start of row i + 1 minus that of row i, minus 1
};

__device__ __forceinline__ float n2_of(const unsigned long long (&p)[8][2], int r, int c) {
  const float2 v = mg::f2_unpack(p[r][c >> 1]);
  return (c & 1) ? v.y : v.x;
}

// The sums as the epilogue uses them: halved on the lean path, where
// n2 / (S_i / 2 + S_j / 2) = 2 n2 / (S_i + S_j) exactly (scaling by 2 commutes
// with rounding while every value is normal, which the lean range
// guarantees), saving the doubling of n2 per output.
template <bool LEAN>
__device__ __forceinline__ float sum_in(const float* __restrict__ Sf, int64_t i) {
  const float s = __ldg(Sf + i);
  return LEAN ? __fmul_rn(0.5f, s) : s;
}

// c2 from n2 and the sum d of two epilogue sums (sum_in)
template <bool LEAN>
__device__ __forceinline__ float metric(float n2, float d) {
  return LEAN ? div_rn_lean(n2, d) : __fdiv_rn(__fadd_rn(n2, n2), d);
}

// One-byte code of c2 (c2_code).  On the lean path its clamp at 255 never
// acts: with v >= 0, n2 <= min(S_i, S_j) <= (S_i + S_j) / 2, and the FP32 n2 (a
// sum of at most 64 mins) and the halved FP32 sums are within 64 and 3 units
// of 2^-24 of their exact values, so c2 <= 1 + 2^-17 and 255 c2 < 255.5,
// which rounds to the clamped code 255 anyway.  Dropping it saves an ALU-pipe
// instruction per output.
template <bool LEAN>
__device__ __forceinline__ unsigned char code_of(float q) {
  if (!LEAN) return c2_code(q);
  return (unsigned char)(__float_as_uint(__fadd_rn(__fmul_rn(255.0f, q), 8388608.0f)) & 0xffu);
}

// Output e (row e / 4, column e % 4) of the previous tile.  Row i + k starts
// k (nv - i - 2) - k (k - 1) / 2 positions after row i in the packed
// triangle (pair (i, j) at P(i) - i - 1 + j).
template <bool U8, bool LEAN>
__device__ __forceinline__ void store_prev(const Prev& pv, int e, bool on, void* __restrict__ out) {
  const int r = e >> 2, c = e & 3;
  const int k = NLanes::kr(r);
  const int64_t o = pv.off0 + (int64_t)k * pv.step0 - (k * (k - 1)) / 2 + NLanes::cs(c);
  const float q = metric<LEAN>(n2_of(pv.n2, r, c), __fadd_rn(pv.Sfi[r], pv.Sfj[c]));
  if (on) {
    if (U8)
      static_cast<unsigned char*>(out)[o] = code_of<LEAN>(q);
    else
      static_cast<float*>(out)[o] = q;
  }
}

__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}

// BK k-steps of the micro-kernel on a landed slice, with the previous tile's
// 32 outputs spread over all but the first K0 of them (stores predicated on
// `on`; the first k-steps give the previous tile's sums, loaded at its end,
// time to arrive: at 32768 vectors and n_f = 16 a delay of 4 of 16 k-steps
// measured 0.900 ms against 0.907 with 2 and 0.921 with 6; at n_f = 64 no
// delay 2.451 ms against 2.474 with 1).  The first k-step sets the sums
// instead of adding to zeros (0 + m = m for the mins m >= 0), which saves
// the zeroing and one packed add per pair of outputs.
template <int BK, bool U8, bool LEAN>
__device__ __forceinline__ void kloop(const NLanes& L, const float* As, const float* Bs,
                                      unsigned long long (&acc)[8][2], const Prev& pv, bool on,
                                      void* __restrict__ out) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    float a[8], b[4];
    L.load(As, Bs, kk, a, b);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int r = 0; r < 8; ++r)
        acc[r][p] = kk == 0 ? f2_pack(fminf(a[r], b[2 * p]), fminf(a[r], b[2 * p + 1]))
                            : mg::f2_add(acc[r][p], fminf(a[r], b[2 * p]), fminf(a[r], b[2 * p + 1]));
    constexpr int K0 = BK >= 64 ? 0 : 64 / BK, KE = BK - K0;
    if (kk >= K0) {
#pragma unroll
      for (int e = (kk - K0) * 32 / KE; e < (kk - K0 + 1) * 32 / KE; ++e) store_prev<U8, LEAN>(pv, e, on, out);
    }
  }
}

template <int BK, int STAGES, bool U8, bool LEAN>
__device__ __forceinline__ void narrow_body(NarrowSmem<BK, STAGES>& sm, const CUtensorMap* mapV, int nv,
                                            const float* __restrict__ Sf, void* __restrict__ out, int T,
                                            int R0, int R1, int G, int64_t ntiles, int* err,
                                            unsigned long long* __restrict__ tile_ctr,
                                            unsigned long long wait_ns, int look) {
  constexpr uint32_t SLICE_BYTES = 2u * BK * BM * sizeof(float);
  const int lane = threadIdx.x & 31;
  const bool producer = threadIdx.x == 0;
  unsigned long long next_claim = 0;
  const int64_t tiles_before = (int64_t)R0 * T - (int64_t)R0 * (R0 - 1) / 2;  // tiles in rows [0, R0)
  if (producer) next_claim = atomicAdd(tile_ctr, 1ull);
  // producer: loads the next tile (waiting until its ring stage is free);
  // false on abort
  auto issue_one = [&]() -> bool {
    const uint32_t g = sm.p_next;
    if (sm.p_done) return true;
    const int s = (int)(g % STAGES);
    const uint32_t ph = (g / STAGES) & 1u;
    if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) return false;
    const unsigned long long t = next_claim;
    if (t < (unsigned long long)ntiles) next_claim = atomicAdd(tile_ctr, 1ull);
    if (t >= (unsigned long long)ntiles) {
      sm.tile_of[s] = make_int2(-1, -1);
      sy::bar_arrive(&sm.full[s]);  // completes the phase with no copies: the warps see -1 and stop
      sm.p_done = 1;
      return true;
    }
    // tile walk: banded (band_tile) for 16- and 32-field slices; row-major
    // for 64-field ones, whose tiles take four times longer (at 32768 vectors
    // n_f = 16: 0.900 ms banded against 0.913 row-major, n_f = 64: 2.452
    // against 2.406).  V fits in L2 at these widths either way.
    int I, J;
    if (BK >= 64)
      mg::tri_tile(tiles_before + (int64_t)t, T, I, J);
    else
      mg::band_tile((int64_t)t, T, R0, R1, G, I, J);
    sm.tile_of[s] = make_int2(I, J);
    sy::bar_arrive_tx(&sm.full[s], SLICE_BYTES);
    sy::tma_load_2d(&sm.A[s][0][0], mapV, I * BM, 0, &sm.full[s]);
    sy::tma_load_2d(&sm.B[s][0][0], mapV, J * BN, 0, &sm.full[s]);
    sm.p_next = g + 1;
    return true;
  };
  bool ok = true;
  if (producer)
    for (int p = 0; p < look && ok; ++p) ok = issue_one();

  const NLanes L;
  // One tile: wait for it, compute it into nx.n2 while the previous tile's
  // metrics (pv, when `have`) are written, release it, and leave in nx what
  // the next tile needs to write this one's metrics -- or, for a diagonal or
  // ragged tile, write them now with guards (rows past nv only occur in
  // diagonal tiles).  False when the schedule has ended or the call aborts.
  auto tile = [&](const Prev& pv, Prev& nx, bool& have, uint32_t lt) -> bool {
    if (producer) ok = issue_one();  // tile lt + look
    const int s = (int)(lt % STAGES);
    const uint32_t ph = (lt / STAGES) & 1u;
    // every lane waits (each gets the barrier's acquire); the warp follows
    // the common verdict so that it never diverges here
    const bool mine = ok && sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns);
    if (!__all_sync(0xffffffffu, mine)) {
      ok = false;
      return false;
    }
    const int2 ij = sm.tile_of[s];
    if (ij.x < 0) return false;  // no tile left
    kloop<BK, U8, LEAN>(L, &sm.A[s][0][0], &sm.B[s][0][0], nx.n2, pv, have, out);
    __syncwarp();
    if (lane == 0) sy::bar_arrive(&sm.empty[s]);
    const int row0 = ij.x * BM, col0 = ij.y * BN;
    if (col0 >= row0 + BM && col0 + BN <= nv) {
      // the lane's 8 rows are consecutive and start at a multiple of 8: two
      // 16-byte loads (rows below col0 < nv, so in bounds)
      const float4 s0 = __ldg(reinterpret_cast<const float4*>(Sf + row0 + L.ra));
      const float4 s1 = __ldg(reinterpret_cast<const float4*>(Sf + row0 + L.ra + 4));
      const float sr[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r) nx.Sfi[r] = LEAN ? __fmul_rn(0.5f, sr[L.kr(r)]) : sr[L.kr(r)];
#pragma unroll
      for (int c = 0; c < 4; ++c) nx.Sfj[c] = sum_in<LEAN>(Sf, col0 + L.cb + L.cs(c));
      const int64_t i = row0 + L.ra;
      nx.off0 = mg::pair_index(nv, i, i + 1) - (i + 1) + col0 + L.cb;
      nx.step0 = nv - (int)i - 2;
      have = true;
      return true;
    }
    have = false;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.ra + L.kr(r);
      if (i >= nv) continue;
      const float Sfi = sum_in<LEAN>(Sf, i);
      const int64_t base = mg::pair_index(nv, i, i + 1) - (i + 1);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = col0 + L.cb + L.cs(c);
        if (j <= i || j >= nv) continue;
        const float q = metric<LEAN>(n2_of(nx.n2, r, c), __fadd_rn(Sfi, sum_in<LEAN>(Sf, j)));
        if (U8)
          static_cast<unsigned char*>(out)[base + j] = code_of<LEAN>(q);
        else
          static_cast<float*>(out)[base + j] = q;
      }
    }
    return true;
  };
  auto flush = [&](const Prev& pv) {
#pragma unroll
    for (int e = 0; e < 32; ++e) store_prev<U8, LEAN>(pv, e, true, out);
  };
  Prev P0, P1;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    P0.n2[r][0] = P0.n2[r][1] = 0ull;
    P0.Sfi[r] = 1.0f;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) P0.Sfj[c] = 1.0f;
  P0.off0 = 0;
  P0.step0 = 0;
  bool have = false;  // warp-uniform: a previous tile's metrics are pending
  // (P1 is copied into P0 after each tile: alternating the two sets instead
  // doubles the unrolled loop body, and the instruction-cache misses cost
  // more than the copies save -- 1.17 vs 1.06 ms at 32768 x 16)
  for (uint32_t lt = 0;; ++lt) {
    if (!tile(P0, P1, have, lt)) {
      if (ok && have) flush(P0);
      break;
    }
    P0 = P1;
  }
}

template <int BK, int STAGES, bool U8>
__global__ void __launch_bounds__(NT, 1)
    mgemm2_narrow_kernel(const __grid_constant__ CUtensorMap mapV, int nv, const float* __restrict__ Sf,
                         const unsigned* __restrict__ lean_words, void* __restrict__ out, int T, int R0,
                         int R1, int G, int64_t ntiles, int* err, unsigned long long* __restrict__ tile_ctr,
                         unsigned long long wait_ns, int look) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  NarrowSmem<BK, STAGES>& sm = *reinterpret_cast<NarrowSmem<BK, STAGES>*>(smem_raw);
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
  // div_rn_lean's range holds for the whole call, or __fdiv_rn everywhere
  if (mg::lean_division_ok(lean_words))
    narrow_body<BK, STAGES, U8, true>(sm, &mapV, nv, Sf, out, T, R0, R1, G, ntiles, err, tile_ctr, wait_ns, look);
  else
    narrow_body<BK, STAGES, U8, false>(sm, &mapV, nv, Sf, out, T, R0, R1, G, ntiles, err, tile_ctr, wait_ns, look);
  __syncthreads();
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
}

template <int BK, int STAGES, bool U8>
cudaError_t run_narrow(ps_ctx* h, const VF32& V, const NarrowPrep& np, void* out, cudaStream_t st, int T, int R0,
                       int R1, int G, int64_t ntiles, int* err, unsigned long long* tile_ctr) {
  constexpr size_t smem = sizeof(NarrowSmem<BK, STAGES>);
  static std::mutex mu;
  static uint64_t attr_done = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    const uint64_t bit = 1ull << (h->device & 63);
    if (!(attr_done & bit)) {
      const cudaError_t e = cudaFuncSetAttribute(mgemm2_narrow_kernel<BK, STAGES, U8>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_done |= bit;
    }
  }
  CUtensorMap map;
  if (!sy::make_map_f32(&map, V.p, V.nv, V.nf, V.ld, BM, BK)) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)h->num_sms);
  // tiles the producer loads ahead of the one the warps compute (it then
  // waits for the release of tile t + look - STAGES)
  const int look = h->tma_lookahead ? std::min(h->tma_lookahead, STAGES - 1) : STAGES - 1;
  mgemm2_narrow_kernel<BK, STAGES, U8><<<grid, NT, smem, st>>>(map, (int)V.nv, np.Sf, np.words, out, T, R0,
                                                               R1, G, ntiles, err, tile_ctr, h->wait_ns, look);
  return cudaGetLastError();
}

}  // namespace

bool narrow_applies(const ps_ctx* h, int64_t nf, int mode) {
  return nf <= 64 && (mode == OUT2_C2_F32 || mode == OUT2_C2_U8) && h->mgemm_narrow != 2 &&
         h->mgemm_tma_dynamic && h->mgemm_tma_sync <= 0;
}

cudaError_t launch_mgemm2_narrow(ps_ctx* h, const VF32& V, const NarrowPrep& np, void* out, int mode,
                                 cudaStream_t st, int T, int R0, int R1, int G, int64_t ntiles, int* err,
                                 unsigned* sync) {
  unsigned long long* tile_ctr = reinterpret_cast<unsigned long long*>(sync + 2);
  cudaError_t e = cudaMemsetAsync(tile_ctr, 0, 8, st);
  if (e != cudaSuccess) return e;
  const bool u8 = mode == OUT2_C2_U8;
#define PS_NARROW(BK, ST)                                                                   \
  (u8 ? run_narrow<BK, ST, true>(h, V, np, out, st, T, R0, R1, G, ntiles, err, tile_ctr) \
      : run_narrow<BK, ST, false>(h, V, np, out, st, T, R0, R1, G, ntiles, err, tile_ctr))
  if (V.nf <= 16) return PS_NARROW(16, 8);
  if (V.nf <= 32) return PS_NARROW(32, 6);
  return PS_NARROW(64, 3);
#undef PS_NARROW
}

}  // namespace ps
