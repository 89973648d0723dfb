// ps_mgemm_impl.cuh -- templated device code of the FP32 min-product kernels.
//
// The paper's "mGEMM" (Section 3.1): (A min B)_{ij} = sum_k min(a_ik, b_kj),
// a GEMM whose multiply is replaced by min.  There is no tensor-core form of
// min on FP32 data, so the inner loop is one FP32 min (FMNMX, ALU pipe) plus
// one FP32 add (FMA pipe) per element pair.
//
// Design (sm_103a):
//  * A warp owns a 64 x 32 output block, 8 x 8 outputs per lane (two 4-wide
//    groups per dimension, so every 128-bit shared load is a conflict-free
//    broadcast).  Tile shapes: 128 x 128 (2 x 4 warps, 1 CTA/SM) and 64 x 64
//    (1 x 2 warps, 4 CTAs/SM; less edge waste on small or 3-way problems).
//  * Operands stream through a 4-stage cp.async (16-byte, zero-filling)
//    shared-memory ring of 16-field slices; zero fill is exact because
//    min(0, x) = 0 for the non-negative data of Section 2.1.
//  * Accumulation: each accumulator sums 64 fields in FP32 ("lo"), then is
//    folded into a running "hi" with an exact TwoSum, leaving the rounding
//    residual in "lo"; hi + lo carries at most 63 roundings of a 64-term
//    non-negative partial sum: relative error <= 64 u (u = 2^-24).
//  * Pairs: only upper-triangle tiles I <= J (Section 3.1, lower-triangle
//    blocks skipped).  Triples: (pivot j, I, K) tiles with rows i < j and
//    columns k > j (Section 3.2: only the part of B_j holding i < j < k); the
//    pivot column v_j is min-ed into each thread's own A chunks as soon as
//    they land (X_j = min(V, v_j) is never materialised).
#pragma once

#include "ps_internal.cuh"

namespace ps {
namespace mg {

constexpr int BK = 16, STAGES = 4;
constexpr int FOLD = 4;  // stages (of BK fields) per compensated fold: 64 fields

// WM x WN warps; a warp owns 64 rows x 4*NJ columns, a lane 8 x NJ outputs
// (NJ = 8: two 4-column groups 16 apart; NJ = 4: one group).
template <int WM_, int WN_, int MINB_, int NJ_ = 8>
struct TileCfg {
  static constexpr int WM = WM_, WN = WN_, NJ = NJ_;
  static constexpr int BM = 64 * WM, BN = 4 * NJ * WN;
  static constexpr int NT = 32 * WM * WN;
  static constexpr int MINB = MINB_;               // resident CTAs per SM
  static constexpr int CHA = BK * BM / 4 / NT;    // 16-byte A chunks per thread
  static constexpr int CHB = BK * BN / 4 / NT;
  static_assert(BM == BN, "square tiles");
  static_assert(CHA * NT * 4 == BK * BM && CHB * NT * 4 == BK * BN, "chunking");
};
using T128 = TileCfg<2, 4, 1>;
using T64 = TileCfg<1, 2, 4>;
using T128W16 = TileCfg<2, 8, 1, 4>;  // 128 x 128, 16 warps of 8 x 4 outputs per lane

template <class C>
struct __align__(16) Smem {
  float A[STAGES][BK][C::BM];
  float B[STAGES][BK][C::BN];
  float P[STAGES][BK];  // pivot value of each slice row
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies of one BK-field slice of the A rows [row0,row0+BM) and B columns
// [col0,col0+BN) into ring buffer `buf`; thread t copies the 16-byte chunks
// t, t+NT, ... of each operand.  With a pivot, the owner of a slice row's
// first chunk also copies that row's pivot value; a row has BM/4 >= 16
// consecutive chunks, so all owners of a row sit in one warp.
template <class C, bool PIVOT>
__device__ __forceinline__ void issue_slice(Smem<C>& sm, int buf, const VF32& V, int row0,
                                            int col0, int k0, int jpiv) {
  const int t = threadIdx.x;
  constexpr int PA = C::BM / 4, PB = C::BN / 4;  // chunks per slice row
#pragma unroll
  for (int h = 0; h < C::CHA; ++h) {
    const int c = t + h * C::NT;
    const int r = c / PA, c4 = (c % PA) * 4;
    const int q = k0 + r;
    const int i = row0 + c4;
    const int bytes = (q < V.nf && i < V.nv) ? min(16, 4 * (V.nv - i)) : 0;
    cp_async16(&sm.A[buf][r][c4], bytes ? V.p + (int64_t)q * V.ld + i : V.p, bytes);
    if (PIVOT && c % PA == 0) {  // the row's first chunk owner copies its pivot value
      const int pb = q < V.nf ? 4 : 0;
      cp_async4(&sm.P[buf][r], pb ? V.p + (int64_t)q * V.ld + jpiv : V.p, pb);
    }
  }
#pragma unroll
  for (int h = 0; h < C::CHB; ++h) {
    const int c = t + h * C::NT;
    const int r = c / PB, c4 = (c % PB) * 4;
    const int q = k0 + r;
    const int jx = col0 + c4;
    const int bytes = (q < V.nf && jx < V.nv) ? min(16, 4 * (V.nv - jx)) : 0;
    cp_async16(&sm.B[buf][r][c4], bytes ? V.p + (int64_t)q * V.ld + jx : V.p, bytes);
  }
}

// X_j = min(V, v_j) on this thread's own A chunks of buffer `buf`.  Every
// thread has waited for its own copies; the warp barrier makes the pivot
// values copied by the row owners in this warp visible.
template <class C>
__device__ __forceinline__ void pivot_min_slice(Smem<C>& sm, int buf) {
  const int t = threadIdx.x;
  constexpr int PA = C::BM / 4;
  static_assert(PA >= 16 && 32 % (PA > 32 ? 32 : PA) == 0, "row owners share a warp");
  __syncwarp();
#pragma unroll
  for (int h = 0; h < C::CHA; ++h) {
    const int c = t + h * C::NT;
    const int r = c / PA, c4 = (c % PA) * 4;
    const float p = sm.P[buf][r];
    float4 a = *reinterpret_cast<float4*>(&sm.A[buf][r][c4]);
    a.x = fminf(a.x, p);
    a.y = fminf(a.y, p);
    a.z = fminf(a.z, p);
    a.w = fminf(a.w, p);
    *reinterpret_cast<float4*>(&sm.A[buf][r][c4]) = a;
  }
}

// Packed FP32 pair add (sm_100+ add.rn.f32x2): two accumulators per issue.
__device__ __forceinline__ unsigned long long f2_add(unsigned long long acc, float x, float y) {
  unsigned long long r;
  asm("{\n\t.reg .b64 t;\n\tmov.b64 t, {%2, %3};\n\tadd.rn.f32x2 %0, %1, t;\n\t}"
      : "=l"(r)
      : "l"(acc), "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// Per-thread accumulators for 8 x NJ outputs: "lo" accumulates up to 64
// fields; fold() moves it into "hi" with an exact TwoSum and leaves the
// rounding residual in "lo".  PACKED adds pairs with one add.rn.f32x2.
template <bool PACKED, int NJ>
struct Acc;

template <int NJ>
struct Acc<true, NJ> {
  static constexpr int NP = NJ / 2;
  unsigned long long hi[8][NP];
  unsigned long long lo[8][NP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NP; ++c) hi[r][c] = lo[r][c] = 0ull;
  }
  __device__ __forceinline__ void step(const float (&a)[8], const float (&b)[NJ]) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NP; ++c)
        lo[r][c] = f2_add(lo[r][c], fminf(a[r], b[2 * c]), fminf(a[r], b[2 * c + 1]));
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const unsigned long long s = f2_add2(hi[r][c], lo[r][c]);
        const unsigned long long bp = f2_sub2(s, hi[r][c]);
        const unsigned long long ap = f2_sub2(s, bp);
        const unsigned long long e = f2_add2(f2_sub2(hi[r][c], ap), f2_sub2(lo[r][c], bp));
        hi[r][c] = s;
        lo[r][c] = e;
      }
  }
  __device__ __forceinline__ float2 hl(int r, int c) const {
    const float2 h = f2_unpack(hi[r][c >> 1]);
    const float2 l = f2_unpack(lo[r][c >> 1]);
    return (c & 1) ? make_float2(h.y, l.y) : make_float2(h.x, l.x);
  }
};

// 8 x 4 accumulators with the adds split between the two forms: columns 0
// and 1 by one packed add.rn.f32x2, columns 2 and 3 by scalar adds (every
// element sees the same round-to-nearest adds in the same order as in
// Acc<true, 4>, so the values are identical).  fold(), hl() as in Acc.  The
// step is written column by column (measured 0.4% faster than row by row in
// the 2-way kernel: 261.7 vs 262.8 ms).
template <int NJ>
struct AccMix {
  static_assert(NJ == 4, "4 columns per lane");
  unsigned long long hp[8], lp[8];  // columns 0, 1
  float hs[8][2], ls[8][2];         // columns 2, 3
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      hp[r] = lp[r] = 0ull;
      hs[r][0] = hs[r][1] = ls[r][0] = ls[r][1] = 0.0f;
    }
  }
  __device__ __forceinline__ void step(const float (&a)[8], const float (&b)[NJ]) {
#pragma unroll
    for (int r = 0; r < 8; ++r) lp[r] = f2_add(lp[r], fminf(a[r], b[0]), fminf(a[r], b[1]));
#pragma unroll
    for (int r = 0; r < 8; ++r) ls[r][0] = __fadd_rn(ls[r][0], fminf(a[r], b[2]));
#pragma unroll
    for (int r = 0; r < 8; ++r) ls[r][1] = __fadd_rn(ls[r][1], fminf(a[r], b[3]));
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const unsigned long long s = f2_add2(hp[r], lp[r]);
      const unsigned long long bp = f2_sub2(s, hp[r]);
      const unsigned long long ap = f2_sub2(s, bp);
      lp[r] = f2_add2(f2_sub2(hp[r], ap), f2_sub2(lp[r], bp));
      hp[r] = s;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float t = __fadd_rn(hs[r][c], ls[r][c]);
        const float bq = __fsub_rn(t, hs[r][c]);
        const float aq = __fsub_rn(t, bq);
        ls[r][c] = __fadd_rn(__fsub_rn(hs[r][c], aq), __fsub_rn(ls[r][c], bq));
        hs[r][c] = t;
      }
    }
  }
  __device__ __forceinline__ float2 hl(int r, int c) const {
    if (c >= 2) return make_float2(hs[r][c - 2], ls[r][c - 2]);
    const float2 h = f2_unpack(hp[r]);
    const float2 l = f2_unpack(lp[r]);
    return (c & 1) ? make_float2(h.y, l.y) : make_float2(h.x, l.x);
  }
};

template <int NJ>
struct Acc<false, NJ> {
  float hi[8][NJ];
  float lo[8][NJ];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NJ; ++c) hi[r][c] = lo[r][c] = 0.0f;
  }
  __device__ __forceinline__ void step(const float (&a)[8], const float (&b)[NJ]) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NJ; ++c) lo[r][c] = __fadd_rn(lo[r][c], fminf(a[r], b[c]));
  }
  // Two consecutive fields at once: a[r], b[c] hold (field k, field k+1) as
  // half2; one packed min, then both halves added to the FP32 accumulator in
  // field order (mixed-precision FP16 + FP32 -> FP32 adds).
  __device__ __forceinline__ void step_h(const uint32_t (&a)[8], const uint32_t (&b)[NJ]) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NJ; ++c) {
        uint32_t m;
        asm("min.f16x2 %0, %1, %2;" : "=r"(m) : "r"(a[r]), "r"(b[c]));
        float x = lo[r][c];
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.f16 %0, l, %0;\n\t"
            "add.rn.f32.f16 %0, h, %0;\n\t}"
            : "+f"(x)
            : "r"(m));
        lo[r][c] = x;
      }
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < NJ; ++c) {
        const float s = __fadd_rn(hi[r][c], lo[r][c]);
        const float bp = __fsub_rn(s, hi[r][c]);
        const float ap = __fsub_rn(s, bp);
        const float e = __fadd_rn(__fsub_rn(hi[r][c], ap), __fsub_rn(lo[r][c], bp));
        hi[r][c] = s;
        lo[r][c] = e;
      }
  }
  __device__ __forceinline__ float2 hl(int r, int c) const { return make_float2(hi[r][c], lo[r][c]); }
};

// BK k-steps of the micro-kernel on ring buffer `buf`, KU steps per loop
// iteration (smaller KU keeps the hot loop in the instruction cache).
template <class C, bool PACKED, int KU, bool HALF = false>
__device__ __forceinline__ void compute_slice(const Smem<C>& sm, int buf, int am, int bn,
                                              Acc<PACKED, C::NJ>& acc) {
  const float* As = &sm.A[buf][0][am];
  const float* Bs = &sm.B[buf][0][bn];
  if constexpr (HALF) {  // 4-byte elements hold half2 field pairs
#pragma unroll KU
    for (int kk = 0; kk < BK; ++kk) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(As + kk * C::BM);
      const uint4 a1 = *reinterpret_cast<const uint4*>(As + kk * C::BM + 32);
      const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const uint4 b0 = *reinterpret_cast<const uint4*>(Bs + kk * C::BN);
      if constexpr (C::NJ == 8) {
        const uint4 b1 = *reinterpret_cast<const uint4*>(Bs + kk * C::BN + 16);
        const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        acc.step_h(a, b);
      } else {
        const uint32_t b[4] = {b0.x, b0.y, b0.z, b0.w};
        acc.step_h(a, b);
      }
    }
    return;
  } else {
#pragma unroll KU
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + kk * C::BM);
    const float4 a1 = *reinterpret_cast<const float4*>(As + kk * C::BM + 32);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * C::BN);
    if constexpr (C::NJ == 8) {
      const float4 b1 = *reinterpret_cast<const float4*>(Bs + kk * C::BN + 16);
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
      acc.step(a, b);
    } else {
      const float b[4] = {b0.x, b0.y, b0.z, b0.w};
      acc.step(a, b);
    }
  }
  }
}

// Full k loop over n_f for one (row0, col0) tile, with optional pivot j.
template <class C, bool PIVOT, bool PACKED, int KU, bool HALF = false>
__device__ __forceinline__ void tile_minsum(Smem<C>& sm, const VF32& V, int row0, int col0,
                                            int jpiv, int am, int bn, Acc<PACKED, C::NJ>& acc,
                                            bool active = true) {
  acc.zero();
  const int nst = (V.nf + BK - 1) / BK;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nst) issue_slice<C, PIVOT>(sm, s, V, row0, col0, s * BK, jpiv);
    cp_async_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int buf = s % STAGES;
    cp_async_wait<STAGES - 2>();
    if (PIVOT) pivot_min_slice<C>(sm, buf);
    __syncthreads();
    const int sn = s + STAGES - 1;
    if (sn < nst) issue_slice<C, PIVOT>(sm, sn % STAGES, V, row0, col0, sn * BK, jpiv);
    cp_async_commit();
    // (a warp with no valid output in this tile only helps stage the ring)
    if (active) compute_slice<C, PACKED, KU, HALF>(sm, buf, am, bn, acc);
    if ((s + 1) % FOLD == 0) acc.fold();
  }
  acc.fold();
  cp_async_wait<0>();
  __syncthreads();  // the ring is reused by the next tile
}

// Thread -> output coordinates inside the tile.
template <class C>
struct Lanes {
  int am, bn;  // smem column offsets of the A / B fragments
  __device__ __forceinline__ Lanes() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp / C::WN, wn = warp % C::WN, lm = lane >> 2, ln = lane & 3;
    am = wm * 64 + lm * 4;
    bn = wn * (4 * C::NJ) + ln * 4;
  }
  __device__ __forceinline__ int row(int r) const { return am + (r < 4 ? r : 28 + r); }
  __device__ __forceinline__ int col(int c) const { return bn + (c < 4 ? c : 12 + c); }
};

// Thread -> output coordinates of the 16-warp 128 x 128 tile (T128W16) in
// the TMA-fed 3-way and batched kernels (same interface as Lanes).  A warp
// owns a 32 x 32 block: lane (lm, ln) = (lane / 8, lane % 8) rows
// 4 lm + {0..3} and 16 + 4 lm + {0..3}, columns 4 ln + {0..3} (the two A
// loads are broadcasts over 4 addresses, the B load 8 consecutive 16-byte
// words).  In a 3-way tile that straddles the pivot, warps whose whole block
// has no row i < j or no column k > j skip the min-add loop; of the block
// shapes a warp of 8 x 4-output lanes can take, 32 x 32 wastes least (at
// nv = 2048 the active blocks hold 95.6% useful outputs, 64 x 16 blocks
// 94.5%).  A skipped warp only helps if another warp on the same scheduler
// (warps w, w+4, w+8, w+12 share one) takes the pipe, so warp w = 4g + s
// (scheduler s) takes block (row block g, column block (g + s) mod 4): every
// scheduler holds one block of each row block and of each column block, and
// skipping whole row blocks at the bottom or whole column blocks at the left
// removes the same number of blocks from every scheduler.
struct Lanes3 {
  static constexpr int BH = 32, BW = 32;  // warp block rows, columns
  static constexpr int RUN = 16;          // offset of a lane's second run of 4 rows
  int am, bn;        // smem column offsets of the A / B fragments
  int wrow0, wcol0;  // first row / column of this warp's block
  __device__ __forceinline__ Lanes3() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp >> 2, s = warp & 3;
    wrow0 = g * BH;
    wcol0 = ((g + s) & 3) * BW;
    am = wrow0 + (lane >> 3) * 4;
    bn = wcol0 + (lane & 7) * 4;
  }
  __device__ __forceinline__ int row(int r) const { return am + (r < 4 ? r : RUN - 4 + r); }
  __device__ __forceinline__ int col(int c) const { return bn + c; }
};

__host__ __device__ __forceinline__ int64_t pair_index(int64_t nv, int64_t i, int64_t j) {
  return i * (2 * nv - i - 1) / 2 + (j - i - 1);
}

// Upper-triangle tile index t -> (I, J), I <= J < T, row-major.
// Row i is the largest with i*T - i(i-1)/2 <= t: an FP32 estimate from the
// quadratic formula (no FP64, whose pipe is slow on this part), made exact by
// the integer steps below.
__host__ __device__ __forceinline__ void tri_tile(int64_t t, int T, int& I, int& J) {
  const float b = 2.0f * (float)T + 1.0f;
  const float disc = fmaxf(b * b - 8.0f * (float)t, 0.0f);
  int i = (int)((b - sqrtf(disc)) * 0.5f);
  i = max(0, min(i, T - 1));
  while (i > 0 && (int64_t)i * T - (int64_t)i * (i - 1) / 2 > t) --i;
  while (i + 1 < T && (int64_t)(i + 1) * T - (int64_t)(i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (int)(t - ((int64_t)i * T - (int64_t)i * (i - 1) / 2));
}

// Tiles of tile rows [R0, R1) of the upper triangle (every J >= I < T), in
// bands of G tile rows: the band's diagonal triangle first, then G-wide
// column chunks from left to right, each chunk column by column.  Consecutive
// indices (the tiles the persistent CTAs hold at one time) then share a band's
// G row panels and a few column panels, which stay in L2; the row-major walk
// re-reads each column panel from DRAM once per tile row instead of once per
// band.  Index t counts from the first tile of row R0.
__host__ __device__ __forceinline__ void band_tile(int64_t t, int T, int R0, int R1, int G, int& I, int& J) {
  auto P = [T](int64_t r) { return r * T - r * (r - 1) / 2; };  // tiles in rows [0, r)
  int gi, gj;
  tri_tile(P(R0) + t, T, gi, gj);
  const int b0 = R0 + ((gi - R0) / G) * G;
  const int g = min(G, R1 - b0);
  int64_t u = P(R0) + t - P(b0);
  const int64_t diag = (int64_t)g * (g + 1) / 2;
  if (u < diag) {
    int li, lj;
    tri_tile(u, g, li, lj);
    I = b0 + li;
    J = b0 + lj;
  } else {
    u -= diag;
    const int64_t c = u / ((int64_t)g * G);
    const int64_t v = u - c * g * G;
    I = b0 + (int)(v % g);
    J = b0 + g + (int)(c * G + v / g);
  }
}

// Section 2.2 eq. (1): n3 = ((n2(ij) + n2(ik)) + n2(jk)) - n3', then
// c3 = (3/2) n3 / d3 with d3 = (S_i + S_j) + S_k, all in FP32 (the FP64
// pipe runs at a small fraction of the FP32 rate on this part).  Exact for
// integer data whose sums stay below 2^24; otherwise a few FP32 roundings:
// per field (a <= b <= c) the n2 terms add to 2a + b <= 1.5 (a + b), so n3
// suffers no cancellation.
__device__ __forceinline__ float c3_value(float2 n3p_hl, float n2ij, float n2ik, float n2jk,
                                          float d3) {
  const float n3p = __fadd_rn(n3p_hl.x, n3p_hl.y);
  const float n3 = __fsub_rn(__fadd_rn(__fadd_rn(n2ij, n2ik), n2jk), n3p);
  return (d3 == 0.0f) ? 0.0f : __fdiv_rn(1.5f * n3, d3);
}

// Pivot-slab offset: sum_{j'=jb}^{j-1} j'(n-1-j') = F(j) - F(jb),
// F(x) = (n-1) x(x-1)/2 - (x-1) x (2x-1)/6.
__host__ __device__ __forceinline__ int64_t slab_offset(int64_t n, int64_t jb, int64_t j) {
  auto F = [n](int64_t x) { return (n - 1) * (x * (x - 1) / 2) - (x - 1) * x * (2 * x - 1) / 6; };
  return F(j) - F(jb);
}

// Tiles (tile width B) of pivot j: I tiles covering rows [0, j) times K tiles
// covering columns (j, nv).
__host__ __device__ __forceinline__ int64_t pivot_tiles(int nv, int64_t j, int B) {
  const int64_t Tk = (nv + B - 1) / B;
  const int64_t nI = (j + B - 1) / B;
  const int64_t nK = (j + 1 < nv) ? (Tk - (j + 1) / B) : 0;
  return nI * nK;
}

// Epilogue of one 2-way tile (Section 2.1): the n2 table (both triangles), or
// c2 = 2 n2 / (S_i + S_j) into the packed strict upper triangle as FP32,
// FP64 or one-byte codes.  FP32 output: d = fl32(fl32(S_i) + fl32(S_j));
// exact, like the FP64 sum, whenever the sums are integers below 2^24 (the
// FP64 pipe, at a small fraction of the FP32 rate, would otherwise bound the
// epilogue at small n_f).  Tiles strictly above the diagonal and inside the
// matrix (every i < j < nv) take a path without per-output checks.  Every
// path gives the same correctly rounded values (store_tile2_lean below
// too).
template <class C, bool PACKED, class LN = Lanes<C>, class ACC = Acc<PACKED, C::NJ>>
__device__ __forceinline__ void store_tile2(const ACC& acc, const LN& L, int row0,
                                            int col0, int64_t nv, const double* __restrict__ S,
                                            void* __restrict__ out, int mode) {
  const bool interior = col0 >= row0 + C::BM && col0 + C::BN <= nv;
  if (mode == OUT2_N2_SQUARE_F32) {
    float* tab = static_cast<float*>(out);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= nv) continue;
#pragma unroll
      for (int c = 0; c < C::NJ; ++c) {
        const int j = col0 + L.col(c);
        if (j <= i || j >= nv) continue;
        const float2 hl = acc.hl(r, c);
        const float n2 = __fadd_rn(hl.x, hl.y);
        tab[(int64_t)i * nv + j] = n2;
        tab[(int64_t)j * nv + i] = n2;
      }
    }
    return;
  }
  if (mode == OUT2_C2_F32 || mode == OUT2_C2_U8) {
    float Sjf[C::NJ];
#pragma unroll
    for (int c = 0; c < C::NJ; ++c) {
      const int j = col0 + L.col(c);
      Sjf[c] = j < nv ? (float)S[j] : 0.0f;
    }
    const bool u8 = mode == OUT2_C2_U8;
    if (interior) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = row0 + L.row(r);
        const float Sif = (float)S[i];
        const int64_t base = pair_index(nv, i, i + 1) - (i + 1);
#pragma unroll
        for (int c = 0; c < C::NJ; ++c) {
          const int j = col0 + L.col(c);
          const float2 hl = acc.hl(r, c);
          const float n2 = __fadd_rn(hl.x, hl.y);
          const float d = __fadd_rn(Sif, Sjf[c]);
          const float c2 = (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
          if (u8)
            static_cast<unsigned char*>(out)[base + j] = c2_code(c2);
          else
            static_cast<float*>(out)[base + j] = c2;
        }
      }
      return;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= nv) continue;
      const float Sif = (float)S[i];
      const int64_t base = pair_index(nv, i, i + 1) - (i + 1);
#pragma unroll
      for (int c = 0; c < C::NJ; ++c) {
        const int j = col0 + L.col(c);
        if (j <= i || j >= nv) continue;
        const float2 hl = acc.hl(r, c);
        const float n2 = __fadd_rn(hl.x, hl.y);
        const float d = __fadd_rn(Sif, Sjf[c]);
        const float c2 = (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
        if (u8)
          static_cast<unsigned char*>(out)[base + j] = c2_code(c2);
        else
          static_cast<float*>(out)[base + j] = c2;
      }
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = row0 + L.row(r);
    if (i >= nv) continue;
    const double Si = S[i];
    double* orow = static_cast<double*>(out) + (pair_index(nv, i, i + 1) - (i + 1));
#pragma unroll
    for (int c = 0; c < C::NJ; ++c) {
      const int j = col0 + L.col(c);
      if (j <= i || j >= nv) continue;
      const float2 hl = acc.hl(r, c);
      const double n2 = (double)hl.x + (double)hl.y;
      const double d = Si + S[j];
      orow[j] = (d == 0.0) ? 0.0 : (2.0 * n2) / d;
    }
  }
}

// Interior-tile epilogue of the small-n_f kernels (FP32 or one-byte
// output): Sfi / Sfj are this lane's rows' and columns' FP32 sums with 1.0 in
// place of 0 (NarrowPrep; an all-zero vector has n2 = 0 with every partner,
// so 0 / (S_j + 1) = 0 is the metric without a test for d = 0), and every
// quotient comes from div_rn_lean, whose range the caller has checked once
// for the whole call.  Values equal store_tile2's bit for bit.  Each row's
// outputs go through one row pointer (no per-output index arithmetic).
template <class C, bool PACKED, bool U8, bool LO_ONLY, class ACC = Acc<PACKED, C::NJ>>
__device__ __forceinline__ void store_tile2_lean(const ACC& acc, const Lanes<C>& L, int row0,
                                                 int col0, int64_t nv, const float (&Sfi)[8],
                                                 const float (&Sfj)[C::NJ], void* __restrict__ out) {
  // packed position of (i, j) = base(i) + j with base(i) = P(i) - i - 1, P(i)
  // the index of pair (i, i + 1); base(i + 1) = base(i) + nv - i - 2.  A
  // lane's rows are two runs of four consecutive rows.
  int64_t base = 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = row0 + L.row(r);
    if (r == 0 || r == 4)
      base = pair_index(nv, i, i + 1) - (i + 1);
    else
      base += nv - i - 1;
    const int64_t off = base + col0 + L.col(0);
#pragma unroll
    for (int c = 0; c < C::NJ; ++c) {
      const float2 hl = acc.hl(r, c);
      // LO_ONLY: nothing was ever folded, hi is 0 and 0 + lo = lo (lo, a sum
      // of non-negative terms from +0, is never -0)
      const float n2 = LO_ONLY ? hl.y : __fadd_rn(hl.x, hl.y);
      const float c2 = div_rn_lean(__fadd_rn(n2, n2), __fadd_rn(Sfi[r], Sfj[c]));
      const int64_t o = off + (L.col(c) - L.col(0));
      if (U8)
        static_cast<unsigned char*>(out)[o] = c2_code(c2);
      else
        static_cast<float*>(out)[o] = c2;
    }
  }
}

// div_rn_lean's range (see there) from NarrowPrep's two words: every
// denominator in [2^-80, 2^101] and every nonzero quotient >= 2^-100.
__device__ __forceinline__ bool lean_division_ok(const unsigned* __restrict__ words) {
  const float vmin = __uint_as_float(__ldg(words)), smax = __uint_as_float(__ldg(words + 1));
  return vmin >= 0x1p-80f && smax <= 0x1p100f && vmin >= smax * 0x1p-100f;
}

// ---------------------------------------------------------------------------
// 2-way: all c2 (or the n2 table) over the upper triangle of tiles.
template <class C, bool PACKED, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    mgemm2_kernel(VF32 V, const double* __restrict__ S, void* __restrict__ out, int mode, int T,
                  int R0, int R1, int G, int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  const Lanes<C> L;
  Acc<PACKED, C::NJ> acc;
  const int64_t nv = V.nv;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    band_tile(t, T, R0, R1, G, I, J);
    const int row0 = I * C::BM, col0 = J * C::BN;
    tile_minsum<C, false, PACKED, KU>(sm, V, row0, col0, 0, L.am, L.bn, acc);
    store_tile2<C, PACKED>(acc, L, row0, col0, nv, S, out, mode);
  }
}

// Epilogue of a thresholded 2-way tile: every pair i < j < nv of this lane
// with c2 >= tau, the value computed exactly as store_tile2's FP32 output, is
// appended warp-aggregated (one atomic per warp and output position) as key
// i << bits | j; appends past `cap` are counted but not stored.  Every lane
// of the warp takes part (the ballots).  NJ: the lane's columns.
template <int NJ, class LN, class ACC>
__device__ __forceinline__ void thresh_append2(const ACC& acc, const LN& L, int row0, int col0, int64_t nv,
                                               const double* __restrict__ S, const ThreshArgs& ta) {
  const int lane = threadIdx.x & 31;
  float Sjf[NJ];
#pragma unroll
  for (int c = 0; c < NJ; ++c) {
    const int j = col0 + L.col(c);
    Sjf[c] = j < nv ? (float)S[j] : 0.0f;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = row0 + L.row(r);
    const float Sif = i < nv ? (float)S[i] : 0.0f;
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
      const int j = col0 + L.col(c);
      float c2 = 0.0f;
      bool hit = false;
      if (i < nv && j > i && j < nv) {
        const float2 hl = acc.hl(r, c);
        const float n2 = __fadd_rn(hl.x, hl.y);
        const float d = __fadd_rn(Sif, Sjf[c]);
        c2 = (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
        hit = c2 >= ta.tau;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(ta.counter, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (hit) {
          const unsigned long long pos = base + (unsigned)__popc(m & ((1u << lane) - 1u));
          if (pos < (unsigned long long)ta.cap) {
            ta.keys[pos] = ((unsigned long long)i << ta.bits) | (unsigned long long)j;
            ta.vals[pos] = c2;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Thresholded 2-way: every pair with c2 >= tau, the value computed exactly as
// mgemm2_kernel's FP32 output.  Hits are appended warp-aggregated (one atomic
// per warp and output position) as key i << bits | j; appends past `cap` are
// counted but not stored.
template <class C, bool PACKED, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    mgemm2_thresh_kernel(VF32 V, const double* __restrict__ S, int T, int G, int64_t ntiles,
                         ThreshArgs ta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  const Lanes<C> L;
  Acc<PACKED, C::NJ> acc;
  const int64_t nv = V.nv;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    band_tile(t, T, 0, T, G, I, J);
    const int row0 = I * C::BM, col0 = J * C::BN;
    tile_minsum<C, false, PACKED, KU>(sm, V, row0, col0, 0, L.am, L.bn, acc);
    thresh_append2<C::NJ>(acc, L, row0, col0, nv, S, ta);
  }
}

// ---------------------------------------------------------------------------
// 2-way on half2 field pairs (PS_PATH_HALF2): V holds (field 2p, field 2p+1)
// of every vector, scaled by a power of two `scale` before rounding to FP16;
// n2 = (hi + lo) / scale is exact rescaling.  Denominators S come from the
// caller's values.
// Epilogue of the half2 kernels: n2 = (hi + lo) / scale (an exact
// power-of-two rescaling of the FP32 sums of the scaled FP16 operands), then
// c2 as in store_tile2 (FP32 with __fdiv_rn, or FP64).
template <class C, class ACC>
__device__ __forceinline__ void store_tile2_half(const ACC& acc, const Lanes<C>& L, int row0, int col0,
                                                 int64_t nv, const double* __restrict__ S,
                                                 void* __restrict__ out, int out_f64, float inv_scale) {
  float Sjf[C::NJ];
#pragma unroll
  for (int c = 0; c < C::NJ; ++c) {
    const int j = col0 + L.col(c);
    Sjf[c] = j < nv ? (float)S[j] : 0.0f;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = row0 + L.row(r);
    if (i >= nv) continue;
    const double Si = S[i];
#pragma unroll
    for (int c = 0; c < C::NJ; ++c) {
      const int j = col0 + L.col(c);
      if (j <= i || j >= nv) continue;
      const float2 hl = acc.hl(r, c);
      if (out_f64) {
        const double n2 = ((double)hl.x + (double)hl.y) * (double)inv_scale;
        const double d = Si + S[j];
        static_cast<double*>(out)[pair_index(nv, i, j)] = (d == 0.0) ? 0.0 : (2.0 * n2) / d;
      } else {
        const float n2 = __fmul_rn(__fadd_rn(hl.x, hl.y), inv_scale);
        const float d = __fadd_rn((float)Si, Sjf[c]);
        static_cast<float*>(out)[pair_index(nv, i, j)] = (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
      }
    }
  }
}

template <class C, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    mgemm2_half_kernel(VF32 V, const double* __restrict__ S, void* __restrict__ out, int out_f64,
                       const float* __restrict__ inv_scale_p, int T, int G, int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  const Lanes<C> L;
  Acc<false, C::NJ> acc;
  const int64_t nv = V.nv;
  const float inv_scale = *inv_scale_p;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    band_tile(t, T, 0, T, G, I, J);
    const int row0 = I * C::BM, col0 = J * C::BN;
    tile_minsum<C, false, false, KU, true>(sm, V, row0, col0, 0, L.am, L.bn, acc);
    store_tile2_half<C>(acc, L, row0, col0, nv, S, out, out_f64, inv_scale);
  }
}

// ---------------------------------------------------------------------------
// 3-way: c3 for pivots [jb, jb+npiv) over (j, I, K) tiles with I*B < j and
// K*B+B-1 > j.  pref[x] = number of tiles of pivots jb .. jb+x-1.
template <class C, bool PACKED, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    mgemm3_kernel(VF32 V, const double* __restrict__ S, const float* __restrict__ n2sq,
                  const int64_t* __restrict__ pref, int npiv, int jb, float* __restrict__ out,
                  int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  const Lanes<C> L;
  Acc<PACKED, C::NJ> acc;
  const int nv = V.nv;
  const int Tk = (nv + C::BN - 1) / C::BN;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = npiv;  // largest x with pref[x] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pref[mid] <= t) lo = mid; else hi = mid;
    }
    const int j = jb + lo;
    const int64_t local = t - pref[lo];
    const int k0t = (j + 1) / C::BN;
    const int nK = Tk - k0t;
    const int row0 = (int)(local / nK) * C::BM, col0 = (k0t + (int)(local % nK)) * C::BN;
    // a warp whose 64 rows all lie at or past the pivot (i >= j) has no
    // output here: it skips the min-add loop, which frees the ALU pipe of
    // its sub-partition for the other warp (the pivot's partial row tile)
    tile_minsum<C, true, PACKED, KU>(sm, V, row0, col0, j, L.am, L.bn, acc,
                                     row0 + (int)(threadIdx.x >> 5) / C::WN * 64 < j);
    const int64_t w = nv - 1 - j;
    const int64_t base = slab_offset(nv, jb, j);
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
            c3_value(acc.hl(r, c), n2ij, n2sq[(int64_t)i * nv + k], n2sq[(int64_t)j * nv + k],
                     __fadd_rn(Sij, Skf[c]));
      }
    }
  }
}

// Epilogue of a thresholded 3-way item (pivot j, tile origin row0, col0):
// every triple i < j < k < nv of this lane with c3 >= tau is appended as a
// lexicographic key of ORIGINAL indices (ta.perm maps a reordered index to
// its original one) and its value.  The three vectors are taken in
// increasing original index, so the sums of eq. (1) are formed in the same
// order as without a reordering and every value is bit-identical to the
// exhaustive search.  NJ: the lane's columns.
template <int NJ, class LN, class ACC>
__device__ __forceinline__ void thresh_append3(const ACC& acc, const LN& L, int row0, int col0, int j, int nv,
                                               const double* __restrict__ S, const float* __restrict__ n2sq,
                                               const ThreshArgs& ta) {
  const int* __restrict__ perm = ta.perm;
  const int oj = perm ? perm[j] : j;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = row0 + L.row(r);
    if (i >= j) continue;
    const int oi = perm ? perm[i] : i;
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
      const int k = col0 + L.col(c);
      if (k <= j || k >= nv) continue;
      int pa = i, pb = j, pc = k, a = oi, bb = oj, cc = perm ? perm[k] : k;
      if (perm) {
        if (a > bb) { int x = a; a = bb; bb = x; x = pa; pa = pb; pb = x; }
        if (bb > cc) { int x = bb; bb = cc; cc = x; x = pb; pb = pc; pc = x; }
        if (a > bb) { int x = a; a = bb; bb = x; x = pa; pa = pb; pb = x; }
      }
      const float v = c3_value(acc.hl(r, c), n2sq[(int64_t)pa * nv + pb], n2sq[(int64_t)pa * nv + pc],
                               n2sq[(int64_t)pb * nv + pc],
                               __fadd_rn(__fadd_rn((float)S[pa], (float)S[pb]), (float)S[pc]));
      if (v >= ta.tau) {
        const unsigned long long pos = atomicAdd(ta.counter, 1ull);
        if (pos < (unsigned long long)ta.cap) {
          ta.keys[pos] = ((unsigned long long)a << (2 * ta.bits)) | ((unsigned long long)bb << ta.bits) |
                         (unsigned long long)cc;
          ta.vals[pos] = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Thresholded 3-way over an explicit list of 128-tile blocks (I, Jt, K),
// I <= Jt <= K: work item = (block, pivot j in tile Jt).  Every triple
// i<j<k with c3 >= tau is appended as a lexicographic key
// (i << 2b | j << b | k) and its value; the counter receives the total even
// beyond `cap`.
template <class C, bool PACKED, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    mgemm3_thresh_kernel(VF32 V, const double* __restrict__ S, const float* __restrict__ n2sq,
                         const int* __restrict__ blocks, int64_t nitems, ThreshArgs ta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  const Lanes<C> L;
  Acc<PACKED, C::NJ> acc;
  const int nv = V.nv;
  constexpr int B = C::BM;
  for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
    const int64_t b = t / B;
    const int I = blocks[3 * b], Jt = blocks[3 * b + 1], K = blocks[3 * b + 2];
    const int j = Jt * B + (int)(t % B);
    const int row0 = I * B, col0 = K * B;
    // CTA-uniform skip: no row i < j or no column k > j in this item
    if (j >= nv || row0 >= j || col0 + B - 1 <= j || col0 >= nv) continue;
    // a warp whose 64 rows all lie at or past the pivot (i >= j) has no
    // output here: it skips the min-add loop, which frees the ALU pipe of
    // its sub-partition for the other warp (the pivot's partial row tile)
    tile_minsum<C, true, PACKED, KU>(sm, V, row0, col0, j, L.am, L.bn, acc,
                                     row0 + (int)(threadIdx.x >> 5) / C::WN * 64 < j);
    thresh_append3<C::NJ>(acc, L, row0, col0, j, nv, S, n2sq, ta);
  }
}

// ---------------------------------------------------------------------------
// Batched persistent kernel: many independent problems of uneven size in one
// launch.  CTAs take items from an atomic work queue over a list ordered
//   [sums blocks] [2-way tiles + n2-table tiles] [3-way pivot tiles],
// each group longest-first.  A tile's epilogue waits (bounded) for its
// problem's sums, a 3-way tile's epilogue for its problem's n2 table; every
// item it waits on sits earlier in the queue and has therefore been taken by
// a running CTA that waits on nothing later, so the waits always end.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *ctr >= target (at most wait_ns of %globaltimer time,
// or until another CTA's wait ran out); the CTA follows its verdict.
__device__ __forceinline__ bool cta_wait_count(const int* ctr, int target, int* err, int* s_flag,
                                               unsigned long long wait_ns) {
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire(ctr) < target) {
      unsigned long long t0;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
      while (ld_acquire(ctr) < target) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t1));
        if (t1 - t0 > wait_ns || *(volatile int*)err) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  const bool ok = *s_flag != 0;
  __syncthreads();
  return ok;
}

__device__ __forceinline__ void cta_signal(int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1);
  }
}

template <class C, bool PACKED, int KU>
__global__ void __launch_bounds__(C::NT, C::MINB)
    batched_kernel(const BatchProb* __restrict__ probs, int nprob, const BatchItem* __restrict__ items,
                   int nitems, int* __restrict__ counters, unsigned long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<C>& sm = *reinterpret_cast<Smem<C>*>(smem_raw);
  __shared__ int s_item, s_flag;
  __shared__ double s_part[8][33];
  const Lanes<C> L;
  Acc<PACKED, C::NJ> acc;
  int* err = counters + 1;
  int* sums_done = counters + 2;
  int* n2_done = counters + 2 + nprob;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&counters[0], 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem w = items[it];
    const BatchProb p = probs[w.prob];
    const VF32 V = p.v;
    const int nv = V.nv;
    if (w.kind == BK_SUMS) {
      // per-vector FP64 sums of 32 vectors in the same fixed order as
      // vector_sums_fm: partial u sums fields u, u+8, ...; partials added
      // in order 0..7 (so results match the single-problem path bit for bit)
      constexpr int NW = C::NT / 32;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const int i = w.a * 32 + lane;
      for (int u = warp; u < 8; u += NW) {
        double sacc = 0.0;
        if (i < nv)
          for (int q = u; q < V.nf; q += 8) sacc += (double)__ldcg(V.p + (int64_t)q * V.ld + i);
        s_part[u][lane] = sacc;
      }
      __syncthreads();
      if (warp == 0 && i < nv) {
        double tsum = s_part[0][lane];
#pragma unroll
        for (int u = 1; u < 8; ++u) tsum += s_part[u][lane];
        p.S[i] = tsum;
      }
      cta_signal(&sums_done[w.prob]);
      continue;
    }
    if (w.kind == BK_TILE2 || w.kind == BK_N2) {
      const int row0 = w.a * C::BM, col0 = w.b * C::BN;
      tile_minsum<C, false, PACKED, KU>(sm, V, row0, col0, 0, L.am, L.bn, acc);
      if (!cta_wait_count(&sums_done[w.prob], p.nsum_blocks, err, &s_flag, wait_ns)) continue;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = row0 + L.row(r);
        if (i >= nv) continue;
        const double Si = __ldcg(p.S + i);
#pragma unroll
        for (int c = 0; c < C::NJ; ++c) {
          const int j = col0 + L.col(c);
          if (j <= i || j >= nv) continue;
          const float2 hl = acc.hl(r, c);
          if (w.kind == BK_N2) {
            const float n2 = __fadd_rn(hl.x, hl.y);
            p.n2[(int64_t)i * nv + j] = n2;
            p.n2[(int64_t)j * nv + i] = n2;
          } else if (p.out_f64) {
            const double n2 = (double)hl.x + (double)hl.y;
            const double d = Si + __ldcg(p.S + j);
            static_cast<double*>(p.out)[pair_index(nv, i, j)] = (d == 0.0) ? 0.0 : (2.0 * n2) / d;
          } else {
            // the denominator as in mgemm2_kernel's FP32 output
            const float n2 = __fadd_rn(hl.x, hl.y);
            const float d = __fadd_rn((float)Si, (float)__ldcg(p.S + j));
            static_cast<float*>(p.out)[pair_index(nv, i, j)] =
                (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
          }
        }
      }
      if (w.kind == BK_N2) cta_signal(&n2_done[w.prob]);
      continue;
    }
    // BK_TILE3: pivot j, tile index b inside the pivot
    const int j = w.a;
    const int Tk = (nv + C::BN - 1) / C::BN;
    const int k0t = (j + 1) / C::BN;
    const int nK = Tk - k0t;
    const int row0 = (w.b / nK) * C::BM, col0 = (k0t + w.b % nK) * C::BN;
    // a warp whose 64 rows all lie at or past the pivot (i >= j) has no
    // output here: it skips the min-add loop, which frees the ALU pipe of
    // its sub-partition for the other warp (the pivot's partial row tile)
    tile_minsum<C, true, PACKED, KU>(sm, V, row0, col0, j, L.am, L.bn, acc,
                                     row0 + (int)(threadIdx.x >> 5) / C::WN * 64 < j);
    if (!cta_wait_count(&n2_done[w.prob], p.n2_tiles, err, &s_flag, wait_ns)) continue;
    const int64_t wdt = nv - 1 - j;
    const int64_t base = slab_offset(nv, 0, j);
    const float Sj = (float)__ldcg(p.S + j);
    float* out = static_cast<float*>(p.out);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= j) continue;
      const float Sij = __fadd_rn((float)__ldcg(p.S + i), Sj);
      const float n2ij = __ldcg(p.n2 + (int64_t)i * nv + j);
#pragma unroll
      for (int c = 0; c < C::NJ; ++c) {
        const int k = col0 + L.col(c);
        if (k <= j || k >= nv) continue;
        out[base + (int64_t)i * wdt + (k - j - 1)] =
            c3_value(acc.hl(r, c), n2ij, __ldcg(p.n2 + (int64_t)i * nv + k), __ldcg(p.n2 + (int64_t)j * nv + k),
                     __fadd_rn(Sij, (float)__ldcg(p.S + k)));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers of one configuration (instantiated per .cu file).
template <class C, bool PACKED, int KU>
struct Launch {
  static constexpr size_t smem = sizeof(Smem<C>);
  static cudaError_t attrs() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(mgemm2_kernel<C, PACKED, KU>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    if ((e = cudaFuncSetAttribute(mgemm3_kernel<C, PACKED, KU>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    return cudaFuncSetAttribute(batched_kernel<C, PACKED, KU>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  static void mgemm2(unsigned grid, cudaStream_t st, const VF32& V, const double* S, void* out,
                     int mode, int T, int R0, int R1, int G, int64_t ntiles) {
    mgemm2_kernel<C, PACKED, KU><<<grid, C::NT, smem, st>>>(V, S, out, mode, T, R0, R1, G, ntiles);
  }
  static void mgemm3(unsigned grid, cudaStream_t st, const VF32& V, const double* S,
                     const float* n2sq, const int64_t* pref, int npiv, int jb, float* out,
                     int64_t ntiles) {
    mgemm3_kernel<C, PACKED, KU><<<grid, C::NT, smem, st>>>(V, S, n2sq, pref, npiv, jb, out,
                                                            ntiles);
  }
  static void batched(unsigned grid, cudaStream_t st, const BatchProb* probs, int nprob,
                      const BatchItem* items, int nitems, int* counters, unsigned long long wait_ns) {
    batched_kernel<C, PACKED, KU><<<grid, C::NT, smem, st>>>(probs, nprob, items, nitems, counters, wait_ns);
  }
};

}  // namespace mg
}  // namespace ps
