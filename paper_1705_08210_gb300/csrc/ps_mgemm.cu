// ps_mgemm.cu -- FP32 min-product matrix kernels on the CUDA cores.
//
// The paper's "mGEMM" (Section 3.1): (A min B)_{ij} = sum_k min(a_ik, b_kj),
// a GEMM whose multiply is replaced by min.  There is no tensor-core form of
// min on FP32 data, so the inner loop is one FP32 min (FMNMX) plus one FP32
// add per element pair, and the kernel is bound by the CUDA-core issue rate.
//
// Design (sm_103a, 152 SMs):
//  * CTA tile 128 x 128 outputs, 256 threads, 8 x 8 outputs per thread;
//    per k step a thread reads 8 + 8 operands (four 128-bit shared loads,
//    broadcast across lanes) and issues 64 min + 64 add.
//  * Operands stream through a 4-stage cp.async (16-byte, zero-filling)
//    shared-memory ring of 16-field slices; zero fill is exact because
//    min(0, x) = 0 for the non-negative data of Section 2.1.
//  * Accumulation: each accumulator sums 64 fields in FP32 ("lo"), then is
//    folded into a running "hi" with an exact TwoSum, leaving the rounding
//    residual in "lo".  hi + lo therefore carries at most 63 roundings of
//    a 64-term partial sum: relative error <= 64 u (u = 2^-24) for the
//    non-negative terms, independent of n_f.
//  * Persistent CTAs (grid = SMs x resident CTAs) walk a static list of
//    non-redundant tiles: the upper triangle I <= J for pairs (Section 3.1,
//    lower-triangle blocks skipped), and for triples the (pivot j, I, K)
//    tiles with rows i < j and columns k > j (Section 3.2: only the part of
//    B_j that holds i < j < k is computed).
//  * 3-way: the pivot column v_j is min-ed into the A slice in shared memory
//    once per slice (X_j = min(V, v_j) of Section 3.2 is never
//    materialised), so the inner loop stays one min + one add.
#include "ps_internal.cuh"

#include <algorithm>
#include <vector>

namespace ps {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, STAGES = 4, NT = 256;
constexpr int FOLD = 4;  // stages (of BK fields) per compensated fold: 64 fields

struct __align__(16) SmemF32 {
  float A[STAGES][BK][BM];
  float B[STAGES][BK][BN];
  float P[STAGES][BK];
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

// Issue the copies of one BK-field slice of the A rows [row0,row0+128) and
// B columns [col0,col0+128) into ring buffer `buf`.  Thread t copies the
// 16-byte chunks t and t+256 of each operand: slice row (t>>5) and
// (t>>5)+8, vector offset 4*(t&31).  With a pivot, lane 0 of warp w also
// copies the pivot values of slice rows w and w+8.
template <bool PIVOT>
__device__ __forceinline__ void issue_slice(SmemF32& sm, int buf, const VF32& V, int row0,
                                            int col0, int k0, int jpiv) {
  const int t = threadIdx.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = t + h * NT;
    const int r = c >> 5, c4 = (c & 31) * 4;
    const int q = k0 + r;
    const bool qok = q < V.nf;
    const int i = row0 + c4;
    int bytes = (qok && i < V.nv) ? min(16, 4 * (V.nv - i)) : 0;
    const float* src = bytes ? V.p + (int64_t)q * V.ld + i : V.p;
    cp_async16(&sm.A[buf][r][c4], src, bytes);
    const int jx = col0 + c4;
    bytes = (qok && jx < V.nv) ? min(16, 4 * (V.nv - jx)) : 0;
    src = bytes ? V.p + (int64_t)q * V.ld + jx : V.p;
    cp_async16(&sm.B[buf][r][c4], src, bytes);
  }
  if (PIVOT && (t & 31) == 0) {
    const int w = t >> 5;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = w + 8 * h, q = k0 + r;
      const int bytes = q < V.nf ? 4 : 0;
      const float* src = bytes ? V.p + (int64_t)q * V.ld + jpiv : V.p;
      cp_async4(&sm.P[buf][r], src, bytes);
    }
  }
}

// X_j = min(V, v_j) on this thread's own two A chunks of buffer `buf`.
__device__ __forceinline__ void pivot_min_slice(SmemF32& sm, int buf) {
  const int t = threadIdx.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = t + h * NT;
    const int r = c >> 5, c4 = (c & 31) * 4;
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

// Per-thread accumulator block for 8 x 8 outputs.  "lo" accumulates up to 64
// fields; fold() moves it into "hi" with an exact TwoSum and leaves the
// rounding residual in "lo".  PACKED adds pairs of accumulators with one
// add.rn.f32x2; otherwise every accumulator takes a scalar FP32 add.
template <bool PACKED>
struct Acc;

template <>
struct Acc<true> {
  unsigned long long hi[8][4];
  unsigned long long lo[8][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) hi[r][c] = lo[r][c] = 0ull;
  }
  __device__ __forceinline__ void step(const float (&a)[8], const float (&b)[8]) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        lo[r][c] = f2_add(lo[r][c], fminf(a[r], b[2 * c]), fminf(a[r], b[2 * c + 1]));
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const unsigned long long s = f2_add2(hi[r][c], lo[r][c]);
        const unsigned long long bp = f2_sub2(s, hi[r][c]);
        const unsigned long long ap = f2_sub2(s, bp);
        const unsigned long long e = f2_add2(f2_sub2(hi[r][c], ap), f2_sub2(lo[r][c], bp));
        hi[r][c] = s;
        lo[r][c] = e;
      }
  }
  // (hi, lo) of output (r, c)
  __device__ __forceinline__ float2 hl(int r, int c) const {
    const float2 h = f2_unpack(hi[r][c >> 1]);
    const float2 l = f2_unpack(lo[r][c >> 1]);
    return (c & 1) ? make_float2(h.y, l.y) : make_float2(h.x, l.x);
  }
};

template <>
struct Acc<false> {
  float hi[8][8];
  float lo[8][8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) hi[r][c] = lo[r][c] = 0.0f;
  }
  __device__ __forceinline__ void step(const float (&a)[8], const float (&b)[8]) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) lo[r][c] = __fadd_rn(lo[r][c], fminf(a[r], b[c]));
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
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

// 16 k steps of the 8 x 8 min-sum micro-kernel on ring buffer `buf`,
// unrolled KU steps at a time (smaller KU keeps the hot loop in the
// instruction cache).
template <bool PACKED, int KU>
__device__ __forceinline__ void compute_slice(const SmemF32& sm, int buf, int am, int bn,
                                              Acc<PACKED>& acc) {
  const float* As = &sm.A[buf][0][am];
  const float* Bs = &sm.B[buf][0][bn];
#pragma unroll KU
  for (int kk = 0; kk < BK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + kk * BM);
    const float4 a1 = *reinterpret_cast<const float4*>(As + kk * BM + 32);
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * BN);
    const float4 b1 = *reinterpret_cast<const float4*>(Bs + kk * BN + 16);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    acc.step(a, b);
  }
}

// Full k loop over n_f for one (row0, col0) tile, with optional pivot j.
template <bool PIVOT, bool PACKED, int KU>
__device__ __forceinline__ void tile_minsum(SmemF32& sm, const VF32& V, int row0, int col0,
                                            int jpiv, int am, int bn, Acc<PACKED>& acc) {
  acc.zero();
  const int nst = (V.nf + BK - 1) / BK;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nst) issue_slice<PIVOT>(sm, s, V, row0, col0, s * BK, jpiv);
    cp_async_commit();
  }
  for (int s = 0; s < nst; ++s) {
    const int buf = s % STAGES;
    cp_async_wait<STAGES - 2>();
    if (PIVOT) {
      __syncwarp();
      pivot_min_slice(sm, buf);
    }
    __syncthreads();
    const int sn = s + STAGES - 1;
    if (sn < nst) issue_slice<PIVOT>(sm, sn % STAGES, V, row0, col0, sn * BK, jpiv);
    cp_async_commit();
    compute_slice<PACKED, KU>(sm, buf, am, bn, acc);
    if ((s + 1) % FOLD == 0) acc.fold();
  }
  acc.fold();
  cp_async_wait<0>();
  __syncthreads();  // the ring is reused by the next tile
}

// Thread -> output coordinates inside the 128 x 128 tile.
struct Lanes {
  int am, bn;  // smem column offsets of the A / B fragments
  __device__ __forceinline__ Lanes() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 2, wn = warp & 3, lm = lane >> 2, ln = lane & 3;
    am = wm * 64 + lm * 4;
    bn = wn * 32 + ln * 4;
  }
  __device__ __forceinline__ int row(int r) const { return am + (r < 4 ? r : 28 + r); }
  __device__ __forceinline__ int col(int c) const { return bn + (c < 4 ? c : 12 + c); }
};

__device__ __forceinline__ int64_t pair_index(int64_t nv, int64_t i, int64_t j) {
  return i * (2 * nv - i - 1) / 2 + (j - i - 1);
}

// Upper-triangle tile index t -> (I, J), I <= J < T, row-major.
__device__ __forceinline__ void tri_tile(int64_t t, int T, int& I, int& J) {
  // rows before I hold I*T - I*(I-1)/2 tiles
  double disc = (2.0 * T + 1) * (2.0 * T + 1) - 8.0 * (double)t;
  int i = (int)floor(((2.0 * T + 1) - sqrt(disc)) * 0.5);
  i = max(0, min(i, T - 1));
  while (i > 0 && (int64_t)i * T - (int64_t)i * (i - 1) / 2 > t) --i;
  while (i + 1 < T && (int64_t)(i + 1) * T - (int64_t)(i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (int)(t - ((int64_t)i * T - (int64_t)i * (i - 1) / 2));
}

// ---------------------------------------------------------------------------
// 2-way: all c2 (or the n2 table) over the upper triangle of tiles.
template <bool PACKED, int KU>
__global__ void __launch_bounds__(NT, 1)
    mgemm2_kernel(VF32 V, const double* __restrict__ S, void* __restrict__ out, int mode,
                  int T, int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32& sm = *reinterpret_cast<SmemF32*>(smem_raw);
  const Lanes L;
  Acc<PACKED> acc;
  const int64_t nv = V.nv;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    tri_tile(t, T, I, J);
    const int row0 = I * BM, col0 = J * BN;
    tile_minsum<false, PACKED, KU>(sm, V, row0, col0, 0, L.am, L.bn, acc);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= nv) continue;
      const double Si = S ? S[i] : 0.0;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = col0 + L.col(c);
        if (j <= i || j >= nv) continue;
        const float2 hl = acc.hl(r, c);
        if (mode == OUT2_C2_F32) {
          const float n2 = __fadd_rn(hl.x, hl.y);
          const float d = (float)(Si + S[j]);
          const float v = (d == 0.0f) ? 0.0f : __fdiv_rn(2.0f * n2, d);
          static_cast<float*>(out)[pair_index(nv, i, j)] = v;
        } else if (mode == OUT2_C2_F64) {
          const double n2 = (double)hl.x + (double)hl.y;
          const double d = Si + S[j];
          static_cast<double*>(out)[pair_index(nv, i, j)] = (d == 0.0) ? 0.0 : (2.0 * n2) / d;
        } else {
          const float n2 = __fadd_rn(hl.x, hl.y);
          float* tab = static_cast<float*>(out);
          tab[(int64_t)i * nv + j] = n2;
          tab[(int64_t)j * nv + i] = n2;
        }
      }
    }
  }
}

// Section 2.2 eq. (1): n3 = n2(ij) + n2(ik) + n2(jk) - n3' in FP64, then
// c3 = (3/2) n3 / d3 rounded to FP32 (d3 = S_i + S_j + S_k from FP64 sums).
__device__ __forceinline__ float c3_value(float2 n3p_hl, double n2ij, double n2ik, double n2jk,
                                          double d3) {
  const double n3p = (double)n3p_hl.x + (double)n3p_hl.y;
  const double n3 = ((n2ij + n2ik) + n2jk) - n3p;
  const float d = (float)d3;
  return (d == 0.0f) ? 0.0f : __fdiv_rn(1.5f * (float)n3, d);
}

// ---------------------------------------------------------------------------
// 3-way: c3 for pivots [jb, je) over (j, I, K) tiles with I*128 < j and
// K*128+127 > j.  pref[x] = number of tiles of pivots jb .. jb+x-1.
__device__ __forceinline__ int64_t slab_offset(int64_t n, int64_t jb, int64_t j) {
  // sum_{j'=jb}^{j-1} j'(n-1-j') = F(j) - F(jb),
  // F(x) = (n-1) x(x-1)/2 - (x-1) x (2x-1)/6
  auto F = [n](int64_t x) { return (n - 1) * (x * (x - 1) / 2) - (x - 1) * x * (2 * x - 1) / 6; };
  return F(j) - F(jb);
}

template <bool PACKED, int KU>
__global__ void __launch_bounds__(NT, 1)
    mgemm3_kernel(VF32 V, const double* __restrict__ S, const float* __restrict__ n2sq,
                  const int64_t* __restrict__ pref, int npiv, int jb, float* __restrict__ out,
                  int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32& sm = *reinterpret_cast<SmemF32*>(smem_raw);
  const Lanes L;
  Acc<PACKED> acc;
  const int nv = V.nv;
  const int Tk = (nv + BN - 1) / BN;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // pivot: largest x with pref[x] <= t
    int lo = 0, hi = npiv;  // pref[0] = 0, pref[npiv] = ntiles
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pref[mid] <= t) lo = mid; else hi = mid;
    }
    const int j = jb + lo;
    const int64_t local = t - pref[lo];
    const int k0t = (j + 1) / BN;
    const int nK = Tk - k0t;
    const int ti = (int)(local / nK), tk = k0t + (int)(local % nK);
    const int row0 = ti * BM, col0 = tk * BN;
    tile_minsum<true, PACKED, KU>(sm, V, row0, col0, j, L.am, L.bn, acc);
    const int64_t w = nv - 1 - j;
    const int64_t base = slab_offset(nv, jb, j);
    const double Sj = S[j];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= j) continue;
      const double Sij = S[i] + Sj;
      const double n2ij = (double)n2sq[(int64_t)i * nv + j];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = col0 + L.col(c);
        if (k <= j || k >= nv) continue;
        const float v = c3_value(acc.hl(r, c), n2ij, (double)n2sq[(int64_t)i * nv + k],
                                 (double)n2sq[(int64_t)j * nv + k], Sij + S[k]);
        out[base + (int64_t)i * w + (k - j - 1)] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Thresholded 3-way over an explicit list of tile blocks (I, Jt, K) with
// I <= Jt <= K (128-wide tiles): work item = (block, pivot j in tile Jt).
// Every triple i<j<k with c3 >= tau is appended as a lexicographic key
// (i << 2b | j << b | k) and its value; counter receives the total even
// beyond `cap`.
__global__ void __launch_bounds__(NT, 1)
    mgemm3_thresh_kernel(VF32 V, const double* __restrict__ S, const float* __restrict__ n2sq,
                         const int* __restrict__ blocks, int64_t nitems, ThreshArgs ta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32& sm = *reinterpret_cast<SmemF32*>(smem_raw);
  const Lanes L;
  Acc<true> acc;
  const int nv = V.nv;
  for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
    const int64_t b = t >> 7;
    const int I = blocks[3 * b], Jt = blocks[3 * b + 1], K = blocks[3 * b + 2];
    const int j = Jt * BM + (int)(t & 127);
    const int row0 = I * BM, col0 = K * BN;
    // CTA-uniform skip: no row i < j or no column k > j in this item
    if (j >= nv || row0 >= j || col0 + BN - 1 <= j || col0 >= nv) continue;
    tile_minsum<true, true, 8>(sm, V, row0, col0, j, L.am, L.bn, acc);
    const double Sj = S[j];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= j) continue;
      const double Sij = S[i] + Sj;
      const double n2ij = (double)n2sq[(int64_t)i * nv + j];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = col0 + L.col(c);
        if (k <= j || k >= nv) continue;
        const float v = c3_value(acc.hl(r, c), n2ij, (double)n2sq[(int64_t)i * nv + k],
                                 (double)n2sq[(int64_t)j * nv + k], Sij + S[k]);
        if (v >= ta.tau) {
          const unsigned long long pos = atomicAdd(ta.counter, 1ull);
          if (pos < (unsigned long long)ta.cap) {
            ta.keys[pos] = ((unsigned long long)i << (2 * ta.bits)) |
                           ((unsigned long long)j << ta.bits) | (unsigned long long)k;
            ta.vals[pos] = v;
          }
        }
      }
    }
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

// Thread 0 waits until *ctr >= target (2 s limit); the CTA follows its verdict.
__device__ __forceinline__ bool cta_wait_count(const int* ctr, int target, int* err, int* s_flag) {
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire(ctr) < target) {
      unsigned long long t0;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
      while (ld_acquire(ctr) < target) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t1));
        if (t1 - t0 > 2000000000ull || *(volatile int*)err) {
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

template <bool PACKED, int KU>
__global__ void __launch_bounds__(NT, 1)
    batched_kernel(const BatchProb* __restrict__ probs, int nprob, const BatchItem* __restrict__ items,
                   int nitems, int* __restrict__ counters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF32& sm = *reinterpret_cast<SmemF32*>(smem_raw);
  __shared__ int s_item, s_flag;
  __shared__ double s_part[8][33];
  const Lanes L;
  Acc<PACKED> acc;
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
      // same fixed summation order as vector_sums_fm
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const int i = w.a * 32 + lane;
      double sacc = 0.0;
      if (i < nv)
        for (int q = warp; q < V.nf; q += 8) sacc += (double)__ldcg(V.p + (int64_t)q * V.ld + i);
      s_part[warp][lane] = sacc;
      __syncthreads();
      if (warp == 0 && i < nv) {
        double t = s_part[0][lane];
#pragma unroll
        for (int u = 1; u < 8; ++u) t += s_part[u][lane];
        p.S[i] = t;
      }
      cta_signal(&sums_done[w.prob]);
      continue;
    }
    if (w.kind == BK_TILE2 || w.kind == BK_N2) {
      const int row0 = w.a * BM, col0 = w.b * BN;
      tile_minsum<false, PACKED, KU>(sm, V, row0, col0, 0, L.am, L.bn, acc);
      if (!cta_wait_count(&sums_done[w.prob], p.nsum_blocks, err, &s_flag)) continue;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int i = row0 + L.row(r);
        if (i >= nv) continue;
        const double Si = __ldcg(p.S + i);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
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
            const float n2 = __fadd_rn(hl.x, hl.y);
            const float d = (float)(Si + __ldcg(p.S + j));
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
    const int Tk = (nv + BN - 1) / BN;
    const int k0t = (j + 1) / BN;
    const int nK = Tk - k0t;
    const int row0 = (w.b / nK) * BM, col0 = (k0t + w.b % nK) * BN;
    tile_minsum<true, PACKED, KU>(sm, V, row0, col0, j, L.am, L.bn, acc);
    if (!cta_wait_count(&n2_done[w.prob], p.n2_tiles, err, &s_flag)) continue;
    const int64_t wdt = nv - 1 - j;
    const int64_t base = slab_offset(nv, 0, j);
    const double Sj = __ldcg(p.S + j);
    float* out = static_cast<float*>(p.out);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = row0 + L.row(r);
      if (i >= j) continue;
      const double Sij = __ldcg(p.S + i) + Sj;
      const double n2ij = (double)__ldcg(p.n2 + (int64_t)i * nv + j);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = col0 + L.col(c);
        if (k <= j || k >= nv) continue;
        const float v = c3_value(acc.hl(r, c), n2ij, (double)__ldcg(p.n2 + (int64_t)i * nv + k),
                                 (double)__ldcg(p.n2 + (int64_t)j * nv + k), Sij + __ldcg(p.S + k));
        out[base + (int64_t)i * wdt + (k - j - 1)] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 CUDA-core path (small problems): 64 x 64 tiles, 4 x 4 per thread.
constexpr int DBM = 64, DBK = 16;

__global__ void __launch_bounds__(256)
    mgemm2_f64_kernel(const double* __restrict__ X, int64_t ld, int nv, int nf,
                      const double* __restrict__ S, void* __restrict__ out, int out_f64, int T,
                      int64_t ntiles) {
  __shared__ double As[DBK][DBM];
  __shared__ double Bs[DBK][DBM];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    tri_tile(t, T, I, J);
    const int row0 = I * DBM, col0 = J * DBM;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < nf; k0 += DBK) {
      for (int e = threadIdx.x; e < DBK * DBM; e += 256) {
        const int r = e / DBM, c = e % DBM, q = k0 + r;
        As[r][c] = (q < nf && row0 + c < nv) ? X[(row0 + c) + (int64_t)q * ld] : 0.0;
        Bs[r][c] = (q < nf && col0 + c < nv) ? X[(col0 + c) + (int64_t)q * ld] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < DBK; ++kk)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] += fmin(As[kk][ty + 16 * r], Bs[kk][tx + 16 * c]);
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = row0 + ty + 16 * r;
      if (i >= nv) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = col0 + tx + 16 * c;
        if (j <= i || j >= nv) continue;
        const double d = S[i] + S[j];
        const double v = (d == 0.0) ? 0.0 : (2.0 * acc[r][c]) / d;
        if (out_f64) static_cast<double*>(out)[pair_index(nv, i, j)] = v;
        else static_cast<float*>(out)[pair_index(nv, i, j)] = (float)v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Issue-rate probe: independent chains x <- x + min(x, y) (one comparison per
// chain step).  Variant 1 adds pairs with add.rn.f32x2.
constexpr int PROBE_CHAINS = 16;

template <int VARIANT>
__global__ void __launch_bounds__(256) probe_kernel(float* out, int iters, float y) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
    if (VARIANT == 0) {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = x[c] + fminf(x[c], y);
    } else {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; c += 2) {
        unsigned long long p;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(x[c]), "f"(x[c + 1]));
        p = f2_add(p, fminf(x[c], y), fminf(x[c + 1], y));
        const float2 u = f2_unpack(p);
        x[c] = u.x;
        x[c + 1] = u.y;
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == 12345.678f) out[threadIdx.x] = s;  // keeps the chains live
}

// Tiles of pivot j: I tiles covering rows [0, j) times K tiles covering
// columns (j, nv).
__host__ __device__ __forceinline__ int64_t pivot_tiles(int nv, int64_t j) {
  const int64_t Tk = (nv + BN - 1) / BN;
  const int64_t nI = (j + BM - 1) / BM;
  const int64_t nK = (j + 1 < nv) ? (Tk - (j + 1) / BN) : 0;
  return nI * nK;
}

int64_t pivot_tile_count(int nv, int64_t jb, int64_t je) {
  int64_t n = 0;
  for (int64_t j = jb; j < je; ++j) n += pivot_tiles(nv, j);
  return n;
}

// pref[x] = tiles of pivots jb .. jb+x-1, x in [0, npiv]; one block.
__global__ void __launch_bounds__(1024) pivot_prefix_kernel(int nv, int jb, int npiv,
                                                            int64_t* __restrict__ pref) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (npiv + 1023) / 1024;
  const int x0 = min(npiv, t * per), x1 = min(npiv, x0 + per);
  int64_t s = 0;
  for (int x = x0; x < x1; ++x) s += pivot_tiles(nv, jb + x);
  part[t] = s;
  __syncthreads();
  if (t == 0) {  // exclusive scan of the 1024 chunk sums
    int64_t run = 0;
    for (int u = 0; u < 1024; ++u) {
      const int64_t v = part[u];
      part[u] = run;
      run += v;
    }
    pref[npiv] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int x = x0; x < x1; ++x) {
    pref[x] = run;
    run += pivot_tiles(nv, jb + x);
  }
}

uint64_t g_mgemm_attr_devices = 0;  // bit d: attributes set on device d

template <bool PACKED, int KU>
cudaError_t set_attrs_one() {
  const int sm = (int)sizeof(SmemF32);
  cudaError_t e = cudaFuncSetAttribute(mgemm2_kernel<PACKED, KU>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mgemm3_kernel<PACKED, KU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(batched_kernel<PACKED, KU>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(mgemm3_thresh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t ensure_attrs(ps_ctx* h) {
  const uint64_t bit = 1ull << (h->device & 63);
  if (g_mgemm_attr_devices & bit) return cudaSuccess;
  cudaError_t e;
  if ((e = set_attrs_one<true, 16>()) || (e = set_attrs_one<true, 8>()) ||
      (e = set_attrs_one<true, 4>()) || (e = set_attrs_one<false, 16>()) ||
      (e = set_attrs_one<false, 8>()) || (e = set_attrs_one<false, 4>()))
    return e;
  g_mgemm_attr_devices |= bit;
  return cudaSuccess;
}

// Kernel variant of the handle: accumulate form x k-unroll depth.
template <bool PACKED, int KU>
void launch2_v(unsigned grid, cudaStream_t st, const VF32& V, const double* S, void* out, int mode,
               int T, int64_t ntiles) {
  mgemm2_kernel<PACKED, KU><<<grid, NT, sizeof(SmemF32), st>>>(V, S, out, mode, T, ntiles);
}
template <bool PACKED, int KU>
void launch3_v(unsigned grid, cudaStream_t st, const VF32& V, const double* S, const float* n2sq,
               const int64_t* pref, int npiv, int jb, float* out, int64_t ntiles) {
  mgemm3_kernel<PACKED, KU><<<grid, NT, sizeof(SmemF32), st>>>(V, S, n2sq, pref, npiv, jb, out,
                                                               ntiles);
}

template <typename F16, typename F8, typename F4>
void by_ku(int ku, F16 f16, F8 f8, F4 f4) {
  if (ku == 16) f16();
  else if (ku == 4) f4();
  else f8();
}

}  // namespace

cudaError_t launch_mgemm2(ps_ctx* h, const VF32& V, const double* S, void* out, int mode,
                          cudaStream_t st) {
  cudaError_t e = ensure_attrs(h);
  if (e != cudaSuccess) return e;
  const int T = (int)ceil_div(V.nv, BM);
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)h->num_sms);
  const unsigned g = (unsigned)grid;
  if (h->mgemm_packed_add)
    by_ku(h->mgemm_ku, [&] { launch2_v<true, 16>(g, st, V, S, out, mode, T, ntiles); },
          [&] { launch2_v<true, 8>(g, st, V, S, out, mode, T, ntiles); },
          [&] { launch2_v<true, 4>(g, st, V, S, out, mode, T, ntiles); });
  else
    by_ku(h->mgemm_ku, [&] { launch2_v<false, 16>(g, st, V, S, out, mode, T, ntiles); },
          [&] { launch2_v<false, 8>(g, st, V, S, out, mode, T, ntiles); },
          [&] { launch2_v<false, 4>(g, st, V, S, out, mode, T, ntiles); });
  return cudaGetLastError();
}

cudaError_t launch_mgemm3(ps_ctx* h, const VF32& V, const double* S, const float* n2sq,
                          int64_t jb, int64_t je, float* out, cudaStream_t st) {
  cudaError_t e = ensure_attrs(h);
  if (e != cudaSuccess) return e;
  const int nv = V.nv;
  const int npiv = (int)(je - jb);
  if (npiv <= 0) return cudaSuccess;
  const int64_t ntiles = pivot_tile_count(nv, jb, je);
  if (ntiles == 0) return cudaSuccess;
  int64_t* dpref = static_cast<int64_t*>(ws_get(h, WS_AUX0, (npiv + 1) * sizeof(int64_t)));
  if (!dpref) return cudaErrorMemoryAllocation;
  pivot_prefix_kernel<<<1, 1024, 0, st>>>(nv, (int)jb, npiv, dpref);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)h->num_sms);
  const unsigned g = (unsigned)grid;
  const int j0 = (int)jb;
  if (h->mgemm_packed_add)
    by_ku(h->mgemm_ku, [&] { launch3_v<true, 16>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); },
          [&] { launch3_v<true, 8>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); },
          [&] { launch3_v<true, 4>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); });
  else
    by_ku(h->mgemm_ku, [&] { launch3_v<false, 16>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); },
          [&] { launch3_v<false, 8>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); },
          [&] { launch3_v<false, 4>(g, st, V, S, n2sq, dpref, npiv, j0, out, ntiles); });
  return cudaGetLastError();
}

cudaError_t launch_batched(ps_ctx* h, int packed, int ku, const BatchProb* probs, int nprob,
                           const BatchItem* items, int nitems, int* counters, cudaStream_t st) {
  cudaError_t e = ensure_attrs(h);
  if (e != cudaSuccess) return e;
  if (nitems == 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min(nitems, h->num_sms);
  const size_t smem = sizeof(SmemF32);
  if (packed)
    by_ku(ku, [&] { batched_kernel<true, 16><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); },
          [&] { batched_kernel<true, 8><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); },
          [&] { batched_kernel<true, 4><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); });
  else
    by_ku(ku, [&] { batched_kernel<false, 16><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); },
          [&] { batched_kernel<false, 8><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); },
          [&] { batched_kernel<false, 4><<<g, NT, smem, st>>>(probs, nprob, items, nitems, counters); });
  return cudaGetLastError();
}

cudaError_t launch_mgemm3_thresh(ps_ctx* h, const VF32& V, const double* S, const float* n2sq,
                                 const int* blocks, int64_t nblocks, const ThreshArgs& ta,
                                 cudaStream_t st) {
  cudaError_t e = ensure_attrs(h);
  if (e != cudaSuccess) return e;
  const int64_t nitems = nblocks * 128;
  if (nitems == 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>(nitems, (int64_t)h->num_sms);
  mgemm3_thresh_kernel<<<(unsigned)grid, NT, sizeof(SmemF32), st>>>(V, S, n2sq, blocks, nitems, ta);
  return cudaGetLastError();
}

cudaError_t launch_mgemm2_f64(ps_ctx* h, const double* X, int64_t ld, int nv, int nf,
                              const double* S, void* out, int out_f64, cudaStream_t st) {
  const int T = (int)ceil_div(nv, DBM);
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)h->num_sms * 4);
  mgemm2_f64_kernel<<<(unsigned)grid, 256, 0, st>>>(X, ld, nv, nf, S, out, out_f64, T, ntiles);
  return cudaGetLastError();
}

cudaError_t probe_minadd(ps_ctx* h, int variant, double* cmp_per_s) {
  float* dout = static_cast<float*>(ws_get(h, WS_AUX1, 256 * sizeof(float)));
  if (!dout) return cudaErrorMemoryAllocation;
  const int iters = 1 << 14;
  const int blocks = h->num_sms * 8;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  float best_ms = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, 0);
    if (variant == 0) probe_kernel<0><<<blocks, 256>>>(dout, iters, 1e-3f);
    else probe_kernel<1><<<blocks, 256>>>(dout, iters, 1e-3f);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best_ms = std::min(best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double cmps = (double)blocks * 256.0 * PROBE_CHAINS * iters;
  *cmp_per_s = cmps / (best_ms * 1e-3);
  return cudaSuccess;
}

}  // namespace ps
