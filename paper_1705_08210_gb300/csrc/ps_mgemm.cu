// ps_mgemm.cu -- dispatch of the FP32 min-product kernels (tile shape x
// accumulate form x unroll depth, see ps_mgemm_impl.cuh), the FP64
// CUDA-core path, the pivot prefix of the 3-way tile walk and the min+add
// issue-rate probe.
#include "ps_mgemm_impl.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace ps {
namespace {

// ---------------------------------------------------------------------------
// FP64 CUDA-core path (small problems): 64 x 64 tiles, 4 x 4 per thread.
constexpr int DBM = 64, DBK = 16;

__global__ void __launch_bounds__(256)
    mgemm2_f64_kernel(const double* __restrict__ X, int64_t ld, int nv, int nf,
                      const double* __restrict__ S, void* __restrict__ out, int out_f64, int T,
                      int64_t tbase, int64_t ntiles) {
  __shared__ double As[DBK][DBM];
  __shared__ double Bs[DBK][DBM];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    mg::tri_tile(tbase + t, T, I, J);
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
        if (out_f64) static_cast<double*>(out)[mg::pair_index(nv, i, j)] = v;
        else static_cast<float*>(out)[mg::pair_index(nv, i, j)] = (float)v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Issue-rate probe: independent chains x <- x + min(x, y) (one comparison per
// chain step).  Variant 1 adds pairs with add.rn.f32x2.  Variant 2 is the
// half2 path's inner operation: one packed min.f16x2 of two field pairs
// (two comparisons), both halves added to FP32 accumulators.
constexpr int PROBE_CHAINS = 16;

template <int VARIANT>
__global__ void __launch_bounds__(256) probe_kernel(float* out, int iters, float y) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  if (VARIANT == 2) {
    // chain c: h[c] is the half2 operand, x[c] the FP32 accumulator
    uint32_t hv[PROBE_CHAINS];
    const __half2 yy = __floats2half2_rn(y, y);
    const uint32_t yb = *reinterpret_cast<const uint32_t*>(&yy);
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
      const __half2 t = __floats2half2_rn(x[c], x[c] + 1e-3f);
      hv[c] = *reinterpret_cast<const uint32_t*>(&t);
    }
    for (int it = 0; it < iters / 2; ++it) {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) {
        uint32_t m;
        asm("min.f16x2 %0, %1, %2;" : "=r"(m) : "r"(hv[c]), "r"(yb));
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.f16 %0, l, %0;\n\t"
            "add.rn.f32.f16 %0, h, %0;\n\t}"
            : "+f"(x[c])
            : "r"(m));
        hv[c] = m;  // the next min depends on this one (an opaque chain)
      }
    }
  }
  for (int it = 0; VARIANT != 2 && it < iters; ++it) {
    if (VARIANT == 3) {
      // the min of two non-negative floats as the signed-integer min of
      // their bit patterns (the same value), scalar FP32 add
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c)
        x[c] = x[c] + __int_as_float(min(__float_as_int(x[c]), __float_as_int(y)));
    } else if (VARIANT == 0) {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = x[c] + fminf(x[c], y);
    } else if (VARIANT == 4) {
      // half the chains with scalar adds, half with packed f32x2 adds
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS / 2; ++c) x[c] = x[c] + fminf(x[c], y);
#pragma unroll
      for (int c = PROBE_CHAINS / 2; c < PROBE_CHAINS; c += 2) {
        unsigned long long p;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(x[c]), "f"(x[c + 1]));
        p = mg::f2_add(p, fminf(x[c], y), fminf(x[c + 1], y));
        const float2 u = mg::f2_unpack(p);
        x[c] = u.x;
        x[c + 1] = u.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; c += 2) {
        unsigned long long p;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(x[c]), "f"(x[c + 1]));
        p = mg::f2_add(p, fminf(x[c], y), fminf(x[c + 1], y));
        const float2 u = mg::f2_unpack(p);
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

// pref[x] = tiles (width B) of pivots jb .. jb+x-1, x in [0, npiv]; one block.
__global__ void __launch_bounds__(1024) pivot_prefix_kernel(int nv, int jb, int npiv, int B,
                                                            int64_t* __restrict__ pref) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (npiv + 1023) / 1024;
  const int x0 = min(npiv, t * per), x1 = min(npiv, x0 + per);
  int64_t s = 0;
  for (int x = x0; x < x1; ++x) s += mg::pivot_tiles(nv, jb + x, B);
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
    run += mg::pivot_tiles(nv, jb + x, B);
  }
}

std::mutex g_attr_mu;
uint64_t g_attr_done[4096] = {};  // per variant code: bit d = attributes set on device d

cudaError_t ensure_attrs(ps_ctx* h, int code, const MgemmVariant* v) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  const uint64_t bit = 1ull << (h->device & 63);
  if (g_attr_done[code] & bit) return cudaSuccess;
  const cudaError_t e = v->attrs();
  if (e == cudaSuccess) g_attr_done[code] |= bit;
  return e;
}

// One block per pivot: its (I, K) tiles in row-major order.
__global__ void __launch_bounds__(256) pivot_items_kernel(int nv, int jb, int B, const int64_t* __restrict__ pref,
                                                          int2* __restrict__ items) {
  const int x = blockIdx.x;
  const int j = jb + x;
  const int Tk = (nv + B - 1) / B;
  const int k0t = (j + 1) / B;
  const int nK = Tk - k0t;
  const int64_t n = pref[x + 1] - pref[x];
  for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
    const int I = (int)(u / nK), K = k0t + (int)(u % nK);
    items[pref[x] + u] = make_int2(j, (I << 16) | K);
  }
}

}  // namespace

cudaError_t launch_pivot_items(int nv, int jb, int npiv, int B, const int64_t* pref, int2* items,
                               cudaStream_t st) {
  if (npiv <= 0) return cudaSuccess;
  if (ceil_div(nv, B) >= 65536) return cudaErrorInvalidValue;  // (I, K) packed in 16 bits each
  pivot_items_kernel<<<npiv, 256, 0, st>>>(nv, jb, B, pref, items);
  return cudaGetLastError();
}

const MgemmVariant* mgemm_variant_of(int code) {
  const int shape = code / 1000, packed = (code / 100) % 10, ku = code % 100;
  if (shape == 1) return mgemm_variant_t64(ku);
  if (shape == 2) return mgemm_variant_t128w16(ku);
  return mgemm_variant_t128(packed, ku);
}

int mgemm_variant_code(const ps_ctx* h, bool two_way) {
  const int warps = h->mgemm_warps ? h->mgemm_warps : (two_way ? 16 : 8);
  const int shape = h->mgemm_tile == 64 ? 1 : (warps == 16 ? 2 : 0);
  const int packed = shape ? 1 : (h->mgemm_packed_add ? 1 : 0);
  return shape * 1000 + packed * 100 + h->mgemm_ku;
}

cudaError_t launch_mgemm2(ps_ctx* h, const VF32& V, const double* S, void* out, int mode,
                          cudaStream_t st, int tile_begin, int tile_end) {
  const int code = mgemm_variant_code(h, true);
  const MgemmVariant* v = mgemm_variant_of(code);
  cudaError_t e = ensure_attrs(h, code, v);
  if (e != cudaSuccess) return e;
  const int T = (int)ceil_div(V.nv, v->tile);
  const int64_t I0 = std::max(0, tile_begin), I1 = tile_end < 0 ? T : std::min(tile_end, T);
  if (I1 <= I0) return cudaSuccess;
  // tiles in rows [0, I) of the triangle: I*T - I(I-1)/2
  const int64_t tbase = I0 * T - I0 * (I0 - 1) / 2;
  const int64_t ntiles = (I1 * T - I1 * (I1 - 1) / 2) - tbase;
  if (code / 1000 == 2 && h->mgemm_feed_tma && V.nf > 0) {
    int* err = async_err_word(h);
    if (!err) return cudaErrorMemoryAllocation;
    return launch_mgemm2_tma(h, V, S, out, mode, st, T, (int)I0, (int)I1, std::max(1, h->mgemm_band), ntiles,
                             err);
  }
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)h->num_sms * v->minb);
  v->mgemm2(grid, st, V, S, out, mode, T, (int)I0, (int)I1, std::max(1, h->mgemm_band), ntiles);
  return cudaGetLastError();
}

void partition_2way(int64_t nv, int nparts, int part, int64_t* row_begin, int64_t* row_end) {
  // pairs in 128-row band b: rows i in [128b, 128b+128), each with nv-1-i
  // partners; bands are assigned so that every part gets ~1/nparts of them
  const int64_t T = ceil_div(nv, 128);
  const double total = (double)nv * (double)(nv - 1) / 2.0;
  auto rows_pairs = [nv](int64_t r) {  // pairs in rows [0, r)
    return (double)r * (double)(nv - 1) - (double)r * (double)(r - 1) / 2.0;
  };
  auto cut = [&](int p) -> int64_t {
    if (p <= 0) return 0;
    if (p >= nparts) return T;
    const double target = total * (double)p / (double)nparts;
    int64_t b = 0;
    while (b < T && rows_pairs(std::min(nv, (b + 1) * 128)) <= target) ++b;
    // nearer of the two band edges around the target
    if (b < T && target - rows_pairs(std::min(nv, b * 128)) > rows_pairs(std::min(nv, (b + 1) * 128)) - target)
      ++b;
    return b;
  };
  *row_begin = std::min(nv, cut(part) * 128);
  *row_end = std::min(nv, cut(part + 1) * 128);
}

void partition_3way(int64_t nv, int nparts, int part, int64_t* j_begin, int64_t* j_end) {
  // pivot j owns j (nv-1-j) triples; equal prefix shares
  const double total = (double)nv * (double)(nv - 1) * (double)(nv - 2) / 6.0;
  auto cut = [&](int p) -> int64_t {
    if (p <= 0) return 0;
    if (p >= nparts) return nv;
    const double target = total * (double)p / (double)nparts;
    double acc = 0.0;
    for (int64_t j = 0; j < nv; ++j) {
      const double w = (double)j * (double)(nv - 1 - j);
      if (acc + w / 2.0 > target) return j;
      acc += w;
    }
    return nv;
  };
  *j_begin = cut(part);
  *j_end = cut(part + 1);
}

int64_t pivot_tile_count(int nv, int64_t jb, int64_t je, int B) {
  int64_t n = 0;
  for (int64_t j = jb; j < je; ++j) n += mg::pivot_tiles(nv, j, B);
  return n;
}

cudaError_t launch_mgemm3(ps_ctx* h, const VF32& V, const double* S, const float* n2sq,
                          int64_t jb, int64_t je, float* out, cudaStream_t st) {
  const int nv = V.nv;
  const int npiv = (int)(je - jb);
  if (npiv <= 0) return cudaSuccess;
  if (h->mgemm3_feed_tma && V.nf > 0) {
    const int64_t ntiles = pivot_tile_count(nv, jb, je, 128);
    if (ntiles == 0) return cudaSuccess;
    int64_t* dpref = static_cast<int64_t*>(ws_get(h, WS_AUX0, (npiv + 1) * sizeof(int64_t)));
    int2* items = static_cast<int2*>(ws_get(h, WS_ITEMS, (size_t)ntiles * sizeof(int2)));
    int* err = async_err_word(h);
    if (!dpref || !items || !err) return cudaErrorMemoryAllocation;
    pivot_prefix_kernel<<<1, 1024, 0, st>>>(nv, (int)jb, npiv, 128, dpref);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pivot_items(nv, (int)jb, npiv, 128, dpref, items, st);
    if (e != cudaSuccess) return e;
    return launch_mgemm3_tma(h, V, S, n2sq, items, (int)jb, out, ntiles, err, st);
  }
  const int code = mgemm_variant_code(h);
  const MgemmVariant* v = mgemm_variant_of(code);
  cudaError_t e = ensure_attrs(h, code, v);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = pivot_tile_count(nv, jb, je, v->tile);
  if (ntiles == 0) return cudaSuccess;
  int64_t* dpref = static_cast<int64_t*>(ws_get(h, WS_AUX0, (npiv + 1) * sizeof(int64_t)));
  if (!dpref) return cudaErrorMemoryAllocation;
  pivot_prefix_kernel<<<1, 1024, 0, st>>>(nv, (int)jb, npiv, v->tile, dpref);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)h->num_sms * v->minb);
  v->mgemm3(grid, st, V, S, n2sq, dpref, npiv, (int)jb, out, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_batched(ps_ctx* h, int code, const BatchProb* probs, int nprob,
                           const BatchItem* items, int nitems, int* counters, cudaStream_t st) {
  const MgemmVariant* v = mgemm_variant_of(code);
  cudaError_t e = ensure_attrs(h, code, v);
  if (e != cudaSuccess) return e;
  if (nitems == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(nitems, (int64_t)h->num_sms * v->minb);
  v->batched(grid, st, probs, nprob, items, nitems, counters, h->wait_ns);
  return cudaGetLastError();
}

cudaError_t launch_mgemm3_thresh(ps_ctx* h, const VF32& V, const double* S, const float* n2sq,
                                 const int* blocks, const int* blocks_host, int64_t nblocks,
                                 const ThreshArgs& ta, cudaStream_t st) {
  if (h->mgemm3_feed_tma && V.nf > 0) {
    // the TMA-fed pipeline of the 3-way kernel (default)
    int* err = async_err_word(h);
    if (!err) return cudaErrorMemoryAllocation;
    return launch_mgemm3_thresh_tma(h, V, S, n2sq, blocks, blocks_host, nblocks, ta, err, st);
  }
  return launch_thresh_t128(h->num_sms, V, S, n2sq, blocks, nblocks, ta, st);
}

cudaError_t launch_mgemm2_f64(ps_ctx* h, const double* X, int64_t ld, int nv, int nf,
                              const double* S, void* out, int out_f64, cudaStream_t st, int64_t row_begin,
                              int64_t row_end) {
  const int T = (int)ceil_div(nv, DBM);
  // tile rows [I0, I1) of the 64-wide triangle; tiles in rows [0, I): I*T - I(I-1)/2
  const int64_t I0 = std::max<int64_t>(0, row_begin) / DBM;
  const int64_t I1 = row_end < 0 ? T : std::min<int64_t>(T, ceil_div(row_end, DBM));
  if (I1 <= I0) return cudaSuccess;
  const int64_t tbase = I0 * T - I0 * (I0 - 1) / 2;
  const int64_t ntiles = (I1 * T - I1 * (I1 - 1) / 2) - tbase;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)h->num_sms * 4);
  mgemm2_f64_kernel<<<(unsigned)grid, 256, 0, st>>>(X, ld, nv, nf, S, out, out_f64, T, tbase, ntiles);
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
    else if (variant == 1) probe_kernel<1><<<blocks, 256>>>(dout, iters, 1e-3f);
    else if (variant == 2) probe_kernel<2><<<blocks, 256>>>(dout, iters, 1e-3f);
    else if (variant == 3) probe_kernel<3><<<blocks, 256>>>(dout, iters, 1e-3f);
    else probe_kernel<4><<<blocks, 256>>>(dout, iters, 1e-3f);
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
