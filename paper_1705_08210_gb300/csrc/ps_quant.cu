// ps_quant.cu -- quantizer and thermometer encoder of the tensor-core path.
//
// Not in the paper.  For integer levels a, b in [0, L-1],
//   min(a, b) = sum_{t=1}^{L-1} [a >= t][b >= t],
// so with each level written as L-1 indicator bits ("thermometer code") the
// min-product sum n2 = sum_q min(a_q, b_q) of Section 2.1 becomes an ordinary
// dot product of 0/1 vectors of length n_f (L-1): a dense GEMM for the tensor
// cores, exact on the quantized data.
//
// Quantizer reading (the library's definition):
//   P     = nearest-rank 99.9th percentile of the nonzero entries,
//           rank r = ceil(0.999 m) of the m nonzeros in ascending order;
//   r32   = fl32((L-1) / P);
//   level = 0 for x == 0, else min(L-1, floor(fl32(fl32(x * r32) + 0.5))).
// P is found exactly with a three-pass radix select over the IEEE bit
// patterns (for x >= 0 the unsigned order of the bits is the numeric order).
#include "ps_internal.cuh"

#include <algorithm>

namespace ps {
namespace {

// Digit of pass p: bits [21,32), [10,21), [0,10).
__host__ __device__ constexpr int sel_shift(int pass) { return pass == 0 ? 21 : (pass == 1 ? 10 : 0); }
__host__ __device__ constexpr int sel_bits(int pass) { return pass == 2 ? 10 : 11; }

// Histogram of one radix digit over the nonzero entries that match the
// prefix selected so far.  Rows (fields) are distributed over blocks, each
// thread walks its columns (vectors) of a row: no index division per entry.
__global__ void __launch_bounds__(256) radix_hist_kernel(VF32 V, int pass,
                                                         const SelectState* __restrict__ st,
                                                         unsigned long long* __restrict__ hist) {
  __shared__ unsigned int sh[2048];
  for (int t = threadIdx.x; t < 2048; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  const int shift = sel_shift(pass), mask = (1 << sel_bits(pass)) - 1;
  const int hi_shift = shift + sel_bits(pass);  // bits above this pass's digit
  const unsigned prefix = pass == 0 ? 0u : st->prefix;
  const bool done = pass > 0 && st->done;
  if (!done) {
    for (int q = blockIdx.x; q < V.nf; q += gridDim.x) {
      const float* row = V.p + (int64_t)q * V.ld;
      for (int i = threadIdx.x; i < V.nv; i += blockDim.x) {
        const float x = row[i];
        if (x == 0.0f) continue;
        const unsigned b = __float_as_uint(x);
        if (pass > 0 && (hi_shift >= 32 ? 0u : (b >> hi_shift)) != prefix) continue;
        atomicAdd(&sh[(b >> shift) & mask], 1u);
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2048; t += blockDim.x)
    if (sh[t]) atomicAdd(&hist[t], (unsigned long long)sh[t]);
}

// One block: choose the digit holding the target rank, extend the prefix.
__global__ void __launch_bounds__(1024) radix_select_kernel(int pass, double p,
                                                            SelectState* __restrict__ st,
                                                            const unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long part[1024];
  const int n = 1 << sel_bits(pass);
  const int t = threadIdx.x;
  // two bins per thread, then an exclusive scan of the 1024 pair sums
  const unsigned long long h0 = (2 * t < n) ? hist[2 * t] : 0ull;
  const unsigned long long h1 = (2 * t + 1 < n) ? hist[2 * t + 1] : 0ull;
  part[t] = h0 + h1;
  __syncthreads();
  if (t == 0) {
    if (pass == 0) {
      unsigned long long m = 0;
      for (int u = 0; u < 1024; ++u) m += part[u];
      st->count = m;
      st->prefix = 0;
      st->done = 0;
      if (m == 0) {
        st->done = 1;
        st->value = 0.0f;
      } else {
        long long r = (long long)ceil(p * (double)m);
        if (r < 1) r = 1;
        if ((unsigned long long)r > m) r = (long long)m;
        st->rank = (unsigned long long)r;
      }
    }
    if (!st->done) {
      unsigned long long cum = 0, rank = st->rank;
      int digit = n - 1;
      for (int u = 0; u < 1024; ++u) {
        if (cum + part[u] >= rank) {
          const unsigned long long a = (2 * u < n) ? hist[2 * u] : 0ull;
          if (cum + a >= rank) {
            digit = 2 * u;
          } else {
            digit = 2 * u + 1;
            cum += a;
          }
          break;
        }
        cum += part[u];
      }
      st->rank = rank - cum;
      st->prefix = (st->prefix << sel_bits(pass)) | (unsigned)digit;
      if (pass == 2) {
        st->value = __uint_as_float(st->prefix);
        st->done = 1;
      }
    }
  }
}

__device__ __forceinline__ int level_of(float x, float r32, int L) {
  if (x == 0.0f || r32 == 0.0f) return 0;
  const float prod = __fmul_rn(x, r32);
  const float f = floorf(__fadd_rn(prod, 0.5f));
  if (f >= (float)(L - 1)) return L - 1;
  return f < 0.0f ? 0 : (int)f;
}

__device__ __forceinline__ float recip_scale(const SelectState* st, int L) {
  const float P = st->value;
  return P > 0.0f ? __fdiv_rn((float)(L - 1), P) : 0.0f;
}

__global__ void quantize_kernel(VF32 V, int L, const SelectState* __restrict__ st,
                                uint8_t* __restrict__ q, int64_t ldq) {
  const float r32 = recip_scale(st, L);
  const int64_t total = (int64_t)V.nf * V.nv;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t qq = t / V.nv, i = t - qq * V.nv;
    q[qq * ldq + i] = (uint8_t)level_of(V.p[qq * V.ld + i], r32, L);
  }
}

// Integer per-vector sums of the levels (the quantized denominators).
__global__ void __launch_bounds__(256) level_sums_kernel(VF32 V, int L,
                                                         const SelectState* __restrict__ st,
                                                         int* __restrict__ SQ) {
  __shared__ int part[8][33];
  const float r32 = recip_scale(st, L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  int s = 0;
  if (i < V.nv)
    for (int64_t q = warp; q < V.nf; q += 8) s += level_of(V.p[q * V.ld + i], r32, L);
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < V.nv) {
    int tsum = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) tsum += part[w][lane];
    SQ[i] = tsum;
  }
}

// Thermometer code T[i][k], k = q (L-1) + (t-1): 1.0 in FP8 E4M3 (0x38) when
// level(i,q) >= t, else 0.  Rows i >= nv and fields q >= nf are zero.  A block
// encodes 32 vectors x 128 fields: levels staged in shared memory, then each
// warp writes whole 16-byte pieces of its rows.
constexpr int ENC_V = 32, ENC_F = 128;

__global__ void __launch_bounds__(256) thermo_encode_kernel(VF32 V, int L,
                                                            const SelectState* __restrict__ st,
                                                            uint8_t* __restrict__ T, int64_t Kpad,
                                                            int nv_pad, int* __restrict__ SQ) {
  __shared__ uint8_t lv[ENC_F][ENC_V];
  const float r32 = recip_scale(st, L);
  const int i0 = blockIdx.x * ENC_V;
  const int q0 = blockIdx.y * ENC_F;
  for (int e = threadIdx.x; e < ENC_F * ENC_V; e += blockDim.x) {
    const int r = e / ENC_V, c = e % ENC_V;
    const int q = q0 + r, i = i0 + c;
    lv[r][c] = (q < V.nf && i < V.nv) ? (uint8_t)level_of(V.p[(int64_t)q * V.ld + i], r32, L) : 0;
  }
  __syncthreads();
  // the quantized denominators: integer level sums (exact in any order)
  if (SQ && threadIdx.x < ENC_V && i0 + (int)threadIdx.x < V.nv) {
    int sacc = 0;
    for (int r = 0; r < ENC_F; ++r) sacc += lv[r][threadIdx.x];
    atomicAdd(&SQ[i0 + threadIdx.x], sacc);
  }
  const int Lm = L - 1;
  const int row_bytes = ENC_F * Lm;  // multiple of 16
  const int pieces = row_bytes / 16;
  for (int e = threadIdx.x; e < ENC_V * pieces; e += blockDim.x) {
    const int pc = e % pieces, r = e / pieces;  // consecutive threads: consecutive pieces of a row
    const int i = i0 + r;
    if (i >= nv_pad) continue;
    // first byte of the piece: field qf, threshold tt (1-based); then step
    int qf = (pc * 16) / Lm;
    int tt = pc * 16 - qf * Lm + 1;
    int lev = lv[qf][r];
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint32_t word = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        word |= (lev >= tt ? 0x38u : 0u) << (8 * b);
        if (++tt > Lm) {
          tt = 1;
          ++qf;
          lev = qf < ENC_F ? lv[qf][r] : 0;
        }
      }
      w[u] = word;
    }
    uint4* dst = reinterpret_cast<uint4*>(T + (int64_t)i * Kpad + (int64_t)q0 * Lm + pc * 16);
    *dst = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

}  // namespace

cudaError_t launch_percentile_nonzero(ps_ctx* h, const VF32& V, double p, SelectState* st,
                                      unsigned long long* hist, cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(V.nf, (int64_t)h->num_sms * 8));
  for (int pass = 0; pass < 3; ++pass) {
    cudaError_t e = cudaMemsetAsync(hist, 0, 2048 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    radix_hist_kernel<<<grid, 256, 0, s>>>(V, pass, st, hist);
    radix_select_kernel<<<1, 1024, 0, s>>>(pass, p, st, hist);
  }
  return cudaGetLastError();
}

cudaError_t launch_quantize(const VF32& V, int levels, const SelectState* st, uint8_t* q,
                            int64_t ldq, cudaStream_t s) {
  const int64_t total = (int64_t)V.nf * V.nv;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16);
  quantize_kernel<<<grid, 256, 0, s>>>(V, levels, st, q, ldq);
  return cudaGetLastError();
}

cudaError_t launch_level_sums(const VF32& V, int levels, const SelectState* st, int* SQ,
                              cudaStream_t s) {
  if (V.nv == 0) return cudaSuccess;
  level_sums_kernel<<<(unsigned)ceil_div(V.nv, 32), 256, 0, s>>>(V, levels, st, SQ);
  return cudaGetLastError();
}

int64_t thermo_kpad(int64_t nf, int levels) { return ceil_div(std::max<int64_t>(nf, 1), ENC_F) * ENC_F * (levels - 1); }

cudaError_t launch_thermo_encode(const VF32& V, int levels, const SelectState* st, uint8_t* T,
                                 int64_t Kpad, int nv_pad, int* SQ, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(nv_pad, ENC_V), (unsigned)(Kpad / ((int64_t)ENC_F * (levels - 1))));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (SQ) {
    const cudaError_t e = cudaMemsetAsync(SQ, 0, (size_t)nv_pad * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  thermo_encode_kernel<<<grid, 256, 0, s>>>(V, levels, st, T, Kpad, nv_pad, SQ);
  return cudaGetLastError();
}

namespace {

// Bit-packed 0/1 vectors (PS_B1) straight into the tensor-core operand: row
// i of T is vector i, byte q = 0x38 (FP8 E4M3 1.0) where bit q is set, zero
// elsewhere and in the padding (q >= nf, i >= nv); SQ[i] = number of ones.
// One warp per row, lane -> word; a word's 32 bits become 32 bytes: each
// nibble is spread to one bit per byte by a multiply whose shifted copies
// of the nibble (shifts 0, 7, 14, 21) occupy disjoint bit ranges.
__global__ void __launch_bounds__(256) b1_encode_kernel(const uint32_t* __restrict__ X, int64_t ld,
                                                        int nv, int64_t nf, uint8_t* __restrict__ T,
                                                        int64_t Kpad, int nv_pad, int* __restrict__ SQ) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nv_pad) return;
  const int64_t nw = Kpad / 32;
  int c = 0;
  for (int64_t w = lane; w < nw; w += 32) {
    uint32_t x = 0;
    if (i < nv && w * 32 < nf) {
      x = __ldg(X + i * ld + w);
      const int64_t rem = nf - w * 32;
      if (rem < 32) x &= (1u << rem) - 1u;
    }
    c += __popc(x);
    uint32_t b[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) b[n] = (((x >> (4 * n)) & 0xFu) * 0x00204081u & 0x01010101u) * 0x38u;
    uint4* dst = reinterpret_cast<uint4*>(T + i * Kpad + w * 32);
    dst[0] = make_uint4(b[0], b[1], b[2], b[3]);
    dst[1] = make_uint4(b[4], b[5], b[6], b[7]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) SQ[i] = c;
}

}  // namespace

cudaError_t launch_b1_encode(const uint32_t* X, int64_t ld, int nv, int64_t nf, uint8_t* T, int64_t Kpad,
                             int nv_pad, int* SQ, cudaStream_t s) {
  if (Kpad % 32 != 0 || nv_pad <= 0) return cudaErrorInvalidValue;
  b1_encode_kernel<<<(unsigned)ceil_div(nv_pad, 8), 256, 0, s>>>(X, ld, nv, nf, T, Kpad, nv_pad, SQ);
  return cudaGetLastError();
}

}  // namespace ps
