// ps_prep.cu -- per-vector FP64 sums and the FP32 field-major repack.
//
// Section 2.1: the denominators need only S_i = sum_q v_{i,q}, O(n_f n_v)
// adds; they are kept in FP64 and computed from the caller's original values
// (also when the numerators run on an FP32 copy).
#include "ps_internal.cuh"

#include <algorithm>

#include <cuda_fp16.h>

namespace ps {
namespace {

template <typename T>
__device__ __forceinline__ double ld_as_double(const T* p) { return (double)__ldg(p); }

// Field-major input, element (i,q) at X[i + q*ld].  A block of 256 threads
// owns 32 consecutive vectors: lane -> vector, warp w sums fields w, w+8, ...
// in FP64; the eight partial sums are combined in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) vector_sums_fm(const T* __restrict__ X, int64_t ld,
                                                      int64_t nv, int64_t nf,
                                                      double* __restrict__ S) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (i < nv) {
    for (int64_t q = warp; q < nf; q += 8) s += ld_as_double(X + i + q * ld);
  }
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < nv) {
    double t = part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += part[w][lane];
    S[i] = t;
  }
}

// Vector-major input, element (i,q) at X[q + i*ld]: one warp per vector,
// lanes stride over q, butterfly reduction (fixed order, deterministic).
template <typename T>
__global__ void __launch_bounds__(256) vector_sums_vm(const T* __restrict__ X, int64_t ld,
                                                      int64_t nv, int64_t nf,
                                                      double* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nv) return;
  double s = 0.0;
  for (int64_t q = lane; q < nf; q += 32) s += ld_as_double(X + q + i * ld);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) S[i] = s;
}

// Field-major -> field-major (FP32 or FP64) with leading dimension ldp,
// zero padding.
template <typename T, typename U>
__global__ void pack_fm(const T* __restrict__ X, int64_t ld, int64_t nv, int64_t nf,
                        U* __restrict__ out, int64_t ldp) {
  const int64_t total = nf * ldp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / ldp, i = t - q * ldp;
    out[t] = (i < nv) ? (U)X[i + q * ld] : (U)0;
  }
}

// Vector-major -> field-major (32 x 32 tile transpose through shared
// memory), zero padding for i in [nv, ldp).
template <typename T, typename U>
__global__ void __launch_bounds__(256) pack_vm(const T* __restrict__ X, int64_t ld, int64_t nv,
                                               int64_t nf, U* __restrict__ out,
                                               int64_t ldp) {
  __shared__ U tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, q0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, q = q0 + tx;
    tile[r][tx] = (i < nv && q < nf) ? (U)X[q + i * ld] : (U)0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t q = q0 + r, i = i0 + tx;
    if (q < nf && i < ldp) out[i + q * ldp] = tile[tx][r];
  }
}

// Bit-packed 0/1 input (PS_B1, Section 2.3's Sorenson case): field q of
// vector i is bit q % 32 of word X[i*ld + q/32]; bits at q >= nf are ignored.
__device__ __forceinline__ uint32_t b1_word(const uint32_t* __restrict__ X, int64_t ld, int64_t i,
                                            int64_t w, int64_t nf) {
  uint32_t x = __ldg(X + i * ld + w);
  const int64_t rem = nf - w * 32;
  if (rem < 32) x &= rem <= 0 ? 0u : ((1u << rem) - 1u);
  return x;
}

// S_i = number of ones of vector i (exact in FP64), one warp per vector.
__global__ void __launch_bounds__(256) vector_sums_b1(const uint32_t* __restrict__ X, int64_t ld,
                                                      int64_t nv, int64_t nf,
                                                      double* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nv) return;
  long long c = 0;
  for (int64_t w = lane; w * 32 < nf; w += 32) c += __popc(b1_word(X, ld, i, w, nf));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) S[i] = (double)c;
}

// Bit-packed -> field-major 0/1 (FP32 or FP64), zero padding for i in
// [nv, ldp): lane -> vector, warp -> word; each warp writes 32 rows q of 32
// consecutive vectors.
template <typename U>
__global__ void __launch_bounds__(256) pack_b1(const uint32_t* __restrict__ X, int64_t ld, int64_t nv,
                                               int64_t nf, U* __restrict__ out, int64_t ldp) {
  const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t w = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5);
  if (w * 32 >= nf || i >= ldp) return;
  const uint32_t x = i < nv ? b1_word(X, ld, i, w, nf) : 0u;
  const int nq = (int)min((int64_t)32, nf - w * 32);
  for (int b = 0; b < nq; ++b) out[(w * 32 + b) * ldp + i] = (U)((x >> b) & 1u);
}

// Largest value of the matrix (non-negative data: unsigned order of the bit
// patterns is the numeric order).
__global__ void max_bits_kernel(VF32 V, unsigned* __restrict__ mx) {
  unsigned m = 0;
  for (int q = blockIdx.x; q < V.nf; q += gridDim.x) {
    const float* row = V.p + (int64_t)q * V.ld;
    for (int i = threadIdx.x; i < V.nv; i += blockDim.x) m = max(m, __float_as_uint(fmaxf(row[i], 0.f)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// out[p*ldo + i] = half2(scale * V[2p][i], scale * V[2p+1][i]) (0 beyond nv / nf);
// scale = 2^e chosen on the device so the largest value lands in [2^13, 2^14).
__global__ void pack_half2_kernel(VF32 V, const unsigned* __restrict__ mx, uint32_t* __restrict__ out,
                                  int64_t ldo, int np, float* __restrict__ inv_scale_out) {
  const float vmax = __uint_as_float(*mx);
  int e = 0;
  if (vmax > 0.f) {
    frexpf(vmax, &e);                     // vmax in [2^(e-1), 2^e)
    e = max(-24, min(24, 14 - e));        // scale 2^e
  }
  const float scale = ldexpf(1.0f, e);
  if (blockIdx.x == 0 && threadIdx.x == 0) *inv_scale_out = ldexpf(1.0f, -e);
  const int64_t total = (int64_t)np * ldo;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / ldo, i = t - p * ldo;
    float x0 = 0.f, x1 = 0.f;
    if (i < V.nv) {
      x0 = V.p[(2 * p) * V.ld + i] * scale;
      if (2 * p + 1 < V.nf) x1 = V.p[(2 * p + 1) * V.ld + i] * scale;
    }
    const __half2 hv = __floats2half2_rn(x0, x1);
    out[t] = *reinterpret_cast<const uint32_t*>(&hv);
  }
}


// Entries that break the paper's precondition v >= 0 (Section 2.1) or are not
// finite: negative, NaN or infinite.  Logical index t = q * nv + i walks the
// matrix in either layout; one atomic per warp.
template <typename T>
__global__ void __launch_bounds__(256) count_invalid(const T* __restrict__ X, int64_t ld, int64_t nv,
                                                     int64_t nf, int field_major,
                                                     unsigned long long* __restrict__ bad) {
  const int64_t total = nv * nf;
  unsigned long long c = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / nv, i = t - q * nv;
    const double x = (double)__ldg(X + (field_major ? i + q * ld : q + i * ld));
    c += !(x >= 0.0 && x <= 1.7976931348623157e308);  // false for NaN, -0.0 passes
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

// Epilogue inputs of the small-n_f 2-way kernels: Sf[i] = fl32(S_i), or 1.0
// for an all-zero vector; words[1] = bits of max Sf; words[0] = bits of the
// smallest nonzero entry of V (non-negative floats order like their bit
// patterns; words are preset to 0x7f7f7f7f and 0 by the launcher).
__global__ void __launch_bounds__(256) narrow_prep_kernel(VF32 V, const double* __restrict__ S,
                                                          float* __restrict__ Sf, unsigned* __restrict__ words) {
  unsigned smax = 0, vmin = 0xffffffffu;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V.nv; i += stride) {
    const float f = S[i] == 0.0 ? 1.0f : (float)S[i];
    Sf[i] = f;
    smax = max(smax, __float_as_uint(f));
  }
  const int64_t total = (int64_t)V.nf * V.nv;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t q = t / V.nv, i = t - q * V.nv;
    const unsigned b = __float_as_uint(__ldg(V.p + q * V.ld + i));
    if (b != 0u) vmin = min(vmin, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (vmin != 0xffffffffu) atomicMin(&words[0], vmin);
    atomicMax(&words[1], smax);
  }
}

}  // namespace

cudaError_t launch_pack_half2(const VF32& V, uint32_t* out, int64_t ldo, unsigned* mx, float* inv_scale,
                              cudaStream_t st) {
  const int np = (V.nf + 1) / 2;
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  max_bits_kernel<<<(unsigned)std::max(1, std::min(V.nf, 152 * 8)), 256, 0, st>>>(V, mx);
  const int64_t total = (int64_t)np * ldo;
  pack_half2_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 152 * 32)), 256,
                      0, st>>>(V, mx, out, ldo, np, inv_scale);
  return cudaGetLastError();
}

cudaError_t launch_count_invalid(const ps_matrix& V, unsigned long long* bad, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || V.nv <= 0 || V.nf <= 0 || V.dtype == PS_B1) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(V.nv * V.nf, 256), 152 * 32);
  const int fm = V.layout == PS_LAYOUT_FIELD_MAJOR;
  if (V.dtype == PS_F32)
    count_invalid<float><<<grid, 256, 0, st>>>((const float*)V.data, V.ld, V.nv, V.nf, fm, bad);
  else
    count_invalid<double><<<grid, 256, 0, st>>>((const double*)V.data, V.ld, V.nv, V.nf, fm, bad);
  return cudaGetLastError();
}

cudaError_t launch_narrow_prep(const VF32& V, const double* S, float* Sf, unsigned* words, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(words, 0x7f, sizeof(unsigned), st);  // 3.4e38: no nonzero value yet
  if (e == cudaSuccess) e = cudaMemsetAsync(words + 1, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || V.nv <= 0) return e;
  const int64_t work = std::max<int64_t>(V.nv, (int64_t)V.nf * V.nv);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), 152 * 16));
  narrow_prep_kernel<<<grid, 256, 0, st>>>(V, S, Sf, words);
  return cudaGetLastError();
}

cudaError_t launch_vector_sums(const ps_matrix& V, double* S, cudaStream_t st) {
  if (V.nv <= 0) return cudaSuccess;
  if (V.dtype == PS_B1) {
    vector_sums_b1<<<(unsigned)ceil_div(V.nv, 8), 256, 0, st>>>((const uint32_t*)V.data, V.ld, V.nv, V.nf, S);
  } else if (V.layout == PS_LAYOUT_FIELD_MAJOR) {
    dim3 grid((unsigned)ceil_div(V.nv, 32));
    if (V.dtype == PS_F32)
      vector_sums_fm<float><<<grid, 256, 0, st>>>((const float*)V.data, V.ld, V.nv, V.nf, S);
    else
      vector_sums_fm<double><<<grid, 256, 0, st>>>((const double*)V.data, V.ld, V.nv, V.nf, S);
  } else {
    dim3 grid((unsigned)ceil_div(V.nv, 8));
    if (V.dtype == PS_F32)
      vector_sums_vm<float><<<grid, 256, 0, st>>>((const float*)V.data, V.ld, V.nv, V.nf, S);
    else
      vector_sums_vm<double><<<grid, 256, 0, st>>>((const double*)V.data, V.ld, V.nv, V.nf, S);
  }
  return cudaGetLastError();
}

template <typename U>
static cudaError_t launch_pack(const ps_matrix& V, U* out, int64_t ldp, cudaStream_t st) {
  if (V.nf <= 0 || ldp <= 0) return cudaSuccess;
  if (V.dtype == PS_B1) {
    if (ceil_div(ceil_div(V.nf, 32), 8) > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)ceil_div(ldp, 32), (unsigned)ceil_div(ceil_div(V.nf, 32), 8));
    pack_b1<U><<<grid, 256, 0, st>>>((const uint32_t*)V.data, V.ld, V.nv, V.nf, out, ldp);
  } else if (V.layout == PS_LAYOUT_FIELD_MAJOR) {
    const int64_t total = V.nf * ldp;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 64);
    if (V.dtype == PS_F32)
      pack_fm<float, U><<<grid, 256, 0, st>>>((const float*)V.data, V.ld, V.nv, V.nf, out, ldp);
    else
      pack_fm<double, U><<<grid, 256, 0, st>>>((const double*)V.data, V.ld, V.nv, V.nf, out, ldp);
  } else {
    if (ceil_div(V.nf, 32) > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)ceil_div(ldp, 32), (unsigned)ceil_div(V.nf, 32));
    if (V.dtype == PS_F32)
      pack_vm<float, U><<<grid, 256, 0, st>>>((const float*)V.data, V.ld, V.nv, V.nf, out, ldp);
    else
      pack_vm<double, U><<<grid, 256, 0, st>>>((const double*)V.data, V.ld, V.nv, V.nf, out, ldp);
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_f32(const ps_matrix& V, float* out, int64_t ldp, cudaStream_t st) {
  return launch_pack<float>(V, out, ldp, st);
}

cudaError_t launch_pack_f64(const ps_matrix& V, double* out, int64_t ldp, cudaStream_t st) {
  return launch_pack<double>(V, out, ldp, st);
}

}  // namespace ps
