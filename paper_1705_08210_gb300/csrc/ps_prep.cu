// ps_prep.cu -- per-vector FP64 sums and the FP32 field-major repack.
//
// Section 2.1: the denominators need only S_i = sum_q v_{i,q}, O(n_f n_v)
// adds; they are kept in FP64 and computed from the caller's original values
// (also when the numerators run on an FP32 copy).
#include "ps_internal.cuh"

#include <algorithm>

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

}  // namespace

cudaError_t launch_vector_sums(const ps_matrix& V, double* S, cudaStream_t st) {
  if (V.nv <= 0) return cudaSuccess;
  if (V.layout == PS_LAYOUT_FIELD_MAJOR) {
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
  if (V.layout == PS_LAYOUT_FIELD_MAJOR) {
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
