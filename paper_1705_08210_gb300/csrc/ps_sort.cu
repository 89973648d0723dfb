// ps_sort.cu -- stable LSD radix sort of (key, value) pairs and the writer of
// the thresholded 3-way result list.
//
// The thresholded search appends hits in whatever order the CTAs finish; the
// result is defined as the list sorted lexicographically by (i, j, k).  Keys
// pack (i, j, k) into i << 2b | j << b | k, so an ascending sort of the keys
// is the lexicographic order.  Each pass sorts on 8 bits:
//   1. per-block digit histograms (hist[digit][block]);
//   2. exclusive scan of the histogram in digit-major order, giving every
//      (digit, block) its first output position;
//   3. stable scatter: each block walks its chunk in rounds of 256 items;
//      warp peers with the same digit are ranked with __match_any_sync and
//      the per-warp counts are combined in warp order.
#include "ps_internal.cuh"

#include <algorithm>

namespace ps {
namespace {

constexpr int SORT_T = 256, SORT_ITEMS = 16, CHUNK = SORT_T * SORT_ITEMS;
constexpr int SCAN_T = 1024;

__device__ __forceinline__ int digit_of(unsigned long long k, int shift) {
  return (int)((k >> shift) & 255ull);
}

__global__ void __launch_bounds__(SORT_T) sort_hist_kernel(const unsigned long long* __restrict__ keys,
                                                           int64_t n, int shift,
                                                           unsigned* __restrict__ hist, int nblocks) {
  __shared__ unsigned cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CHUNK;
  for (int it = 0; it < SORT_ITEMS; ++it) {
    const int64_t e = base + it * SORT_T + threadIdx.x;
    if (e < n) atomicAdd(&cnt[digit_of(keys[e], shift)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of x[0..n) in chunks of SCAN_T; chunk totals to sums.
__global__ void __launch_bounds__(SCAN_T) scan_chunks_kernel(unsigned* __restrict__ x, int64_t n,
                                                             unsigned* __restrict__ sums) {
  __shared__ unsigned s[SCAN_T];
  const int64_t e = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  const unsigned v = e < n ? x[e] : 0u;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_T; off <<= 1) {  // Hillis-Steele inclusive scan
    const unsigned a = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
    __syncthreads();
    s[threadIdx.x] += a;
    __syncthreads();
  }
  if (e < n) x[e] = s[threadIdx.x] - v;
  if (threadIdx.x == SCAN_T - 1) sums[blockIdx.x] = s[threadIdx.x];
}

// One block: exclusive scan of the chunk totals (sequential over chunks of
// SCAN_T, each scanned in parallel).
__global__ void __launch_bounds__(SCAN_T) scan_sums_kernel(unsigned* __restrict__ sums, int64_t n) {
  __shared__ unsigned s[SCAN_T];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < n; b0 += SCAN_T) {
    const int64_t e = b0 + threadIdx.x;
    const unsigned v = e < n ? sums[e] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
      const unsigned a = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
      __syncthreads();
      s[threadIdx.x] += a;
      __syncthreads();
    }
    if (e < n) sums[e] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == SCAN_T - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_T) add_sums_kernel(unsigned* __restrict__ x, int64_t n,
                                                          const unsigned* __restrict__ sums) {
  const int64_t e = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  if (e < n) x[e] += sums[blockIdx.x];
}

__global__ void __launch_bounds__(SORT_T) sort_scatter_kernel(
    const unsigned long long* __restrict__ kin, const float* __restrict__ vin, int64_t n, int shift,
    const unsigned* __restrict__ offs, int nblocks, unsigned long long* __restrict__ kout,
    float* __restrict__ vout) {
  __shared__ unsigned running[256];
  __shared__ unsigned wcnt[SORT_T / 32][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
#pragma unroll
  for (int w = 0; w < SORT_T / 32; ++w) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * CHUNK;
  for (int it = 0; it < SORT_ITEMS; ++it) {
    const int64_t e = base + it * SORT_T + threadIdx.x;
    const bool valid = e < n;
    unsigned long long k = 0;
    float v = 0.f;
    int d = 256;  // distinct value for the tail
    if (valid) {
      k = kin[e];
      v = vin[e];
      d = digit_of(k, shift);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned pos = running[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    unsigned tot = 0;
#pragma unroll
    for (int w = 0; w < SORT_T / 32; ++w) {
      tot += wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = 0;
    }
    running[threadIdx.x] += tot;
    __syncthreads();
  }
}

__global__ void write_triples_kernel(const unsigned long long* __restrict__ keys,
                                     const float* __restrict__ vals, int64_t n, int bits,
                                     ps_triple* __restrict__ out) {
  const unsigned long long mask = (1ull << bits) - 1ull;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    ps_triple t;
    t.i = (int32_t)(k >> (2 * bits));
    t.j = (int32_t)((k >> bits) & mask);
    t.k = (int32_t)(k & mask);
    t.value = vals[p];
    out[p] = t;
  }
}

__global__ void write_pairs_kernel(const unsigned long long* __restrict__ keys,
                                   const float* __restrict__ vals, int64_t n, int bits,
                                   ps_pair* __restrict__ out) {
  const unsigned long long mask = (1ull << bits) - 1ull;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    ps_pair q;
    q.i = (int32_t)(k >> bits);
    q.j = (int32_t)(k & mask);
    q.value = vals[p];
    out[p] = q;
  }
}

}  // namespace

size_t radix_sort_scratch_words(int64_t n) {
  const int64_t nblocks = std::max<int64_t>(1, ceil_div(n, CHUNK));
  const int64_t hist = 256 * nblocks;
  return (size_t)(hist + ceil_div(hist, SCAN_T) + 64);
}

cudaError_t launch_radix_sort(ps_ctx* h, unsigned long long* keys, float* vals,
                              unsigned long long* keys_tmp, float* vals_tmp, int64_t n, int key_bits,
                              unsigned* scratch, size_t scratch_words, cudaStream_t st) {
  (void)h;
  if (n <= 1) return cudaSuccess;
  if (n > 0xFFFFFFFFll) return cudaErrorInvalidValue;  // positions are 32-bit
  const int nblocks = (int)ceil_div(n, CHUNK);
  const int64_t nh = 256ll * nblocks;
  const int nchunks = (int)ceil_div(nh, SCAN_T);
  if ((size_t)(nh + nchunks) > scratch_words) return cudaErrorInvalidValue;
  unsigned* hist = scratch;
  unsigned* sums = scratch + nh;
  unsigned long long *ka = keys, *kb = keys_tmp;
  float *va = vals, *vb = vals_tmp;
  const int passes = (key_bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    sort_hist_kernel<<<nblocks, SORT_T, 0, st>>>(ka, n, shift, hist, nblocks);
    scan_chunks_kernel<<<nchunks, SCAN_T, 0, st>>>(hist, nh, sums);
    scan_sums_kernel<<<1, SCAN_T, 0, st>>>(sums, nchunks);
    add_sums_kernel<<<nchunks, SCAN_T, 0, st>>>(hist, nh, sums);
    sort_scatter_kernel<<<nblocks, SORT_T, 0, st>>>(ka, va, n, shift, hist, nblocks, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ka != keys) {  // odd number of passes: result is in the temporaries
    e = cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, va, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

cudaError_t launch_write_pairs(const unsigned long long* keys, const float* vals, int64_t n,
                               int bits, ps_pair* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
  write_pairs_kernel<<<grid, 256, 0, st>>>(keys, vals, n, bits, out);
  return cudaGetLastError();
}

cudaError_t launch_write_triples(const unsigned long long* keys, const float* vals, int64_t n,
                                 int bits, ps_triple* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
  write_triples_kernel<<<grid, 256, 0, st>>>(keys, vals, n, bits, out);
  return cudaGetLastError();
}

}  // namespace ps
