// ps_mlp.cu -- the encoder of the learned block proposal: forward, pair-loss
// backward and Adam kernels.
//
// Not in the paper.  e_i = W2 relu(W1 x_i + b1) + b2 with x_i = log1p(v_i)
// (d_in = n_f inputs, 256 hidden, 64 outputs), BF16 weights in the forward
// and backward products, FP32 accumulation, FP32 master weights for Adam.
// A pair (i, j) is scored z_ij = e_i . e_j + beta; training minimises the
// logistic loss of z against the label "the pair belongs to a triple with
// c3 >= tau" (labels come from the exact thresholded search).
//
// The products are small (n x d_in x 256 with n <= 8192): a shared-memory
// tiled CUDA-core GEMM with FP32 accumulation is used for all of them; the
// encoder costs well under 1% of the proposal pipeline.
#include "ps_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace ps {
namespace {

constexpr int GT = 64, GK = 16;  // GEMM tile (GT x GT outputs), k slice

// C[m][n] = sum_k A(m, k) * B(n, k), then epi(m, n, acc).  256 threads, each
// 4 x 4 outputs (rows ty + 16 r, columns tx + 16 c).
template <class AccA, class AccB, class Epi>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, AccA A, AccB B, Epi epi) {
  __shared__ float As[GK][GT + 1];
  __shared__ float Bs[GK][GT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e / GT, r = e % GT;
      const int k = k0 + kk;
      As[kk][r] = (k < K && m0 + r < M) ? A(m0 + r, k) : 0.f;
      Bs[kk][r] = (k < K && n0 + r < N) ? B(n0 + r, k) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(As[kk][ty + 16 * r], Bs[kk][tx + 16 * c], acc[r][c]);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < N) epi(m, n, acc[r][c]);
    }
}

template <class AccA, class AccB, class Epi>
cudaError_t gemm(int M, int N, int K, AccA A, AccB B, Epi epi, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(N, GT), (unsigned)ceil_div(M, GT));
  gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, B, epi);
  return cudaGetLastError();
}

// ---- operand accessors ----
struct XLog {  // x(i, q) = log1p(V[q*ld + i])
  const float* p;
  int64_t ld;
  __device__ float operator()(int i, int q) const { return log1pf(__ldg(p + (int64_t)q * ld + i)); }
};
struct XLogT {  // x(q, i) (k = vector index)
  const float* p;
  int64_t ld;
  __device__ float operator()(int q, int i) const { return log1pf(__ldg(p + (int64_t)q * ld + i)); }
};
struct RowBF {  // w(r, c) = W[r*ld + c] in BF16
  const __nv_bfloat16* p;
  int ld;
  __device__ float operator()(int r, int c) const { return __bfloat162float(p[(int64_t)r * ld + c]); }
};
struct ColBF {  // w(c, r) = W[r*ld + c]
  const __nv_bfloat16* p;
  int ld;
  __device__ float operator()(int c, int r) const { return __bfloat162float(p[(int64_t)r * ld + c]); }
};
struct RowF {  // a(r, c) = A[r*ld + c]
  const float* p;
  int ld;
  __device__ float operator()(int r, int c) const { return p[(int64_t)r * ld + c]; }
};
struct ColF {  // a(c, r) = A[r*ld + c]
  const float* p;
  int ld;
  __device__ float operator()(int c, int r) const { return p[(int64_t)r * ld + c]; }
};

// ---- epilogues ----
struct EpiHidden {  // Hpre = acc + b1, H = relu(Hpre)
  const float* b1;
  float* Hpre;
  float* H;
  __device__ void operator()(int i, int h, float acc) const {
    const float v = acc + b1[h];
    Hpre[(int64_t)i * MLP_HIDDEN + h] = v;
    H[(int64_t)i * MLP_HIDDEN + h] = v > 0.f ? v : 0.f;
  }
};
struct EpiOut {  // E = acc + b2
  const float* b2;
  float* E;
  __device__ void operator()(int i, int o, float acc) const { E[(int64_t)i * MLP_OUT + o] = acc + b2[o]; }
};
struct EpiStore {  // G[m][n] = acc
  float* G;
  int ld;
  __device__ void operator()(int m, int n, float acc) const { G[(int64_t)m * ld + n] = acc; }
};
struct EpiReluGrad {  // dH = acc * [Hpre > 0]
  const float* Hpre;
  float* dH;
  __device__ void operator()(int i, int h, float acc) const {
    const int64_t o = (int64_t)i * MLP_HIDDEN + h;
    dH[o] = Hpre[o] > 0.f ? acc : 0.f;
  }
};

// Column sums of G (rows x cols) into out[cols] (fixed order per column).
__global__ void colsum_kernel(const float* __restrict__ G, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += G[(int64_t)r * cols + c];
  out[c] = s;
}

// Pair logistic loss: z = e_i . e_j + beta; dz = (sigmoid(z) - y) / npairs.
// dE rows accumulate dz * e_other; the loss and d beta are reduced per block.
__global__ void pair_loss_kernel(const float* __restrict__ E, const int* __restrict__ pairs,
                                 const float* __restrict__ y, int64_t npairs,
                                 const float* __restrict__ beta_p,
                                 float* __restrict__ dE, double* __restrict__ loss,
                                 float* __restrict__ dbeta) {
  __shared__ double sl[256];
  __shared__ float sb[256];
  double l = 0.0;
  float gb = 0.f;
  const float inv = 1.0f / (float)npairs;
  const float beta = *beta_p;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    const float* ei = E + (int64_t)i * MLP_OUT;
    const float* ej = E + (int64_t)j * MLP_OUT;
    float z = beta;
    for (int d = 0; d < MLP_OUT; ++d) z = fmaf(ei[d], ej[d], z);
    const float t = y[p];
    // log(1 + exp(-|z|)) + max(z, 0) - t z
    l += (double)(log1pf(expf(-fabsf(z))) + fmaxf(z, 0.f) - t * z);
    const float s = 1.f / (1.f + expf(-z));
    const float g = (s - t) * inv;
    gb += g;
    for (int d = 0; d < MLP_OUT; ++d) {
      atomicAdd(&dE[(int64_t)i * MLP_OUT + d], g * ej[d]);
      atomicAdd(&dE[(int64_t)j * MLP_OUT + d], g * ei[d]);
    }
  }
  sl[threadIdx.x] = l;
  sb[threadIdx.x] = gb;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sl[threadIdx.x] += sl[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(loss, sl[0] / (double)npairs);
    atomicAdd(dbeta, sb[0]);
  }
}

// Adam on the FP32 master weights; BF16 copies for the products.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    const float wt = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    w[t] = wt;
    if (wb) wb[t] = __float2bfloat16_rn(wt);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    wb[t] = __float2bfloat16_rn(w[t]);
}

}  // namespace

// Parameter layout (FP32, contiguous): W1 [256][d_in], b1 [256], W2 [64][256],
// b2 [64], beta [1].
int64_t mlp_param_count(int d_in) {
  return (int64_t)MLP_HIDDEN * d_in + MLP_HIDDEN + (int64_t)MLP_OUT * MLP_HIDDEN + MLP_OUT + 1;
}

cudaError_t mlp_sync_bf16(MlpState& M, cudaStream_t st) {
  const int64_t n1 = (int64_t)MLP_HIDDEN * M.d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  to_bf16_kernel<<<256, 256, 0, st>>>(M.w, M.w1b, n1);
  to_bf16_kernel<<<64, 256, 0, st>>>(M.w + n1 + MLP_HIDDEN, M.w2b, n2);
  return cudaGetLastError();
}

// E (n x 64) for the n vectors of the FP32 field-major view V (n = V.nv).
cudaError_t mlp_forward(MlpState& M, const VF32& V, float* Hpre, float* H, float* E, cudaStream_t st) {
  const float* b1 = M.w + (int64_t)MLP_HIDDEN * M.d_in;
  const float* b2 = b1 + MLP_HIDDEN + (int64_t)MLP_OUT * MLP_HIDDEN;
  cudaError_t e = gemm(V.nv, MLP_HIDDEN, M.d_in, XLog{V.p, V.ld}, RowBF{M.w1b, M.d_in},
                       EpiHidden{b1, Hpre, H}, st);
  if (e != cudaSuccess) return e;
  return gemm(V.nv, MLP_OUT, MLP_HIDDEN, RowF{H, MLP_HIDDEN}, RowBF{M.w2b, MLP_HIDDEN}, EpiOut{b2, E},
              st);
}

// Gradient of the mean pair loss w.r.t. all parameters (layout as above);
// loss receives the mean loss.  Buffers: Hpre, H (n x 256), E, dE (n x 64),
// dH (n x 256).
cudaError_t mlp_pair_grad(MlpState& M, const VF32& V, const int* pairs, const float* y, int64_t npairs,
                          float* Hpre, float* H, float* E, float* dE, float* dH, float* grad,
                          double* loss, cudaStream_t st) {
  cudaError_t e = mlp_forward(M, V, Hpre, H, E, st);
  if (e != cudaSuccess) return e;
  const int n = V.nv;
  const int64_t n1 = (int64_t)MLP_HIDDEN * M.d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  float* gW1 = grad;
  float* gb1 = grad + n1;
  float* gW2 = gb1 + MLP_HIDDEN;
  float* gb2 = gW2 + n2;
  float* gbeta = gb2 + MLP_OUT;
  if ((e = cudaMemsetAsync(dE, 0, (size_t)n * MLP_OUT * sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(gbeta, 0, sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st))) return e;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(npairs, 256), 1024));
  const float* beta = M.w + mlp_param_count(M.d_in) - 1;
  pair_loss_kernel<<<g, 256, 0, st>>>(E, pairs, y, npairs, beta, dE, loss, gbeta);
  if ((e = cudaGetLastError())) return e;
  // dW2[o][h] = sum_i dE[i][o] H[i][h];  db2 = colsum(dE)
  if ((e = gemm(MLP_OUT, MLP_HIDDEN, n, ColF{dE, MLP_OUT}, ColF{H, MLP_HIDDEN}, EpiStore{gW2, MLP_HIDDEN}, st)))
    return e;
  colsum_kernel<<<1, 64, 0, st>>>(dE, n, MLP_OUT, gb2);
  // dH = (dE W2) * relu'(Hpre)
  if ((e = gemm(n, MLP_HIDDEN, MLP_OUT, RowF{dE, MLP_OUT}, ColBF{M.w2b, MLP_HIDDEN},
                EpiReluGrad{Hpre, dH}, st)))
    return e;
  // dW1[h][q] = sum_i dH[i][h] x[i][q];  db1 = colsum(dH)
  if ((e = gemm(MLP_HIDDEN, M.d_in, n, ColF{dH, MLP_HIDDEN}, XLogT{V.p, V.ld}, EpiStore{gW1, M.d_in}, st)))
    return e;
  colsum_kernel<<<1, 256, 0, st>>>(dH, n, MLP_HIDDEN, gb1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(MlpState& M, const float* grad, float lr, cudaStream_t st) {
  M.step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)M.step), c2 = 1.f - powf(b2, (float)M.step);
  const int64_t n = mlp_param_count(M.d_in);
  adam_kernel<<<512, 256, 0, st>>>(M.w, grad, M.m, M.v, nullptr, n, lr, b1, b2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return mlp_sync_bf16(M, st);
}

}  // namespace ps
