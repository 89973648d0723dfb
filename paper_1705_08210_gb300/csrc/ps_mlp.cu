// ps_mlp.cu -- the encoder of the learned block proposal: element-wise and
// reduction kernels, the pair loss and its backward pass, Adam.
//
// Not in the paper.  e_i = W2 relu(W1 x_i + b1) + b2 with x_iq =
// log1p(v_iq n_f / S_i) (scale-free input) (d_in = n_f inputs, 256 hidden,
// 64 outputs).  The five products of the forward and backward passes run on
// the tensor cores (ps_mlp_tc.cu: BF16 operands, FP32 accumulation); FP32
// master weights for Adam.  p_i = softmax(e_i) is a soft assignment to 64
// learned clusters; a pair is scored P_ij = p_i . p_j (probability of sharing
// a cluster), and training minimises the binary cross-entropy of P against
// the label "the pair belongs to a triple with c3 >= tau" (labels from the
// exact search).
#include "ps_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace ps {
namespace {

using bf16 = __nv_bfloat16;

// r[i] = n_f / S_i (0 for an all-zero vector): the encoder input
// log1p(v_iq * r_i) does not change when a vector is scaled.
__global__ void input_scale_kernel(const double* __restrict__ S, int n, int nf, float* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = S[i] > 0.0 ? (float)((double)nf / S[i]) : 0.f;
}

// Column sums of G (rows x cols, row-major) into out[cols]: block b covers
// columns 32b .. 32b + 31; thread (slice, column) adds rows slice, slice + 8,
// ...; the eight partials are added in a fixed order (deterministic).
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ G, int rows, int cols,
                                                     float* __restrict__ out) {
  __shared__ float part[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), sl = threadIdx.x >> 5;
  float s = 0.f;
  if (c < cols)
    for (int r = sl; r < rows; r += 8) s += G[(int64_t)r * cols + c];
  part[sl][threadIdx.x & 31] = s;
  __syncthreads();
  if (sl == 0 && c < cols) {
    float t = part[0][threadIdx.x];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += part[k][threadIdx.x];
    out[c] = t;
  }
}

// Row softmax P = softmax(E) (n x 64), one warp per row.
__global__ void softmax_kernel(const float* __restrict__ E, int n, float* __restrict__ Pm) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const float a = E[(int64_t)row * MLP_OUT + lane], b = E[(int64_t)row * MLP_OUT + 32 + lane];
  float mx = fmaxf(a, b);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float ea = expf(a - mx), eb = expf(b - mx);
  float s = ea + eb;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  Pm[(int64_t)row * MLP_OUT + lane] = ea / s;
  Pm[(int64_t)row * MLP_OUT + 32 + lane] = eb / s;
}

// Pair loss: P = p_i . p_j clamped to [1e-6, 1 - 1e-6],
// loss = -(y log P + (1-y) log(1-P)), mean over pairs; dPm accumulates
// dloss/dP * p_other into both rows.
__global__ void pair_loss_kernel(const float* __restrict__ Pm, const int* __restrict__ pairs,
                                 const float* __restrict__ y, int64_t npairs, float* __restrict__ dPm,
                                 double* __restrict__ loss) {
  __shared__ double sl[256];
  double l = 0.0;
  const float inv = 1.0f / (float)npairs;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    const float* pi = Pm + (int64_t)i * MLP_OUT;
    const float* pj = Pm + (int64_t)j * MLP_OUT;
    float P = 0.f;
    for (int d = 0; d < MLP_OUT; ++d) P = fmaf(pi[d], pj[d], P);
    const float Pc = fminf(fmaxf(P, 1e-6f), 1.f - 1e-6f);
    const float t = y[p];
    l += (double)(-(t * logf(Pc) + (1.f - t) * log1pf(-Pc)));
    // d/dP of the clamped loss (zero outside the clamp)
    float g = (P > 1e-6f && P < 1.f - 1e-6f) ? (-t / Pc + (1.f - t) / (1.f - Pc)) : 0.f;
    g *= inv;
    for (int d = 0; d < MLP_OUT; ++d) {
      atomicAdd(&dPm[(int64_t)i * MLP_OUT + d], g * pj[d]);
      atomicAdd(&dPm[(int64_t)j * MLP_OUT + d], g * pi[d]);
    }
  }
  sl[threadIdx.x] = l;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sl[threadIdx.x] += sl[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, sl[0] / (double)npairs);
}

// dE = p * (dP - (p . dP)) per row (softmax Jacobian), one warp per row; also
// the BF16 operands of the backward products: dEb (n x 64) and dEbT
// (64 x ldn).
__global__ void softmax_backward_kernel(const float* __restrict__ Pm, const float* dPm, int n, float* dE,
                                        bf16* __restrict__ dEb, bf16* __restrict__ dEbT, int64_t ldn) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const int64_t o = (int64_t)row * MLP_OUT;
  const float pa = Pm[o + lane], pb = Pm[o + 32 + lane];
  const float ga = dPm[o + lane], gb = dPm[o + 32 + lane];
  float dot = pa * ga + pb * gb;
  for (int s = 16; s > 0; s >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, s);
  const float da = pa * (ga - dot), db = pb * (gb - dot);
  dE[o + lane] = da;
  dE[o + 32 + lane] = db;
  const bf16 ba = __float2bfloat16_rn(da), bb = __float2bfloat16_rn(db);
  dEb[o + lane] = ba;
  dEb[o + 32 + lane] = bb;
  dEbT[(int64_t)lane * ldn + row] = ba;
  dEbT[(int64_t)(32 + lane) * ldn + row] = bb;
}

// The step counter of Adam lives on the device, so that a training step can
// be replayed from a CUDA graph.
__global__ void adam_step_kernel(int* __restrict__ step) { *step += 1; }

// Adam on the FP32 master weights, step t = *step (bias corrections
// 1 - b1^t and 1 - b2^t).
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            const int* __restrict__ step) {
  const float t1 = (float)*step;
  const float c1 = 1.f - powf(b1, t1), c2 = 1.f - powf(b2, t1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    w[t] = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

// BF16 copies of the weights for the products: W1 (rows of pitch ld1), W2 and
// its transpose.
__global__ void to_bf16_kernel(const float* __restrict__ W1, int d_in, int64_t ld1, const float* __restrict__ W2,
                               bf16* __restrict__ w1b, bf16* __restrict__ w2b, bf16* __restrict__ w2bt) {
  const int64_t n1 = (int64_t)MLP_HIDDEN * d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < n1) {
      const int64_t h = t / d_in, q = t - h * d_in;
      w1b[h * ld1 + q] = __float2bfloat16_rn(W1[t]);
    } else {
      const int64_t u = t - n1, o = u / MLP_HIDDEN, h = u - o * MLP_HIDDEN;
      const bf16 b = __float2bfloat16_rn(W2[u]);
      w2b[u] = b;
      w2bt[h * MLP_OUT + o] = b;
    }
  }
}

}  // namespace

// Parameter layout (FP32, contiguous): W1 [256][d_in], b1 [256], W2 [64][256],
// b2 [64].
int64_t mlp_param_count(int d_in) {
  return (int64_t)MLP_HIDDEN * d_in + MLP_HIDDEN + (int64_t)MLP_OUT * MLP_HIDDEN + MLP_OUT;
}

cudaError_t mlp_softmax(const float* E, int n, float* Pm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  softmax_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(E, n, Pm);
  return cudaGetLastError();
}

cudaError_t mlp_sync_bf16(MlpState& M, cudaStream_t st) {
  const float* W2 = M.w + (int64_t)MLP_HIDDEN * M.d_in + MLP_HIDDEN;
  to_bf16_kernel<<<512, 256, 0, st>>>(M.w, M.d_in, round_up(M.d_in, 8), W2, M.w1b, M.w2b, M.w2bt);
  return cudaGetLastError();
}

cudaError_t mlp_input_scale(const double* S, int n, int nf, float* r, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  input_scale_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(S, n, nf, r);
  return cudaGetLastError();
}

cudaError_t mlp_pair_grad(MlpState& M, const MlpBufs& B, const int* pairs, const float* y, int64_t npairs,
                          float* grad, double* loss, cudaStream_t st) {
  cudaError_t e = mlp_forward_tc(M, B, true, st);
  if (e != cudaSuccess) return e;
  const int n = B.n;
  const int64_t n1 = (int64_t)MLP_HIDDEN * M.d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  float* gW1 = grad;
  float* gb1 = grad + n1;
  float* gW2 = gb1 + MLP_HIDDEN;
  float* gb2 = gW2 + n2;
  if ((e = mlp_softmax(B.E, n, B.Pm, st))) return e;
  if ((e = cudaMemsetAsync(B.dE, 0, (size_t)n * MLP_OUT * sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st))) return e;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(npairs, 256), 1024));
  pair_loss_kernel<<<g, 256, 0, st>>>(B.Pm, pairs, y, npairs, B.dE, loss);
  if ((e = cudaGetLastError())) return e;
  // dP -> dE in place (each row reads its own dP before writing)
  softmax_backward_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(B.Pm, B.dE, n, B.dE, B.dEb, B.dEbT, B.ldn);
  if ((e = cudaGetLastError())) return e;
  colsum_kernel<<<MLP_OUT / 32, 256, 0, st>>>(B.dE, n, MLP_OUT, gb2);  // db2
  if ((e = cudaGetLastError())) return e;
  if ((e = mlp_backward_tc(M, B, gW1, gW2, st))) return e;             // dW2, dH, dW1
  colsum_kernel<<<MLP_HIDDEN / 32, 256, 0, st>>>(B.dH, n, MLP_HIDDEN, gb1);  // db1
  return cudaGetLastError();
}

cudaError_t mlp_adam(MlpState& M, const float* grad, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int64_t n = mlp_param_count(M.d_in);
  adam_step_kernel<<<1, 1, 0, st>>>(M.dstep);
  adam_kernel<<<512, 256, 0, st>>>(M.w, grad, M.m, M.v, n, lr, b1, b2, eps, M.dstep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return mlp_sync_bf16(M, st);
}

}  // namespace ps
