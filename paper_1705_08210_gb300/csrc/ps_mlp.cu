// ps_mlp.cu -- the encoder of the learned block proposal: forward, pair-loss
// backward and Adam kernels.
//
// Not in the paper.  e_i = W2 relu(W1 x_i + b1) + b2 with x_iq =
// log1p(v_iq n_f / S_i) (scale-free input)
// (d_in = n_f inputs, 256 hidden, 64 outputs), BF16 weights in the forward
// and backward products, FP32 accumulation, FP32 master weights for Adam.
// p_i = softmax(e_i) is a soft assignment to 64 learned clusters; a pair is
// scored P_ij = p_i . p_j (probability of sharing a cluster), and training
// minimises the binary cross-entropy of P against the label "the pair
// belongs to a triple with c3 >= tau" (labels from the exact search).
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
struct XLog {  // x(i, q) = log1p(V[q*ld + i] * r[i]),  r[i] = n_f / S_i
  const float* p;
  int64_t ld;
  const float* r;
  __device__ float operator()(int i, int q) const { return log1pf(__ldg(p + (int64_t)q * ld + i) * r[i]); }
};
struct XLogT {  // x(q, i) (k = vector index)
  const float* p;
  int64_t ld;
  const float* r;
  __device__ float operator()(int q, int i) const { return log1pf(__ldg(p + (int64_t)q * ld + i) * r[i]); }
};

// r[i] = n_f / S_i (0 for an all-zero vector): the encoder input
// log1p(v_iq * r_i) does not change when a vector is scaled.
__global__ void input_scale_kernel(const double* __restrict__ S, int n, int nf, float* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = S[i] > 0.0 ? (float)((double)nf / S[i]) : 0.f;
}
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

// dE = p * (dP - (p . dP)) per row (softmax Jacobian), one warp per row.
__global__ void softmax_backward_kernel(const float* __restrict__ Pm, const float* dPm, int n,
                                        float* dE) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const int64_t o = (int64_t)row * MLP_OUT;
  const float pa = Pm[o + lane], pb = Pm[o + 32 + lane];
  const float ga = dPm[o + lane], gb = dPm[o + 32 + lane];
  float dot = pa * ga + pb * gb;
  for (int s = 16; s > 0; s >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, s);
  dE[o + lane] = pa * (ga - dot);
  dE[o + 32 + lane] = pb * (gb - dot);
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
  const int64_t n1 = (int64_t)MLP_HIDDEN * M.d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  to_bf16_kernel<<<256, 256, 0, st>>>(M.w, M.w1b, n1);
  to_bf16_kernel<<<64, 256, 0, st>>>(M.w + n1 + MLP_HIDDEN, M.w2b, n2);
  return cudaGetLastError();
}

cudaError_t mlp_input_scale(const double* S, int n, int nf, float* r, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  input_scale_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(S, n, nf, r);
  return cudaGetLastError();
}

// E (n x 64) for the n vectors of the FP32 field-major view V (n = V.nv);
// r: per-vector input scales (mlp_input_scale).
cudaError_t mlp_forward(MlpState& M, const VF32& V, const float* r, float* Hpre, float* H, float* E,
                        cudaStream_t st) {
  const float* b1 = M.w + (int64_t)MLP_HIDDEN * M.d_in;
  const float* b2 = b1 + MLP_HIDDEN + (int64_t)MLP_OUT * MLP_HIDDEN;
  cudaError_t e = gemm(V.nv, MLP_HIDDEN, M.d_in, XLog{V.p, V.ld, r}, RowBF{M.w1b, M.d_in},
                       EpiHidden{b1, Hpre, H}, st);
  if (e != cudaSuccess) return e;
  return gemm(V.nv, MLP_OUT, MLP_HIDDEN, RowF{H, MLP_HIDDEN}, RowBF{M.w2b, MLP_HIDDEN}, EpiOut{b2, E},
              st);
}

// Gradient of the mean pair loss w.r.t. all parameters (layout as above);
// loss receives the mean loss.  Buffers: Hpre, H, dH (n x 256), E, Pm, dE
// (n x 64); dE is also used for dP.
cudaError_t mlp_pair_grad(MlpState& M, const VF32& V, const float* r, const int* pairs, const float* y,
                          int64_t npairs, float* Hpre, float* H, float* E, float* Pm, float* dE, float* dH,
                          float* grad, double* loss, cudaStream_t st) {
  cudaError_t e = mlp_forward(M, V, r, Hpre, H, E, st);
  if (e != cudaSuccess) return e;
  const int n = V.nv;
  const int64_t n1 = (int64_t)MLP_HIDDEN * M.d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  float* gW1 = grad;
  float* gb1 = grad + n1;
  float* gW2 = gb1 + MLP_HIDDEN;
  float* gb2 = gW2 + n2;
  if ((e = mlp_softmax(E, n, Pm, st))) return e;
  if ((e = cudaMemsetAsync(dE, 0, (size_t)n * MLP_OUT * sizeof(float), st))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st))) return e;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(npairs, 256), 1024));
  pair_loss_kernel<<<g, 256, 0, st>>>(Pm, pairs, y, npairs, dE, loss);
  if ((e = cudaGetLastError())) return e;
  // dP -> dE in place (each row reads its own dP before writing)
  softmax_backward_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(Pm, dE, n, dE);
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
  if ((e = gemm(MLP_HIDDEN, M.d_in, n, ColF{dH, MLP_HIDDEN}, XLogT{V.p, V.ld, r}, EpiStore{gW1, M.d_in}, st)))
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
