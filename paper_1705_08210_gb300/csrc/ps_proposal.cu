// ps_proposal.cu -- block proposals for the thresholded 3-way search.
//
// Not in the paper.  The exact thresholded search visits every 128-tile
// block (I <= J <= K) of the tetrahedron.  Two ways to visit fewer:
//
//  * learned (use_proposal = 1): the encoder of ps_mlp.cu assigns every
//    vector a soft cluster p = softmax(e) over 64 learned clusters; vectors
//    are reordered by their most likely cluster, so vectors that form
//    high-c3 triples land in the same tiles; for every tile pair the maximum
//    pair score P = p_a . p_b is taken, and a block is proposed when its
//    three tile pairs all reach the threshold theta calibrated on the
//    training data.  Recall is measured against the exhaustive search.
//  * bound (use_proposal = 2, lossless): from min(a,b,c) >= min(a,b) +
//    min(a,c) - a, n3' >= n2(ij) + n2(ik) - S_i (and its two rotations), so
//    c3 <= 1.5 min(n2ij+n2ik+n2jk, n2jk+S_i, n2ik+S_j, n2ij+S_k) / d3.
//    A block is kept when any of its triples reaches tau under this bound
//    (evaluated on the pair table the search needs anyway).  Reordered by
//    the encoder when one is trained, else in input order.
//
// The selected blocks then run through the same exact kernel as the
// exhaustive search; its epilogue forms eq. (1) in original index order, so
// every reported value equals the exhaustive one bit for bit.
#include "ps_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_set>
#include <vector>

namespace ps {
namespace {

constexpr int PT = 128;  // tile width of the block lists

__global__ void cluster_keys_kernel(const float* __restrict__ E, int n, unsigned long long* keys,
                                    float* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int best = 0;
  float bv = E[(int64_t)i * MLP_OUT];
  for (int d = 1; d < MLP_OUT; ++d) {
    const float v = E[(int64_t)i * MLP_OUT + d];
    if (v > bv) {
      bv = v;
      best = d;
    }
  }
  keys[i] = ((unsigned long long)best << 32) | (unsigned long long)i;
  vals[i] = __int_as_float(i);
}

__global__ void perm_from_vals_kernel(const float* __restrict__ vals, int n, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) perm[i] = __float_as_int(vals[i]);
}

// out[q*ldo + p] = V[q*ld + perm[p]] (zero for p >= nv); Sp[p] = S[perm[p]].
__global__ void gather_kernel(VF32 V, const double* __restrict__ S, const int* __restrict__ perm,
                              float* __restrict__ out, int64_t ldo, double* __restrict__ Sp) {
  const int64_t total = (int64_t)V.nf * ldo;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / ldo, p = t - q * ldo;
    out[t] = p < V.nv ? V.p[q * V.ld + perm[p]] : 0.0f;
    if (q == 0 && p < V.nv) Sp[p] = S[perm[p]];
  }
}

// Tmax[A][B] = Tmax[B][A] = max over a in tile A, b in tile B (a < b) of
// P = p_a . p_b (p: cluster probabilities); one block per tile pair A <= B.
__global__ void __launch_bounds__(256) tile_pair_max_kernel(const float* __restrict__ E, int n, int T,
                                                            float* __restrict__ Tmax) {
  __shared__ float ea[PT][MLP_OUT + 1];
  __shared__ float eb[PT][MLP_OUT + 1];
  __shared__ float red[256];
  // upper-triangle index -> (A, B)
  const int64_t t = blockIdx.x;
  int A = 0;
  while ((int64_t)(A + 1) * T - (int64_t)(A + 1) * A / 2 <= t) ++A;
  const int B = A + (int)(t - ((int64_t)A * T - (int64_t)A * (A - 1) / 2));
  for (int e = threadIdx.x; e < PT * MLP_OUT; e += 256) {
    const int r = e / MLP_OUT, d = e % MLP_OUT;
    const int ia = A * PT + r, ib = B * PT + r;
    ea[r][d] = ia < n ? E[(int64_t)ia * MLP_OUT + d] : 0.f;
    eb[r][d] = ib < n ? E[(int64_t)ib * MLP_OUT + d] : 0.f;
  }
  __syncthreads();
  float best = -INFINITY;
  for (int e = threadIdx.x; e < PT * PT; e += 256) {
    const int r = e / PT, c = e % PT;
    const int ia = A * PT + r, ib = B * PT + c;
    if (ia >= n || ib >= n || ia >= ib) continue;
    float z = 0.f;
#pragma unroll 16
    for (int d = 0; d < MLP_OUT; ++d) z = fmaf(ea[r][d], eb[c][d], z);
    best = fmaxf(best, z);
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Tmax[(int64_t)A * T + B] = red[0];
    Tmax[(int64_t)B * T + A] = red[0];
  }
}

// Pair scores P = p_i . p_j for a list of pairs.
__global__ void pair_score_kernel(const float* __restrict__ E, const int* __restrict__ pairs, int64_t np,
                                  float* __restrict__ z) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float* ei = E + (int64_t)pairs[2 * p] * MLP_OUT;
    const float* ej = E + (int64_t)pairs[2 * p + 1] * MLP_OUT;
    float s = 0.f;
    for (int d = 0; d < MLP_OUT; ++d) s = fmaf(ei[d], ej[d], s);
    z[p] = s;
  }
}

// Lossless block filter: flag[b] = 1 if some triple i<j<k of block b has
// 1.5 min(n2ij+n2ik+n2jk, n2jk+S_i, n2ik+S_j, n2ij+S_k) >= tau' d3.
constexpr int BF_THREADS = 256;
struct BoundSmem {
  float ik[PT][PT + 1];
  float jk[PT][PT + 1];
  float si[PT], sj[PT], sk[PT];
  int found;
};

__global__ void __launch_bounds__(BF_THREADS) bound_filter_kernel(const float* __restrict__ n2, const double* __restrict__ S,
                                                                  int nv, const int* __restrict__ blocks,
                                                                  float thr, int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char raw[];
  BoundSmem& sm = *reinterpret_cast<BoundSmem*>(raw);
  const int b = blockIdx.x;
  const int I = blocks[3 * b], J = blocks[3 * b + 1], K = blocks[3 * b + 2];
  const int i0 = I * PT, j0 = J * PT, k0 = K * PT;
  for (int e = threadIdx.x; e < PT * PT; e += BF_THREADS) {
    const int r = e / PT, c = e % PT;
    const int i = i0 + r, j = j0 + r, k = k0 + c;
    sm.ik[r][c] = (i < nv && k < nv) ? n2[(int64_t)i * nv + k] : 0.f;
    sm.jk[r][c] = (j < nv && k < nv) ? n2[(int64_t)j * nv + k] : 0.f;
  }
  for (int r = threadIdx.x; r < PT; r += BF_THREADS) {
    sm.si[r] = i0 + r < nv ? (float)S[i0 + r] : 0.f;
    sm.sj[r] = j0 + r < nv ? (float)S[j0 + r] : 0.f;
    sm.sk[r] = k0 + r < nv ? (float)S[k0 + r] : 0.f;
  }
  if (threadIdx.x == 0) sm.found = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < PT * PT; e += BF_THREADS) {
    if (*(volatile int*)&sm.found) break;
    const int r = e / PT, c = e % PT;
    const int i = i0 + r, j = j0 + c;
    if (i >= j || j >= nv) continue;
    const float nij = n2[(int64_t)i * nv + j];
    const float si = sm.si[r], sj = sm.sj[c];
    const int kstart = max(0, j + 1 - k0);
    for (int kk = kstart; kk < PT && k0 + kk < nv; ++kk) {
      const float nik = sm.ik[r][kk], njk = sm.jk[c][kk], sk = sm.sk[kk];
      const float m = fminf(fminf(nij + nik + njk, njk + si), fminf(nik + sj, nij + sk));
      if (m >= thr * (si + sj + sk)) {
        sm.found = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) flags[b] = sm.found;
}

// splitmix64: the host generator of negative pairs
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct DevBuf {  // small owned device allocations of the training loop
  std::vector<void*> ptrs;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return p;
  }
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
};

ps_status mlp_alloc(ps_ctx* h, int d_in, uint64_t seed) {
  MlpState& M = h->mlp;
  if (M.w) {
    cudaFree(M.w);
    M.w = nullptr;
  }
  M = MlpState();
  M.d_in = d_in;
  M.device = h->device;
  const int64_t n = mlp_param_count(d_in);
  const int64_t n1 = (int64_t)MLP_HIDDEN * d_in, n2 = (int64_t)MLP_OUT * MLP_HIDDEN;
  const int64_t n1p = (int64_t)MLP_HIDDEN * round_up(d_in, 8);  // W1 in BF16, rows padded to 16 bytes
  char* mem = nullptr;
  const size_t bytes = (size_t)n * 12 + (size_t)(n1p + 2 * n2) * 2 + 4096;
  PS_CUDA_TRY(h, cudaMalloc(&mem, bytes));
  PS_CUDA_TRY(h, cudaMemset(mem, 0, bytes));
  M.w = reinterpret_cast<float*>(mem);
  M.m = M.w + n;
  M.v = M.m + n;
  M.w1b = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<uintptr_t>(M.v + n + 64) & ~(uintptr_t)255);
  M.w2b = reinterpret_cast<__nv_bfloat16*>(round_up((int64_t)reinterpret_cast<uintptr_t>(M.w1b + n1p), 256));
  M.w2bt = M.w2b + n2;
  M.err = reinterpret_cast<int*>(round_up((int64_t)reinterpret_cast<uintptr_t>(M.w2bt + n2), 256));
  M.dstep = M.err + 32;
  // Glorot-uniform weights, zero biases (host generator)
  std::vector<float> w((size_t)n, 0.f);
  uint64_t s = seed;
  const float a1 = std::sqrt(6.f / (float)(d_in + MLP_HIDDEN)), a2 = std::sqrt(6.f / (float)(MLP_HIDDEN + MLP_OUT));
  for (int64_t t = 0; t < n1; ++t) w[t] = a1 * (2.f * (float)((splitmix(s) >> 11) * 0x1.0p-53) - 1.f);
  for (int64_t t = 0; t < n2; ++t)
    w[n1 + MLP_HIDDEN + t] = a2 * (2.f * (float)((splitmix(s) >> 11) * 0x1.0p-53) - 1.f);
  PS_CUDA_TRY(h, cudaMemcpy(M.w, w.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
  PS_CUDA_TRY(h, cudaMemset(M.m, 0, (size_t)n * 8));
  PS_CUDA_TRY(h, mlp_sync_bf16(M, 0));
  PS_CUDA_TRY(h, cudaDeviceSynchronize());
  return PS_OK;
}

}  // namespace

void mlp_free(ps_ctx* h) {
  if (h->mlp.w) cudaFree(h->mlp.w);
  h->mlp = MlpState();
}

// The tensor-core products' error word: PS_ERR_TIMEOUT (and cleared) if a
// pipeline wait ran out since the last check.  Synchronises `st`.
ps_status mlp_take_error(ps_ctx* h, cudaStream_t st) {
  int e = 0;
  PS_CUDA_TRY(h, cudaMemcpyAsync(&e, h->mlp.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  if (e) {
    PS_CUDA_TRY(h, cudaMemsetAsync(h->mlp.err, 0, sizeof(int), st));
    return fail(h, PS_ERR_TIMEOUT, "encoder: a tensor-core pipeline wait timed out");
  }
  return PS_OK;
}

// Encoder outputs E of the n vectors of v (sums S) into buffers from WS_MLP.
ps_status mlp_encode(ps_ctx* h, const VF32& v, const double* S, cudaStream_t st, MlpBufs* out) {
  MlpState& M = h->mlp;
  M.wait_ns = h->wait_ns;
  const int n = v.nv;
  void* base = ws_get(h, WS_MLP, mlp_bufs_bytes(n, M.d_in, true));
  if (!base) return PS_ERR_OOM;
  const MlpBufs B = mlp_bufs_at(base, n, M.d_in, true);
  PS_CUDA_TRY(h, mlp_input_scale(S, n, v.nf, B.r, st));
  PS_CUDA_TRY(h, mlp_prep_x(v, B.r, B.Xb, B.ldx, nullptr, B.ldn, st));
  PS_CUDA_TRY(h, mlp_forward_tc(M, B, false, st));
  *out = B;
  return mlp_take_error(h, st);
}

// Reorder by learned cluster: perm, the reordered FP32 view and sums.
ps_status proposal_reorder(ps_ctx* h, const VF32& v, const double* S, cudaStream_t st, VF32* vp,
                           double** Sp, int** perm) {
  MlpState& M = h->mlp;
  const int n = v.nv;
  if (v.nf != M.d_in)
    return fail(h, PS_ERR_INVALID_ARG, "encoder expects nf=%d, matrix has nf=%d", M.d_in, v.nf);
  const int64_t ldp = round_up(n, 4);
  float* vperm = static_cast<float*>(ws_get(h, WS_PERMV, (size_t)v.nf * ldp * 4 + (size_t)n * 8 + 256));
  unsigned char* sortb = static_cast<unsigned char*>(ws_get(h, WS_HITS, (size_t)n * 24 + 256));
  int* dperm = static_cast<int*>(ws_get(h, WS_PERM, (size_t)n * 4 + 256));
  const size_t words = radix_sort_scratch_words(n);
  unsigned* scratch = static_cast<unsigned*>(ws_get(h, WS_SORT, words * 4));
  if (!vperm || !sortb || !dperm || !scratch) return PS_ERR_OOM;
  MlpBufs B;
  {
    ScopedTimer tm(h, "proposal_encode", st);
    const ps_status es = mlp_encode(h, v, S, st, &B);
    if (es != PS_OK) return es;
  }
  const float* E = B.E;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(sortb);
  unsigned long long* ktmp = keys + n;
  float* vals = reinterpret_cast<float*>(ktmp + n);
  float* vtmp = vals + n;
  cluster_keys_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(E, n, keys, vals);
  PS_CUDA_TRY(h, cudaGetLastError());
  PS_CUDA_TRY(h, launch_radix_sort(h, keys, vals, ktmp, vtmp, n, 40, scratch, words, st));
  perm_from_vals_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(vals, n, dperm);
  double* dS = reinterpret_cast<double*>(vperm + (size_t)v.nf * ldp + 64);
  dS = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(dS) & ~(uintptr_t)15);
  const int64_t total = (int64_t)v.nf * ldp;
  gather_kernel<<<(unsigned)std::min<int64_t>(std::max<int64_t>(1, ceil_div(total, 256)), 152 * 32), 256,
                  0, st>>>(v, S, dperm, vperm, ldp, dS);
  PS_CUDA_TRY(h, cudaGetLastError());
  *vp = VF32{vperm, ldp, n, v.nf};
  *Sp = dS;
  *perm = dperm;
  return PS_OK;
}

// Learned proposal on the reordered view: blocks whose three tile pairs
// reach theta.  Returns the fraction of blocks kept in *kept.
ps_status proposal_blocks_learned(ps_ctx* h, const VF32& vp, const double* Sp, cudaStream_t st,
                                  std::vector<int>* blk, double* kept) {
  MlpState& M = h->mlp;
  const int n = vp.nv;
  const int T = (int)ceil_div(n, PT);
  float* tmax = static_cast<float*>(ws_get(h, WS_AUX2, (size_t)T * T * 4 + 256));
  if (!tmax) return PS_ERR_OOM;
  {
    ScopedTimer tm(h, "proposal_score", st);
    MlpBufs B;
    const ps_status es = mlp_encode(h, vp, Sp, st, &B);
    if (es != PS_OK) return es;
    PS_CUDA_TRY(h, mlp_softmax(B.E, n, B.Pm, st));
    tile_pair_max_kernel<<<(unsigned)((int64_t)T * (T + 1) / 2), 256, 0, st>>>(B.Pm, n, T, tmax);
    PS_CUDA_TRY(h, cudaGetLastError());
  }
  std::vector<float> tm_h((size_t)T * T);
  PS_CUDA_TRY(h, cudaMemcpyAsync(tm_h.data(), tmax, tm_h.size() * 4, cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  int64_t all = 0;
  blk->clear();
  for (int I = 0; I < T; ++I)
    for (int K = I; K < T; ++K)
      for (int J = I; J <= K; ++J) {
        ++all;
        if (tm_h[(size_t)I * T + J] >= M.theta && tm_h[(size_t)I * T + K] >= M.theta &&
            tm_h[(size_t)J * T + K] >= M.theta) {
          blk->push_back(I);
          blk->push_back(J);
          blk->push_back(K);
        }
      }
  *kept = all ? (double)(blk->size() / 3) / (double)all : 0.0;
  return PS_OK;
}

// Lossless bound filter over all blocks of the (possibly reordered) view.
ps_status proposal_blocks_bound(ps_ctx* h, const VF32& vp, const double* Sp, const float* n2, float tau,
                                cudaStream_t st, std::vector<int>* blk, double* kept) {
  const int n = vp.nv;
  const int T = (int)ceil_div(n, PT);
  std::vector<int> all;
  for (int I = 0; I < T; ++I)
    for (int K = I; K < T; ++K)
      for (int J = I; J <= K; ++J) {
        all.push_back(I);
        all.push_back(J);
        all.push_back(K);
      }
  const int nb = (int)(all.size() / 3);
  int* dblk = static_cast<int*>(ws_get(h, WS_BLOCKS, all.size() * 4 + 256));
  int* flags = static_cast<int*>(ws_get(h, WS_AUX2, (size_t)nb * 4 + 256));
  if (!dblk || !flags) return PS_ERR_OOM;
  PS_CUDA_TRY(h, cudaMemcpyAsync(dblk, all.data(), all.size() * 4, cudaMemcpyHostToDevice, st));
  static bool attr = false;
  if (!attr) {
    PS_CUDA_TRY(h, cudaFuncSetAttribute(bound_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(BoundSmem)));
    attr = true;
  }
  // a small margin keeps the FP32 bound on the safe side of the FP32 c3
  const float thr = (float)(tau / 1.5) * (1.0f - 1e-4f);
  {
    ScopedTimer tm(h, "proposal_bound", st);
    bound_filter_kernel<<<nb, BF_THREADS, sizeof(BoundSmem), st>>>(n2, Sp, n, dblk, thr, flags);
    PS_CUDA_TRY(h, cudaGetLastError());
  }
  std::vector<int> f((size_t)nb);
  PS_CUDA_TRY(h, cudaMemcpyAsync(f.data(), flags, (size_t)nb * 4, cudaMemcpyDeviceToHost, st));
  PS_CUDA_TRY(h, cudaStreamSynchronize(st));
  blk->clear();
  for (int b = 0; b < nb; ++b)
    if (f[b]) {
      blk->push_back(all[3 * b]);
      blk->push_back(all[3 * b + 1]);
      blk->push_back(all[3 * b + 2]);
    }
  *kept = nb ? (double)(blk->size() / 3) / nb : 0.0;
  return PS_OK;
}

}  // namespace ps

using namespace ps;

extern "C" ps_status ps_proposal_init(ps_handle h, int32_t d_in, uint64_t seed) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (d_in < 1 || d_in > (1 << 20)) return fail(h, PS_ERR_INVALID_ARG, "d_in=%d", d_in);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  const ps_status s = mlp_alloc(h, d_in, seed);
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

extern "C" int64_t ps_proposal_param_count(ps_handle h) {
  return (h && h->mlp.w) ? mlp_param_count(h->mlp.d_in) : -1;
}

extern "C" ps_status ps_proposal_params(ps_handle h, int32_t set, float* params, int64_t n,
                                        float* theta) {
  if (!h || !h->mlp.w) return fail(h, PS_ERR_INVALID_ARG, "no encoder (ps_proposal_init first)");
  if (!params || n != mlp_param_count(h->mlp.d_in))
    return fail(h, PS_ERR_INVALID_ARG, "params: expected %lld floats",
                (long long)mlp_param_count(h->mlp.d_in));
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaError_t e;
  if (set) {
    e = cudaMemcpy(h->mlp.w, params, (size_t)n * 4, cudaMemcpyDefault);
    if (e == cudaSuccess) e = mlp_sync_bf16(h->mlp, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (theta) {
      h->mlp.theta = *theta;
      h->mlp.trained = true;
    }
  } else {
    e = cudaMemcpy(params, h->mlp.w, (size_t)n * 4, cudaMemcpyDefault);
    if (theta) *theta = h->mlp.theta;
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(h, e, "ps_proposal_params");
  return PS_OK;
}

// Forward pass and the gradient of the mean pair loss (test hooks).
extern "C" ps_status ps_proposal_pair_grad(ps_handle h, const ps_matrix* V, const int32_t* pairs,
                                           const float* labels, int64_t npairs, float* E_out,
                                           float* grad, double* loss, ps_stream stream) {
  if (!h || !h->mlp.w) return fail(h, PS_ERR_INVALID_ARG, "no encoder (ps_proposal_init first)");
  if (!V || V->dtype != PS_F32 || V->layout != PS_LAYOUT_FIELD_MAJOR || V->nf != h->mlp.d_in)
    return fail(h, PS_ERR_INVALID_ARG, "pair_grad: FP32 field-major device matrix with nf = d_in");
  if (npairs < 0 || (npairs > 0 && (!pairs || !labels))) return fail(h, PS_ERR_INVALID_ARG, "pairs");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)V->nv;
  const VF32 v{static_cast<const float*>(V->data), V->ld, n, (int)V->nf};
  h->mlp.wait_ns = h->wait_ns;
  void* base = ws_get(h, WS_MLP, mlp_bufs_bytes(n, h->mlp.d_in, true));
  double* dloss = static_cast<double*>(ws_get(h, WS_AUX3, 256));
  double* dS = static_cast<double*>(ws_get(h, WS_SUMS, (size_t)std::max(n, 1) * 8));
  if (!base || !dloss || !dS) return PS_ERR_OOM;
  const MlpBufs B = mlp_bufs_at(base, n, h->mlp.d_in, true);
  cudaError_t e = launch_vector_sums(*V, dS, st);
  if (e == cudaSuccess) e = mlp_input_scale(dS, n, (int)V->nf, B.r, st);
  if (e == cudaSuccess) e = mlp_prep_x(v, B.r, B.Xb, B.ldx, B.XbT, B.ldn, st);
  if (e != cudaSuccess) {
  } else if (grad && npairs > 0) {
    e = mlp_pair_grad(h->mlp, B, pairs, labels, npairs, grad, dloss, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, dloss, 8, cudaMemcpyDefault, st);
  } else {
    e = mlp_forward_tc(h->mlp, B, false, st);
  }
  if (e == cudaSuccess && E_out) e = cudaMemcpyAsync(E_out, B.E, (size_t)n * MLP_OUT * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  ps_status s = e == cudaSuccess ? mlp_take_error(h, st) : cuda_fail(h, e, "ps_proposal_pair_grad");
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

extern "C" ps_status ps_proposal_train(ps_handle h, const ps_matrix* train, int32_t ntrain, float tau,
                                       int32_t steps, float lr, float target_recall, uint64_t seed,
                                       double* final_loss, ps_stream stream) {
  if (!h) return fail(nullptr, PS_ERR_INVALID_ARG, "null handle");
  if (!train || ntrain <= 0 || steps < 0 || !(lr > 0.f) || !(target_recall > 0.f && target_recall <= 1.f))
    return fail(h, PS_ERR_INVALID_ARG, "ps_proposal_train: bad arguments");
  for (int t = 0; t < ntrain; ++t)
    if (train[t].dtype != PS_F32 || train[t].layout != PS_LAYOUT_FIELD_MAJOR || train[t].nv < 3 ||
        train[t].nf != train[0].nf || train[t].ld % 4 != 0)
      return fail(h, PS_ERR_INVALID_ARG,
                  "ps_proposal_train: FP32 field-major device matrices (ld %% 4 == 0) with one nf");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ps_status s = PS_OK;
  if (!h->mlp.w || h->mlp.d_in != train[0].nf) s = mlp_alloc(h, (int)train[0].nf, seed ^ 0x5eedull);
  DevBuf mem;
  struct Set {
    VF32 v;
    float* r;
    __nv_bfloat16* Xb;   // encoder inputs in BF16 (n x ldx) and field-major (d_in x ldn)
    __nv_bfloat16* XbT;
    int* pairs;
    float* y;
    int64_t np;
    int* pos;
    int64_t npos;
  };
  h->mlp.wait_ns = h->wait_ns;
  std::vector<Set> sets;
  uint64_t rs = seed;
  for (int t = 0; t < ntrain && s == PS_OK; ++t) {
    const ps_matrix& V = train[t];
    const int n = (int)V.nv;
    // exact labels: every triple with c3 >= tau
    const int64_t cap = 1 << 22;
    ps_triple* dh = static_cast<ps_triple*>(mem.get((size_t)cap * sizeof(ps_triple)));
    int64_t* dcount = static_cast<int64_t*>(mem.get(8));
    if (!dh || !dcount) {
      s = fail(h, PS_ERR_OOM, "training buffers");
      break;
    }
    ps_status ts;
    {
      ScopedTimer tm(h, "proposal_labels", st);
      ts = ps_threshold_3way(h, &V, tau, 0, dh, cap, dcount, stream);
    }
    if (ts != PS_OK && ts != PS_ERR_CAPACITY) {
      s = ts;
      break;
    }
    int64_t count = 0;
    cudaMemcpy(&count, dcount, 8, cudaMemcpyDeviceToHost);
    count = std::min(count, cap);
    std::vector<ps_triple> hits((size_t)count);
    cudaMemcpy(hits.data(), dh, (size_t)count * sizeof(ps_triple), cudaMemcpyDeviceToHost);
    std::unordered_set<uint64_t> posset;
    auto key = [](int a, int b) { return ((uint64_t)std::min(a, b) << 32) | (uint64_t)std::max(a, b); };
    for (const ps_triple& x : hits) {
      posset.insert(key(x.i, x.j));
      posset.insert(key(x.i, x.k));
      posset.insert(key(x.j, x.k));
    }
    std::vector<int> pr;
    std::vector<float> yy;
    std::vector<int> pos;
    for (uint64_t kk : posset) {
      pr.push_back((int)(kk >> 32));
      pr.push_back((int)(kk & 0xffffffffu));
      yy.push_back(1.f);
    }
    pos = pr;
    const int64_t nneg = std::max<int64_t>(4 * (int64_t)posset.size(), 4096);
    for (int64_t c = 0; c < nneg;) {
      const int a = (int)(splitmix(rs) % (uint64_t)n), b = (int)(splitmix(rs) % (uint64_t)n);
      if (a == b || posset.count(key(a, b))) continue;
      pr.push_back(std::min(a, b));
      pr.push_back(std::max(a, b));
      yy.push_back(0.f);
      ++c;
    }
    Set S;
    S.v = VF32{static_cast<const float*>(V.data), V.ld, n, (int)V.nf};
    double* sums = static_cast<double*>(mem.get((size_t)n * 8));
    S.r = static_cast<float*>(mem.get((size_t)n * 4));
    if (!sums || !S.r) {
      s = fail(h, PS_ERR_OOM, "training scales");
      break;
    }
    const int64_t ldn = round_up(n, 8), ldx = round_up(V.nf, 8);
    S.Xb = static_cast<__nv_bfloat16*>(mem.get((size_t)n * ldx * 2));
    S.XbT = static_cast<__nv_bfloat16*>(mem.get((size_t)V.nf * ldn * 2));
    if (!S.Xb || !S.XbT) {
      s = fail(h, PS_ERR_OOM, "training inputs");
      break;
    }
    if (launch_vector_sums(V, sums, st) != cudaSuccess || mlp_input_scale(sums, n, (int)V.nf, S.r, st) != cudaSuccess ||
        mlp_prep_x(S.v, S.r, S.Xb, ldx, S.XbT, ldn, st) != cudaSuccess) {
      s = fail(h, PS_ERR_CUDA, "training scales");
      break;
    }
    S.np = (int64_t)yy.size();
    S.npos = (int64_t)posset.size();
    S.pairs = static_cast<int*>(mem.get(pr.size() * 4));
    S.y = static_cast<float*>(mem.get(yy.size() * 4));
    S.pos = S.pairs;  // positives come first
    if (!S.pairs || !S.y) {
      s = fail(h, PS_ERR_OOM, "training pairs");
      break;
    }
    cudaMemcpy(S.pairs, pr.data(), pr.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(S.y, yy.data(), yy.size() * 4, cudaMemcpyHostToDevice);
    sets.push_back(S);
  }
  if (s == PS_OK) {
    int nmax = 0;
    for (const Set& S : sets) nmax = std::max(nmax, S.v.nv);
    const int64_t np_all = mlp_param_count(h->mlp.d_in);
    void* buf = mem.get(mlp_bufs_bytes(nmax, h->mlp.d_in, false));
    float* grad = static_cast<float*>(mem.get((size_t)np_all * 4));
    double* dloss = static_cast<double*>(mem.get(8));
    if (!buf || !grad || !dloss) s = fail(h, PS_ERR_OOM, "training state");
    // activations of set S (its own inputs)
    auto bufs_of = [&](const Set& S) {
      MlpBufs B = mlp_bufs_at(buf, S.v.nv, h->mlp.d_in, false);
      B.Xb = S.Xb;
      B.XbT = S.XbT;
      return B;
    };
    double last = 0.0;
    // One CUDA graph per training matrix holds a whole step (forward,
    // backward, Adam); the steps replay them in turn.  A gradient pass
    // outside the capture first sets the kernels' attributes.
    std::vector<cudaGraphExec_t> gx;
    cudaStream_t cs = nullptr;
    if (s == PS_OK && steps > 0) {
      cudaError_t e = mlp_pair_grad(h->mlp, bufs_of(sets[0]), sets[0].pairs, sets[0].y, sets[0].np, grad, dloss, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      for (size_t k = 0; k < sets.size() && e == cudaSuccess; ++k) {
        const Set& S = sets[k];
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t e1 = mlp_pair_grad(h->mlp, bufs_of(S), S.pairs, S.y, S.np, grad, dloss, cs);
        if (e1 == cudaSuccess) e1 = mlp_adam(h->mlp, grad, lr, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e1;
        cudaGraphExec_t x = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) gx.push_back(x);
      }
      if (e != cudaSuccess) s = cuda_fail(h, e, "training step graphs");
    }
    {
      ScopedTimer tm(h, "proposal_steps", st);  // the Adam steps, as one record
      for (int it = 0; it < steps && s == PS_OK; ++it) {
        cudaError_t e = cudaGraphLaunch(gx[(size_t)it % gx.size()], st);
        if (e != cudaSuccess) s = cuda_fail(h, e, "training step");
        if (it == steps - 1 && s == PS_OK) {
          cudaMemcpyAsync(&last, dloss, 8, cudaMemcpyDeviceToHost, st);
          cudaStreamSynchronize(st);
        }
      }
    }
    cudaStreamSynchronize(st);
    for (cudaGraphExec_t x : gx) cudaGraphExecDestroy(x);
    if (cs) cudaStreamDestroy(cs);
    // theta: the (1 - target_recall) quantile of the positive pair scores
    std::vector<float> zs;
    for (const Set& S : sets) {
      if (s != PS_OK) break;
      const int n = S.v.nv;
      const MlpBufs B = bufs_of(S);
      float* zz = static_cast<float*>(mem.get((size_t)std::max<int64_t>(S.npos, 1) * 4));
      cudaError_t e = mlp_forward_tc(h->mlp, B, false, st);
      if (e == cudaSuccess) e = mlp_softmax(B.E, n, B.Pm, st);
      if (e == cudaSuccess && S.npos > 0) {
        pair_score_kernel<<<256, 256, 0, st>>>(B.Pm, S.pos, S.npos, zz);
        e = cudaGetLastError();
      }
      std::vector<float> hz((size_t)S.npos);
      if (e == cudaSuccess && S.npos > 0) e = cudaMemcpyAsync(hz.data(), zz, (size_t)S.npos * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(h, e, "calibration");
      zs.insert(zs.end(), hz.begin(), hz.end());
    }
    if (s == PS_OK) s = mlp_take_error(h, st);
    if (s == PS_OK) {
      std::sort(zs.begin(), zs.end());
      float theta = -INFINITY;
      if (!zs.empty()) {
        const size_t q = (size_t)std::floor((1.0 - (double)target_recall) * (double)zs.size());
        theta = zs[std::min(q, zs.size() - 1)];
        theta *= 0.999f;
      }
      h->mlp.theta = theta;
      h->mlp.trained = true;
      if (final_loss) *final_loss = last;
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}
