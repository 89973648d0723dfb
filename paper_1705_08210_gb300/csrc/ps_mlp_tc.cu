// ps_mlp_tc.cu -- the encoder's products on the 5th-generation tensor cores.
//
// Not in the paper (the encoder belongs to the learned block proposal).
// C[M x N] = A[M x K] . B[N x K]^T with A and B in BF16, both K-major (row
// i of A and row n of B hold their K values contiguously, pitch a multiple of
// 8 elements), FP32 accumulation in tensor memory, and an epilogue functor
// applied to every (row, column, value) of the tile.
//
// Kernel: one CTA per 128 x TN output tile, 6 warps.
//   warp 0      TMA producer: per K-block of 64 elements (128 bytes) one
//               128 x 128-byte box of A and one TN x 128-byte box of B, with
//               the 128-byte swizzle, into a 4-stage mbarrier ring;
//   warp 1      allocates TN tensor-memory columns and issues, per K-block,
//               four tcgen05.mma.kind::f16 (M = 128, N = TN, K = 16);
//               tcgen05.commit frees the stage, and after the last block
//               signals the accumulator;
//   warps 2..5  epilogue: each warp reads its 32-lane quadrant of the
//               accumulator with tcgen05.ld (thread = output row) and calls
//               the functor.
// Rows past M and columns past N or K are zero-filled by the TMA and never
// passed to the functor.  Every wait is bounded (the handle's wait limit);
// on a timeout the CTA raises `err`, lets issued copies and products finish,
// frees its tensor memory and returns.
#include "ps_internal.cuh"
#include "ps_sync.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace ps {
namespace tc {

constexpr int TM = 128, KB = 64, KBYTES = 128, TSTAGES = 4, NTHREADS = 192;

template <int TN>
struct __align__(1024) SmemG {
  uint8_t A[TSTAGES][TM * KBYTES];
  uint8_t B[TSTAGES][TN * KBYTES];
  unsigned long long full[TSTAGES];
  unsigned long long empty[TSTAGES];
  unsigned long long done;
  uint32_t tmem_base;
  int abort;
};

// UMMA shared-memory descriptor of a K-major operand written by the TMA with
// the 128-byte swizzle: 8-row x 128-byte atoms, 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                      // leading offset (unused for swizzled K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;  // stride offset: the next 8-row atom
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// M = 128, N = TN.
template <int TN>
constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   sy::smem_addr(bar))
               : "memory");
}

// 32 lanes x 32 columns of FP32 from tensor memory: thread t gets row
// (lane base + t), columns c .. c + 31.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
}

template <int TN, class Epi>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                     int N, int K, Epi epi, int* err, unsigned long long wait_ns) {
  extern __shared__ unsigned char smem_raw[];
  SmemG<TN>& sm = *reinterpret_cast<SmemG<TN>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int nkb = (K + KB - 1) / KB;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      sy::bar_init(&sm.full[s], 1);
      sy::bar_init(&sm.empty[s], 1);
    }
    sy::bar_init(&sm.done, 1);
    sm.abort = 0;
    sy::bar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sy::smem_addr(&sm.tmem_base)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer ----
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TSTAGES;
        const uint32_t ph = (kb / TSTAGES) & 1u;
        if (!sy::bar_wait(&sm.empty[s], ph ^ 1u, &sm.abort, err, wait_ns)) break;
        sy::bar_arrive_tx(&sm.full[s], (uint32_t)(TM + TN) * KBYTES);
        sy::tma_load_2d(sm.A[s], &mapA, kb * KBYTES, m0, &sm.full[s]);
        sy::tma_load_2d(sm.B[s], &mapB, kb * KBYTES, n0, &sm.full[s]);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer ----
      constexpr uint32_t IDESC = idesc_bf16<TN>();
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TSTAGES;
        const uint32_t ph = (kb / TSTAGES) & 1u;
        if (!sy::bar_wait(&sm.full[s], ph, &sm.abort, err, wait_ns)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = sy::smem_addr(sm.A[s]), b0 = sy::smem_addr(sm.B[s]);
#pragma unroll
        for (int kk = 0; kk < KBYTES / 32; ++kk)  // K = 16 BF16 = 32 bytes per product
          umma_bf16(tmem, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), IDESC, (kb | kk) ? 1u : 0u);
        umma_commit(&sm.empty[s]);
      }
      if (ok) umma_commit(&sm.done);
    }
    __syncwarp();
  } else {  // ---- epilogue: warps 2..5 ----
    const int quad = warp & 3;  // the tensor-memory lane quadrant this warp may read
    int ok = 0;
    if (lane == 0) ok = sy::bar_wait(&sm.done, 0, &sm.abort, err, wait_ns) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + quad * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + (uint32_t)c0 + ((uint32_t)(quad * 32) << 16), v);
        if (row < M) {
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (n0 + c0 + c < N) epi(row, n0 + c0 + c, v[c]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // let copies and products already issued finish before the memory goes away
  if (*(volatile int*)&sm.abort) sy::drain_after_abort();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TN)
                 : "memory");
}

template <int TN, class Epi>
cudaError_t gemm_bf16(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N, int K,
                      Epi epi, int* err, unsigned long long wait_ns, int device, cudaStream_t st) {
  static std::mutex mu;
  static uint64_t attr_done = 0;
  const size_t smem = sizeof(SmemG<TN>) + 1024;
  {
    std::lock_guard<std::mutex> lk(mu);
    const uint64_t bit = 1ull << (device & 63);
    if (!(attr_done & bit)) {
      const cudaError_t e =
          cudaFuncSetAttribute(gemm_bf16_kernel<TN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_done |= bit;
    }
  }
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // K-major BF16 operands seen as byte matrices (rows of pitch 2 ld bytes,
  // 2 K valid bytes), boxes of 128 bytes x (128 or TN) rows, 128-byte swizzle
  if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || lda % 8 || ldb % 8) return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!sy::make_map_u8_sw128(&mA, A, 2 * (int64_t)K, M, 2 * lda, KBYTES, TM) ||
      !sy::make_map_u8_sw128(&mB, B, 2 * (int64_t)K, N, 2 * ldb, KBYTES, TN))
    return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ceil_div(N, TN), (unsigned)ceil_div(M, TM));
  gemm_bf16_kernel<TN, Epi><<<grid, NTHREADS, smem, st>>>(mA, mB, M, N, K, epi, err, wait_ns);
  return cudaGetLastError();
}

}  // namespace tc

namespace {

using bf16 = __nv_bfloat16;

// ---- epilogues of the five products ----
struct EpiHidden {  // Hpre = acc + b1, H = relu(Hpre) in BF16 (and transposed)
  const float* b1;
  float* Hpre;
  bf16* Hb;
  bf16* HbT;  // may be null
  int64_t ldn;
  __device__ void operator()(int i, int h, float acc) const {
    const float v = acc + b1[h];
    Hpre[(int64_t)i * MLP_HIDDEN + h] = v;
    const bf16 hb = __float2bfloat16_rn(v > 0.f ? v : 0.f);
    Hb[(int64_t)i * MLP_HIDDEN + h] = hb;
    if (HbT) HbT[(int64_t)h * ldn + i] = hb;
  }
};
struct EpiOut {  // E = acc + b2
  const float* b2;
  float* E;
  __device__ void operator()(int i, int o, float acc) const { E[(int64_t)i * MLP_OUT + o] = acc + b2[o]; }
};
struct EpiStoreT {  // G[col][row] = acc
  float* G;
  int64_t ld;
  __device__ void operator()(int r, int c, float acc) const { G[(int64_t)c * ld + r] = acc; }
};
struct EpiStore {  // G[row][col] = acc
  float* G;
  int64_t ld;
  __device__ void operator()(int r, int c, float acc) const { G[(int64_t)r * ld + c] = acc; }
};
struct EpiReluGrad {  // dH = acc [Hpre > 0] (FP32, and transposed in BF16)
  const float* Hpre;
  float* dH;
  bf16* dHbT;
  int64_t ldn;
  __device__ void operator()(int i, int h, float acc) const {
    const int64_t o = (int64_t)i * MLP_HIDDEN + h;
    const float d = Hpre[o] > 0.f ? acc : 0.f;
    dH[o] = d;
    dHbT[(int64_t)h * ldn + i] = __float2bfloat16_rn(d);
  }
};

// Encoder input x_iq = log1p(v_iq r_i) in BF16, vector-major (Xb, n x ldx)
// and, when XbT is not null, field-major (XbT, d_in x ldn); 32 x 32 tiles
// through shared memory.
__global__ void __launch_bounds__(256) prep_x_kernel(VF32 V, const float* __restrict__ r, bf16* __restrict__ Xb,
                                                     int64_t ldx, bf16* __restrict__ XbT, int64_t ldn) {
  __shared__ bf16 tile[32][34];
  const int i0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int q = q0 + k, i = i0 + tx;
    bf16 x = __float2bfloat16_rn(0.f);
    if (q < V.nf && i < V.nv) x = __float2bfloat16_rn(log1pf(__ldg(V.p + (int64_t)q * V.ld + i) * r[i]));
    tile[k][tx] = x;
    if (XbT && q < V.nf && i < V.nv) XbT[(int64_t)q * ldn + i] = x;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int i = i0 + k, q = q0 + tx;
    if (i < V.nv && q < V.nf) Xb[(int64_t)i * ldx + q] = tile[tx][k];
  }
}

}  // namespace

// The three forward / backward activations' BF16 operands and FP32 values of
// n vectors, carved from one buffer of mlp_bufs_bytes(n, d_in) bytes.
size_t mlp_bufs_bytes(int n, int d_in, bool with_x) {
  const int64_t ldn = round_up(n, 8), ldx = round_up(d_in, 8);
  size_t b = 0;
  auto add = [&b](int64_t bytes) { b += (size_t)round_up(bytes, 256); };
  add((int64_t)n * MLP_HIDDEN * 4);  // Hpre
  add((int64_t)n * MLP_OUT * 4);     // E
  add((int64_t)n * MLP_OUT * 4);     // Pm
  add((int64_t)n * MLP_OUT * 4);     // dE
  add((int64_t)n * MLP_HIDDEN * 4);  // dH
  add((int64_t)n * 4);               // r
  add((int64_t)n * MLP_HIDDEN * 2);  // Hb
  add((int64_t)MLP_HIDDEN * ldn * 2);  // HbT
  add((int64_t)n * MLP_OUT * 2);     // dEb
  add((int64_t)MLP_OUT * ldn * 2);   // dEbT
  add((int64_t)MLP_HIDDEN * ldn * 2);  // dHbT
  if (with_x) {
    add((int64_t)n * ldx * 2);       // Xb
    add((int64_t)d_in * ldn * 2);    // XbT
  }
  return b + 256;
}

MlpBufs mlp_bufs_at(void* base, int n, int d_in, bool with_x) {
  const int64_t ldn = round_up(n, 8), ldx = round_up(d_in, 8);
  char* p = reinterpret_cast<char*>(round_up((int64_t)reinterpret_cast<uintptr_t>(base), 256));
  auto take = [&p](int64_t bytes) {
    char* q = p;
    p += round_up(bytes, 256);
    return q;
  };
  MlpBufs B;
  B.n = n;
  B.ldn = ldn;
  B.ldx = ldx;
  B.Hpre = reinterpret_cast<float*>(take((int64_t)n * MLP_HIDDEN * 4));
  B.E = reinterpret_cast<float*>(take((int64_t)n * MLP_OUT * 4));
  B.Pm = reinterpret_cast<float*>(take((int64_t)n * MLP_OUT * 4));
  B.dE = reinterpret_cast<float*>(take((int64_t)n * MLP_OUT * 4));
  B.dH = reinterpret_cast<float*>(take((int64_t)n * MLP_HIDDEN * 4));
  B.r = reinterpret_cast<float*>(take((int64_t)n * 4));
  B.Hb = reinterpret_cast<bf16*>(take((int64_t)n * MLP_HIDDEN * 2));
  B.HbT = reinterpret_cast<bf16*>(take((int64_t)MLP_HIDDEN * ldn * 2));
  B.dEb = reinterpret_cast<bf16*>(take((int64_t)n * MLP_OUT * 2));
  B.dEbT = reinterpret_cast<bf16*>(take((int64_t)MLP_OUT * ldn * 2));
  B.dHbT = reinterpret_cast<bf16*>(take((int64_t)MLP_HIDDEN * ldn * 2));
  if (with_x) {
    B.Xb = reinterpret_cast<bf16*>(take((int64_t)n * ldx * 2));
    B.XbT = reinterpret_cast<bf16*>(take((int64_t)d_in * ldn * 2));
  }
  return B;
}

cudaError_t mlp_prep_x(const VF32& V, const float* r, bf16* Xb, int64_t ldx, bf16* XbT, int64_t ldn,
                       cudaStream_t st) {
  if (V.nv <= 0 || V.nf <= 0) return cudaSuccess;
  if (ceil_div(V.nf, 32) > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)ceil_div(V.nv, 32), (unsigned)ceil_div(V.nf, 32));
  prep_x_kernel<<<grid, 256, 0, st>>>(V, r, Xb, ldx, XbT, ldn);
  return cudaGetLastError();
}

// Hpre, Hb (and HbT when with_t) and E of the n vectors whose inputs are in
// B.Xb: the first two products on the tensor cores.
cudaError_t mlp_forward_tc(const MlpState& M, const MlpBufs& B, bool with_t, cudaStream_t st) {
  const float* b1 = M.w + (int64_t)MLP_HIDDEN * M.d_in;
  const float* b2 = b1 + MLP_HIDDEN + (int64_t)MLP_OUT * MLP_HIDDEN;
  cudaError_t e = tc::gemm_bf16<128>(B.Xb, B.ldx, M.w1b, round_up(M.d_in, 8), B.n, MLP_HIDDEN, M.d_in,
                                     EpiHidden{b1, B.Hpre, B.Hb, with_t ? B.HbT : nullptr, B.ldn}, M.err,
                                     M.wait_ns, M.device, st);
  if (e != cudaSuccess) return e;
  return tc::gemm_bf16<64>(B.Hb, MLP_HIDDEN, M.w2b, MLP_HIDDEN, B.n, MLP_OUT, MLP_HIDDEN, EpiOut{b2, B.E},
                           M.err, M.wait_ns, M.device, st);
}

// The three weight-side products of the backward pass: dW2^T = H^T dE (stored
// transposed into dW2), dH = (dE W2) [Hpre > 0] and dW1 = dH^T X.
cudaError_t mlp_backward_tc(const MlpState& M, const MlpBufs& B, float* gW1, float* gW2, cudaStream_t st) {
  cudaError_t e = tc::gemm_bf16<64>(B.HbT, B.ldn, B.dEbT, B.ldn, MLP_HIDDEN, MLP_OUT, B.n, EpiStoreT{gW2, MLP_HIDDEN},
                                    M.err, M.wait_ns, M.device, st);
  if (e != cudaSuccess) return e;
  e = tc::gemm_bf16<128>(B.dEb, MLP_OUT, M.w2bt, MLP_OUT, B.n, MLP_HIDDEN, MLP_OUT,
                         EpiReluGrad{B.Hpre, B.dH, B.dHbT, B.ldn}, M.err, M.wait_ns, M.device, st);
  if (e != cudaSuccess) return e;
  return tc::gemm_bf16<128>(B.dHbT, B.ldn, B.XbT, B.ldn, MLP_HIDDEN, M.d_in, B.n, EpiStore{gW1, M.d_in}, M.err,
                            M.wait_ns, M.device, st);
}

}  // namespace ps
