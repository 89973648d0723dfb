// ps_mgemm_t128.cu -- 128 x 128-tile instantiations of the FP32 min-product
// kernels (8 warps, one CTA per SM), plus the thresholded 3-way kernel.
#include "ps_mgemm_impl.cuh"

namespace ps {

template <bool P, int KU>
static MgemmVariant make_t128() {
  using L = mg::Launch<mg::T128, P, KU>;
  return MgemmVariant{&L::attrs, &L::mgemm2, &L::mgemm3, &L::batched, mg::T128::BM, mg::T128::MINB};
}

const MgemmVariant* mgemm_variant_t128(int packed, int ku) {
  static const MgemmVariant v[6] = {make_t128<true, 16>(),  make_t128<true, 8>(),
                                    make_t128<true, 4>(),   make_t128<false, 16>(),
                                    make_t128<false, 8>(),  make_t128<false, 4>()};
  const int k = ku == 16 ? 0 : (ku == 4 ? 2 : 1);
  return &v[(packed ? 0 : 3) + k];
}

template <class C>
static cudaError_t launch_half(int num_sms, int band, const VF32& Vh, const double* S, void* out, int out_f64,
                               const float* inv_scale, cudaStream_t st) {
  static bool attrs_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(mg::Smem<C>);
  if (!attrs_done[dev & 63]) {
    cudaError_t e = cudaFuncSetAttribute(mg::mgemm2_half_kernel<C, 8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attrs_done[dev & 63] = true;
  }
  const int T = (int)ceil_div(Vh.nv, C::BM);
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)num_sms * C::MINB);
  mg::mgemm2_half_kernel<C, 8><<<grid, C::NT, smem, st>>>(Vh, S, out, out_f64, inv_scale, T, std::max(1, band),
                                                         ntiles);
  return cudaGetLastError();
}

cudaError_t launch_mgemm2_half(int num_sms, int band, int warps, const VF32& Vh, const double* S, void* out,
                               int out_f64, const float* inv_scale, cudaStream_t st) {
  // 8 warps unless 16 are asked for: 209.9 vs 213.1 ms at 32768 x 8192
  if (warps == 16) return launch_half<mg::T128W16>(num_sms, band, Vh, S, out, out_f64, inv_scale, st);
  return launch_half<mg::T128>(num_sms, band, Vh, S, out, out_f64, inv_scale, st);
}

cudaError_t launch_thresh_t128(int num_sms, const VF32& V, const double* S, const float* n2sq,
                               const int* blocks, int64_t nblocks, const ThreshArgs& ta,
                               cudaStream_t st) {
  using C = mg::T128;
  static bool attrs_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(mg::Smem<C>);
  if (!attrs_done[dev & 63]) {
    cudaError_t e = cudaFuncSetAttribute(mg::mgemm3_thresh_kernel<C, true, 8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attrs_done[dev & 63] = true;
  }
  const int64_t nitems = nblocks * C::BM;
  if (nitems == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(nitems, (int64_t)num_sms * C::MINB);
  mg::mgemm3_thresh_kernel<C, true, 8><<<grid, C::NT, smem, st>>>(V, S, n2sq, blocks, nitems, ta);
  return cudaGetLastError();
}

cudaError_t launch_mgemm2_thresh(int num_sms, int band, const VF32& V, const double* S,
                                 const ThreshArgs& ta, cudaStream_t st) {
  using C = mg::T128;
  static bool attrs_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(mg::Smem<C>);
  if (!attrs_done[dev & 63]) {
    cudaError_t e = cudaFuncSetAttribute(mg::mgemm2_thresh_kernel<C, true, 8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attrs_done[dev & 63] = true;
  }
  const int T = (int)ceil_div(V.nv, C::BM);
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)num_sms * C::MINB);
  mg::mgemm2_thresh_kernel<C, true, 8><<<grid, C::NT, smem, st>>>(V, S, T, std::max(1, band), ntiles, ta);
  return cudaGetLastError();
}

}  // namespace ps
