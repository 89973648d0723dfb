// ps_mgemm_t64.cu -- 64 x 64-tile instantiations of the FP32 min-product
// kernels (2 warps per CTA, four CTAs per SM): a quarter of the tile area,
// so less work is wasted in the ragged edge tiles of small problems and of
// the per-pivot 3-way rectangles.
#include "ps_mgemm_impl.cuh"

namespace ps {

template <int KU>
static MgemmVariant make_t64() {
  using L = mg::Launch<mg::T64, true, KU>;
  return MgemmVariant{&L::attrs, &L::mgemm2, &L::mgemm3, &L::batched, mg::T64::BM, mg::T64::MINB};
}

const MgemmVariant* mgemm_variant_t64(int ku) {
  static const MgemmVariant v[3] = {make_t64<16>(), make_t64<8>(), make_t64<4>()};
  return &v[ku == 16 ? 0 : (ku == 4 ? 2 : 1)];
}

}  // namespace ps
