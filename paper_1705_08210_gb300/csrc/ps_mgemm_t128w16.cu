// ps_mgemm_t128w16.cu -- 128 x 128-tile instantiations run by 16 warps
// (8 x 4 outputs per lane, <= 128 registers): twice the warps per scheduler
// of the 8-warp tile, to hide the min -> add dependency latency.
#include "ps_mgemm_impl.cuh"

namespace ps {

template <int KU>
static MgemmVariant make_t128w16() {
  using L = mg::Launch<mg::T128W16, true, KU>;
  return MgemmVariant{&L::attrs, &L::mgemm2, &L::mgemm3, &L::batched, mg::T128W16::BM,
                      mg::T128W16::MINB};
}

const MgemmVariant* mgemm_variant_t128w16(int ku) {
  static const MgemmVariant v[3] = {make_t128w16<16>(), make_t128w16<8>(), make_t128w16<4>()};
  return &v[ku == 16 ? 0 : (ku == 4 ? 2 : 1)];
}

}  // namespace ps
