// Stage-kernel instantiations for PrecFP32.
#include "hbe_stage.cuh"
#include "hbe_variants.h"

namespace hbe {
namespace {
template <class C>
KernelInfo info() {
  return KernelInfo{reinterpret_cast<const void *>(&stage_kernel<C>), C::THREADS, C::SMEM, C::RING,
                    C::TX, C::TY, C::VEC, C::VY, C::NW};
}
// NW5: consumer warps of the stages 1+2 kernel (its tile is 32 V x NW5 VY)
template <class PR, int V, int VY, int NW, int B, int MB, int NW5 = NW>
void add(VariantTable &t) {
  KernelInfo *k = t.k[t.count++];
  k[0] = info<StageCfg<PR, V, VY, NW, B, MB, 1>>();
  k[1] = info<StageCfg<PR, V, VY, NW, B, MB, 2>>();
  k[2] = info<StageCfg<PR, V, VY, NW, B, MB, 3>>();
  k[3] = info<StageCfg<PR, V, VY, NW, B, MB, 4>>();
  k[4] = info<StageCfg<PR, V, VY, NW5, B, MB, 5>>();
  k[5] = info<StageCfg<PR, V, VY, NW, B, MB, 6>>();
  k[6] = info<StageCfg<PR, V, VY, NW5, B, MB, 5, true>>();
}
}  // namespace

const VariantTable &variants_fp32() {
  static const VariantTable table = [] {
    using PR = PrecFP32;
    VariantTable t{};
    // <precision, x points per lane, rows per warp, consumer warps, smem budget, min blocks/SM>
    add<PR, 4, 1, 11, 226 * 1024, 1>(t);  // 128 x 11 tile, 12 warps, one CTA per SM
    // the same, with stages 1+2 on a 128 x 15 tile, 16 warps at <= 128 registers
    add<PR, 4, 1, 11, 226 * 1024, 1, 15>(t);
    add<PR, 4, 1, 8, 220 * 1024, 1>(t);   // 128 x 8 tile, 9 warps, one CTA per SM
    add<PR, 2, 1, 11, 220 * 1024, 1>(t);  // 64 x 11 tile, 12 warps, one CTA per SM
    add<PR, 2, 1, 4, 110 * 1024, 2>(t);   // 64 x 4 tile, 5 warps, two CTAs per SM
    return t;
  }();
  return table;
}

}  // namespace hbe
