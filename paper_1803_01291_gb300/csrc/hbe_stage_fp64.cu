// Stage-kernel instantiations for PrecFP64.
#include "hbe_stage.cuh"
#include "hbe_variants.h"

namespace hbe {
namespace {
template <class C>
KernelInfo info() {
  return KernelInfo{reinterpret_cast<const void *>(&stage_kernel<C>), C::THREADS, C::SMEM, C::RING,
                    C::TX, C::TY, C::VEC, C::VY, C::NW};
}
template <class PR, int V, int VY, int NW, int B, int MB>
void add(VariantTable &t) {
  KernelInfo *k = t.k[t.count++];
  k[0] = info<StageCfg<PR, V, VY, NW, B, MB, 1>>();
  k[1] = info<StageCfg<PR, V, VY, NW, B, MB, 2>>();
  k[2] = info<StageCfg<PR, V, VY, NW, B, MB, 3>>();
  k[3] = info<StageCfg<PR, V, VY, NW, B, MB, 4>>();
  k[4] = info<StageCfg<PR, V, VY, NW, B, MB, 5>>();
  k[5] = info<StageCfg<PR, V, VY, NW, B, MB, 6>>();
  k[6] = info<StageCfg<PR, V, VY, NW, B, MB, 5, true>>();
}
}  // namespace

const VariantTable &variants_fp64() {
  static const VariantTable table = [] {
    using PR = PrecFP64;
    VariantTable t{};
    // <precision, x points per lane, rows per warp, consumer warps, smem budget, min blocks/SM>
    add<PR, 1, 2, 8, 110 * 1024, 1>(t);  // 32 x 16 tile, 9 warps
    add<PR, 2, 1, 8, 110 * 1024, 1>(t);  // 64 x 8 tile, 9 warps
    add<PR, 2, 1, 4, 110 * 1024, 1>(t);  // 64 x 4 tile, 5 warps
    return t;
  }();
  return table;
}

}  // namespace hbe
