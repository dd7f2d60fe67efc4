// Stage-kernel instantiations for PrecFP32.
#include "hbe_stage.cuh"
#include "hbe_variants.h"

namespace hbe {
namespace {
template <class C>
KernelInfo info() {
  return KernelInfo{reinterpret_cast<const void *>(&stage_kernel<C>), C::THREADS, C::SMEM, C::RING,
                    C::TX, C::TY};
}
template <class PR, int TX, int TY, int B>
void add(VariantTable &t) {
  KernelInfo *k = t.k[t.count++];
  k[0] = info<StageCfg<PR, TX, TY, B, 1>>();
  k[1] = info<StageCfg<PR, TX, TY, B, 2>>();
  k[2] = info<StageCfg<PR, TX, TY, B, 3>>();
  k[3] = info<StageCfg<PR, TX, TY, B, 4>>();
}
}  // namespace

const VariantTable &variants_fp32() {
  static const VariantTable table = [] {
    using PR = PrecFP32;
    VariantTable t{};
    add<PR, 32, 16, 110 * 1024>(t);   // 128 threads, 2 blocks / SM
    add<PR, 32, 8, 55 * 1024>(t);     //  64 threads, 4 blocks / SM
    add<PR, 64, 8, 110 * 1024>(t);    // 128 threads, 2 blocks / SM
    add<PR, 64, 16, 220 * 1024>(t);   // 256 threads, 1 block / SM
    return t;
  }();
  return table;
}

}  // namespace hbe
