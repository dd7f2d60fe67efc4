// hbe_variants.h -- tile variants of the stage kernels, per precision.
#pragma once

namespace hbe {

struct KernelInfo {
  const void *fn;   // __global__ stage_kernel<...>
  int threads;
  int smem;         // dynamic shared memory bytes
  int ring;         // z-planes in the TMA ring
  int tx, ty;       // tile in x and y
  int vec;          // consecutive x points per lane
  int vy;           // rows per consumer warp
  int nw;           // consumer warps
};

constexpr int kMaxVariants = 6;

struct VariantTable {
  int count;
  // [variant][0..3] one RK stage per launch; [4] stages 1+2; [5] stages 3+4 + combine.
  // Every kernel of a variant has the same tile except [4], which may be taller.
  KernelInfo k[kMaxVariants][7];  // [6]: [4] with the Laplacian monitor
};

const VariantTable &variants_fp64();
const VariantTable &variants_fp32();
const VariantTable &variants_bf16();
const VariantTable &variants_fp32_plain();

}  // namespace hbe
