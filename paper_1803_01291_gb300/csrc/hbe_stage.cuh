// hbe_stage.cuh -- the fused RK4 stage kernels (the hot path).
//
// Method (Sec. 2.1 of arXiv:1803.01291): v = (p, q) = (phi, phi_t), f(t, v) =
// (q, G(t, p, q)) with (Eq. rhs)
//     G(t, P, Q) = -3 Q + e^{-2t} h^{-2} Lambda(P) + mu^2 P - lambda P^3,
//     Lambda(P)  = sum over x, y, z of (-1/12 P[-2] + 4/3 P[-1] - 5/2 P[0] + 4/3 P[+1] - 1/12 P[+2]),
// advanced by the classic RK4 step.  Because the p-component of f is q itself,
// the four stages need only the q-components G_s of k_s, and the stage
// arguments are recomputed from (p, q, G) instead of being stored:
//     stage 1: G1 = G(t,        p,                          q)
//     stage 2: G2 = G(t + dt/2, p + dt/2 q,                 q + dt/2 G1)
//     stage 3: G3 = G(t + dt/2, p + dt/2 q + dt^2/4 G1,     q + dt/2 G2)
//     stage 4: G4 = G(t + dt,   p + dt q + dt^2/2 G2,       q + dt G3)
//     p' = p + dt q + dt^2/6 (G1 + G2 + G3),   q' = q + dt/6 (G1 + 2 G2 + 2 G3 + G4)
// which is RK4 exactly (k_{p,s} is the q-argument of stage s, and
// q + 2(q + dt/2 G1) + 2(q + dt/2 G2) + (q + dt G3) = 6q + dt (G1 + G2 + G3)).
// Stage 4 writes the new state to the other buffer set (ping-pong), so no
// field a stage reads with a halo is written by that stage.
//
// Kernel shape (one launch per stage or per fused pair of stages -- stages
// 1+2 and stages 3+4 with the combine, which share the p, q tiles -- with
// persistent blocks over a work list):
//   * a block owns a TX x TY tile in x-y (TX = 32 VEC: one warp spans the row,
//     each lane VEC consecutive x points) and marches along z over a chunk;
//   * one producer warp streams every z-plane of every input field into a
//     shared-memory ring with the TMA unit (cp.async.bulk.tensor, completion
//     on a "full" mbarrier per slot); fields that enter the stencil come with a
//     2-row / 16-byte halo, zero filled by the TMA unit outside the box in z;
//   * NW consumer warps each own VY rows of the tile.  A consumer forms the
//     stage argument P of its own points once per plane into a 5-deep register
//     window (z-2..z+2); x neighbours come from the neighbouring lanes by warp
//     shuffles, y neighbours from the warp's own rows in registers or, for the
//     two rows above and below its strip, from the ring; z neighbours from the
//     window.  When a warp is done with a slot it arrives on the slot's
//     "empty" mbarrier; the producer refills a slot once all consumers have
//     released it.  There is no block-wide synchronisation in the plane loop.
//   * results are stored as interior points only; the periodic ghost copies
//     are made by a separate launch after the stage (hbe_aux.cu).
#pragma once
#include <cuda_bf16.h>
#include <type_traits>


#include "hbe_common.cuh"

namespace hbe {

// ---------------------------------------------------------------- precisions
struct PrecFP64 {
  using TS = double; using TG = double; using TM = double;
  static constexpr bool KAHAN = false;
  static constexpr bool DIFF = false;   // merged-centre stencil (fewest FP64 ops)
  // plane loop unrolled 5 times over a rotating register window (no register
  // moves) where that measured faster than shifting the window: the FP32-math
  // paths (FP64 spills with it)
  static constexpr bool ROTATE = false;
};
struct PrecFP32 {
  using TS = float; using TG = float; using TM = float;
  static constexpr bool KAHAN = true;
  static constexpr bool DIFF = true;    // neighbour-minus-centre stencil (less cancellation)
  static constexpr bool ROTATE = true;
};
struct PrecBF16 {
  using TS = float; using TG = __nv_bfloat16; using TM = float;
  static constexpr bool KAHAN = true;
  static constexpr bool DIFF = true;
  static constexpr bool ROTATE = true;
};
struct PrecFP32Plain {
  using TS = float; using TG = float; using TM = float;
  static constexpr bool KAHAN = false;
  static constexpr bool DIFF = true;
  static constexpr bool ROTATE = true;
};

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <class PR, int VEC_, int VY_, int NW_, int BUDGET_, int MINB_, int S_, bool MON_ = false>
struct StageCfg {
  using TS = typename PR::TS;
  using TG = typename PR::TG;
  using TM = typename PR::TM;
  static constexpr bool KAHAN = PR::KAHAN;
  static constexpr bool DIFF = PR::DIFF;
  static constexpr int S = S_;
  static constexpr int VEC = VEC_;                 // consecutive x points per lane
  static constexpr int VY = VY_;                   // rows per consumer warp
  static constexpr int NW = NW_;                   // consumer warps
  static constexpr int TX = 32 * VEC, TY = NW * VY;
  static constexpr int THREADS = 32 * (NW + 1);    // + one producer warp
  static constexpr int HXS = 16 / (int)sizeof(TS);
  static constexpr int HXG = 16 / (int)sizeof(TG);
  static constexpr int BY = TY + 4;
  static constexpr int BXS = TX + 2 * HXS, BXG = TX + 2 * HXG;
  // S = 1..4: one RK stage per launch; S = 5: stages 1 and 2 in one launch;
  // S = 6: stages 3 and 4 (with the RK4 combine) in one launch.
  static constexpr bool PAIR = S >= 5;
  // ring slot composition: halo tiles of the fields that enter a stencil, then
  // interior tiles of the fields read at the point only
  static constexpr int NHS = (S == 1) ? 1 : 2;                                  // p [, q]
  static constexpr int NHG = (S == 3 || S == 4) ? 1 : (S == 6 ? 2 : 0);         // G1 | G2 | G1, G2
  static constexpr int NIG = (S == 1 || S >= 5) ? 0 : ((S == 4) ? 2 : 1);       // G1 | G2 | G1, G3
  static constexpr int HS_RAW = BY * BXS * (int)sizeof(TS);
  static constexpr int HG_RAW = BY * BXG * (int)sizeof(TG);
  static constexpr int IS_RAW = TY * TX * (int)sizeof(TS);
  static constexpr int IG_RAW = TY * TX * (int)sizeof(TG);
  static constexpr int HS_BYTES = align128(HS_RAW), HG_BYTES = align128(HG_RAW);
  static constexpr int IS_BYTES = align128(IS_RAW), IG_BYTES = align128(IG_RAW);
  static constexpr int HEADER = 384;  // 2 x 16 mbarriers, flags, 2 x 4 mbarriers
  static constexpr int ring_of(int budget, int slot) { return cmax(4, cmin(16, budget / slot)); }
  // Stages 3+4 read the compensation terms at the output point only.  A slot
  // is held for three plane steps (its tiles feed the stencils of planes m,
  // m+1 and m+2), so where a ring with those tiles inside would hold at most 5
  // slots (two planes in flight), they get a ring of their own of 3 slots, each
  // held for one step: the main ring then holds one plane more.  Deeper rings
  // keep them inside, where their lead is that of the main ring.
  static constexpr int MAIN_BYTES = NHS * HS_BYTES + NHG * HG_BYTES + NIG * IG_BYTES;
  static constexpr bool LO_TERMS = (S == 4 || S == 6) && KAHAN;
  static constexpr int RING_IN = ring_of(BUDGET_ - HEADER, MAIN_BYTES + (LO_TERMS ? 2 * IS_BYTES : 0));
  static constexpr int RING_SPLIT = ring_of(BUDGET_ - HEADER - 3 * 2 * IS_BYTES, MAIN_BYTES);
  static constexpr bool LOR = S == 6 && KAHAN && RING_IN <= 5 && RING_SPLIT > RING_IN;
  static constexpr int NIS = (S == 1) ? 1 : ((LO_TERMS && !LOR) ? 2 : 0);
  static constexpr int OFF_HG = NHS * HS_BYTES;
  static constexpr int OFF_IS = OFF_HG + NHG * HG_BYTES;
  static constexpr int OFF_IG = OFF_IS + NIS * IS_BYTES;
  static constexpr int SLOT_BYTES = OFF_IG + NIG * IG_BYTES;
  static constexpr uint32_t TX_BYTES =
      (uint32_t)(NHS * HS_RAW + NHG * HG_RAW + NIS * IS_RAW + NIG * IG_RAW);
  static constexpr int LO_BAR = 36;  // compensation full barriers at header byte 288, empty at 320
  static constexpr int LO_SLOT = LOR ? 2 * IS_BYTES : 0;
  static constexpr uint32_t LO_TX = LOR ? (uint32_t)(2 * IS_RAW) : 0u;
  static constexpr int RING_LO = LOR ? 3 : 0;  // compensation slots (lead of two planes)
  static constexpr int RING = LOR ? RING_SPLIT : RING_IN;
  static constexpr int OFF_LO = HEADER + RING * SLOT_BYTES;  // compensation ring
  static constexpr int SMEM = OFF_LO + RING_LO * LO_SLOT;
  static_assert(SLOT_BYTES == MAIN_BYTES + NIS * IS_BYTES, "slot composition");
  static_assert(SMEM <= 227 * 1024, "ring of 4 slots does not fit in 227 KB of shared memory");
  static_assert(RING_LO <= 4 && 8 * (LO_BAR + 4 + RING_LO) <= HEADER, "barrier area");
  static constexpr int MINB = MINB_;  // blocks per SM the registers must allow
  static constexpr bool ROTATE = PR::ROTATE;
  // packed FP32 arithmetic for pairs of x points (FP32 math, even VEC, difference form)
  static constexpr bool PACKED = sizeof(TM) == 4 && VEC % 2 == 0 && DIFF;
  // one row per warp with packed arithmetic: the 13-point sums are formed part
  // by part (z pairs, rows +-1, rows +-2, x pairs), so fewer neighbour values
  // are live at once
  static constexpr bool INCR = PACKED && VY_ == 1 && PAIR;
  // fused pairs: the x neighbours of both stage arguments are formed from the
  // ring's halo columns by every lane instead of exchanged by warp shuffles
  static constexpr bool XLDS = PACKED && PAIR;
  // fused pairs: stage arguments formed by packed FMAs.  In the stages 3+4
  // kernel each of these three alone spills on the 128 x 11 tile; together
  // they fit (158 registers FP32, 156 BF16)
  static constexpr bool PCOMB = PACKED && PAIR;
  // stages 1+2 with the Laplacian monitor of Sec. 3: max over the grid of
  // |Delta_h phi| of the step's starting state (stage 1's argument is phi)
  static constexpr bool MON = MON_ && S_ == 5;
  static_assert(!MON_ || S_ == 5, "the monitor rides on the stages 1+2 kernel");
  static_assert(!MON || INCR || !PACKED, "monitor: packed kernels form the sums part by part");
  static_assert(VEC == 1 || VEC == 2 || VEC == 4, "1, 2 or 4 x points per lane");
  static_assert(VEC * (int)sizeof(TM) <= 16, "lane vector of <= 16 bytes");
  static_assert(HXS >= 2 && HXG >= 2 && HXS % VEC == 0 && HXG % VEC == 0, "halo alignment");
  static_assert(BXG <= 256 && BXS <= 256 && BY <= 256, "TMA box limit");
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for a barrier phase for at most ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0u && global_ns() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

// ---------------------------------------------------------------- vectors
// Aligned loads/stores of n = 1, 2 or 4 consecutive elements as one access.
template <class T, int n> struct Raw;
template <> struct Raw<float, 1> { using type = float; };
template <> struct Raw<float, 2> { using type = float2; };
template <> struct Raw<float, 4> { using type = float4; };
template <> struct Raw<double, 1> { using type = double; };
template <> struct Raw<double, 2> { using type = double2; };
template <> struct Raw<__nv_bfloat16, 1> { using type = unsigned short; };
template <> struct Raw<__nv_bfloat16, 2> { using type = unsigned int; };
template <> struct Raw<__nv_bfloat16, 4> { using type = uint2; };

template <class T, class TM, int n>
__device__ __forceinline__ void load_as(const T *p, TM (&v)[n]) {
  using R = typename Raw<T, n>::type;
  const R raw = *reinterpret_cast<const R *>(p);
  const T *e = reinterpret_cast<const T *>(&raw);
#pragma unroll
  for (int j = 0; j < n; ++j) {
    if constexpr (sizeof(T) == sizeof(TM)) v[j] = e[j];
    else v[j] = __bfloat162float(e[j]);  // exact widening
  }
}
template <class T, class TM>
__device__ __forceinline__ T narrow(TM v) {
  if constexpr (sizeof(T) == sizeof(TM)) return v;
  else return __float2bfloat16_rn(v);  // round to nearest even
}
template <class T, class TM, int n>
__device__ __forceinline__ void store_as(T *p, const TM (&v)[n]) {
  using R = typename Raw<T, n>::type;
  R raw;
  T *e = reinterpret_cast<T *>(&raw);
#pragma unroll
  for (int j = 0; j < n; ++j) e[j] = narrow<T>(v[j]);
  *reinterpret_cast<R *>(p) = raw;
}

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

// Error-free sum s + e = a + b (Knuth's TwoSum).
template <class T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
  s = a + b;
  const T bb = s - a;
  const T aa = s - bb;
  e = (a - aa) + (b - bb);
}

// Store VEC values of a field at interior point x of a row of the padded
// layout (`row` points at the row's x = 0) in a tile that crosses x = N: the
// points at x >= N are skipped.  (Periodic ghost copies are written by a
// separate launch after the stage, so the stage kernels store interior points
// only.)
template <class T, class TM, int VEC>
__device__ __forceinline__ void store_ragged(T *row, int N, int x, const TM (&v)[VEC]) {
  if (x + VEC <= N) {
    store_as<T, TM, VEC>(row + x, v);
  } else {
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      if (x + j < N) row[x + j] = narrow<T>(v[j]);
  }
}

// ---------------------------------------------------------------- the kernel
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Whether a work item's context takes this step (the same answer in every
// warp: n_base/n_end are fixed during a launch, and the stop rule of stage 1
// reads the previous step's maximum, written by an earlier launch).
template <int S>
__device__ __forceinline__ bool item_active(Desc *d, int k, bool leader) {
  const long long n = d->n_base + k;
  if (n >= d->n_end || __ldcg(&d->stop_k) <= k) return false;
  if ((S == 1 || S == 5) && k > 0) {
    const double m = __longlong_as_double((long long)__ldcg(d->maxabs + k - 1));
    if (!(m <= 1.7976931348623157e308) || (d->stop_thr > 0.0 && m > d->stop_thr)) {
      if (leader) atomicMin(&d->stop_k, (long long)k);
      return false;
    }
  }
  return true;
}

template <class TM>
__device__ __forceinline__ TM shfl_idx(TM v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <class TM>
__device__ __forceinline__ TM shfl_up1(TM v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <class TM>
__device__ __forceinline__ TM shfl_dn1(TM v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

// ---------------------------------------------------------------- producer warp
template <class C>
__device__ __forceinline__ void produce(const StageParams &prm, uint64_t *full, uint64_t *empty,
                                        unsigned char *ring, volatile int *abort_flag) {
  constexpr int S = C::S, RING = C::RING, TX = C::TX, TY = C::TY;
  const int nitems = *prm.nitems;
  int slot = 0;
  uint32_t fill = 0;  // fill count of `slot` (phase = fill & 1)
  uint32_t issued_slots = 0;
  // compensation ring (stages 3+4): slot, fill count, slots ever filled
  uint64_t *lo_full = full + C::LO_BAR, *lo_empty = full + C::LO_BAR + 4;
  unsigned char *lo_ring = ring - C::HEADER + C::OFF_LO;
  int lslot = 0;
  uint32_t lfill = 0, lo_issued = 0;
  bool bad = false;
  for (int it = blockIdx.x; it < nitems && !bad; it += gridDim.x) {
    const WorkItem w = prm.items[it];
    Desc *d = prm.descs + w.x;
    if (!item_active<S>(d, prm.k, false)) continue;
    const CUtensorMap *tm = d->tmaps;
    for (int t = 0; t < NUM_TMAPS; ++t) tmap_acquire(tm + t);
    const int nz = d->nz, zoff = d->zoff;
    const bool zwrap = d->zwrap != 0;
    const int set = (int)((d->n_base + prm.k) & 1);
    const CUtensorMap *mp = tm + (S == 5 ? (set ? TM_P_H1_P : TM_P_H0_P) : (set ? TM_P_H1 : TM_P_H0));
    const CUtensorMap *mq = tm + (S == 5 ? (set ? TM_Q_H1_P : TM_Q_H0_P) : (set ? TM_Q_H1 : TM_Q_H0));
    const CUtensorMap *mg = tm + (S == 3 ? TM_G1_H : TM_G2_H);
    const CUtensorMap *mi0 = tm + (S == 1 ? (set ? TM_Q_I1 : TM_Q_I0)
                                          : (S == 2 ? TM_G1_I : (S == 3 ? TM_G2_I : TM_G1_I)));
    const CUtensorMap *mi1 = tm + TM_G3_I;
    const CUtensorMap *mlp = tm + (set ? TM_PLO_I1 : TM_PLO_I0);
    const CUtensorMap *mlq = tm + (set ? TM_QLO_I1 : TM_QLO_I0);
    const int x0 = (w.y & 0xffff) * TX, y0 = (w.y >> 16) * TY;
    const int z0 = w.z, nplanes = w.w + 4;
    for (int m = 0; m < nplanes; ++m) {
      if (fill >= 1 && !mbar_wait_bounded(&empty[slot], (fill - 1) & 1u)) { bad = true; break; }
      if (*abort_flag) { bad = true; break; }
      if constexpr (S == 5) {
        if (d->withhold && blockIdx.x == 0 && it == 0 && m == 0) {  // test hook (Desc::withhold)
          if (++slot == RING) { slot = 0; ++fill; }
          continue;
        }
      }
      unsigned char *base = ring + slot * C::SLOT_BYTES;
      uint64_t *bar = &full[slot];
      int z = z0 - 2 + m;
      if (zwrap) z = (z % nz + nz) % nz;
      z += zoff;
      mbar_expect_tx(bar, C::TX_BYTES);
      tma_load_3d(base, mp, bar, x0, y0, z);
      if constexpr (C::NHS == 2) tma_load_3d(base + C::HS_BYTES, mq, bar, x0, y0, z);
      if constexpr (C::NHG == 1 && !C::PAIR) tma_load_3d(base + C::OFF_HG, mg, bar, x0, y0, z);
      constexpr int HXS = C::HXS, HXG = C::HXG;
      if constexpr (S == 6) {
        tma_load_3d(base + C::OFF_HG, tm + TM_G1_H, bar, x0, y0, z);
        tma_load_3d(base + C::OFF_HG + C::HG_BYTES, tm + TM_G2_H, bar, x0, y0, z);
        if constexpr (C::KAHAN && !C::LOR) {
          tma_load_3d(base + C::OFF_IS, mlp, bar, x0 + HXS, y0 + 2, z);
          tma_load_3d(base + C::OFF_IS + C::IS_BYTES, mlq, bar, x0 + HXS, y0 + 2, z);
        }
      }
      if constexpr (S == 1) tma_load_3d(base + C::OFF_IS, mi0, bar, x0 + HXS, y0 + 2, z);
      if constexpr (S >= 2 && S <= 4) tma_load_3d(base + C::OFF_IG, mi0, bar, x0 + HXG, y0 + 2, z);
      if constexpr (S == 4) {
        tma_load_3d(base + C::OFF_IG + C::IG_BYTES, mi1, bar, x0 + HXG, y0 + 2, z);
        if constexpr (C::KAHAN) {
          tma_load_3d(base + C::OFF_IS, mlp, bar, x0 + HXS, y0 + 2, z);
          tma_load_3d(base + C::OFF_IS + C::IS_BYTES, mlq, bar, x0 + HXS, y0 + 2, z);
        }
      }
      issued_slots |= 1u << slot;
      if (++slot == RING) { slot = 0; ++fill; }
      if constexpr (C::LOR) {
        // the compensation terms of output plane m - 2 (needed at step m);
        // the slot's previous tile was consumed at step m - 3
        if (m >= 4) {
          if (lfill >= 1 && !mbar_wait_bounded(&lo_empty[lslot], (lfill - 1) & 1u)) { bad = true; break; }
          int zl = z0 - 4 + m;
          if (zwrap) zl = (zl % nz + nz) % nz;
          zl += zoff;
          unsigned char *lb = lo_ring + lslot * C::LO_SLOT;
          uint64_t *lbar = &lo_full[lslot];
          mbar_expect_tx(lbar, C::LO_TX);
          tma_load_3d(lb, mlp, lbar, x0 + HXS, y0 + 2, zl);
          tma_load_3d(lb + C::IS_BYTES, mlq, lbar, x0 + HXS, y0 + 2, zl);
          lo_issued |= 1u << lslot;
          if (++lslot == C::RING_LO) { lslot = 0; ++lfill; }
        }
      }
    }
  }
  if (bad) {
    *abort_flag = 1;
    atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
  }
  // every copy issued must land before the block's shared memory goes away:
  // the last fill of slot r has fill count fill (r < slot) or fill - 1 (r >= slot)
  for (int r = 0; r < RING; ++r) {
    if (!(issued_slots >> r & 1u)) continue;
    const uint32_t f = r < slot ? fill : fill - 1;
    (void)mbar_wait_bounded(&full[r], f & 1u);
  }
  for (int r = 0; r < C::RING_LO; ++r) {
    if (!(lo_issued >> r & 1u)) continue;
    const uint32_t f = r < lslot ? lfill : lfill - 1;
    (void)mbar_wait_bounded(&lo_full[r], f & 1u);
  }
}

// ---------------------------------------------------------------- consumer warps
// Coefficients of the stage(s) one launch evaluates, formed in double
// precision.  Kind k = 0 (and 1 for a fused pair) is one RK stage:
//   stage argument  P_k = p + kq[k] q + kg[k] G(tile k),
//   stencil         c43[k], cm12[k], ccen[k],
//   point argument  Q_0 = q + q0 X (X = the stage's G input, or 0),
//                   Q_1 = q + q1 * (result of kind 0).
template <class TM>
struct UCoef {
  TM c43[2], cm12[2], ccen[2];
  TM kq[2], kg[2];
  TM q0, q1;
  TM nlam, m3;
  TM b6, d6, dt;
};

// Value `lane` of UCoef (in member order) for step `kstep` of the batch, from
// the FP64 table of coef_kernel (stage times t, t + dt/2, t + dt/2, t + dt of
// step n_base + kstep), rounded to the math type: each lane reads one entry,
// and the warp assembles the struct with shuffles.
template <class C>
__device__ __forceinline__ typename C::TM coef_entry(const Desc *d, int kstep, int lane) {
  using TM = typename C::TM;
  constexpr int S = C::S;
  const int s0 = S <= 4 ? S - 1 : (S == 5 ? 0 : 2);  // stage of kind 0
  const int s1 = (s0 + 1) & 3;                        // stage of kind 1
  const int st = kstep * kCoefPerStep, cc = kMaxK * kCoefPerStep;
  // offset into the table; -1: mu^2 (the centre weight of the difference
  // form), -2: the constant -3
  int off;
  switch (lane) {
    case 0: off = st + s0 * kCoefPerStage; break;            // c43[0] = 4/3 c
    case 1: off = st + s1 * kCoefPerStage; break;            // c43[1]
    case 2: off = st + s0 * kCoefPerStage + 1; break;        // cm12[0] = -c/12
    case 3: off = st + s1 * kCoefPerStage + 1; break;        // cm12[1]
    case 4: off = C::DIFF ? -1 : st + s0 * kCoefPerStage + 2; break;  // ccen[0]
    case 5: off = C::DIFF ? -1 : st + s1 * kCoefPerStage + 2; break;  // ccen[1]
    case 6: off = cc + kCoefSq + s0; break;                  // kq[0]: q weight of P
    case 7: off = cc + kCoefSq + s1; break;                  // kq[1]
    case 8: off = cc + kCoefSg + s0; break;                  // kg[0]: G weight of P
    case 9: off = cc + kCoefSg + s1; break;                  // kg[1]
    case 10: off = cc + kCoefSp + s0; break;                 // q0: G weight of Q
    case 11: off = cc + kCoefSp + s1; break;                 // q1
    case 12: off = cc + kCoefNlam; break;                    // -lambda
    case 13: off = -2; break;                                // m3 = -3
    case 14: off = cc + kCoefB6; break;                      // dt^2/6
    case 15: off = cc + kCoefD6; break;                      // dt/6
    case 16: off = cc + kCoefDt; break;                      // dt
    default: off = -2; break;
  }
  const double v = off >= 0 ? __ldcg(d->coef + off) : (off == -1 ? d->mu2 : -3.0);
  return (TM)v;
}

template <class TM>
__device__ __forceinline__ TM lap_g(TM c43, TM cm12, TM ccen, TM nlam, TM m3, bool diff, TM P0,
                                    TM xm2, TM xm1, TM xp1, TM xp2, TM ym2, TM ym1, TM yp1,
                                    TM yp2, TM zm2, TM zm1, TM zp1, TM zp2, TM Q,
                                    TM *lap_h2 = nullptr) {
  TM s1, s2;
  if (diff) {
    s1 = ((xm1 - P0) + (xp1 - P0)) + (((ym1 - P0) + (yp1 - P0)) + ((zm1 - P0) + (zp1 - P0)));
    s2 = ((xm2 - P0) + (xp2 - P0)) + (((ym2 - P0) + (yp2 - P0)) + ((zm2 - P0) + (zp2 - P0)));
  } else {
    s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
    s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
  }
  // h^2 Delta_h P (Sec. 2.1 weights; the difference form folds the centre in)
  if (lap_h2)
    *lap_h2 = diff ? fmaT((TM)(4.0 / 3.0), s1, (TM)(-1.0 / 12.0) * s2)
                   : fmaT((TM)(4.0 / 3.0), s1, fmaT((TM)(-1.0 / 12.0), s2, (TM)(-7.5) * P0));
  // reaction and centre terms as (ccen - lambda P0^2) P0 - 3 Q
  TM g = fmaT(fmaT(nlam, P0 * P0, ccen), P0, m3 * Q);
  g = fmaT(cm12, s2, g);
  return fmaT(c43, s1, g);
}

// The same evaluation for two neighbouring x points at once with the packed
// FP32 instructions of sm_100 and later (two lanes of arithmetic per
// instruction, each rounded exactly as the scalar operation: a - b is formed
// as fma(b, -1, a), one rounding of the exact difference).  Difference form
// only (the FP32 paths).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// The reaction and damping terms and the weighted pair sums s1 (distance 1)
// and s2 (distance 2) of the difference-form stencil, on two points at once.
__device__ __forceinline__ float2 lap_tail2(float2 c43, float2 cm12, float2 ccen, float2 nlam,
                                           float2 m3, float2 P0, float2 s1, float2 s2,
                                           float2 Q) {
  float2 g = __ffma2_rn(__ffma2_rn(nlam, __fmul2_rn(P0, P0), ccen), P0, __fmul2_rn(m3, Q));
  g = __ffma2_rn(cm12, s2, g);
  return __ffma2_rn(c43, s1, g);
}
__device__ __forceinline__ float2 lap_g2(float2 c43, float2 cm12, float2 ccen, float2 nlam,
                                         float2 m3, float2 P0, float2 xm2, float2 xm1,
                                         float2 xp1, float2 xp2, float2 ym2, float2 ym1,
                                         float2 yp1, float2 yp2, float2 zm2, float2 zm1,
                                         float2 zp1, float2 zp2, float2 Q) {
  const float2 s1 = __fadd2_rn(__fadd2_rn(sub2(xm1, P0), sub2(xp1, P0)),
                               __fadd2_rn(__fadd2_rn(sub2(ym1, P0), sub2(yp1, P0)),
                                          __fadd2_rn(sub2(zm1, P0), sub2(zp1, P0))));
  const float2 s2 = __fadd2_rn(__fadd2_rn(sub2(xm2, P0), sub2(xp2, P0)),
                               __fadd2_rn(__fadd2_rn(sub2(ym2, P0), sub2(yp2, P0)),
                                          __fadd2_rn(sub2(zm2, P0), sub2(zp2, P0))));
  return lap_tail2(c43, cm12, ccen, nlam, m3, P0, s1, s2, Q);
}
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// One consumer warp.  Kinds (KN = 1 for one stage, 2 for a fused pair) share
// the ring tiles; the register window holds P of every kind at planes
// z-2..z+2 for the warp's own points (rotating or shifted, see plane()).
template <class C>
struct Consumer {
  using TS = typename C::TS;
  using TG = typename C::TG;
  using TM = typename C::TM;
  static constexpr int S = C::S, VEC = C::VEC, VY = C::VY, TX = C::TX, RING = C::RING;
  static constexpr int BXS = C::BXS, BXG = C::BXG, HXS = C::HXS, HXG = C::HXG;
  static constexpr int KN = C::PAIR ? 2 : 1;

  // G tile (halo) that enters the stage argument of kind k, or -1
  __host__ __device__ static constexpr int gtile(int kk) {
    return (S == 3 || S == 4) ? (kk == 0 ? 0 : -1) : (S == 6 ? kk : -1);
  }
  __host__ __device__ static constexpr bool uses_q(int kk) { return !(S == 1 || (S == 5 && kk == 0)); }

  const unsigned char *ring;
  UCoef<TM> k;
  int lane, lx0, ly0;

  // Stage arguments of every kind at n consecutive tile positions from (lx, ly).
  template <int n>
  __device__ __forceinline__ void comb(const unsigned char *base, int lx, int ly,
                                       TM (&out)[KN][n]) const {
    TM pv[n], qv[n] = {};
    load_as<TS, TM, n>(reinterpret_cast<const TS *>(base) + (ly + 2) * BXS + lx + HXS, pv);
    if constexpr (uses_q(0) || (KN == 2 && uses_q(1)))
      load_as<TS, TM, n>(reinterpret_cast<const TS *>(base + C::HS_BYTES) + (ly + 2) * BXS + lx + HXS, qv);
#pragma unroll
    for (int kk = 0; kk < KN; ++kk) {
      TM gv[n] = {};
      if (gtile(kk) >= 0)
        load_as<TG, TM, n>(reinterpret_cast<const TG *>(base + C::OFF_HG + gtile(kk) * C::HG_BYTES) +
                               (ly + 2) * BXG + lx + HXG, gv);
      if constexpr (C::PCOMB && n % 2 == 0) {
        // pairs of points per packed FMA (each element rounded as fmaf)
#pragma unroll
        for (int j = 0; j < n; j += 2) {
          float2 v = f2(pv[j], pv[j + 1]);
          if (uses_q(kk)) v = __ffma2_rn(f2(k.kq[kk]), f2(qv[j], qv[j + 1]), v);
          if (gtile(kk) >= 0) v = __ffma2_rn(f2(k.kg[kk]), f2(gv[j], gv[j + 1]), v);
          out[kk][j] = v.x;
          out[kk][j + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < n; ++j) {
          TM v = pv[j];
          if (uses_q(kk)) v = fmaT(k.kq[kk], qv[j], v);
          if (gtile(kk) >= 0) v = fmaT(k.kg[kk], gv[j], v);
          out[kk][j] = v;
        }
      }
    }
  }

  // x neighbours e[kk][i] = P_kk at x - 2 + i (i = 0 .. VEC + 3) of the lane's
  // points in row ly, given the own values c.
  __device__ __forceinline__ void xnb(const unsigned char *base, int ly, const TM (&c)[KN][VEC],
                                      TM (&e)[KN][VEC + 4]) const {
#pragma unroll
    for (int kk = 0; kk < KN; ++kk)
#pragma unroll
      for (int j = 0; j < VEC; ++j) e[kk][2 + j] = c[kk][j];
    if constexpr (C::XLDS) {
      // every lane forms its four x neighbours of each kind from the halo
      // columns of the ring tiles (the same values the neighbouring lanes hold)
      TM l[KN][2], rr[KN][2];
      comb<2>(base, lx0 - 2, ly, l);
      comb<2>(base, lx0 + VEC, ly, rr);
#pragma unroll
      for (int kk = 0; kk < KN; ++kk) {
        e[kk][0] = l[kk][0]; e[kk][1] = l[kk][1];
        e[kk][VEC + 2] = rr[kk][0]; e[kk][VEC + 3] = rr[kk][1];
      }
    } else if constexpr (S == 1) {
      // P = p: neighbours straight from the halo tile
      const TS *hp = reinterpret_cast<const TS *>(base) + (ly + 2) * BXS + lx0 + HXS;
      if constexpr (VEC >= 2) {
        TM a[2], b[2];
        load_as<TS, TM, 2>(hp - 2, a);
        load_as<TS, TM, 2>(hp + VEC, b);
        e[0][0] = a[0]; e[0][1] = a[1]; e[0][VEC + 2] = b[0]; e[0][VEC + 3] = b[1];
      } else {
        e[0][0] = (TM)hp[-2]; e[0][1] = (TM)hp[-1]; e[0][3] = (TM)hp[1]; e[0][4] = (TM)hp[2];
      }
    } else if constexpr (VEC >= 2) {
      TM l0[KN], l1[KN], r0[KN], r1[KN];
#pragma unroll
      for (int kk = 0; kk < KN; ++kk) {
        l0[kk] = shfl_up1(c[kk][VEC - 2], 1);
        l1[kk] = shfl_up1(c[kk][VEC - 1], 1);
        r0[kk] = shfl_dn1(c[kk][0], 1);
        r1[kk] = shfl_dn1(c[kk][1], 1);
      }
      if (lane == 0 || lane == 31) {
        TM h[KN][2];
        comb<2>(base, lane == 0 ? -2 : TX, ly, h);
#pragma unroll
        for (int kk = 0; kk < KN; ++kk) {
          if (lane == 0) { l0[kk] = h[kk][0]; l1[kk] = h[kk][1]; }
          else { r0[kk] = h[kk][0]; r1[kk] = h[kk][1]; }
        }
      }
#pragma unroll
      for (int kk = 0; kk < KN; ++kk) {
        e[kk][0] = l0[kk]; e[kk][1] = l1[kk]; e[kk][VEC + 2] = r0[kk]; e[kk][VEC + 3] = r1[kk];
      }
    } else {
      TM h[KN][1];
#pragma unroll
      for (int kk = 0; kk < KN; ++kk) h[kk][0] = c[kk][0];
      if (lane < 2 || lane >= 30) comb<1>(base, lane < 2 ? lane - 2 : TX + lane - 30, ly, h);
#pragma unroll
      for (int kk = 0; kk < KN; ++kk) {
        const TM u2 = shfl_up1(c[kk][0], 2), u1 = shfl_up1(c[kk][0], 1);
        const TM d2 = shfl_dn1(c[kk][0], 2), d1 = shfl_dn1(c[kk][0], 1);
        const TM h1 = shfl_idx(h[kk][0], 1), h30 = shfl_idx(h[kk][0], 30);
        e[kk][0] = lane < 2 ? h[kk][0] : u2;
        e[kk][1] = lane == 0 ? h1 : u1;
        e[kk][3] = lane == 31 ? h30 : d1;
        e[kk][4] = lane >= 30 ? h[kk][0] : d2;
      }
    }
  }

  struct Item {
    int N, x, z0, zoff, nplanes, set;
    bool ragged, xok;
    int64_t pitch_s, plane_s, pitch_g, plane_g, row_s, row_g;
    int y0;
    TG *outG0, *outG1;
    TS *outP, *outQ, *outPL, *outQL;
  };

  // One z-plane: plane m of the item enters the window (slot `slot`); for
  // m >= 4 the output plane m - 4 (loaded as plane m - 2, slot s2) is computed.
  // ROT >= 0: plane j lives at window index j mod 5 and m mod 5 == ROT (the
  // plane loop is unrolled 5 times, so no register moves); ROT < 0: the window
  // is shifted by one plane first and the newest plane is at index 4.
  template <int ROT>
  __device__ __forceinline__ void plane(const Item &it, int m, int slot, int s2,
                                        const unsigned char *lob, TM (&win)[5][KN][VY][VEC],
                                        TM &run_max, bool &bad) const {
    constexpr int R0 = ROT < 0 ? 4 : ROT;
    constexpr int W0 = R0 % 5, WM1 = (R0 + 4) % 5, WM2 = (R0 + 3) % 5, WM3 = (R0 + 2) % 5,
                  WM4 = (R0 + 1) % 5;
    if constexpr (ROT < 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int kk = 0; kk < KN; ++kk)
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int j = 0; j < VEC; ++j) win[a][kk][r][j] = win[a + 1][kk][r][j];
    }
    const unsigned char *base = ring + slot * C::SLOT_BYTES;
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      TM t[KN][VEC];
      comb<VEC>(base, lx0, ly0 + r, t);
#pragma unroll
      for (int kk = 0; kk < KN; ++kk)
#pragma unroll
        for (int j = 0; j < VEC; ++j) win[W0][kk][r][j] = t[kk][j];
    }
    if (m < 4) return;
    // ---- output plane z = z0 + m - 4 (window: z-2 = W(m-4), z-1 = W(m-3),
    // z = W(m-2), z+1 = W(m-1), z+2 = W(m))
    const int z = it.z0 + m - 4 + it.zoff;  // storage plane of the output
    const unsigned char *b2 = ring + s2 * C::SLOT_BYTES;
    TM R[KN][4][VEC];  // rows ly0-2, ly0-1, ly0+VY, ly0+VY+1 of P at plane z (not INCR)
    if constexpr (!C::INCR) {
      TM t[KN][VEC];
      const int rows[4] = {ly0 - 2, ly0 - 1, ly0 + VY, ly0 + VY + 1};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        comb<VEC>(b2, lx0, rows[i], t);
#pragma unroll
        for (int kk = 0; kk < KN; ++kk)
#pragma unroll
          for (int j = 0; j < VEC; ++j) R[kk][i][j] = t[kk][j];
      }
    }
    // P of kind kk, row offset dy (in [-2, VY+1]) at plane z, lane point j
    auto Pz = [&](int kk, int rr, int j) -> TM {
      return rr < 0 ? R[kk][rr + 2][j] : (rr >= VY ? R[kk][rr - VY + 2][j] : win[WM2][kk][rr][j]);
    };
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      const int ly = ly0 + r;
      const int y = it.y0 + ly;
      TM c[KN][VEC];
#pragma unroll
      for (int kk = 0; kk < KN; ++kk)
#pragma unroll
        for (int j = 0; j < VEC; ++j) c[kk][j] = win[WM2][kk][r][j];
      TM e[KN][VEC + 4];
      if constexpr (!C::INCR) xnb(b2, ly, c, e);
      const int hoff = (ly + 2) * BXS + lx0 + HXS;
      const int ioff = ly * TX + lx0;
      // point-only values of plane z
      TM qS[VEC], X[VEC] = {}, g1[VEC] = {}, g2[VEC] = {}, g3[VEC] = {}, lp[VEC] = {},
                                lq[VEC] = {};
      if constexpr (S == 1) {
        load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2 + C::OFF_IS) + ioff, qS);
      } else {
        load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2 + C::HS_BYTES) + hoff, qS);
      }
      if constexpr (S == 2 || S == 3)  // G1 | G2 at the point
        load_as<TG, TM, VEC>(reinterpret_cast<const TG *>(b2 + C::OFF_IG) + ioff, X);
      if constexpr (S == 4) {
        const TG *ig = reinterpret_cast<const TG *>(b2 + C::OFF_IG) + ioff;
        load_as<TG, TM, VEC>(ig, g1);
        load_as<TG, TM, VEC>(ig + C::IG_BYTES / (int)sizeof(TG), g3);
        load_as<TG, TM, VEC>(reinterpret_cast<const TG *>(b2 + C::OFF_HG) + (ly + 2) * BXG + lx0 + HXG, g2);
#pragma unroll
        for (int j = 0; j < VEC; ++j) X[j] = g3[j];
      }
      if constexpr (S == 6) {
        const TG *hg = reinterpret_cast<const TG *>(b2 + C::OFF_HG) + (ly + 2) * BXG + lx0 + HXG;
        load_as<TG, TM, VEC>(hg, g1);
        load_as<TG, TM, VEC>(hg + C::HG_BYTES / (int)sizeof(TG), g2);
#pragma unroll
        for (int j = 0; j < VEC; ++j) X[j] = g2[j];
      }
      if constexpr (C::LOR) {  // compensation terms of plane z, from their own ring
        const TS *is = reinterpret_cast<const TS *>(lob) + ioff;
        load_as<TS, TM, VEC>(is, lp);
        load_as<TS, TM, VEC>(is + C::IS_BYTES / (int)sizeof(TS), lq);
      } else if constexpr ((S == 4 || S == 6) && C::KAHAN) {
        const TS *is = reinterpret_cast<const TS *>(b2 + C::OFF_IS) + ioff;
        load_as<TS, TM, VEC>(is, lp);
        load_as<TS, TM, VEC>(is + C::IS_BYTES / (int)sizeof(TS), lq);
      }
      TM res[KN][VEC];
      if constexpr (C::INCR) {
        // the pair sums of lap_g2 in its association, formed part by part:
        // s1 = x1 + (y1 + z1), s2 = x2 + (y2 + z2)
        constexpr int NP = VEC / 2;
        float2 P0[KN][NP], A1[KN][NP], A2[KN][NP];
#pragma unroll
        for (int kk = 0; kk < KN; ++kk)
#pragma unroll
          for (int jp = 0; jp < NP; ++jp) {
            const int j = 2 * jp;
            P0[kk][jp] = f2(c[kk][j], c[kk][j + 1]);
            A1[kk][jp] = __fadd2_rn(sub2(f2(win[WM3][kk][0][j], win[WM3][kk][0][j + 1]), P0[kk][jp]),
                                    sub2(f2(win[WM1][kk][0][j], win[WM1][kk][0][j + 1]), P0[kk][jp]));
            A2[kk][jp] = __fadd2_rn(sub2(f2(win[WM4][kk][0][j], win[WM4][kk][0][j + 1]), P0[kk][jp]),
                                    sub2(f2(win[W0][kk][0][j], win[W0][kk][0][j + 1]), P0[kk][jp]));
          }
#pragma unroll
        for (int d = 1; d <= 2; ++d) {
          TM a[KN][VEC], b[KN][VEC];
          comb<VEC>(b2, lx0, ly - d, a);
          comb<VEC>(b2, lx0, ly + d, b);
#pragma unroll
          for (int kk = 0; kk < KN; ++kk)
#pragma unroll
            for (int jp = 0; jp < NP; ++jp) {
              const int j = 2 * jp;
              const float2 yy = __fadd2_rn(sub2(f2(a[kk][j], a[kk][j + 1]), P0[kk][jp]),
                                           sub2(f2(b[kk][j], b[kk][j + 1]), P0[kk][jp]));
              if (d == 1) A1[kk][jp] = __fadd2_rn(yy, A1[kk][jp]);
              else A2[kk][jp] = __fadd2_rn(yy, A2[kk][jp]);
            }
        }
        xnb(b2, ly, c, e);
#pragma unroll
        for (int kk = 0; kk < KN; ++kk) {
#pragma unroll
          for (int jp = 0; jp < NP; ++jp) {
            const int j = 2 * jp;
            const float2 s1 = __fadd2_rn(__fadd2_rn(sub2(f2(e[kk][j + 1], e[kk][j + 2]), P0[kk][jp]),
                                                    sub2(f2(e[kk][j + 3], e[kk][j + 4]), P0[kk][jp])),
                                         A1[kk][jp]);
            const float2 s2 = __fadd2_rn(__fadd2_rn(sub2(f2(e[kk][j], e[kk][j + 1]), P0[kk][jp]),
                                                    sub2(f2(e[kk][j + 4], e[kk][j + 5]), P0[kk][jp])),
                                         A2[kk][jp]);
            float2 Q;
            if (kk == 0)
              Q = (S == 1 || S == 5) ? f2(qS[j], qS[j + 1])
                                     : __ffma2_rn(f2(k.q0), f2(X[j], X[j + 1]), f2(qS[j], qS[j + 1]));
            else
              Q = __ffma2_rn(f2(k.q1), f2(res[0][j], res[0][j + 1]), f2(qS[j], qS[j + 1]));
            const float2 g = lap_tail2(f2(k.c43[kk]), f2(k.cm12[kk]), f2(k.ccen[kk]), f2(k.nlam),
                                       f2(k.m3), P0[kk][jp], s1, s2, Q);
            res[kk][j] = g.x;
            res[kk][j + 1] = g.y;
            if constexpr (C::MON) {
              if (kk == 0) {
                // h^2 Delta_h phi at the two points; the largest |.| over valid points
                const float2 lap = __ffma2_rn(f2(4.0f / 3.0f), s1,
                                              __fmul2_rn(f2(-1.0f / 12.0f), s2));
                const bool ok = it.xok && it.y0 + ly < it.N;
                const float a0 = (ok && it.x + j < it.N) ? fabsf(lap.x) : 0.f;
                const float a1 = (ok && it.x + j + 1 < it.N) ? fabsf(lap.y) : 0.f;
                run_max = fmaxf(run_max, fmaxf(a0, a1));
              }
            }
          }
        }
      } else if constexpr (C::PACKED) {
        // two x points per packed instruction (bitwise the scalar results)
#pragma unroll
        for (int kk = 0; kk < KN; ++kk) {
#pragma unroll
          for (int j = 0; j < VEC; j += 2) {
            float2 Q;
            if (kk == 0)
              Q = (S == 1 || S == 5) ? f2(qS[j], qS[j + 1])
                                     : __ffma2_rn(f2(k.q0), f2(X[j], X[j + 1]), f2(qS[j], qS[j + 1]));
            else
              Q = __ffma2_rn(f2(k.q1), f2(res[0][j], res[0][j + 1]), f2(qS[j], qS[j + 1]));
            const float2 g = lap_g2(
                f2(k.c43[kk]), f2(k.cm12[kk]), f2(k.ccen[kk]), f2(k.nlam), f2(k.m3),
                f2(c[kk][j], c[kk][j + 1]), f2(e[kk][j], e[kk][j + 1]),
                f2(e[kk][j + 1], e[kk][j + 2]), f2(e[kk][j + 3], e[kk][j + 4]),
                f2(e[kk][j + 4], e[kk][j + 5]), f2(Pz(kk, r - 2, j), Pz(kk, r - 2, j + 1)),
                f2(Pz(kk, r - 1, j), Pz(kk, r - 1, j + 1)), f2(Pz(kk, r + 1, j), Pz(kk, r + 1, j + 1)),
                f2(Pz(kk, r + 2, j), Pz(kk, r + 2, j + 1)),
                f2(win[WM4][kk][r][j], win[WM4][kk][r][j + 1]),
                f2(win[WM3][kk][r][j], win[WM3][kk][r][j + 1]),
                f2(win[WM1][kk][r][j], win[WM1][kk][r][j + 1]),
                f2(win[W0][kk][r][j], win[W0][kk][r][j + 1]), Q);
            res[kk][j] = g.x;
            res[kk][j + 1] = g.y;
          }
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < KN; ++kk) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            TM Q;
            if (kk == 0) Q = (S == 1 || S == 5) ? qS[j] : fmaT(k.q0, X[j], qS[j]);
            else Q = fmaT(k.q1, res[0][j], qS[j]);
            TM lap = (TM)0;
            res[kk][j] = lap_g(k.c43[kk], k.cm12[kk], k.ccen[kk], k.nlam, k.m3, C::DIFF, c[kk][j],
                               e[kk][j], e[kk][j + 1], e[kk][j + 3], e[kk][j + 4], Pz(kk, r - 2, j),
                               Pz(kk, r - 1, j), Pz(kk, r + 1, j), Pz(kk, r + 2, j),
                               win[WM4][kk][r][j], win[WM3][kk][r][j], win[WM1][kk][r][j],
                               win[W0][kk][r][j], Q, (C::MON && kk == 0) ? &lap : nullptr);
            if constexpr (C::MON) {
              if (kk == 0 && it.xok && y < it.N && it.x + j < it.N) {
                const TM a = lap < (TM)0 ? -lap : lap;
                run_max = a > run_max ? a : run_max;
              }
            }
          }
        }
      }
      const bool rok = it.xok && y < it.N;
      const bool fast = rok && !it.ragged;
      if constexpr (S <= 3 || S == 5) {
        const int64_t off = (int64_t)z * it.plane_g + it.row_g + r * it.pitch_g;
        if (fast) {
          store_as<TG, TM, VEC>(it.outG0 + off, res[0]);
          if constexpr (S == 5) store_as<TG, TM, VEC>(it.outG1 + off, res[KN - 1]);
        } else if (rok) {
          store_ragged<TG, TM, VEC>(it.outG0 + off - it.x, it.N, it.x, res[0]);
          if constexpr (S == 5) store_ragged<TG, TM, VEC>(it.outG1 + off - it.x, it.N, it.x, res[KN - 1]);
        }
      } else {
        // RK4 combine (Sec. 2.1): p' = p + dt q + dt^2/6 (G1 + G2 + G3),
        //                         q' = q + dt/6 (G1 + 2 G2 + 2 G3 + G4)
        if constexpr (S == 6) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) g3[j] = res[0][j];
        }
        const TM *G4 = res[KN - 1];
        TM pS[VEC];
        load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2) + hoff, pS);
        TM pn[VEC], qn[VEC], pl[VEC], ql[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          const TM dp = fmaT(k.b6, (g1[j] + g2[j]) + g3[j], k.dt * qS[j]);
          // 2 x is exact, so the FMA rounds 2 (g2 + g3) + (g1 + G4) once, as before
          const TM dq = k.d6 * fmaT((TM)2, g2[j] + g3[j], g1[j] + G4[j]);
          if constexpr (C::KAHAN) {
            two_sum(pS[j], dp + lp[j], pn[j], pl[j]);
            two_sum(qS[j], dq + lq[j], qn[j], ql[j]);
          } else {
            pn[j] = pS[j] + dp;
            qn[j] = qS[j] + dq;
          }
          // running max of |p'| over valid points; NaN and overflow read as +inf
          TM av = pn[j] < (TM)0 ? -pn[j] : pn[j];
          av = (av == av) ? av : (TM)INFINITY;
          av = (rok && it.x + j < it.N) ? av : (TM)0;
          run_max = av > run_max ? av : run_max;
        }
        const int64_t off = (int64_t)z * it.plane_s + it.row_s + r * it.pitch_s;
        if (fast) {
          store_as<TS, TM, VEC>(it.outP + off, pn);
          store_as<TS, TM, VEC>(it.outQ + off, qn);
          if constexpr (C::KAHAN) {
            store_as<TS, TM, VEC>(it.outPL + off, pl);
            store_as<TS, TM, VEC>(it.outQL + off, ql);
          }
        } else if (rok) {
          store_ragged<TS, TM, VEC>(it.outP + off - it.x, it.N, it.x, pn);
          store_ragged<TS, TM, VEC>(it.outQ + off - it.x, it.N, it.x, qn);
          if constexpr (C::KAHAN) {
            store_ragged<TS, TM, VEC>(it.outPL + off - it.x, it.N, it.x, pl);
            store_ragged<TS, TM, VEC>(it.outQL + off - it.x, it.N, it.x, ql);
          }
        }
      }
    }
    (void)bad;
  }

  static __device__ __forceinline__ void run(const StageParams &prm, uint64_t *full,
                                             uint64_t *empty, const unsigned char *ring_,
                                             volatile int *abort_flag, int warp, int lane_) {
    Consumer self;
    self.ring = ring_;
    self.lane = lane_;
    self.lx0 = lane_ * VEC;
    self.ly0 = warp * VY;
    const int nitems = *prm.nitems;
    int slot = 0;
    uint32_t phase = 0;
    uint64_t *lo_full = full + C::LO_BAR, *lo_empty = full + C::LO_BAR + 4;
    const unsigned char *lo_ring = ring_ - C::HEADER + C::OFF_LO;
    int lslot = 0;
    uint32_t lphase = 0;
    const Desc *coef_d = nullptr;
    long long coef_n = -1;
    for (int itx = blockIdx.x; itx < nitems; itx += gridDim.x) {
      const WorkItem w = prm.items[itx];
      Desc *d = prm.descs + w.x;
      if (!item_active<S>(d, prm.k, warp == 0 && lane_ == 0)) continue;
      const long long n = d->n_base + prm.k;
      if (d != coef_d || n != coef_n) {
        // the coefficients of (context, step): read once per warp and launch
        // when every work item belongs to one context
        coef_d = d;
        coef_n = n;
        static_assert(sizeof(UCoef<TM>) / sizeof(TM) == 17, "coef_entry covers UCoef");
        const TM mine = coef_entry<C>(d, prm.k, lane_);
        TM *dst = reinterpret_cast<TM *>(&self.k);
#pragma unroll
        for (int i = 0; i < 17; ++i) dst[i] = shfl_idx(mine, i);
      }
      Item it;
      it.N = d->N;
      it.set = (int)(n & 1);
      const int so = it.set ^ 1;
      const int x0 = (w.y & 0xffff) * TX;
      it.y0 = (w.y >> 16) * C::TY;
      it.z0 = w.z;
      it.zoff = d->zoff;
      it.nplanes = w.w + 4;
      it.ragged = x0 + TX > it.N;
      it.x = x0 + self.lx0;
      it.xok = it.x < it.N;
      it.pitch_s = d->pitch_s; it.plane_s = d->plane_s;
      it.pitch_g = d->pitch_g; it.plane_g = d->plane_g;
      it.row_s = (int64_t)(it.y0 + self.ly0 + 2) * it.pitch_s + HXS + it.x;
      it.row_g = (int64_t)(it.y0 + self.ly0 + 2) * it.pitch_g + HXG + it.x;
      it.outG0 = it.outG1 = nullptr;
      it.outP = it.outQ = it.outPL = it.outQL = nullptr;
      if constexpr (S <= 3) it.outG0 = reinterpret_cast<TG *>(d->f[S == 1 ? F_G1 : (S == 2 ? F_G2 : F_G3)]);
      if constexpr (S == 5) {
        it.outG0 = reinterpret_cast<TG *>(d->f[F_G1]);
        it.outG1 = reinterpret_cast<TG *>(d->f[F_G2]);
      }
      if constexpr (S == 4 || S == 6) {
        it.outP = reinterpret_cast<TS *>(d->f[F_P0 + so]);
        it.outQ = reinterpret_cast<TS *>(d->f[F_Q0 + so]);
        if constexpr (C::KAHAN) {
          it.outPL = reinterpret_cast<TS *>(d->f[F_PLO0 + so]);
          it.outQL = reinterpret_cast<TS *>(d->f[F_QLO0 + so]);
        }
      }
      TM win[5][KN][VY][VEC];
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int kk = 0; kk < KN; ++kk)
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int j = 0; j < VEC; ++j) win[a][kk][r][j] = (TM)0;
      TM run_max = (TM)0;
      bool bad = false;
      // one plane: wait for its slot, compute, release what is no longer needed
      auto step = [&](auto rot, int m) -> bool {
        if (!mbar_wait_bounded(&full[slot], phase)) {
          *abort_flag = 1;
          atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
          return false;
        }
        const bool lo = C::LOR && m >= 4;  // an output plane: its compensation slot
        if (lo && !mbar_wait_bounded(&lo_full[lslot], lphase)) {
          *abort_flag = 1;
          atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
          return false;
        }
        if (*abort_flag) return false;
        const int s2 = slot >= 2 ? slot - 2 : slot + RING - 2;  // slot of plane m - 2
        self.template plane<decltype(rot)::value>(it, m, slot, s2, lo_ring + lslot * C::LO_SLOT,
                                                  win, run_max, bad);
        __syncwarp();
        if (self.lane == 0) {
          if (m < 2 || m >= it.nplanes - 2) mbar_arrive(&empty[slot]);
          if (m >= 4) mbar_arrive(&empty[s2]);
          if (lo) mbar_arrive(&lo_empty[lslot]);
        }
        if (++slot == RING) { slot = 0; phase ^= 1u; }
        if (lo && ++lslot == C::RING_LO) { lslot = 0; lphase ^= 1u; }
        return true;
      };
      bool ok = true;
      using I0 = std::integral_constant<int, 0>;
      using I1 = std::integral_constant<int, 1>;
      using I2 = std::integral_constant<int, 2>;
      using I3 = std::integral_constant<int, 3>;
      using I4 = std::integral_constant<int, 4>;
      int m = 0;
      if constexpr (C::ROTATE) {
        for (; ok && m + 5 <= it.nplanes; m += 5)
          ok = step(I0{}, m) && step(I1{}, m + 1) && step(I2{}, m + 2) && step(I3{}, m + 3) &&
               step(I4{}, m + 4);
        if (ok && m < it.nplanes) ok = step(I0{}, m++);
        if (ok && m < it.nplanes) ok = step(I1{}, m++);
        if (ok && m < it.nplanes) ok = step(I2{}, m++);
        if (ok && m < it.nplanes) ok = step(I3{}, m++);
      } else {
        for (; ok && m < it.nplanes; ++m) ok = step(std::integral_constant<int, -1>{}, m);
      }
      if (!ok) return;
      if constexpr (S == 4 || S == 6 || C::MON) {
        double v = (double)run_max;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        unsigned long long *dst = d->maxabs + prm.k;
        if constexpr (C::MON) dst = d->mon + (n % d->mon_cap);  // the step's monitor entry
        if (lane_ == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
      }
    }
  }
};

template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    stage_kernel(const StageParams prm) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty = reinterpret_cast<uint64_t *>(smem + 128);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 256);
  unsigned char *ring = smem + C::HEADER;
  static_assert(C::RING <= 16, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int r = 0; r < C::RING; ++r) {
      mbar_init(&full[r], 1);
      mbar_init(&empty[r], C::NW);
    }
    for (int r = 0; r < C::RING_LO; ++r) {
      mbar_init(&full[C::LO_BAR + r], 1);
      mbar_init(&full[C::LO_BAR + 4 + r], C::NW);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (warp == C::NW) {
    if (lane == 0) produce<C>(prm, full, empty, ring, abort_flag);
  } else {
    Consumer<C>::run(prm, full, empty, ring, abort_flag, warp, lane);
  }
}

}  // namespace hbe
