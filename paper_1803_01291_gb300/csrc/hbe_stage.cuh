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
// Kernel shape (one launch per stage, persistent blocks over a work list):
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
#pragma once
#include <cuda_bf16.h>

#include "hbe_common.cuh"

namespace hbe {

// ---------------------------------------------------------------- precisions
struct PrecFP64 {
  using TS = double; using TG = double; using TM = double;
  static constexpr bool KAHAN = false;
  static constexpr bool DIFF = false;   // merged-centre stencil (fewest FP64 ops)
};
struct PrecFP32 {
  using TS = float; using TG = float; using TM = float;
  static constexpr bool KAHAN = true;
  static constexpr bool DIFF = true;    // neighbour-minus-centre stencil (less cancellation)
};
struct PrecBF16 {
  using TS = float; using TG = __nv_bfloat16; using TM = float;
  static constexpr bool KAHAN = true;
  static constexpr bool DIFF = true;
};
struct PrecFP32Plain {
  using TS = float; using TG = float; using TM = float;
  static constexpr bool KAHAN = false;
  static constexpr bool DIFF = true;
};

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <class PR, int VEC_, int VY_, int NW_, int BUDGET_, int MINB_, int S_>
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
  static constexpr int NIS = (S == 1) ? 1 : (((S == 4 || S == 6) && KAHAN) ? 2 : 0);
  static constexpr int NIG = (S == 1 || S >= 5) ? 0 : ((S == 4) ? 2 : 1);       // G1 | G2 | G1, G3
  static constexpr int HS_RAW = BY * BXS * (int)sizeof(TS);
  static constexpr int HG_RAW = BY * BXG * (int)sizeof(TG);
  static constexpr int IS_RAW = TY * TX * (int)sizeof(TS);
  static constexpr int IG_RAW = TY * TX * (int)sizeof(TG);
  static constexpr int HS_BYTES = align128(HS_RAW), HG_BYTES = align128(HG_RAW);
  static constexpr int IS_BYTES = align128(IS_RAW), IG_BYTES = align128(IG_RAW);
  static constexpr int OFF_HG = NHS * HS_BYTES;
  static constexpr int OFF_IS = OFF_HG + NHG * HG_BYTES;
  static constexpr int OFF_IG = OFF_IS + NIS * IS_BYTES;
  static constexpr int SLOT_BYTES = OFF_IG + NIG * IG_BYTES;
  static constexpr uint32_t TX_BYTES =
      (uint32_t)(NHS * HS_RAW + NHG * HG_RAW + NIS * IS_RAW + NIG * IG_RAW);
  static constexpr int HEADER = 384;  // 2 x 16 mbarriers, flags
  static constexpr int RING = cmax(4, cmin(16, (BUDGET_ - HEADER) / SLOT_BYTES));
  static constexpr int SMEM = HEADER + RING * SLOT_BYTES;
  static constexpr int MINB = MINB_;  // blocks per SM the registers must allow
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
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
template <class TM, int n>
__device__ __forceinline__ void lds(const TM *p, TM (&v)[n]) { load_as<TM, TM, n>(p, v); }
template <class TM, int n>
__device__ __forceinline__ void sts(TM *p, const TM (&v)[n]) { store_as<TM, TM, n>(p, v); }

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

// Store VEC values of a field at interior point (x, y) of a plane of the padded
// layout (`row` points at the row's x = 0).  `ragged`: the tile may cross x = N
// (mask); `edge`: periodic tile touching a wrap band (write the ghost copies).
template <class T, class TM, int VEC>
__device__ __forceinline__ void store_point(T *row, int64_t pitch, int N, bool ragged, bool edge,
                                            int x, int y, const TM (&v)[VEC]) {
  if (!ragged || x + VEC <= N) {
    store_as<T, TM, VEC>(row + x, v);
  } else {
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      if (x + j < N) row[x + j] = narrow<T>(v[j]);
  }
  if (edge) {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int xx = x + j;
      if (xx >= N) continue;
      const T val = narrow<T>(v[j]);
      if (xx < 2) row[xx + N] = val;
      if (xx >= N - 2) row[xx - N] = val;
      if (y < 2) row[(int64_t)N * pitch + xx] = val;
      if (y >= N - 2) row[-(int64_t)N * pitch + xx] = val;
    }
  }
}

// Coefficients of one stage, formed in double precision by one thread.
template <class TM>
struct Coef {
  TM c43, cm12, ccen, nlam, a1, a2, m3;   // stencil / combine
  TM b6, d6;                              // stage-4 combine
};

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

// Stage coefficients in double precision, narrowed to the math type.
template <class C>
__device__ __forceinline__ Coef<typename C::TM> stage_coef(const Desc *d, long long n) {
  using TM = typename C::TM;
  constexpr int S = C::S;
  const double dt = d->dt;
  const double tn = d->t0 + (double)n * dt;
  const double ts = tn + (S == 1 ? 0.0 : (S == 4 ? dt : 0.5 * dt));
  const double c = exp(-2.0 * ts) * d->inv_h2;
  Coef<TM> cf;
  cf.c43 = (TM)(4.0 / 3.0 * c);
  cf.cm12 = (TM)(-c / 12.0);
  cf.ccen = C::DIFF ? (TM)d->mu2 : (TM)(d->mu2 - 7.5 * c);
  cf.nlam = (TM)(-d->lambda);
  cf.m3 = (TM)(-3.0);
  cf.a1 = (TM)(S == 1 ? 0.0 : (S == 4 ? dt : 0.5 * dt));
  cf.a2 = (TM)(S == 3 ? 0.25 * dt * dt : (S == 4 ? 0.5 * dt * dt : 0.0));
  cf.b6 = (TM)(dt * dt / 6.0);
  cf.d6 = (TM)(dt / 6.0);
  return cf;
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
  bool bad = false;
  for (int it = blockIdx.x; it < nitems && !bad; it += gridDim.x) {
    const WorkItem w = prm.items[it];
    Desc *d = prm.descs + w.x;
    if (!item_active<S>(d, prm.k, false)) continue;
    const CUtensorMap *tm = d->tmaps;
    for (int t = 0; t < NUM_TMAPS; ++t) tmap_acquire(tm + t);
    const int N = d->N;
    const bool periodic = d->bc == 1;
    const int set = (int)((d->n_base + prm.k) & 1);
    const CUtensorMap *mp = tm + (set ? TM_P_H1 : TM_P_H0);
    const CUtensorMap *mq = tm + (set ? TM_Q_H1 : TM_Q_H0);
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
      unsigned char *base = ring + slot * C::SLOT_BYTES;
      uint64_t *bar = &full[slot];
      int z = z0 - 2 + m;
      if (periodic) z = (z % N + N) % N;
      mbar_expect_tx(bar, C::TX_BYTES);
      tma_load_3d(base, mp, bar, x0, y0, z);
      if constexpr (C::NHS == 2) tma_load_3d(base + C::HS_BYTES, mq, bar, x0, y0, z);
      if constexpr (C::NHG == 1 && !C::PAIR) tma_load_3d(base + C::OFF_HG, mg, bar, x0, y0, z);
      constexpr int HXS = C::HXS, HXG = C::HXG;
      if constexpr (S == 6) {
        tma_load_3d(base + C::OFF_HG, tm + TM_G1_H, bar, x0, y0, z);
        tma_load_3d(base + C::OFF_HG + C::HG_BYTES, tm + TM_G2_H, bar, x0, y0, z);
        if constexpr (C::KAHAN) {
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
}

// ---------------------------------------------------------------- consumer warps
template <class C>
struct Consumer {
  using TS = typename C::TS;
  using TG = typename C::TG;
  using TM = typename C::TM;
  static constexpr int S = C::S, VEC = C::VEC, VY = C::VY, TX = C::TX;
  static constexpr int BXS = C::BXS, BXG = C::BXG, HXS = C::HXS, HXG = C::HXG;
  static constexpr int NI = C::NIS + C::NIG;  // point-only input fields

  // Stage argument P at n consecutive tile positions from (lx, ly) (ly in
  // [-2, TY+2)), formed from the ring tiles.
  template <int n>
  static __device__ __forceinline__ void comb_n(const unsigned char *base, const Coef<TM> &cf,
                                                int lx, int ly, TM (&out)[n]) {
    load_as<TS, TM, n>(reinterpret_cast<const TS *>(base) + (ly + 2) * BXS + lx + HXS, out);
    if constexpr (S >= 2) {
      TM qv[n];
      load_as<TS, TM, n>(reinterpret_cast<const TS *>(base + C::HS_BYTES) + (ly + 2) * BXS + lx + HXS, qv);
#pragma unroll
      for (int j = 0; j < n; ++j) out[j] = fmaT(cf.a1, qv[j], out[j]);
    }
    if constexpr (S >= 3) {
      TM gv[n];
      load_as<TG, TM, n>(reinterpret_cast<const TG *>(base + C::OFF_HG) + (ly + 2) * BXG + lx + HXG, gv);
#pragma unroll
      for (int j = 0; j < n; ++j) out[j] = fmaT(cf.a2, gv[j], out[j]);
    }
  }
  static __device__ __forceinline__ void comb(const unsigned char *base, const Coef<TM> &cf,
                                              int lx, int ly, TM (&out)[VEC]) {
    comb_n<VEC>(base, cf, lx, ly, out);
  }

  // x neighbours (x-2, x-1, x+1, x+2) of the lane's VEC points in tile row ly,
  // whose own P values are c.
  static __device__ __forceinline__ void xnb(const unsigned char *base, const Coef<TM> &cf,
                                             int lane, int lx0, int ly, const TM (&c)[VEC],
                                             TM (&m2)[VEC], TM (&m1)[VEC], TM (&p1)[VEC],
                                             TM (&p2)[VEC]) {
    if constexpr (S == 1) {
      // P = p: read the neighbours straight from the halo tile
      const TS *hp = reinterpret_cast<const TS *>(base) + (ly + 2) * BXS + lx0 + HXS;
      if constexpr (VEC == 4) {
        TM a[4], b[4];
        load_as<TS, TM, 4>(hp - 4, a);
        load_as<TS, TM, 4>(hp + 4, b);
        const TM e[8] = {a[2], a[3], c[0], c[1], c[2], c[3], b[0], b[1]};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          m2[j] = e[j]; m1[j] = e[j + 1]; p1[j] = e[j + 3]; p2[j] = e[j + 4];
        }
      } else if constexpr (VEC == 2) {
        TM a[2], b[2];
        load_as<TS, TM, 2>(hp - 2, a);
        load_as<TS, TM, 2>(hp + 2, b);
        m2[0] = a[0]; m1[0] = a[1]; p1[0] = c[1]; p2[0] = b[0];
        m2[1] = a[1]; m1[1] = c[0]; p1[1] = b[0]; p2[1] = b[1];
      } else {
        m2[0] = (TM)hp[-2]; m1[0] = (TM)hp[-1]; p1[0] = (TM)hp[1]; p2[0] = (TM)hp[2];
      }
    } else if constexpr (VEC == 4) {
      // the two points each side come from the neighbouring lanes, or from the
      // halo columns for the first and last lane
      TM pc = shfl_up1(c[2], 1), pd = shfl_up1(c[3], 1);
      TM na = shfl_dn1(c[0], 1), nb = shfl_dn1(c[1], 1);
      if (lane == 0) {
        TM hv[2];
        Consumer::template comb_n<2>(base, cf, -2, ly, hv);
        pc = hv[0]; pd = hv[1];
      } else if (lane == 31) {
        TM hv[2];
        Consumer::template comb_n<2>(base, cf, TX, ly, hv);
        na = hv[0]; nb = hv[1];
      }
      const TM e[8] = {pc, pd, c[0], c[1], c[2], c[3], na, nb};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        m2[j] = e[j]; m1[j] = e[j + 1]; p1[j] = e[j + 3]; p2[j] = e[j + 4];
      }
    } else if constexpr (VEC == 2) {
      TM pa = shfl_up1(c[0], 1), pb = shfl_up1(c[1], 1);
      TM na = shfl_dn1(c[0], 1), nb = shfl_dn1(c[1], 1);
      if (lane == 0) {
        TM hv[2];
        comb(base, cf, -2, ly, hv);
        pa = hv[0]; pb = hv[1];
      } else if (lane == 31) {
        TM hv[2];
        comb(base, cf, TX, ly, hv);
        na = hv[0]; nb = hv[1];
      }
      m2[0] = pa; m1[0] = pb; p1[0] = c[1]; p2[0] = na;
      m2[1] = pb; m1[1] = c[0]; p1[1] = na; p2[1] = nb;
    } else {
      TM hv[1] = {c[0]};
      if (lane < 2) comb(base, cf, lane - 2, ly, hv);
      else if (lane >= 30) comb(base, cf, TX + lane - 30, ly, hv);
      const TM up2 = shfl_up1(c[0], 2), up1 = shfl_up1(c[0], 1);
      const TM dn2 = shfl_dn1(c[0], 2), dn1 = shfl_dn1(c[0], 1);
      const TM h1 = shfl_idx(hv[0], 1), h30 = shfl_idx(hv[0], 30);
      m2[0] = lane < 2 ? hv[0] : up2;
      m1[0] = lane == 0 ? h1 : up1;
      p2[0] = lane >= 30 ? hv[0] : dn2;
      p1[0] = lane == 31 ? h30 : dn1;
    }
  }

  static __device__ __forceinline__ TM lap_g(const Coef<TM> &cf, TM P0, TM xm2, TM xm1, TM xp1,
                                             TM xp2, TM ym2, TM ym1, TM yp1, TM yp2, TM zm2,
                                             TM zm1, TM zp1, TM zp2, TM Q) {
    TM s1, s2;
    if constexpr (C::DIFF) {
      s1 = ((xm1 - P0) + (xp1 - P0)) + (((ym1 - P0) + (yp1 - P0)) + ((zm1 - P0) + (zp1 - P0)));
      s2 = ((xm2 - P0) + (xp2 - P0)) + (((ym2 - P0) + (yp2 - P0)) + ((zm2 - P0) + (zp2 - P0)));
    } else {
      s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
      s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
    }
    TM g = fmaT(cf.nlam * (P0 * P0), P0, cf.m3 * Q);
    g = fmaT(cf.ccen, P0, g);
    g = fmaT(cf.cm12, s2, g);
    return fmaT(cf.c43, s1, g);
  }

  static __device__ __forceinline__ void run(const StageParams &prm, uint64_t *full,
                                             uint64_t *empty, const unsigned char *ring,
                                             volatile int *abort_flag, int warp, int lane) {
    constexpr int RING = C::RING;
    const int nitems = *prm.nitems;
    const int lx0 = lane * VEC, ly0 = warp * VY;
    int slot = 0;
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      const WorkItem w = prm.items[it];
      Desc *d = prm.descs + w.x;
      if (!item_active<S>(d, prm.k, warp == 0 && lane == 0)) continue;
      const long long n = d->n_base + prm.k;
      Coef<TM> cf;
      {
        Coef<TM> c0;
        if (lane == 0) c0 = stage_coef<C>(d, n);
        const TM *src = reinterpret_cast<const TM *>(&c0);
        TM *dst = reinterpret_cast<TM *>(&cf);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(Coef<TM>) / sizeof(TM)); ++i) dst[i] = shfl_idx(src[i], 0);
      }
      // ---- everything the item needs from the descriptor, held in registers
      const int N = d->N;
      const bool periodic = d->bc == 1;
      const int set = (int)(n & 1);
      const int so = set ^ 1;
      const int x0 = (w.y & 0xffff) * TX, y0 = (w.y >> 16) * C::TY;
      const int z0 = w.z, len = w.w, nplanes = len + 4;
      const bool ragged = x0 + TX > N;
      const int x = x0 + lx0;
      // periodic ghost copies are written only by the lanes / rows next to a wrap
      const bool lane_edge = periodic && (x < 2 || x + VEC > N - 2);
      const int64_t pitch_s = d->pitch_s, plane_s = d->plane_s;
      const int64_t pitch_g = d->pitch_g, plane_g = d->plane_g;
      const int64_t row_s = (int64_t)(y0 + ly0 + 2) * pitch_s + HXS + x;  // row r: + r pitch
      const int64_t row_g = (int64_t)(y0 + ly0 + 2) * pitch_g + HXG + x;
      const bool xok = x < N;
      (void)len;
      // outputs
      TG *outG = nullptr;
      TS *outP = nullptr, *outQ = nullptr, *outPL = nullptr, *outQL = nullptr;
      if constexpr (S <= 3) outG = reinterpret_cast<TG *>(d->f[S == 1 ? F_G1 : (S == 2 ? F_G2 : F_G3)]);
      if constexpr (S == 4) {
        outP = reinterpret_cast<TS *>(d->f[F_P0 + so]);
        outQ = reinterpret_cast<TS *>(d->f[F_Q0 + so]);
        if constexpr (C::KAHAN) {
          outPL = reinterpret_cast<TS *>(d->f[F_PLO0 + so]);
          outQL = reinterpret_cast<TS *>(d->f[F_QLO0 + so]);
        }
      }
      bool rok[VY];
#pragma unroll
      for (int r = 0; r < VY; ++r) rok[r] = xok && (y0 + ly0 + r < N);

      TM win[5][VY][VEC];
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int r = 0; r < VY; ++r)
#pragma unroll
          for (int j = 0; j < VEC; ++j) win[a][r][j] = (TM)0;
      TM run_max = (TM)0;

      for (int m = 0; m < nplanes; ++m) {
        if (!mbar_wait_bounded(&full[slot], phase)) {
          *abort_flag = 1;
          atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
          return;
        }
        if (*abort_flag) return;
        const unsigned char *base = ring + slot * C::SLOT_BYTES;
        // own rows at plane z0 - 2 + m enter the window
#pragma unroll
        for (int r = 0; r < VY; ++r) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < VEC; ++j) win[a][r][j] = win[a + 1][r][j];
          comb(base, cf, lx0, ly0 + r, win[4][r]);
        }
        const int s2 = slot >= 2 ? slot - 2 : slot + RING - 2;  // slot of plane m - 2
        if (m >= 4) {
          // ---- output plane z0 + m - 4, loaded as plane m - 2
          const int z = z0 + m - 4;
          const unsigned char *b2 = ring + s2 * C::SLOT_BYTES;
          TM R[VY + 4][VEC];  // rows ly0-2 .. ly0+VY+1 of P at plane z
          comb(b2, cf, lx0, ly0 - 2, R[0]);
          comb(b2, cf, lx0, ly0 - 1, R[1]);
          comb(b2, cf, lx0, ly0 + VY, R[VY + 2]);
          comb(b2, cf, lx0, ly0 + VY + 1, R[VY + 3]);
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int j = 0; j < VEC; ++j) R[r + 2][j] = win[2][r][j];
#pragma unroll
          for (int r = 0; r < VY; ++r) {
            const int ly = ly0 + r;
            const int y = y0 + ly;
            TM m2[VEC], m1[VEC], p1[VEC], p2[VEC];
            xnb(b2, cf, lane, lx0, ly, win[2][r], m2, m1, p1, p2);
            const int hoff = (ly + 2) * BXS + lx0 + HXS;
            const int ioff = ly * TX + lx0;
            // point-only inputs from the interior tiles
            TM cur[NI > 0 ? NI : 1][VEC];
            if constexpr (S == 1) {
              load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2 + C::OFF_IS) + ioff, cur[0]);
            } else {
              const TG *ig = reinterpret_cast<const TG *>(b2 + C::OFF_IG) + ioff;
              load_as<TG, TM, VEC>(ig, cur[0]);  // S2: G1, S3: G2, S4: G1
              if constexpr (S == 4) {
                load_as<TG, TM, VEC>(ig + C::IG_BYTES / (int)sizeof(TG), cur[1]);  // G3
                if constexpr (C::KAHAN) {
                  const TS *is = reinterpret_cast<const TS *>(b2 + C::OFF_IS) + ioff;
                  load_as<TS, TM, VEC>(is, cur[2]);
                  load_as<TS, TM, VEC>(is + C::IS_BYTES / (int)sizeof(TS), cur[3]);
                }
              }
            }
            TM Q[VEC], qS[VEC];
            if constexpr (S == 1) {
#pragma unroll
              for (int j = 0; j < VEC; ++j) Q[j] = cur[0][j];
            } else {
              load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2 + C::HS_BYTES) + hoff, qS);
              // S2: q + dt/2 G1, S3: q + dt/2 G2, S4: q + dt G3
              const int gi = (S == 4) ? 1 : 0;
#pragma unroll
              for (int j = 0; j < VEC; ++j) Q[j] = fmaT(cf.a1, cur[gi][j], qS[j]);
            }
            TM Gout[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j)
              Gout[j] = lap_g(cf, win[2][r][j], m2[j], m1[j], p1[j], p2[j], R[r][j], R[r + 1][j],
                              R[r + 3][j], R[r + 4][j], win[0][r][j], win[1][r][j], win[3][r][j],
                              win[4][r][j], Q[j]);
            if (!rok[r]) continue;
            const bool edge = lane_edge || (periodic && (y < 2 || y >= N - 2));
            if constexpr (S <= 3) {
              TG *row = outG + ((int64_t)z * plane_g + row_g + r * pitch_g - x);
              store_point<TG, TM, VEC>(row, pitch_g, N, ragged, edge, x, y, Gout);
            } else {
              // RK4 combine (Sec. 2.1): p' = p + dt q + dt^2/6 (G1 + G2 + G3),
              //                         q' = q + dt/6 (G1 + 2 G2 + 2 G3 + G4)
              TM pS[VEC], G2h[VEC];
              load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2) + hoff, pS);
              load_as<TG, TM, VEC>(reinterpret_cast<const TG *>(b2 + C::OFF_HG) +
                                       (ly + 2) * BXG + lx0 + HXG, G2h);
              TM pn[VEC], qn[VEC], pl[VEC], ql[VEC];
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                const TM g1 = cur[0][j], g3 = cur[1][j];
                const TM dp = fmaT(cf.b6, (g1 + G2h[j]) + g3, cf.a1 * qS[j]);
                const TM dq = cf.d6 * ((g1 + Gout[j]) + (TM)2 * (G2h[j] + g3));
                if constexpr (C::KAHAN) {
                  two_sum(pS[j], dp + cur[2][j], pn[j], pl[j]);
                  two_sum(qS[j], dq + cur[3][j], qn[j], ql[j]);
                } else {
                  pn[j] = pS[j] + dp;
                  qn[j] = qS[j] + dq;
                }
                if (x + j < N) {
                  const TM a = pn[j] < (TM)0 ? -pn[j] : pn[j];
                  // NaN and overflow both read as +inf in the running max
                  run_max = (a <= run_max) ? run_max : ((a == a) ? a : (TM)INFINITY);
                }
              }
              const int64_t off = (int64_t)z * plane_s + row_s + r * pitch_s - x;
              store_point<TS, TM, VEC>(outP + off, pitch_s, N, ragged, edge, x, y, pn);
              store_point<TS, TM, VEC>(outQ + off, pitch_s, N, ragged, edge, x, y, qn);
              if constexpr (C::KAHAN) {
                store_point<TS, TM, VEC>(outPL + off, pitch_s, N, ragged, edge, x, y, pl);
                store_point<TS, TM, VEC>(outQL + off, pitch_s, N, ragged, edge, x, y, ql);
              }
            }
          }
        }
        // release the slots this warp no longer needs
        __syncwarp();
        if (lane == 0) {
          if (m < 2 || m >= nplanes - 2) mbar_arrive(&empty[slot]);
          if (m >= 4) mbar_arrive(&empty[s2]);
        }
        if (++slot == RING) { slot = 0; phase ^= 1u; }
      }
      if constexpr (S == 4) {
        double v = (double)run_max;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMax(d->maxabs + prm.k, (unsigned long long)__double_as_longlong(v));
      }
    }
  }
};

// Coefficients of a fused pair of stages, formed in double precision.
template <class TM>
struct PairCoef {
  TM c43a, cm12a, ccena;  // stencil coefficients of the first stage of the pair
  TM c43b, cm12b, ccenb;  // and of the second
  TM nlam, m3;
  TM aq, ag;              // Pa = p + aq q + ag G1          (pair 3+4)
  TM bq, bg;              // Pb = p + bq q + bg G2          (pair 1+2: bg = 0)
  TM qa;                  // Qa = q + qa G2                 (pair 3+4)
  TM qb;                  // Qb = q + qb * (first stage's G)
  TM b6, d6, dt;          // RK4 combine (pair 3+4)
};

template <class C>
__device__ __forceinline__ PairCoef<typename C::TM> pair_coef(const Desc *d, long long n) {
  using TM = typename C::TM;
  const bool second = C::S == 6;
  const double dt = d->dt;
  const double tn = d->t0 + (double)n * dt;
  const double ta = second ? tn + 0.5 * dt : tn;        // stage 3 | stage 1
  const double tb = second ? tn + dt : tn + 0.5 * dt;   // stage 4 | stage 2
  const double ca = exp(-2.0 * ta) * d->inv_h2, cb = exp(-2.0 * tb) * d->inv_h2;
  PairCoef<TM> k;
  k.c43a = (TM)(4.0 / 3.0 * ca); k.cm12a = (TM)(-ca / 12.0);
  k.ccena = C::DIFF ? (TM)d->mu2 : (TM)(d->mu2 - 7.5 * ca);
  k.c43b = (TM)(4.0 / 3.0 * cb); k.cm12b = (TM)(-cb / 12.0);
  k.ccenb = C::DIFF ? (TM)d->mu2 : (TM)(d->mu2 - 7.5 * cb);
  k.nlam = (TM)(-d->lambda);
  k.m3 = (TM)(-3.0);
  k.aq = (TM)(second ? 0.5 * dt : 0.0);
  k.ag = (TM)(second ? 0.25 * dt * dt : 0.0);
  k.bq = (TM)(second ? dt : 0.5 * dt);
  k.bg = (TM)(second ? 0.5 * dt * dt : 0.0);
  k.qa = (TM)(second ? 0.5 * dt : 0.0);
  k.qb = (TM)(second ? dt : 0.5 * dt);
  k.b6 = (TM)(dt * dt / 6.0);
  k.d6 = (TM)(dt / 6.0);
  k.dt = (TM)dt;
  return k;
}

template <class TM>
__device__ __forceinline__ TM lap_g2(TM c43, TM cm12, TM ccen, TM nlam, TM m3, bool diff, TM P0,
                                     TM xm2, TM xm1, TM xp1, TM xp2, TM ym2, TM ym1, TM yp1,
                                     TM yp2, TM zm2, TM zm1, TM zp1, TM zp2, TM Q) {
  TM s1, s2;
  if (diff) {
    s1 = ((xm1 - P0) + (xp1 - P0)) + (((ym1 - P0) + (yp1 - P0)) + ((zm1 - P0) + (zp1 - P0)));
    s2 = ((xm2 - P0) + (xp2 - P0)) + (((ym2 - P0) + (yp2 - P0)) + ((zm2 - P0) + (zp2 - P0)));
  } else {
    s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
    s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
  }
  TM g = fmaT(nlam * (P0 * P0), P0, m3 * Q);
  g = fmaT(ccen, P0, g);
  g = fmaT(cm12, s2, g);
  return fmaT(c43, s1, g);
}

// Two RK stages per launch.  Pair 1+2: G1 = G(t, p, q) and
// G2 = G(t + dt/2, p + dt/2 q, q + dt/2 G1) need p and q (with halo) only, and
// G1 enters G2 at the point.  Pair 3+4: G3 = G(t + dt/2, p + dt/2 q + dt^2/4 G1,
// q + dt/2 G2) and G4 = G(t + dt, p + dt q + dt^2/2 G2, q + dt G3) need p, q,
// G1, G2 (with halo) and G3 only at the point, so G3 never leaves the SM; the
// RK4 combine follows.  Both stage arguments of a pair are formed from the same
// ring tiles.
template <class C>
struct PairConsumer {
  using TS = typename C::TS;
  using TG = typename C::TG;
  using TM = typename C::TM;
  static constexpr int S = C::S, VEC = C::VEC, VY = C::VY, TX = C::TX;
  static constexpr int BXS = C::BXS, BXG = C::BXG, HXS = C::HXS, HXG = C::HXG;

  // Both stage arguments at n consecutive positions from (lx, ly).
  template <int n>
  static __device__ __forceinline__ void comb2(const unsigned char *base, const PairCoef<TM> &k,
                                               int lx, int ly, TM (&pa)[n], TM (&pb)[n]) {
    TM pv[n], qv[n];
    load_as<TS, TM, n>(reinterpret_cast<const TS *>(base) + (ly + 2) * BXS + lx + HXS, pv);
    load_as<TS, TM, n>(reinterpret_cast<const TS *>(base + C::HS_BYTES) + (ly + 2) * BXS + lx + HXS, qv);
    if constexpr (S == 5) {
#pragma unroll
      for (int j = 0; j < n; ++j) { pa[j] = pv[j]; pb[j] = fmaT(k.bq, qv[j], pv[j]); }
    } else {
      TM g1[n], g2[n];
      const TG *hg = reinterpret_cast<const TG *>(base + C::OFF_HG) + (ly + 2) * BXG + lx + HXG;
      load_as<TG, TM, n>(hg, g1);
      load_as<TG, TM, n>(hg + C::HG_BYTES / (int)sizeof(TG), g2);
#pragma unroll
      for (int j = 0; j < n; ++j) {
        pa[j] = fmaT(k.ag, g1[j], fmaT(k.aq, qv[j], pv[j]));
        pb[j] = fmaT(k.bg, g2[j], fmaT(k.bq, qv[j], pv[j]));
      }
    }
  }

  // x neighbours of both stage arguments for the lane's VEC points in row ly.
  static __device__ __forceinline__ void xnb2(const unsigned char *base, const PairCoef<TM> &k,
                                              int lane, int ly, const TM (&ca)[VEC],
                                              const TM (&cb)[VEC], TM (&ea)[VEC + 4],
                                              TM (&eb)[VEC + 4]) {
    // e[i] = P at x - 2 + i, i = 0 .. VEC + 3
    if constexpr (VEC >= 2) {
      TM la0 = shfl_up1(ca[VEC - 2], 1), la1 = shfl_up1(ca[VEC - 1], 1);
      TM lb0 = shfl_up1(cb[VEC - 2], 1), lb1 = shfl_up1(cb[VEC - 1], 1);
      TM ra0 = shfl_dn1(ca[0], 1), ra1 = shfl_dn1(ca[1], 1);
      TM rb0 = shfl_dn1(cb[0], 1), rb1 = shfl_dn1(cb[1], 1);
      if (lane == 0) {
        TM ha[2], hb[2];
        comb2<2>(base, k, -2, ly, ha, hb);
        la0 = ha[0]; la1 = ha[1]; lb0 = hb[0]; lb1 = hb[1];
      } else if (lane == 31) {
        TM ha[2], hb[2];
        comb2<2>(base, k, TX, ly, ha, hb);
        ra0 = ha[0]; ra1 = ha[1]; rb0 = hb[0]; rb1 = hb[1];
      }
      ea[0] = la0; ea[1] = la1; eb[0] = lb0; eb[1] = lb1;
#pragma unroll
      for (int j = 0; j < VEC; ++j) { ea[2 + j] = ca[j]; eb[2 + j] = cb[j]; }
      ea[VEC + 2] = ra0; ea[VEC + 3] = ra1; eb[VEC + 2] = rb0; eb[VEC + 3] = rb1;
    } else {
      TM ha[1] = {ca[0]}, hb[1] = {cb[0]};
      if (lane < 2) comb2<1>(base, k, lane - 2, ly, ha, hb);
      else if (lane >= 30) comb2<1>(base, k, TX + lane - 30, ly, ha, hb);
      const TM a_u2 = shfl_up1(ca[0], 2), a_u1 = shfl_up1(ca[0], 1);
      const TM a_d2 = shfl_dn1(ca[0], 2), a_d1 = shfl_dn1(ca[0], 1);
      const TM b_u2 = shfl_up1(cb[0], 2), b_u1 = shfl_up1(cb[0], 1);
      const TM b_d2 = shfl_dn1(cb[0], 2), b_d1 = shfl_dn1(cb[0], 1);
      const TM a_h1 = shfl_idx(ha[0], 1), a_h30 = shfl_idx(ha[0], 30);
      const TM b_h1 = shfl_idx(hb[0], 1), b_h30 = shfl_idx(hb[0], 30);
      ea[0] = lane < 2 ? ha[0] : a_u2;
      ea[1] = lane == 0 ? a_h1 : a_u1;
      ea[2] = ca[0];
      ea[3] = lane == 31 ? a_h30 : a_d1;
      ea[4] = lane >= 30 ? ha[0] : a_d2;
      eb[0] = lane < 2 ? hb[0] : b_u2;
      eb[1] = lane == 0 ? b_h1 : b_u1;
      eb[2] = cb[0];
      eb[3] = lane == 31 ? b_h30 : b_d1;
      eb[4] = lane >= 30 ? hb[0] : b_d2;
    }
  }

  static __device__ __forceinline__ void run(const StageParams &prm, uint64_t *full,
                                             uint64_t *empty, const unsigned char *ring,
                                             volatile int *abort_flag, int warp, int lane) {
    constexpr int RING = C::RING;
    const int nitems = *prm.nitems;
    const int lx0 = lane * VEC, ly0 = warp * VY;
    int slot = 0;
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      const WorkItem w = prm.items[it];
      Desc *d = prm.descs + w.x;
      if (!item_active<S>(d, prm.k, warp == 0 && lane == 0)) continue;
      const long long n = d->n_base + prm.k;
      PairCoef<TM> k;
      {
        PairCoef<TM> c0;
        if (lane == 0) c0 = pair_coef<C>(d, n);
        const TM *src = reinterpret_cast<const TM *>(&c0);
        TM *dst = reinterpret_cast<TM *>(&k);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(PairCoef<TM>) / sizeof(TM)); ++i)
          dst[i] = shfl_idx(src[i], 0);
      }
      const int N = d->N;
      const bool periodic = d->bc == 1;
      const int set = (int)(n & 1);
      const int so = set ^ 1;
      const int x0 = (w.y & 0xffff) * TX, y0 = (w.y >> 16) * C::TY;
      const int z0 = w.z, nplanes = w.w + 4;
      const bool ragged = x0 + TX > N;
      const int x = x0 + lx0;
      const bool lane_edge = periodic && (x < 2 || x + VEC > N - 2);
      const int64_t pitch_s = d->pitch_s, plane_s = d->plane_s;
      const int64_t pitch_g = d->pitch_g, plane_g = d->plane_g;
      const int64_t row_s = (int64_t)(y0 + ly0 + 2) * pitch_s + HXS + x;
      const int64_t row_g = (int64_t)(y0 + ly0 + 2) * pitch_g + HXG + x;
      const bool xok = x < N;
      TG *outG1 = nullptr, *outG2 = nullptr;
      TS *outP = nullptr, *outQ = nullptr, *outPL = nullptr, *outQL = nullptr;
      if constexpr (S == 5) {
        outG1 = reinterpret_cast<TG *>(d->f[F_G1]);
        outG2 = reinterpret_cast<TG *>(d->f[F_G2]);
      } else {
        outP = reinterpret_cast<TS *>(d->f[F_P0 + so]);
        outQ = reinterpret_cast<TS *>(d->f[F_Q0 + so]);
        if constexpr (C::KAHAN) {
          outPL = reinterpret_cast<TS *>(d->f[F_PLO0 + so]);
          outQL = reinterpret_cast<TS *>(d->f[F_QLO0 + so]);
        }
      }
      bool rok[VY];
#pragma unroll
      for (int r = 0; r < VY; ++r) rok[r] = xok && (y0 + ly0 + r < N);

      TM wa[5][VY][VEC], wb[5][VY][VEC];
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int r = 0; r < VY; ++r)
#pragma unroll
          for (int j = 0; j < VEC; ++j) { wa[a][r][j] = (TM)0; wb[a][r][j] = (TM)0; }
      TM run_max = (TM)0;

      for (int m = 0; m < nplanes; ++m) {
        if (!mbar_wait_bounded(&full[slot], phase)) {
          *abort_flag = 1;
          atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
          return;
        }
        if (*abort_flag) return;
        const unsigned char *base = ring + slot * C::SLOT_BYTES;
#pragma unroll
        for (int r = 0; r < VY; ++r) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < VEC; ++j) { wa[a][r][j] = wa[a + 1][r][j]; wb[a][r][j] = wb[a + 1][r][j]; }
          comb2<VEC>(base, k, lx0, ly0 + r, wa[4][r], wb[4][r]);
        }
        const int s2 = slot >= 2 ? slot - 2 : slot + RING - 2;
        if (m >= 4) {
          const int z = z0 + m - 4;
          const unsigned char *b2 = ring + s2 * C::SLOT_BYTES;
          TM Ra[VY + 4][VEC], Rb[VY + 4][VEC];
          comb2<VEC>(b2, k, lx0, ly0 - 2, Ra[0], Rb[0]);
          comb2<VEC>(b2, k, lx0, ly0 - 1, Ra[1], Rb[1]);
          comb2<VEC>(b2, k, lx0, ly0 + VY, Ra[VY + 2], Rb[VY + 2]);
          comb2<VEC>(b2, k, lx0, ly0 + VY + 1, Ra[VY + 3], Rb[VY + 3]);
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int j = 0; j < VEC; ++j) { Ra[r + 2][j] = wa[2][r][j]; Rb[r + 2][j] = wb[2][r][j]; }
#pragma unroll
          for (int r = 0; r < VY; ++r) {
            const int ly = ly0 + r;
            const int y = y0 + ly;
            TM ea[VEC + 4], eb[VEC + 4];
            xnb2(b2, k, lane, ly, wa[2][r], wb[2][r], ea, eb);
            const int hoff = (ly + 2) * BXS + lx0 + HXS;
            TM qS[VEC];
            load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2 + C::HS_BYTES) + hoff, qS);
            TM Ga[VEC], Gb[VEC], g1[VEC], g2[VEC];
            if constexpr (S == 6) {
              const TG *hg = reinterpret_cast<const TG *>(b2 + C::OFF_HG) + (ly + 2) * BXG + lx0 + HXG;
              load_as<TG, TM, VEC>(hg, g1);
              load_as<TG, TM, VEC>(hg + C::HG_BYTES / (int)sizeof(TG), g2);
            }
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
              const TM Qa = (S == 6) ? fmaT(k.qa, g2[j], qS[j]) : qS[j];
              Ga[j] = lap_g2(k.c43a, k.cm12a, k.ccena, k.nlam, k.m3, C::DIFF, wa[2][r][j], ea[j],
                             ea[j + 1], ea[j + 3], ea[j + 4], Ra[r][j], Ra[r + 1][j], Ra[r + 3][j],
                             Ra[r + 4][j], wa[0][r][j], wa[1][r][j], wa[3][r][j], wa[4][r][j], Qa);
              const TM Qb = fmaT(k.qb, Ga[j], qS[j]);
              Gb[j] = lap_g2(k.c43b, k.cm12b, k.ccenb, k.nlam, k.m3, C::DIFF, wb[2][r][j], eb[j],
                             eb[j + 1], eb[j + 3], eb[j + 4], Rb[r][j], Rb[r + 1][j], Rb[r + 3][j],
                             Rb[r + 4][j], wb[0][r][j], wb[1][r][j], wb[3][r][j], wb[4][r][j], Qb);
            }
            if (!rok[r]) continue;
            const bool edge = lane_edge || (periodic && (y < 2 || y >= N - 2));
            if constexpr (S == 5) {
              const int64_t off = (int64_t)z * plane_g + row_g + r * pitch_g - x;
              store_point<TG, TM, VEC>(outG1 + off, pitch_g, N, ragged, edge, x, y, Ga);
              store_point<TG, TM, VEC>(outG2 + off, pitch_g, N, ragged, edge, x, y, Gb);
            } else {
              // RK4 combine (Sec. 2.1) with G3 = Ga, G4 = Gb
              TM pS[VEC], lp[VEC], lq[VEC];
              load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(b2) + hoff, pS);
              if constexpr (C::KAHAN) {
                const TS *is = reinterpret_cast<const TS *>(b2 + C::OFF_IS) + ly * TX + lx0;
                load_as<TS, TM, VEC>(is, lp);
                load_as<TS, TM, VEC>(is + C::IS_BYTES / (int)sizeof(TS), lq);
              }
              TM pn[VEC], qn[VEC], pl[VEC], ql[VEC];
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                const TM dp = fmaT(k.b6, (g1[j] + g2[j]) + Ga[j], k.dt * qS[j]);
                const TM dq = k.d6 * ((g1[j] + Gb[j]) + (TM)2 * (g2[j] + Ga[j]));
                if constexpr (C::KAHAN) {
                  two_sum(pS[j], dp + lp[j], pn[j], pl[j]);
                  two_sum(qS[j], dq + lq[j], qn[j], ql[j]);
                } else {
                  pn[j] = pS[j] + dp;
                  qn[j] = qS[j] + dq;
                }
                if (x + j < N) {
                  const TM av = pn[j] < (TM)0 ? -pn[j] : pn[j];
                  run_max = (av <= run_max) ? run_max : ((av == av) ? av : (TM)INFINITY);
                }
              }
              const int64_t off = (int64_t)z * plane_s + row_s + r * pitch_s - x;
              store_point<TS, TM, VEC>(outP + off, pitch_s, N, ragged, edge, x, y, pn);
              store_point<TS, TM, VEC>(outQ + off, pitch_s, N, ragged, edge, x, y, qn);
              if constexpr (C::KAHAN) {
                store_point<TS, TM, VEC>(outPL + off, pitch_s, N, ragged, edge, x, y, pl);
                store_point<TS, TM, VEC>(outQL + off, pitch_s, N, ragged, edge, x, y, ql);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) {
          if (m < 2 || m >= nplanes - 2) mbar_arrive(&empty[slot]);
          if (m >= 4) mbar_arrive(&empty[s2]);
        }
        if (++slot == RING) { slot = 0; phase ^= 1u; }
      }
      if constexpr (S == 6) {
        double v = (double)run_max;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMax(d->maxabs + prm.k, (unsigned long long)__double_as_longlong(v));
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
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (warp == C::NW) {
    if (lane == 0) produce<C>(prm, full, empty, ring, abort_flag);
  } else if constexpr (C::PAIR) {
    PairConsumer<C>::run(prm, full, empty, ring, abort_flag, warp, lane);
  } else {
    Consumer<C>::run(prm, full, empty, ring, abort_flag, warp, lane);
  }
}

}  // namespace hbe
