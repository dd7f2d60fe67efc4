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
//   * a block owns a TX x TY tile in x-y and marches along z over a chunk;
//   * each z-plane of every input field is brought into a shared-memory ring
//     by the TMA unit (cp.async.bulk.tensor, completion on an mbarrier); the
//     fields that enter the stencil come with a 2-row / HX-column halo, zero
//     filled by the TMA unit outside the box in z (Dirichlet);
//   * the stage argument P is formed once per loaded point: for the thread's
//     own column it enters a 5-deep register window (z-2..z+2), for the x-y
//     halo ring it is written with the own values to a shared P-plane;
//   * the 13-point stencil reads x/y neighbours from the P-plane (128-bit
//     loads) and z neighbours from registers; each thread owns VEC consecutive
//     x points (16 bytes of the math type), stores are 128-bit where possible.
//   * one __syncthreads per plane; the slot of plane m-3 is refilled right
//     after it, so up to RING-3 planes are in flight ahead of the consumer.
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

template <class PR, int TX_, int TY_, int BUDGET_, int S_>
struct StageCfg {
  using TS = typename PR::TS;
  using TG = typename PR::TG;
  using TM = typename PR::TM;
  static constexpr bool KAHAN = PR::KAHAN;
  static constexpr bool DIFF = PR::DIFF;
  static constexpr int S = S_;
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int VEC = 16 / (int)sizeof(TM);
  static constexpr int TPR = TX / VEC;
  static constexpr int THREADS = TPR * TY;
  static constexpr int HXS = 16 / (int)sizeof(TS);
  static constexpr int HXG = 16 / (int)sizeof(TG);
  static constexpr int HXM = 16 / (int)sizeof(TM);
  static constexpr int BY = TY + 4;
  static constexpr int BXS = TX + 2 * HXS, BXG = TX + 2 * HXG, BXM = TX + 2 * HXM;
  // ring slot composition
  static constexpr int NHS = (S == 1) ? 1 : 2;                           // p [, q]
  static constexpr int NHG = (S >= 3) ? 1 : 0;                           // G1 (S3) / G2 (S4)
  static constexpr int NIS = (S == 1) ? 1 : ((S == 4 && KAHAN) ? 2 : 0); // q (S1) / plo, qlo (S4)
  static constexpr int NIG = (S == 1) ? 0 : ((S == 4) ? 2 : 1);          // G1 | G2 | G1, G3
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
  static constexpr int PPLANE_BYTES = align128(BY * BXM * (int)sizeof(TM));
  static constexpr int HEADER = 256;  // mbarriers + coefficients + flags
  static constexpr int RING = cmax(4, cmin(12, (BUDGET_ - HEADER - 2 * PPLANE_BYTES) / SLOT_BYTES));
  static constexpr int SMEM = HEADER + 2 * PPLANE_BYTES + RING * SLOT_BYTES;
  static constexpr int NHALO = 4 * TPR + 2 * TY;  // halo vector items per plane
  static_assert(TX % VEC == 0, "tile width must hold whole vectors");
  static_assert(HXS >= 2 && HXG >= 2, "halo of 2 needed");
  static_assert(TX + 2 * HXG <= 256 && BY <= 256, "TMA box limit");
  static_assert(RING * 8 <= 128, "barrier area");
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
template <class T> struct VecIO;
template <> struct VecIO<float> {  // 4 floats = 16 bytes
  static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void store(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct VecIO<double> {  // 2 doubles = 16 bytes
  static __device__ __forceinline__ void load(const double *p, double (&v)[2]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    v[0] = a.x; v[1] = a.y;
  }
  static __device__ __forceinline__ void store(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};

// Load VEC values of storage type T at p (aligned) and widen to TM.
template <class T, class TM, int VEC>
__device__ __forceinline__ void load_as(const T *p, TM (&v)[VEC]) {
  if constexpr (sizeof(T) == sizeof(TM)) {
    VecIO<TM>::load(reinterpret_cast<const TM *>(p), v);
  } else {  // bfloat16 x 4 -> float x 4 (exact)
    static_assert(VEC == 4, "bf16 path uses float math");
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&raw.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&raw.y);
    v[0] = __low2float(a); v[1] = __high2float(a);
    v[2] = __low2float(b); v[3] = __high2float(b);
  }
}
template <class T, class TM>
__device__ __forceinline__ T narrow(TM v) {
  if constexpr (sizeof(T) == sizeof(TM)) return v;
  else return __float2bfloat16_rn(v);  // round to nearest even
}
template <class T, class TM, int VEC>
__device__ __forceinline__ void store_as(T *p, const TM (&v)[VEC]) {
  if constexpr (sizeof(T) == sizeof(TM)) {
    VecIO<TM>::store(reinterpret_cast<TM *>(p), v);
  } else {
    __nv_bfloat162 a, b;
    a.x = narrow<T>(v[0]); a.y = narrow<T>(v[1]);
    b.x = narrow<T>(v[2]); b.y = narrow<T>(v[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t *>(&a);
    raw.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
  }
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

// Store VEC values of a field at interior point (x, y, z) of the padded layout,
// masking x >= N and writing the periodic ghost copies.
template <class T, class TM, int VEC>
__device__ __forceinline__ void store_point(T *base, int pitch, int64_t plane, int hx, int N,
                                            bool periodic, int x, int y, int z,
                                            const TM (&v)[VEC]) {
  T *row = base + (int64_t)z * plane + (int64_t)(y + 2) * pitch + hx;
  if (x + VEC <= N) {
    store_as<T, TM, VEC>(row + x, v);
  } else {
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      if (x + j < N) row[x + j] = narrow<T>(v[j]);
  }
  if (periodic) {
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
template <class C>
__global__ void __launch_bounds__(C::THREADS)
    stage_kernel(const StageParams prm) {
  using TS = typename C::TS;
  using TG = typename C::TG;
  using TM = typename C::TM;
  constexpr int S = C::S, VEC = C::VEC, TX = C::TX, TY = C::TY, TPR = C::TPR;
  constexpr int RING = C::RING, BXM = C::BXM, HXM = C::HXM;
  constexpr int BXS = C::BXS, BXG = C::BXG, HXS = C::HXS, HXG = C::HXG;

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  Coef<TM> *coef = reinterpret_cast<Coef<TM> *>(smem + 128);
  int *flags = reinterpret_cast<int *>(smem + 240);   // [0] skip item, [1] abort
  static_assert(128 + sizeof(Coef<TM>) <= 240, "header layout");
  TM *pplane[2] = {reinterpret_cast<TM *>(smem + C::HEADER),
                   reinterpret_cast<TM *>(smem + C::HEADER + C::PPLANE_BYTES)};
  unsigned char *ring = smem + C::HEADER + 2 * C::PPLANE_BYTES;
  __shared__ double warp_max[32];

  const int tid = threadIdx.x;
  const int txt = tid % TPR, tyt = tid / TPR;
  const int lx0 = txt * VEC;

  if (tid == 0) {
    for (int r = 0; r < RING; ++r) mbar_init(&bars[r], 1);
    fence_barrier_init();
  }
  __syncthreads();

  uint32_t gplane = 0;  // planes consumed by this block so far (slot / phase bookkeeping)
  const int nitems = *prm.nitems;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = prm.items[it];
    Desc *d = prm.descs + w.x;
    // ---- per-item decisions and coefficients, by thread 0 (uniform via smem)
    if (tid == 0) {
      const long long n = d->n_base + prm.k;
      int skip = (n >= d->n_end) || (d->stop_k <= prm.k);
      if (S == 1 && !skip && prm.k > 0) {
        const double m = __longlong_as_double((long long)d->maxabs[prm.k - 1]);
        const bool nonfin = !(m <= 1.7976931348623157e308);
        if (nonfin || (d->stop_thr > 0.0 && m > d->stop_thr)) {
          atomicMin(&d->stop_k, (long long)prm.k);
          skip = 1;
        }
      }
      flags[0] = skip;
      flags[1] = 0;
      if (!skip) {
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
        if (S == 2) { cf.a1 = (TM)(0.5 * dt); cf.a2 = (TM)0; }
        if (S == 3) { cf.a1 = (TM)(0.5 * dt); cf.a2 = (TM)(0.25 * dt * dt); }
        if (S == 4) { cf.a1 = (TM)dt; cf.a2 = (TM)(0.5 * dt * dt); }
        if (S == 1) { cf.a1 = (TM)0; cf.a2 = (TM)0; }
        cf.b6 = (TM)(dt * dt / 6.0);
        cf.d6 = (TM)(dt / 6.0);
        *coef = cf;
        for (int t = 0; t < NUM_TMAPS; ++t) tmap_acquire(d->tmaps + t);
      }
    }
    __syncthreads();
    if (flags[0]) continue;
    const Coef<TM> cf = *coef;
    const int N = d->N;
    const bool periodic = d->bc == 1;
    const long long n = d->n_base + prm.k;
    const int set = (int)(n & 1);
    const int x0 = (w.y & 0xffff) * TX, y0 = (w.y >> 16) * TY;
    const int z0 = w.z, len = w.w;
    const int nplanes = len + 4;
    const CUtensorMap *tm = d->tmaps;

    // ---- TMA producer (thread 0): plane m of this item into its ring slot
    auto issue = [&](int m) {
      const uint32_t gp = gplane + (uint32_t)m;
      const int slot = (int)(gp % RING);
      uint64_t *bar = &bars[slot];
      unsigned char *base = ring + slot * C::SLOT_BYTES;
      int z = z0 - 2 + m;
      if (periodic) z = (z % N + N) % N;
      fence_proxy_async();
      mbar_expect_tx(bar, C::TX_BYTES);
      tma_load_3d(base, tm + (set ? TM_P_H1 : TM_P_H0), bar, x0, y0, z);
      if constexpr (C::NHS == 2)
        tma_load_3d(base + C::HS_BYTES, tm + (set ? TM_Q_H1 : TM_Q_H0), bar, x0, y0, z);
      if constexpr (C::NHG == 1)
        tma_load_3d(base + C::OFF_HG, tm + (S == 3 ? TM_G1_H : TM_G2_H), bar, x0, y0, z);
      if constexpr (S == 1)
        tma_load_3d(base + C::OFF_IS, tm + (set ? TM_Q_I1 : TM_Q_I0), bar, x0 + HXS, y0 + 2, z);
      if constexpr (S == 4 && C::KAHAN) {
        tma_load_3d(base + C::OFF_IS, tm + (set ? TM_PLO_I1 : TM_PLO_I0), bar, x0 + HXS, y0 + 2, z);
        tma_load_3d(base + C::OFF_IS + C::IS_BYTES, tm + (set ? TM_QLO_I1 : TM_QLO_I0), bar,
                    x0 + HXS, y0 + 2, z);
      }
      if constexpr (S == 2)
        tma_load_3d(base + C::OFF_IG, tm + TM_G1_I, bar, x0 + HXG, y0 + 2, z);
      if constexpr (S == 3)
        tma_load_3d(base + C::OFF_IG, tm + TM_G2_I, bar, x0 + HXG, y0 + 2, z);
      if constexpr (S == 4) {
        tma_load_3d(base + C::OFF_IG, tm + TM_G1_I, bar, x0 + HXG, y0 + 2, z);
        tma_load_3d(base + C::OFF_IG + C::IG_BYTES, tm + TM_G3_I, bar, x0 + HXG, y0 + 2, z);
      }
    };
    // P = stage argument at halo-tile position (row, col of the state tiles)
    auto combine_at = [&](const unsigned char *base, int lx, int ly, TM (&out)[VEC]) {
      const TS *hp = reinterpret_cast<const TS *>(base);
      load_as<TS, TM, VEC>(hp + (ly + 2) * BXS + lx + HXS, out);
      if constexpr (S >= 2) {
        TM qv[VEC];
        const TS *hq = reinterpret_cast<const TS *>(base + C::HS_BYTES);
        load_as<TS, TM, VEC>(hq + (ly + 2) * BXS + lx + HXS, qv);
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = fmaT(cf.a1, qv[j], out[j]);
      }
      if constexpr (S >= 3) {
        TM gv[VEC];
        const TG *hg = reinterpret_cast<const TG *>(base + C::OFF_HG);
        load_as<TG, TM, VEC>(hg + (ly + 2) * BXG + lx + HXG, gv);
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = fmaT(cf.a2, gv[j], out[j]);
      }
    };

    int issued = cmin(RING, nplanes);
    if (tid == 0)
      for (int m = 0; m < issued; ++m) issue(m);

    TM win[5][VEC];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int j = 0; j < VEC; ++j) win[a][j] = (TM)0;
    TM run_max = (TM)0;
    bool aborted = false;

    int consumed = 0;
    for (int m = 0; m < nplanes; ++m) {
      const uint32_t gp = gplane + (uint32_t)m;
      consumed = m + 1;
      const int slot = (int)(gp % RING);
      if (!mbar_wait_bounded(&bars[slot], (gp / RING) & 1u)) {
        flags[1] = 1;
        atomicOr(prm.err, (unsigned)DEV_ERR_TIMEOUT);
      }
      const unsigned char *base = ring + slot * C::SLOT_BYTES;
      // own column: P at plane z0-2+m enters the window
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int j = 0; j < VEC; ++j) win[a][j] = win[a + 1][j];
      combine_at(base, lx0, tyt, win[4]);
      const bool out = m >= 4;
      // slot of the output plane z0 + m - 4 (loaded as plane m - 2)
      const unsigned char *obase = ring + (int)((gp + (uint32_t)(2 * RING - 2)) % RING) * C::SLOT_BYTES;
      TM *pp = pplane[m & 1];
      if (out) {
        VecIO<TM>::store(pp + (tyt + 2) * BXM + HXM + lx0, win[2]);
        for (int hix = tid; hix < C::NHALO; hix += C::THREADS) {
          int lx, ly;
          if (hix < 4 * TPR) {
            const int r = hix / TPR;
            ly = (r < 2) ? r - 2 : TY + (r - 2);
            lx = (hix % TPR) * VEC;
          } else {
            const int h2 = hix - 4 * TPR;
            ly = h2 % TY;
            lx = (h2 / TY) ? TX : -VEC;
          }
          TM v[VEC];
          combine_at(obase, lx, ly, v);
          VecIO<TM>::store(pp + (ly + 2) * BXM + HXM + lx, v);
        }
      }
      __syncthreads();
      if (flags[1]) { aborted = true; break; }
      if (tid == 0 && m >= 3) {
        const int pn = m - 3 + RING;
        if (pn < nplanes) { issue(pn); issued = pn + 1; }
      }
      if (!out) continue;

      // ---- stencil at plane z = z0 + m - 4 for the thread's VEC points
      const int z = z0 + m - 4;
      const int x = x0 + lx0, y = y0 + tyt;
      const TM *prow = pp + (tyt + 2) * BXM + HXM + lx0;
      TM E[3 * VEC];
      {
        TM a[VEC], c[VEC];
        VecIO<TM>::load(prow - VEC, a);
        VecIO<TM>::load(prow + VEC, c);
#pragma unroll
        for (int j = 0; j < VEC; ++j) { E[j] = a[j]; E[VEC + j] = win[2][j]; E[2 * VEC + j] = c[j]; }
      }
      TM ym1[VEC], yp1[VEC], ym2[VEC], yp2[VEC];
      VecIO<TM>::load(prow - BXM, ym1);
      VecIO<TM>::load(prow + BXM, yp1);
      VecIO<TM>::load(prow - 2 * BXM, ym2);
      VecIO<TM>::load(prow + 2 * BXM, yp2);

      // pointwise inputs at the output plane
      TM Q[VEC], Gint0[VEC], Gint1[VEC], pS[VEC], qS[VEC], loP[VEC], loQ[VEC];
      {
        const TS *hp = reinterpret_cast<const TS *>(obase);
        const int hoff = (tyt + 2) * BXS + lx0 + HXS;
        if constexpr (S == 1) {
          load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(obase + C::OFF_IS) + tyt * TX + lx0, Q);
        } else {
          load_as<TS, TM, VEC>(reinterpret_cast<const TS *>(obase + C::HS_BYTES) + hoff, qS);
          const TG *ig = reinterpret_cast<const TG *>(obase + C::OFF_IG) + tyt * TX + lx0;
          load_as<TG, TM, VEC>(ig, Gint0);   // S2: G1, S3: G2, S4: G1
          if constexpr (S == 4) load_as<TG, TM, VEC>(ig + C::IG_BYTES / (int)sizeof(TG), Gint1);  // G3
          if constexpr (S == 2 || S == 3) {  // q + dt/2 G1 (S2), q + dt/2 G2 (S3)
#pragma unroll
            for (int j = 0; j < VEC; ++j) Q[j] = fmaT(cf.a1, Gint0[j], qS[j]);
          }
          if constexpr (S == 4) {
            load_as<TS, TM, VEC>(hp + hoff, pS);
#pragma unroll
            for (int j = 0; j < VEC; ++j) Q[j] = fmaT(cf.a1, Gint1[j], qS[j]);  // q + dt G3
            if constexpr (C::KAHAN) {
              const TS *is = reinterpret_cast<const TS *>(obase + C::OFF_IS) + tyt * TX + lx0;
              load_as<TS, TM, VEC>(is, loP);
              load_as<TS, TM, VEC>(is + C::IS_BYTES / (int)sizeof(TS), loQ);
            }
          }
        }
      }
      TM Gout[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const TM P0 = E[VEC + j];
        TM s1, s2;
        if constexpr (C::DIFF) {
          s1 = ((E[VEC + j - 1] - P0) + (E[VEC + j + 1] - P0)) +
               (((ym1[j] - P0) + (yp1[j] - P0)) + ((win[1][j] - P0) + (win[3][j] - P0)));
          s2 = ((E[VEC + j - 2] - P0) + (E[VEC + j + 2] - P0)) +
               (((ym2[j] - P0) + (yp2[j] - P0)) + ((win[0][j] - P0) + (win[4][j] - P0)));
        } else {
          s1 = ((E[VEC + j - 1] + E[VEC + j + 1]) + (ym1[j] + yp1[j])) + (win[1][j] + win[3][j]);
          s2 = ((E[VEC + j - 2] + E[VEC + j + 2]) + (ym2[j] + yp2[j])) + (win[0][j] + win[4][j]);
        }
        TM g = fmaT(cf.nlam * (P0 * P0), P0, cf.m3 * Q[j]);
        g = fmaT(cf.ccen, P0, g);
        g = fmaT(cf.cm12, s2, g);
        Gout[j] = fmaT(cf.c43, s1, g);
      }

      const bool yok = y < N;
      if constexpr (S <= 3) {
        if (yok && x < N) {
          TG *gbase = reinterpret_cast<TG *>(d->f[S == 1 ? F_G1 : (S == 2 ? F_G2 : F_G3)]);
          store_point<TG, TM, VEC>(gbase, d->pitch_g, d->plane_g, HXG, N, periodic, x, y, z, Gout);
        }
      } else {
        // RK4 combine (Sec. 2.1): p' = p + dt q + dt^2/6 (G1 + G2 + G3),
        //                         q' = q + dt/6 (G1 + 2 G2 + 2 G3 + G4)
        TM G2v[VEC];
        {
          const TG *hg = reinterpret_cast<const TG *>(obase + C::OFF_HG);
          load_as<TG, TM, VEC>(hg + (tyt + 2) * BXG + lx0 + HXG, G2v);
        }
        TM pn[VEC], qn[VEC], pl[VEC], ql[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          const TM dp = fmaT(cf.b6, (Gint0[j] + G2v[j]) + Gint1[j], cf.a1 * qS[j]);
          const TM dq = cf.d6 * ((Gint0[j] + Gout[j]) + (TM)2 * (G2v[j] + Gint1[j]));
          if constexpr (C::KAHAN) {
            two_sum(pS[j], dp + loP[j], pn[j], pl[j]);
            two_sum(qS[j], dq + loQ[j], qn[j], ql[j]);
          } else {
            pn[j] = pS[j] + dp;
            qn[j] = qS[j] + dq;
          }
        }
        if (yok && x < N) {
          const int so = set ? 0 : 1;  // write the other buffer set
          store_point<TS, TM, VEC>(reinterpret_cast<TS *>(d->f[F_P0 + so]), d->pitch_s,
                                   d->plane_s, HXS, N, periodic, x, y, z, pn);
          store_point<TS, TM, VEC>(reinterpret_cast<TS *>(d->f[F_Q0 + so]), d->pitch_s,
                                   d->plane_s, HXS, N, periodic, x, y, z, qn);
          if constexpr (C::KAHAN) {
            store_point<TS, TM, VEC>(reinterpret_cast<TS *>(d->f[F_PLO0 + so]), d->pitch_s,
                                     d->plane_s, HXS, N, periodic, x, y, z, pl);
            store_point<TS, TM, VEC>(reinterpret_cast<TS *>(d->f[F_QLO0 + so]), d->pitch_s,
                                     d->plane_s, HXS, N, periodic, x, y, z, ql);
          }
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            if (x + j < N) {
              const TM a = pn[j] < (TM)0 ? -pn[j] : pn[j];
              // NaN and overflow both read as +inf in the running max
              run_max = (a <= run_max) ? run_max : ((a == a) ? a : (TM)INFINITY);
            }
          }
        }
      }
    }
    if (aborted) {
      // let the copies already in flight land before the block exits
      if (tid == 0) {
        for (int m2 = consumed; m2 < issued; ++m2) {
          const uint32_t gp2 = gplane + (uint32_t)m2;
          (void)mbar_wait_bounded(&bars[gp2 % RING], (gp2 / RING) & 1u);
        }
      }
      return;
    }
    gplane += (uint32_t)nplanes;
    if constexpr (S == 4) {
      // block max of |p'| -> one atomicMax on the double bit pattern (non-negative)
      double v = (double)run_max;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((tid & 31) == 0) warp_max[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double mx = 0.0;
        for (int wi = 0; wi < (C::THREADS + 31) / 32; ++wi) mx = fmax(mx, warp_max[wi]);
        atomicMax(d->maxabs + prm.k, (unsigned long long)__double_as_longlong(mx));
      }
    }
  }
}

}  // namespace hbe
