// hbe_aux.cu -- kernels around the stage kernels: field packing, per-batch
// step bookkeeping, and the diagnostics of Sec. 1 / Sec. 3 (max|phi|, sign
// masks, connected components of the sign sets = bubbles).
#include <cuda_bf16.h>

#include "hbe_aux.h"

namespace hbe {

// ---------------------------------------------------------------- packing
// Dense N^3 doubles -> padded field (hi, and lo = residual when lo != nullptr).
// Every padded position is written: interior, periodic ghost copies (edge
// ghosts only; the star stencil never reads corners), zeros elsewhere.
template <class T>
__global__ void pack_kernel(const double *__restrict__ src, T *__restrict__ hi,
                            T *__restrict__ lo, int N, int pitch, int hx, int periodic,
                            int z_begin, int z_count) {
  const int64_t plane = (int64_t)(N + 4) * pitch;
  const int64_t total = plane * z_count;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int zl = (int)(i / plane);
    const int64_t r = i - (int64_t)zl * plane;
    const int yp = (int)(r / pitch), xp = (int)(r - (int64_t)yp * pitch);
    int x = xp - hx, y = yp - 2;
    const bool xin = x >= 0 && x < N, yin = y >= 0 && y < N;
    double v = 0.0;
    bool have = false;
    if (xin && yin) {
      have = true;
    } else if (periodic) {
      if (yin && x >= -2 && x < N + 2) { x = (x + N) % N; have = true; }
      else if (xin && y >= -2 && y < N + 2) { y = (y + N) % N; have = true; }
    }
    if (have) v = src[((int64_t)zl * N + y) * N + x];
    const int64_t o = (int64_t)(z_begin + zl) * plane + r;
    const T h = (T)v;
    hi[o] = h;
    if (lo) lo[o] = (T)(v - (double)h);
  }
}

template <class T>
__global__ void unpack_kernel(const T *__restrict__ hi, const T *__restrict__ lo,
                              double *__restrict__ dst, int N, int pitch, int hx, int z_begin,
                              int z_count) {
  const int64_t plane = (int64_t)(N + 4) * pitch;
  const int64_t total = (int64_t)N * N * z_count;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int zl = (int)(i / ((int64_t)N * N));
    const int64_t r = i - (int64_t)zl * N * N;
    const int y = (int)(r / N), x = (int)(r - (int64_t)y * N);
    const int64_t o = (int64_t)(z_begin + zl) * plane + (int64_t)(y + 2) * pitch + x + hx;
    double v = (double)hi[o];
    if (lo) v += (double)lo[o];
    dst[i] = v;
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_pack(int prec, const double *src, void *hi, void *lo, int N, int pitch, int hx,
                        int periodic, int z_begin, int z_count, cudaStream_t st) {
  const int64_t n = (int64_t)(N + 4) * pitch * z_count;
  if (prec == 0) {
    pack_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
        src, (double *)hi, (double *)lo, N, pitch, hx, periodic, z_begin, z_count);
  } else {
    pack_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
        src, (float *)hi, (float *)lo, N, pitch, hx, periodic, z_begin, z_count);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(int prec, const void *hi, const void *lo, double *dst, int N, int pitch,
                          int hx, int z_begin, int z_count, cudaStream_t st) {
  const int64_t n = (int64_t)N * N * z_count;
  if (prec == 0) {
    unpack_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
        (const double *)hi, (const double *)lo, dst, N, pitch, hx, z_begin, z_count);
  } else {
    unpack_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
        (const float *)hi, (const float *)lo, dst, N, pitch, hx, z_begin, z_count);
  }
  return cudaGetLastError();
}

// Sum of bumps A exp(-1 / (1 - r^2/R^2)) (r < R) at every padded position of
// a field (the initial-data family of Sec. 3, Eq. bump, in box coordinates).
// Node i sits at (i - c) h with c = (N-1)/2 (Dirichlet) or N/2 (periodic);
// periodic ghosts take the wrapped node's value, other ghosts stay 0.
template <class T>
__global__ void bumps_kernel(T *__restrict__ hi, T *__restrict__ lo, int N, int pitch, int hx,
                             int periodic, double h, int nb, const double *__restrict__ prm) {
  const int64_t plane = (int64_t)(N + 4) * pitch;
  const int64_t total = plane * N;
  const double cen = periodic ? 0.5 * N : 0.5 * (N - 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(i / plane);
    const int64_t r = i - (int64_t)z * plane;
    const int yp = (int)(r / pitch), xp = (int)(r - (int64_t)yp * pitch);
    int x = xp - hx, y = yp - 2;
    const bool xin = x >= 0 && x < N, yin = y >= 0 && y < N;
    bool have = xin && yin;
    if (!have && periodic) {
      if (yin && x >= -2 && x < N + 2) { x = (x + N) % N; have = true; }
      else if (xin && y >= -2 && y < N + 2) { y = (y + N) % N; have = true; }
    }
    double v = 0.0;
    if (have) {
      const double px = ((double)x - cen) * h, py = ((double)y - cen) * h,
                   pz = ((double)z - cen) * h;
      for (int b = 0; b < nb; ++b) {
        const double A = prm[5 * b], R = prm[5 * b + 1];
        const double dx = px - prm[5 * b + 2], dy = py - prm[5 * b + 3], dz = pz - prm[5 * b + 4];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < R * R) v = v + A * exp(-1.0 / (1.0 - r2 / (R * R)));
      }
    }
    const T hv = (T)v;
    hi[i] = hv;
    if (lo) lo[i] = (T)(v - (double)hv);
  }
}

cudaError_t launch_bumps(int prec, void *hi, void *lo, int N, int pitch, int hx, int periodic,
                         double h, int nb, const double *d_prm, cudaStream_t st) {
  const int64_t n = (int64_t)(N + 4) * pitch * N;
  if (prec == 0)
    bumps_kernel<double><<<grid_for(n, 256), 256, 0, st>>>((double *)hi, (double *)lo, N, pitch,
                                                           hx, periodic, h, nb, d_prm);
  else
    bumps_kernel<float><<<grid_for(n, 256), 256, 0, st>>>((float *)hi, (float *)lo, N, pitch, hx,
                                                          periodic, h, nb, d_prm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- bookkeeping
// After K steps of a batch: count the steps each context executed, apply the
// stop rule to the last of them, advance n_base, and clear the per-step maxima.
__global__ void advance_kernel(Desc *descs, const int *ndesc, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *ndesc) return;
  Desc &d = descs[i];
  long long exec = K;
  if (d.n_end - d.n_base < exec) exec = d.n_end - d.n_base;
  if (d.stop_k < exec) exec = d.stop_k;
  if (exec < 0) exec = 0;
  int status = ST_RUNNING;
  if (exec > 0) {
    const double m = __longlong_as_double((long long)d.maxabs[exec - 1]);
    if (!(m <= 1.7976931348623157e308)) status = ST_NONFINITE;
    else if (d.stop_thr > 0.0 && m > d.stop_thr) status = ST_STOPPED;
  }
  d.n_base += exec;
  d.last_done = exec;
  if (status != ST_RUNNING) {
    d.status = status;
    d.n_end = d.n_base;  // nothing more until the host asks again
  }
  d.stop_k = kNoStop;
  for (int k = 0; k < K; ++k) d.maxabs[k] = 0ull;
  // monitor entries of the steps any next replay may take start from 0
  if (d.mon)
    for (int k = 0; k < kMaxK; ++k) d.mon[(d.n_base + k) % d.mon_cap] = 0ull;
}

// The step coefficients of steps k = 0 .. K-1 of the coming batch (t from the
// context's t0, dt and n_base, all in FP64), and the dt-only constants.  One
// thread per (context, step); run before the batch's first stage launch.
__global__ void coef_kernel(Desc *descs, const int *ndesc, int K) {
  const int i = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *ndesc || k >= K) return;
  const Desc &d = descs[i];
  double *c = d.coef;
  const double dt = d.dt;
  const double tn = d.t0 + (double)(d.n_base + k) * dt;
  const double st[4] = {tn, tn + 0.5 * dt, tn + 0.5 * dt, tn + dt};
  for (int s = 0; s < 4; ++s) {
    const double e = exp(-2.0 * st[s]) * d.inv_h2;
    double *o = c + k * kCoefPerStep + s * kCoefPerStage;
    o[0] = 4.0 / 3.0 * e;
    o[1] = -e / 12.0;
    o[2] = d.mu2 - 7.5 * e;
  }
  if (k == 0) {
    double *o = c + kMaxK * kCoefPerStep;
    const double sq[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
    const double sg[4] = {0.0, 0.0, 0.25 * dt * dt, 0.5 * dt * dt};
    for (int s = 0; s < 4; ++s) {
      o[kCoefSq + s] = sq[s];
      o[kCoefSg + s] = sg[s];
      o[kCoefSp + s] = sq[s];
    }
    o[kCoefB6] = dt * dt / 6.0;
    o[kCoefD6] = dt / 6.0;
    o[kCoefDt] = dt;
    o[kCoefNlam] = -d.lambda;
  }
}

cudaError_t launch_coef(Desc *descs, const int *ndesc, int max_desc, int K, cudaStream_t st) {
  coef_kernel<<<dim3((K + 63) / 64, max_desc), 64, 0, st>>>(descs, ndesc, K);
  return cudaGetLastError();
}

cudaError_t launch_advance(Desc *descs, const int *ndesc, int max_desc, int K, cudaStream_t st) {
  const int threads = 128;
  advance_kernel<<<(max_desc + threads - 1) / threads, threads, 0, st>>>(descs, ndesc, K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- periodic ghosts
// After a stage launch of a periodic context, the ghost cells of the fields it
// wrote that later launches read with a halo receive the wrapped copies:
// columns -2, -1 <- N-2, N-1 and N, N+1 <- 0, 1 of every row, and rows
// -2, -1 <- N-2, N-1 and N, N+1 <- 0, 1 of every plane (x in [0, N)).  The
// fields: stage 1 -> G1, stage 2 -> G2, stages 4 and 6 -> phi, psi of the new
// state, stage 5 (stages 1 + 2) -> G1, G2; G3 and the compensation parts are
// read at the point only.  Elements are moved as raw bits.
template <class E> struct Pair;
template <> struct Pair<unsigned long long> { using type = ulonglong2; };
template <> struct Pair<unsigned> { using type = uint2; };
template <> struct Pair<unsigned short> { using type = unsigned; };

// Work unit u of a plane stack covers (a) the four ghost columns of interior
// row u (u < N^2) and (b) piece u of the ghost rows: 16-byte vectors when a
// row is a whole number of them (rows start 16-byte aligned), else single
// elements, over x in [0, N) of the 4 ghost rows of every plane.  A thread
// loads everything its unit needs from both fields before it stores anything,
// so all its scattered loads are in flight at once.  Reads and writes never
// overlap: ghost rows are written only at x in [0, N) from interior rows,
// ghost columns only in interior rows from interior columns.
template <class E>
__device__ void wrap_pair(void *va, void *vb, int N, int nzp, int zoff, int pitch, int64_t plane,
                          int hx, long long tid, long long nth) {
  E *fa = static_cast<E *>(va), *fb = static_cast<E *>(vb);
  const bool two = fb != nullptr;
  using P = typename Pair<E>::type;
  constexpr int VE = 16 / (int)sizeof(E);
  const bool vec = N % VE == 0;
  const int nv = vec ? N / VE : N;                       // row pieces per ghost row
  const long long nc = (long long)nzp * N, nr = 4LL * nzp * nv;  // nzp planes from zoff
  const long long nu = nc > nr ? nc : nr;
  const bool even = (N & 1) == 0;                        // column pairs aligned
  for (long long u = tid; u < nu; u += nth) {
    // (b) ghost rows: padded rows 0, 1 <- N, N+1 (y = N-2, N-1), N+2, N+3 <- 2, 3 (y = 0, 1)
    const bool hr = u < nr;
    int64_t rs = 0, rd = 0;
    if (hr) {
      const int piece = (int)(u % nv);
      const long long r = u / nv;
      const int z = (int)(r >> 2) + zoff, g = (int)(r & 3);
      const int dst = g < 2 ? g : N + g, src = g < 2 ? N + g : g;
      const int64_t cb = (int64_t)z * plane + hx + (int64_t)piece * (vec ? VE : 1);
      rs = cb + (int64_t)src * pitch;
      rd = cb + (int64_t)dst * pitch;
    }
    uint4 va4 = {}, vb4 = {};
    E sa = E(0), sb = E(0);
    if (hr) {
      if (vec) {
        va4 = *reinterpret_cast<const uint4 *>(fa + rs);
        if (two) vb4 = *reinterpret_cast<const uint4 *>(fb + rs);
      } else {
        sa = fa[rs];
        if (two) sb = fb[rs];
      }
    }
    // (a) ghost columns of row (zc, y): -2, -1 <- N-2, N-1 and N, N+1 <- 0, 1
    const bool hc = u < nc;
    int64_t ro = 0;
    E a[4] = {}, b[4] = {};
    P alo = {}, ahi = {}, blo = {}, bhi = {};
    if (hc) {
      const int zc = (int)(u / N) + zoff, y = (int)(u % N);
      ro = (int64_t)zc * plane + (int64_t)(y + 2) * pitch + hx;
      if (even) {
        alo = *reinterpret_cast<const P *>(fa + ro);
        ahi = *reinterpret_cast<const P *>(fa + ro + N - 2);
        if (two) {
          blo = *reinterpret_cast<const P *>(fb + ro);
          bhi = *reinterpret_cast<const P *>(fb + ro + N - 2);
        }
      } else {
        const int cs[4] = {0, 1, N - 2, N - 1};
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = fa[ro + cs[i]];
        if (two) {
#pragma unroll
          for (int i = 0; i < 4; ++i) b[i] = fb[ro + cs[i]];
        }
      }
    }
    if (hr) {
      if (vec) {
        *reinterpret_cast<uint4 *>(fa + rd) = va4;
        if (two) *reinterpret_cast<uint4 *>(fb + rd) = vb4;
      } else {
        fa[rd] = sa;
        if (two) fb[rd] = sb;
      }
    }
    if (hc) {
      if (even) {
        *reinterpret_cast<P *>(fa + ro - 2) = ahi;
        *reinterpret_cast<P *>(fa + ro + N) = alo;
        if (two) {
          *reinterpret_cast<P *>(fb + ro - 2) = bhi;
          *reinterpret_cast<P *>(fb + ro + N) = blo;
        }
      } else {
        fa[ro - 2] = a[2]; fa[ro - 1] = a[3]; fa[ro + N] = a[0]; fa[ro + N + 1] = a[1];
        if (two) {
          fb[ro - 2] = b[2]; fb[ro - 1] = b[3]; fb[ro + N] = b[0]; fb[ro + N + 1] = b[1];
        }
      }
    }
  }
}

__global__ void wrap_kernel(Desc *descs, const int *ndesc, int k, int stage) {
  if ((int)blockIdx.y >= *ndesc) return;
  const Desc *d = descs + blockIdx.y;
  if (d->bc != 1) return;
  const long long n = d->n_base + k;
  if (n >= d->n_end || __ldcg(&d->stop_k) <= k) return;  // the step was not taken
  const int so = (int)(n & 1) ^ 1;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const int N = d->N;
  const int es = d->prec == 0 ? 8 : 4, eg = d->prec == 0 ? 8 : (d->prec == 2 ? 2 : 4);
  void *fa, *fb = nullptr;
  int esz;
  if (stage == 4 || stage == 6) {
    fa = d->f[F_P0 + so];
    fb = d->f[F_Q0 + so];
    esz = es;
  } else if (stage == 1 || stage == 2 || stage == 5) {
    fa = d->f[stage == 2 ? F_G2 : F_G1];
    if (stage == 5) fb = d->f[F_G2];
    esz = eg;
  } else {
    return;
  }
  const bool state = stage == 4 || stage == 6;
  const int pitch = state ? d->pitch_s : d->pitch_g;
  const int64_t plane = state ? d->plane_s : d->plane_g;
  const int hx = 16 / esz;
  const int nz = d->nz, zoff = d->zoff;
  if (esz == 8) wrap_pair<unsigned long long>(fa, fb, N, nz, zoff, pitch, plane, hx, tid, nth);
  else if (esz == 4) wrap_pair<unsigned>(fa, fb, N, nz, zoff, pitch, plane, hx, tid, nth);
  else wrap_pair<unsigned short>(fa, fb, N, nz, zoff, pitch, plane, hx, tid, nth);
}

// ---------------------------------------------------------------- z-slab halos
// The stage pairs read phi, psi (stages 1+2) and phi, psi, G1, G2 (stages 3+4)
// two planes beyond a slab in z, so after each pair the two planes next to a
// slab boundary are copied into the neighbour's halo planes: plain 16-byte
// copies of whole padded planes (their periodic x/y ghosts included, the
// ghost-copy launch having run before).  Block row y = one transfer.
__global__ void halo_kernel(const Desc *descs, const HaloCopy *copies, int k, int stage) {
  const HaloCopy c = copies[blockIdx.y];
  const Desc &s = descs[c.src];
  const Desc &d = descs[c.dst];
  const long long n = s.n_base + k;
  if (n >= s.n_end || __ldcg(&s.stop_k) <= k) return;  // the step was not taken
  const bool state = stage == 6;
  const int es = state ? (s.prec == 0 ? 8 : 4) : (s.prec == 0 ? 8 : (s.prec == 2 ? 2 : 4));
  const int64_t pb = (state ? s.plane_s : s.plane_g) * es;  // bytes per stored plane
  const int so = (int)(n & 1) ^ 1;
  const int fields[2] = {state ? F_P0 + so : F_G1, state ? F_Q0 + so : F_G2};
  const int64_t units = 2 * pb / 16;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const char *>(s.f[fields[f]]) +
                                                       c.src_plane * pb);
    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<char *>(d.f[fields[f]]) + c.dst_plane * pb);
    for (int64_t i = tid; i < units; i += nth) dst[i] = src[i];
  }
}

cudaError_t launch_halo(const Desc *descs, const HaloCopy *copies, int n, int k, int stage,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  halo_kernel<<<dim3(32, n), 256, 0, st>>>(descs, copies, k, stage);
  return cudaGetLastError();
}

bool stage_needs_wrap(int stage) { return stage == 1 || stage == 2 || stage >= 4; }

cudaError_t launch_wrap(Desc *descs, const int *ndesc, int max_desc, int k, int stage,
                        int blocks, cudaStream_t st) {
  wrap_kernel<<<dim3(blocks, max_desc), 256, 0, st>>>(descs, ndesc, k, stage);
  return cudaGetLastError();
}

// Host-requested changes to a running context, applied in stream order.
__global__ void set_run_kernel(Desc *d, long long add_steps, double t0, double dt, double thr,
                               int reset) {
  if (reset) {
    d->n_end = d->n_base;
    d->status = ST_RUNNING;
    d->stop_k = kNoStop;
    d->t0 = t0;
    d->dt = dt;
    d->stop_thr = thr;
  }
  d->n_end += add_steps;
}

cudaError_t launch_set_run(Desc *d, long long add_steps, double t0, double dt, double thr,
                           int reset, cudaStream_t st) {
  set_run_kernel<<<1, 1, 0, st>>>(d, add_steps, t0, dt, thr, reset);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- diagnostics
template <class T>
__device__ __forceinline__ double state_at(const T *hi, const T *lo, int64_t o) {
  double v = (double)hi[o];
  if (lo) v += (double)lo[o];
  return v;
}

// One warp per (y, z, word): bit x%32 of word x/32 of the two masks, plus the
// running max of |phi| (NaN and inf read as +inf) as a double bit pattern.
template <class T>
__global__ void signpack_kernel(const T *__restrict__ hi, const T *__restrict__ lo, int N,
                                int pitch, int hx, double eps, uint32_t *__restrict__ pos,
                                uint32_t *__restrict__ neg, unsigned long long *maxbits) {
  const int W = (N + 31) / 32;
  const int64_t nwords = (int64_t)N * N * W;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t plane = (int64_t)(N + 4) * pitch;
  double mx = 0.0;
  for (int64_t wi = warp0; wi < nwords; wi += nwarps) {
    const int64_t row = wi / W;
    const int wx = (int)(wi - row * W);
    const int z = (int)(row / N), y = (int)(row - (int64_t)z * N);
    const int x = wx * 32 + lane;
    double v = 0.0;
    if (x < N) v = state_at(hi, lo, (int64_t)z * plane + (int64_t)(y + 2) * pitch + x + hx);
    const unsigned bp = __ballot_sync(0xffffffffu, x < N && v > eps);
    const unsigned bn = __ballot_sync(0xffffffffu, x < N && v < -eps);
    if (lane == 0) { pos[wi] = bp; neg[wi] = bn; }
    const double a = fabs(v);
    mx = (a <= mx) ? mx : ((a == a) ? a : (double)INFINITY);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(mx));
}

__device__ __forceinline__ bool mask_bit(const uint32_t *m, int W, int N, int x, int y, int z) {
  return (m[((int64_t)z * N + y) * W + (x >> 5)] >> (x & 31)) & 1u;
}

__device__ __forceinline__ int find_root(const int *L, int x) {
  int y = __ldcg(L + x);
  while (y != x) {
    x = y;
    y = __ldcg(L + x);
  }
  return x;
}

// Union of the sets of a and b: link the larger root under the smaller one
// (labels only decrease, so every find terminates).  Bounded retries.
__device__ __forceinline__ void unite(int *L, int a, int b, unsigned *err) {
  for (int it = 0; it < (1 << 24); ++it) {
    a = find_root(L, a);
    b = find_root(L, b);
    if (a == b) return;
    if (a < b) {
      const int old = atomicMin(L + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(L + a, b);
      if (old == a) return;
      a = old;
    }
  }
  atomicOr(err, (unsigned)DEV_ERR_UNIONFIND);
}

__global__ void ccl_init_kernel(const uint32_t *m, int N, int *L) {
  const int W = (N + 31) / 32;
  const int64_t n3 = (int64_t)N * N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % N);
    const int64_t r = i / N;
    const int y = (int)(r % N), z = (int)(r / N);
    L[i] = mask_bit(m, W, N, x, y, z) ? (int)i : -1;
  }
}

// 6-connectivity: each set voxel joins its -x, -y, -z neighbours (and, when
// periodic, the wrapped neighbour across the low face).
__global__ void ccl_merge_kernel(const uint32_t *m, int N, int periodic, int *L, unsigned *err) {
  const int W = (N + 31) / 32;
  const int64_t n3 = (int64_t)N * N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(L + i) < 0) continue;
    const int x = (int)(i % N);
    const int64_t r = i / N;
    const int y = (int)(r % N), z = (int)(r / N);
    const int xm = x > 0 ? x - 1 : (periodic ? N - 1 : -1);
    const int ym = y > 0 ? y - 1 : (periodic ? N - 1 : -1);
    const int zm = z > 0 ? z - 1 : (periodic ? N - 1 : -1);
    if (xm >= 0 && mask_bit(m, W, N, xm, y, z)) unite(L, (int)i, (int)(((int64_t)z * N + y) * N + xm), err);
    if (ym >= 0 && mask_bit(m, W, N, x, ym, z)) unite(L, (int)i, (int)(((int64_t)z * N + ym) * N + x), err);
    if (zm >= 0 && mask_bit(m, W, N, x, y, zm)) unite(L, (int)i, (int)(((int64_t)zm * N + y) * N + x), err);
  }
}

__global__ void ccl_count_kernel(const int *L, int64_t n3, unsigned long long *count) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x)
    c += (L[i] == (int)i) ? 1ull : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_signpack(int prec, const void *hi, const void *lo, int N, int pitch, int hx,
                            double eps, uint32_t *pos, uint32_t *neg, unsigned long long *maxbits,
                            cudaStream_t st) {
  const int64_t words = (int64_t)N * N * ((N + 31) / 32);
  const int blocks = grid_for(words * 32, 256);
  if (prec == 0)
    signpack_kernel<double><<<blocks, 256, 0, st>>>((const double *)hi, (const double *)lo, N,
                                                    pitch, hx, eps, pos, neg, maxbits);
  else
    signpack_kernel<float><<<blocks, 256, 0, st>>>((const float *)hi, (const float *)lo, N, pitch,
                                                   hx, eps, pos, neg, maxbits);
  return cudaGetLastError();
}

cudaError_t launch_ccl(const uint32_t *mask, int N, int periodic, int *labels,
                       unsigned long long *count, unsigned *err, cudaStream_t st) {
  const int64_t n3 = (int64_t)N * N * N;
  const int blocks = grid_for(n3, 256);
  ccl_init_kernel<<<blocks, 256, 0, st>>>(mask, N, labels);
  ccl_merge_kernel<<<blocks, 256, 0, st>>>(mask, N, periodic, labels, err);
  ccl_count_kernel<<<blocks, 256, 0, st>>>(labels, n3, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- analysis
// Per-block partial reductions of the paper's analysis quantities over the
// N^3 unknowns of the current state (double precision):
//   [0] sum phi, [1] sum phi^3, [2] max |FD4 Laplacian of phi| (as double bits),
//   [3] points with |phi| + |psi| > eps ("support"), [4] support points where
//   m phi + psi >= 0 (the first bubble condition fails), m = 3/2 + sqrt(9/4 + mu^2).
// A second single-block pass adds the partials in a fixed order, so the
// result does not depend on scheduling.
template <class T>
__global__ void analysis_kernel(const T *__restrict__ phi, const T *__restrict__ phlo,
                                const T *__restrict__ psi, const T *__restrict__ pslo, int N,
                                int pitch, int hx, int periodic, double inv_h2, double mcoef,
                                double eps, double *__restrict__ part) {
  const int64_t plane = (int64_t)(N + 4) * pitch;
  const int64_t n3 = (int64_t)N * N * N;
  double s1 = 0.0, s3 = 0.0, lmax = 0.0, sup = 0.0, bad = 0.0;
  auto at = [&](int x, int y, int z) -> double {
    // outside the box: 0 (Dirichlet; the stored ghost layers are 0 too) or the
    // wrapped node (periodic), indexed directly so that nothing depends on the
    // ghost copies of the compensation parts
    if (periodic) {
      x = (x + N) % N;
      y = (y + N) % N;
      z = (z + N) % N;
    } else if (z < 0 || z >= N) {
      return 0.0;
    }
    const int64_t o = (int64_t)z * plane + (int64_t)(y + 2) * pitch + x + hx;
    double v = (double)phi[o];
    if (phlo) v += (double)phlo[o];
    return v;
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % N);
    const int64_t r = i / N;
    const int y = (int)(r % N), z = (int)(r / N);
    const double c = at(x, y, z);
    const int64_t o = (int64_t)z * plane + (int64_t)(y + 2) * pitch + x + hx;
    double q = (double)psi[o];
    if (pslo) q += (double)pslo[o];
    double lap = 0.0;
    lap += -1.0 / 12.0 * (at(x - 2, y, z) + at(x + 2, y, z)) + 4.0 / 3.0 * (at(x - 1, y, z) + at(x + 1, y, z)) - 2.5 * c;
    lap += -1.0 / 12.0 * (at(x, y - 2, z) + at(x, y + 2, z)) + 4.0 / 3.0 * (at(x, y - 1, z) + at(x, y + 1, z)) - 2.5 * c;
    lap += -1.0 / 12.0 * (at(x, y, z - 2) + at(x, y, z + 2)) + 4.0 / 3.0 * (at(x, y, z - 1) + at(x, y, z + 1)) - 2.5 * c;
    lap = fabs(lap * inv_h2);
    s1 += c;
    s3 += c * c * c;
    lmax = (lap <= lmax) ? lmax : ((lap == lap) ? lap : (double)INFINITY);
    if (fabs(c) + fabs(q) > eps) {
      sup += 1.0;
      if (mcoef * c + q >= 0.0) bad += 1.0;
    }
  }
  __shared__ double red[5][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    sup += __shfl_xor_sync(0xffffffffu, sup, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) { red[0][wid] = s1; red[1][wid] = s3; red[2][wid] = lmax; red[3][wid] = sup; red[4][wid] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a[0] += red[0][w]; a[1] += red[1][w]; a[2] = fmax(a[2], red[2][w]);
      a[3] += red[3][w]; a[4] += red[4][w];
    }
    for (int k = 0; k < 5; ++k) part[(int64_t)k * gridDim.x + blockIdx.x] = a[k];
  }
}

__global__ void analysis_finish_kernel(const double *part, int nblocks, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    a[0] += part[b]; a[1] += part[nblocks + b]; a[2] = fmax(a[2], part[2 * nblocks + b]);
    a[3] += part[3 * nblocks + b]; a[4] += part[4 * nblocks + b];
  }
  for (int k = 0; k < 5; ++k) out[k] = a[k];
}

int analysis_blocks() { return 152 * 4; }

cudaError_t launch_analysis(int prec, const void *phi, const void *phlo, const void *psi,
                            const void *pslo, int N, int pitch, int hx, int periodic,
                            double inv_h2, double mcoef, double eps, double *part, double *out,
                            cudaStream_t st) {
  const int blocks = analysis_blocks();
  if (prec == 0)
    analysis_kernel<double><<<blocks, 256, 0, st>>>((const double *)phi, (const double *)phlo,
                                                    (const double *)psi, (const double *)pslo, N,
                                                    pitch, hx, periodic, inv_h2, mcoef, eps, part);
  else
    analysis_kernel<float><<<blocks, 256, 0, st>>>((const float *)phi, (const float *)phlo,
                                                   (const float *)psi, (const float *)pslo, N,
                                                   pitch, hx, periodic, inv_h2, mcoef, eps, part);
  analysis_finish_kernel<<<1, 32, 0, st>>>(part, blocks, out);
  return cudaGetLastError();
}

}  // namespace hbe
