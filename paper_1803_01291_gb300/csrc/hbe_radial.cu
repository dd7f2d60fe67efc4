// Batched solver for radial solutions of the HBE (Sec. 2.2, Eq. radial):
//
//   phi_tt - e^{-2t} (phi_rr + (2/r) phi_r) + 3 phi_t = mu^2 phi - lambda phi^3,
//   0 <= r <= R,  phi_r(0, t) = 0,  phi(R, t) = 0.
//
// Nodes r_i = i dr, dr = R/n, unknowns i = 0 .. n-1.  Interior nodes use the
// fourth-order second difference of Sec. 2.1 and the fourth-order central first
// difference; the ghosts are the even reflection phi(-r) = phi(r) at the origin
// and zero from the wall on.  At r = 0 the operator is 3 phi_rr(0) (L'Hospital,
// Sec. 2.2) with the even closure (-5/2 phi_0 + 8/3 phi_1 - 1/6 phi_2) / dr^2.
// Time: classic RK4 in the recompute form (only the psi-components G_s of the
// stages are kept; the stage arguments are rebuilt from p, q and G).
//
// One CTA integrates one problem of the batch for all its steps: the state
// (p, q, G1..G3) of a thread's 8 nodes lives in registers, the stage argument of
// every node (with its ghosts) in one of two shared-memory buffers, so a step
// costs four block barriers and no global-memory traffic.  The stage
// coefficients e^{-2 t_s} / dr^2 are computed in double precision, 64 steps at
// a time, into shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "hbe.h"

namespace hbe_radial {

constexpr int kMaxThreads = 512;
constexpr int kCoefChunk = 64;  // steps whose stage coefficients are tabled at once

struct Args {
  int n;
  double dr;
  const double *mu, *lambda, *phi0, *phi1;
  double t0, dt;
  int64_t nsteps;
  int record_every;
  int64_t nrec;
  double stop, eps;
  double *phi, *psi, *records;
  int64_t *steps;
  int32_t *status;
};

template <typename T>
struct Shared {
  double coef[kCoefChunk][4];
  T wmax[kMaxThreads / 32];
  int first[kMaxThreads], last[kMaxThreads], changes[kMaxThreads];
  int any_nonfinite;
};

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// a * b + c with one rounding (the library is built without automatic contraction)
__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fm(double a, double b, double c) { return __fma_rn(a, b, c); }

// G = -3 Q + c Lap + mu^2 P - lambda P^3 (Eq. rhs, radial form)
template <typename T>
__device__ __forceinline__ T rhs_g(T Q, T c, T lap, T P, T mu2, T lam) {
  const T P2 = P * P;
  return fm(c, lap, fm(T(-3), Q, P * fm(-lam, P2, mu2)));
}

// Laplacian of the stage argument A (node i at A[i + 2]) times dr^2:
// D2 + (2/i) D1 in the interior, 3 x the even closure at the origin.  The
// weights of D2 and of the closure sum to zero, so both are formed from
// differences to the centre value (same operator in exact arithmetic; in FP32
// it avoids the cancellation of terms 1/dr^2 times larger than the result).
template <typename T>
__device__ __forceinline__ T lap_dr2(const T *A, int i, T two_over_i) {
  const T c0 = A[i + 2];
  if (i == 0)
    return T(3) * fm(T(8.0 / 3.0), A[3] - c0, T(-1.0 / 6.0) * (A[4] - c0));
  const T m2 = A[i], m1 = A[i + 1], p1 = A[i + 3], p2 = A[i + 4];
  const T d2 = fm(T(-1.0 / 12.0), (m2 - c0) + (p2 - c0), T(4.0 / 3.0) * ((m1 - c0) + (p1 - c0)));
  const T d1 = fm(T(2.0 / 3.0), p1 - m1, T(-1.0 / 12.0) * (p2 - m2));
  return fm(two_over_i, d1, d2);
}

// store a node's stage argument, and the mirrored ghost for nodes 1 and 2
template <typename T>
__device__ __forceinline__ void put(T *A, int i, T v) {
  A[i + 2] = v;
  if (i == 1) A[1] = v;
  if (i == 2) A[0] = v;
}

// NPT nodes a thread (node i = thread + j x blockDim), at most TH threads, MINB
// CTAs per SM the registers must allow
template <typename T, int NPT, int TH, int MINB>
__global__ void __launch_bounds__(TH, MINB) radial_kernel(Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T> &sh = *reinterpret_cast<Shared<T> *>(smem_raw);
  T *A0 = reinterpret_cast<T *>(smem_raw + ((sizeof(Shared<T>) + 15) / 16) * 16);
  T *A1 = A0 + (a.n + 4);
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x, b = blockIdx.x;
  const T mu2 = T(a.mu[b] * a.mu[b]), lam = T(a.lambda[b]);
  const T dt = T(a.dt), hdt = T(0.5 * a.dt), qdt2 = T(0.25 * a.dt * a.dt),
          hdt2 = T(0.5 * a.dt * a.dt), sdt2 = T(a.dt * a.dt / 6.0), sdt = T(a.dt / 6.0);

  T p[NPT], q[NPT], g1[NPT], g2[NPT], g3[NPT], w[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int i = tid + j * nt;
    p[j] = q[j] = g1[j] = g2[j] = g3[j] = T(0);
    w[j] = i > 0 ? T(2.0 / (double)i) : T(0);
    if (i < n) {
      p[j] = T(a.phi0[(size_t)b * n + i]);
      q[j] = T(a.phi1[(size_t)b * n + i]);
      put(A0, i, p[j]);
    }
  }
  if (tid == 0) {
    A0[n + 2] = A0[n + 3] = A1[n + 2] = A1[n + 3] = T(0);
    sh.any_nonfinite = 0;
  }

  int64_t k = 0;
  int status = 0;
  const double inv_dr2 = 1.0 / (a.dr * a.dr);
  for (; k < a.nsteps; ++k) {
    const int kc = (int)(k % kCoefChunk);
    if (kc == 0) {
      // table e^{-2 t_s} / dr^2 for the next steps (t_n = t0 + n dt, Sec. 2.1)
      for (int e = tid; e < 4 * kCoefChunk; e += nt) {
        const int s = e & 3, kk = e >> 2;
        const double t = a.t0 + (double)(k + kk) * a.dt;
        const double ts = s == 0 ? t : (s == 3 ? t + a.dt : t + a.dt / 2);
        sh.coef[kk][s] = exp(-2.0 * ts) * inv_dr2;
      }
      __syncthreads();
    }
    const T c1 = T(sh.coef[kc][0]), c2 = T(sh.coef[kc][1]), c3 = T(sh.coef[kc][2]),
            c4 = T(sh.coef[kc][3]);
    // stage 1: argument p (A0) -> G1; forms P2 = p + dt/2 q into A1
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int i = tid + j * nt;
      if (i < n) {
        const T P = p[j];
        g1[j] = rhs_g(q[j], c1, lap_dr2(A0, i, w[j]), P, mu2, lam);
        put(A1, i, fm(hdt, q[j], p[j]));
      }
    }
    __syncthreads();
    // stage 2: argument P2 (A1), Q2 = q + dt/2 G1 -> G2; forms P3 into A0
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int i = tid + j * nt;
      if (i < n) {
        const T P = A1[i + 2], Q = fm(hdt, g1[j], q[j]);
        g2[j] = rhs_g(Q, c2, lap_dr2(A1, i, w[j]), P, mu2, lam);
        put(A0, i, fm(qdt2, g1[j], fm(hdt, q[j], p[j])));
      }
    }
    __syncthreads();
    // stage 3: argument P3 (A0), Q3 = q + dt/2 G2 -> G3; forms P4 into A1
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int i = tid + j * nt;
      if (i < n) {
        const T P = A0[i + 2], Q = fm(hdt, g2[j], q[j]);
        g3[j] = rhs_g(Q, c3, lap_dr2(A0, i, w[j]), P, mu2, lam);
        put(A1, i, fm(hdt2, g2[j], fm(dt, q[j], p[j])));
      }
    }
    __syncthreads();
    // stage 4: argument P4 (A1), Q4 = q + dt G3 -> G4; RK4 combine; p' into A0
    T lmax = T(0);
    int bad = 0;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int i = tid + j * nt;
      if (i < n) {
        const T P = A1[i + 2], Q = fm(dt, g3[j], q[j]);
        const T g4 = rhs_g(Q, c4, lap_dr2(A1, i, w[j]), P, mu2, lam);
        const T s3 = g1[j] + g2[j] + g3[j];
        p[j] = fm(sdt2, s3, fm(dt, q[j], p[j]));
        q[j] = fm(sdt, fm(T(2), g2[j] + g3[j], g1[j] + g4), q[j]);
        put(A0, i, p[j]);
        const T m = fabs(p[j]);
        if (!(m <= m) || isinf(m)) bad = 1;  // NaN or infinite
        lmax = tmax(lmax, m);
      }
    }
    const bool over = a.stop > 0.0 && (double)lmax > a.stop;
    const int any = __syncthreads_or(bad || over);
    const int64_t done = k + 1;
    if (a.record_every > 0 && done % a.record_every == 0) {
      // max|phi| and the number of strict sign changes along r (|phi| <= eps ignored)
      T m = lmax;
      for (int o = 16; o > 0; o >>= 1) m = tmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((tid & 31) == 0) sh.wmax[tid >> 5] = m;
      const int per = (n + nt - 1) / nt, lo = tid * per, hi = min(n, lo + per);
      int f = 0, l = 0, c = 0;
      for (int i = lo; i < hi; ++i) {
        const double v = (double)A0[i + 2];
        const int s = v > a.eps ? 1 : (v < -a.eps ? -1 : 0);
        if (s == 0) continue;
        if (f == 0) f = s;
        else if (s != l) ++c;
        l = s;
      }
      sh.first[tid] = f;
      sh.last[tid] = l;
      sh.changes[tid] = c;
      __syncthreads();
      if (tid == 0) {
        T mm = T(0);
        for (int wi = 0; wi < (nt + 31) / 32; ++wi) mm = tmax(mm, sh.wmax[wi]);
        int prev = 0, total = 0;
        for (int t = 0; t < nt; ++t) {
          total += sh.changes[t];
          if (sh.first[t] != 0) {
            if (prev != 0 && prev != sh.first[t]) ++total;
            prev = sh.last[t];
          }
        }
        const int64_t r = done / a.record_every - 1;
        if (a.records && r < a.nrec) {
          double *rec = a.records + ((size_t)b * a.nrec + r) * 3;
          rec[0] = a.t0 + (double)done * a.dt;
          rec[1] = (double)mm;
          rec[2] = (double)total;
        }
      }
    }
    if (any) {
      if (bad) atomicOr(&sh.any_nonfinite, 1);
      __syncthreads();
      status = sh.any_nonfinite ? 2 : 1;
      ++k;
      break;
    }
  }

#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int i = tid + j * nt;
    if (i < n) {
      a.phi[(size_t)b * n + i] = (double)p[j];
      a.psi[(size_t)b * n + i] = (double)q[j];
    }
  }
  if (tid == 0) {
    if (a.steps) a.steps[b] = k;
    if (a.status) a.status[b] = status;
  }
}

template <typename T>
size_t smem_bytes(int n) {
  return ((sizeof(Shared<T>) + 15) / 16) * 16 + 2 * (size_t)(n + 4) * sizeof(T);
}

template <typename T, int NPT, int TH, int MINB>
cudaError_t launch(const Args &a, int batch, cudaStream_t st) {
  const int threads = std::max(32, ((a.n + NPT - 1) / NPT + 31) / 32 * 32);
  if (threads > TH) return cudaErrorInvalidConfiguration;
  const size_t sm = smem_bytes<T>(a.n);
  cudaError_t e = cudaFuncSetAttribute(radial_kernel<T, NPT, TH, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  radial_kernel<T, NPT, TH, MINB><<<batch, threads, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hbe_radial

extern "C" int hbe_radial_max_n(int prec) {
  return (prec == HBE_FP64 || prec == HBE_FP32) ? 8 * hbe_radial::kMaxThreads : 0;
}

extern "C" hbe_status hbe_radial_run(int batch, int n, double R, const double *d_mu,
                                     const double *d_lambda, const double *d_phi0,
                                     const double *d_phi1, double t0, double dt, int64_t nsteps,
                                     int prec, int record_every, double stop, double eps,
                                     double *d_phi, double *d_psi, double *d_records,
                                     int64_t *d_steps, int32_t *d_status, void *stream) {
  using namespace hbe_radial;
  if (batch < 1 || n < 4 || n > hbe_radial_max_n(prec)) return HBE_EINVAL;
  if (!(R > 0.0) || !std::isfinite(R) || !(dt > 0.0) || !std::isfinite(dt) ||
      !std::isfinite(t0) || nsteps < 0 || record_every < 0 || !(stop >= 0.0) || !(eps >= 0.0))
    return HBE_EINVAL;
  if (!d_mu || !d_lambda || !d_phi0 || !d_phi1 || !d_phi || !d_psi) return HBE_EINVAL;
  if (batch > (1 << 30)) return HBE_EINVAL;
  Args a;
  a.n = n;
  a.dr = R / n;
  a.mu = d_mu;
  a.lambda = d_lambda;
  a.phi0 = d_phi0;
  a.phi1 = d_phi1;
  a.t0 = t0;
  a.dt = dt;
  a.nsteps = nsteps;
  a.record_every = record_every;
  a.nrec = record_every > 0 ? nsteps / record_every : 0;
  a.stop = stop;
  a.eps = eps;
  a.phi = d_phi;
  a.psi = d_psi;
  a.records = a.nrec > 0 ? d_records : nullptr;
  a.steps = d_steps;
  a.status = d_status;
  if (a.nrec > 0 && !d_records) return HBE_EINVAL;
  // 8 nodes a thread; up to 2048 nodes a CTA of <= 256 threads, two CTAs per SM
  // for FP32 (measured 1.3x over one CTA of 512 threads with 4 nodes each;
  // FP64 is bound by the FP64 pipe either way)
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prec == HBE_FP64)
    e = n <= 2048 ? launch<double, 8, 256, 1>(a, batch, st) : launch<double, 8, 512, 1>(a, batch, st);
  else
    e = n <= 2048 ? launch<float, 8, 256, 2>(a, batch, st) : launch<float, 8, 512, 1>(a, batch, st);
  return e == cudaSuccess ? HBE_OK : HBE_ECUDA;
}
