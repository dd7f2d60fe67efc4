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
// One CTA integrates one problem of the batch for all its steps.  Each thread
// owns 8 consecutive nodes and keeps their state (p, q, G1..G3) and stage
// arguments in registers; the two neighbours on each side come from the
// adjacent lanes by warp shuffles and, at warp boundaries, through a small
// exchange in shared memory, so a step costs four block barriers and no
// global-memory traffic beyond 16 bytes of stage coefficients a step.  The
// coefficients e^{-2 t_s} / dr^2 are the same for every problem of the batch:
// a small kernel forms them in double precision once per step and stage
// (t_n = t0 + n dt) and rounds them to the solver's type; each CTA copies
// them into shared memory 64 steps at a time.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "hbe.h"

namespace hbe_radial {

constexpr int kMaxThreads = 512;
constexpr int kCoefChunk = 64;  // steps whose stage coefficients are tabled at once
static_assert((kCoefChunk & (kCoefChunk - 1)) == 0, "a power of two");

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
  const void *ctab;  // [nsteps][4] stage coefficients, in the solver's type
};

// ctab[4 n + s] = e^{-2 t_s} / dr^2 for stage s of step n (stage times t_n,
// t_n + dt/2, t_n + dt/2, t_n + dt; t_n = t0 + n dt), formed in double.
template <typename T>
__global__ void radial_coef_kernel(T *ctab, double t0, double dt, double inv_dr2, int64_t nsteps) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 4 * nsteps;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e & 3);
    const double t = t0 + (double)(e >> 2) * dt;
    const double ts = s == 0 ? t : (s == 3 ? t + dt : t + dt / 2);
    ctab[e] = T(exp(-2.0 * ts) * inv_dr2);
  }
}

template <typename T>
struct Shared {
  T coef[kCoefChunk][4];  // e^{-2 t_s} / dr^2 formed in double, rounded once to T
  // stage-argument values at the ends of each warp's run of nodes, double
  // buffered by stage: [buffer][0: last two nodes, 1: first two][warp][2]
  T edge[2][2][kMaxThreads / 32][2];
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

// Laplacian times dr^2 at node i from the stage argument at nodes i-2 .. i+2:
// D2 + (2/i) D1 in the interior, 3 x the even closure at the origin (where
// p1, p2 are the values at nodes 1 and 2).  The weights of D2 and of the
// closure sum to zero, so both are formed from differences to the centre
// value (same operator in exact arithmetic; in FP32 it avoids the
// cancellation of terms 1/dr^2 times larger than the result).
template <typename T>
__device__ __forceinline__ T lap_dr2(T m2, T m1, T c0, T p1, T p2, bool origin, T two_over_i) {
  if (origin) return T(3) * fm(T(8.0 / 3.0), p1 - c0, T(-1.0 / 6.0) * (p2 - c0));
  const T d2 = fm(T(-1.0 / 12.0), (m2 - c0) + (p2 - c0), T(4.0 / 3.0) * ((m1 - c0) + (p1 - c0)));
  const T d1 = fm(T(2.0 / 3.0), p1 - m1, T(-1.0 / 12.0) * (p2 - m2));
  return fm(two_over_i, d1, d2);
}

// The FP32 evaluation of two neighbouring nodes (j, j+1 of a thread) at once
// with Blackwell's packed FP32 instructions; every element is rounded as the
// scalar operation above (a - b as fma(b, -1, a)), so the results are the same
// bits.  Interior nodes only: the caller replaces the origin's value.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
template <int V>
__device__ __forceinline__ float2 g_pair(const float (&E)[V + 4], int j, float2 w, float2 Q,
                                         float c, float2 P, float mu2, float lam) {
  const float2 m2 = p2(E[j], E[j + 1]), m1 = p2(E[j + 1], E[j + 2]), c0 = p2(E[j + 2], E[j + 3]),
               p1 = p2(E[j + 3], E[j + 4]), q2 = p2(E[j + 4], E[j + 5]);
  const float2 d2 = __ffma2_rn(p2(-1.0f / 12.0f), __fadd2_rn(sub2(m2, c0), sub2(q2, c0)),
                               __fmul2_rn(p2(4.0f / 3.0f), __fadd2_rn(sub2(m1, c0), sub2(p1, c0))));
  const float2 d1 = __ffma2_rn(p2(2.0f / 3.0f), sub2(p1, m1), __fmul2_rn(p2(-1.0f / 12.0f), sub2(q2, m2)));
  const float2 lap = __ffma2_rn(w, d1, d2);
  const float2 PP = __fmul2_rn(P, P);
  const float2 t = __fmul2_rn(P, __ffma2_rn(p2(-lam), PP, p2(mu2)));
  return __ffma2_rn(p2(c), lap, __ffma2_rn(p2(-3.0f), Q, t));
}

// Thread t owns the V consecutive nodes V t .. V t + V - 1 (those below n) and
// keeps their state in registers; a stage's neighbour values come from the
// adjacent lanes by shuffles and, across warps, from the `edge` exchange in
// shared memory, behind one block barrier per stage.  TH: most threads a
// block, MINB: CTAs per SM the registers must allow.
// out[j] = a * x[j] + y[j] for the V owned nodes, each with one rounding; two
// nodes per packed instruction in FP32 (the same bits as the scalar FMA)
template <typename T, int V>
__device__ __forceinline__ void axpy(T (&out)[V], T a, const T (&x)[V], const T (&y)[V]) {
  if constexpr (std::is_same<T, float>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V; j += 2) {
      const float2 r = __ffma2_rn(p2(a), p2(x[j], x[j + 1]), p2(y[j], y[j + 1]));
      out[j] = r.x;
      out[j + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) out[j] = fm(a, x[j], y[j]);
  }
}

template <typename T, int V, int TH, int MINB>
__global__ void __launch_bounds__(TH, MINB) radial_kernel(Args a) {
  static_assert(V >= 3, "the origin mirror reads nodes 1 and 2 from thread 0");
  __shared__ Shared<T> sh;
  const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5, b = blockIdx.x, i0 = tid * V;
  const unsigned full = 0xffffffffu;
  const T mu2 = T(a.mu[b] * a.mu[b]), lam = T(a.lambda[b]);
  const T dt = T(a.dt), hdt = T(0.5 * a.dt), qdt2 = T(0.25 * a.dt * a.dt),
          hdt2 = T(0.5 * a.dt * a.dt), sdt2 = T(a.dt * a.dt / 6.0), sdt = T(a.dt / 6.0);

  // nodes at or beyond n hold 0 in every field: the wall value and its ghosts
  T p[V], q[V], g1[V], g2[V], g3[V], w[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = i0 + j;
    p[j] = q[j] = g1[j] = g2[j] = g3[j] = T(0);
    w[j] = i > 0 ? T(2.0 / (double)i) : T(0);
    if (i < n) {
      p[j] = T(a.phi0[(size_t)b * n + i]);
      q[j] = T(a.phi1[(size_t)b * n + i]);
    }
  }
  if (tid == 0) sh.any_nonfinite = 0;

  // E[0 .. V+3] = stage argument at nodes i0-2 .. i0+V+1; the barrier returns
  // the OR of `flag` over the block
  int buf = 0;
  auto exchange = [&](const T (&P)[V], T (&E)[V + 4], int flag) -> int {
#pragma unroll
    for (int j = 0; j < V; ++j) E[j + 2] = P[j];
    if (lane == 31) { sh.edge[buf][0][warp][0] = P[V - 2]; sh.edge[buf][0][warp][1] = P[V - 1]; }
    if (lane == 0) { sh.edge[buf][1][warp][0] = P[0]; sh.edge[buf][1][warp][1] = P[1]; }
    T l2 = __shfl_up_sync(full, P[V - 2], 1), l1 = __shfl_up_sync(full, P[V - 1], 1);
    T r1 = __shfl_down_sync(full, P[0], 1), r2 = __shfl_down_sync(full, P[1], 1);
    const int any = __syncthreads_or(flag);
    if (lane == 0) {
      if (warp > 0) { l2 = sh.edge[buf][0][warp - 1][0]; l1 = sh.edge[buf][0][warp - 1][1]; }
      else { l2 = P[2]; l1 = P[1]; }  // phi(-r) = phi(r) at the origin
    }
    if (lane == 31) {
      if (warp + 1 < nw) { r1 = sh.edge[buf][1][warp + 1][0]; r2 = sh.edge[buf][1][warp + 1][1]; }
      else { r1 = r2 = T(0); }
    }
    E[0] = l2; E[1] = l1; E[V + 2] = r1; E[V + 3] = r2;
    buf ^= 1;
    return any;
  };
  auto lap = [&](const T (&E)[V + 4], int j) -> T {
    return lap_dr2(E[j], E[j + 1], E[j + 2], E[j + 3], E[j + 4], tid == 0 && j == 0, w[j]);
  };

  // (double)x > stop for a T value x  <=>  x > stop rounded toward -inf in T
  const bool use_stop = a.stop > 0.0;
  T stop_t;
  if constexpr (std::is_same<T, float>::value) stop_t = __double2float_rd(a.stop);
  else stop_t = a.stop;
  int64_t k = 0;
  int status = 0, flag = 0, bad = 0;
  int64_t pending = 0;  // 1 + index of a record whose partial results await combining
  // steps to the next record and records taken (no 64-bit division per step)
  int rec_left = a.record_every;
  int64_t rec_done = 0;
  T E[V + 4], P[V];
  for (;; ++k) {
    const int kc = (int)(k & (kCoefChunk - 1));  // k >= 0, kCoefChunk a power of 2
    if (kc == 0 && k < a.nsteps) {
      // the next steps' e^{-2 t_s} / dr^2 (t_n = t0 + n dt, Sec. 2.1) from the
      // table; the barrier of the exchange below publishes them
      const T *ctab = static_cast<const T *>(a.ctab);
      for (int e = tid; e < 4 * kCoefChunk; e += blockDim.x)
        if (4 * k + e < 4 * a.nsteps) (&sh.coef[0][0])[e] = ctab[4 * k + e];
    }
    // stage 1 exchange; its barrier also ends step k - 1 (stop rule, records)
    const int any = exchange(p, E, flag);
    if (pending && tid == 0) {
      T mm = T(0);
      for (int wi = 0; wi < nw; ++wi) mm = tmax(mm, sh.wmax[wi]);
      int prev = 0, total = 0;
      for (int t = 0; t < (int)blockDim.x; ++t) {
        total += sh.changes[t];
        if (sh.first[t] != 0) {
          if (prev != 0 && prev != sh.first[t]) ++total;
          prev = sh.last[t];
        }
      }
      double *rec = a.records + ((size_t)b * a.nrec + (pending - 1)) * 3;
      rec[0] = a.t0 + (double)k * a.dt;
      rec[1] = (double)mm;
      rec[2] = (double)total;
    }
    pending = 0;
    if (any) {
      status = sh.any_nonfinite ? 2 : 1;
      break;
    }
    if (k >= a.nsteps) break;
    const T c1 = sh.coef[kc][0], c2 = sh.coef[kc][1], c3 = sh.coef[kc][2], c4 = sh.coef[kc][3];
    // G of every owned node from the stage argument (in E and A) and the point
    // argument Q; nodes at or beyond n keep 0
    auto eval = [&](T (&out)[V], const T (&A)[V], const T (&Qv)[V], T c) {
      if constexpr (std::is_same<T, float>::value && V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
          const float2 g = g_pair<V>(E, j, p2(w[j], w[j + 1]), p2(Qv[j], Qv[j + 1]), c,
                                     p2(A[j], A[j + 1]), mu2, lam);
          out[j] = g.x;
          out[j + 1] = g.y;
        }
        if (tid == 0) out[0] = rhs_g(Qv[0], c, lap(E, 0), A[0], mu2, lam);  // the origin
        // nodes at or beyond the wall keep 0 (only the thread that holds the wall)
        if (i0 + V > n) {
#pragma unroll
          for (int j = 0; j < V; ++j)
            if (i0 + j >= n) out[j] = T(0);
        }
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (i0 + j < n) out[j] = rhs_g(Qv[j], c, lap(E, j), A[j], mu2, lam);
      }
    };
    T Qs[V];
    // stage 1: argument p -> G1
    eval(g1, p, q, c1);
    // stage 2: argument P2 = p + dt/2 q, Q2 = q + dt/2 G1 -> G2
    T H[V];  // p + dt/2 q, shared by stages 2 and 3
    axpy(H, hdt, q, p);
    exchange(H, E, 0);
    axpy(Qs, hdt, g1, q);
    eval(g2, H, Qs, c2);
    // stage 3: argument P3 = p + dt/2 q + dt^2/4 G1, Q3 = q + dt/2 G2 -> G3
    axpy(P, qdt2, g1, H);
    exchange(P, E, 0);
    axpy(Qs, hdt, g2, q);
    eval(g3, P, Qs, c3);
    // stage 4: argument P4 = p + dt q + dt^2/2 G2, Q4 = q + dt G3 -> G4; RK4 combine
    T D[V];  // p + dt q, shared by stage 4 and the combine
    axpy(D, dt, q, p);
    axpy(P, hdt2, g2, D);
    exchange(P, E, 0);
    T lmax = T(0);
    T g4v[V] = {};  // 0 at and beyond the wall (the FP64 evaluation skips those nodes)
    axpy(Qs, dt, g3, q);
    eval(g4v, P, Qs, c4);
    // every field is 0 at and beyond the wall, so the combine keeps it 0 there
    T s3[V], s4[V], s23[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      s3[j] = g1[j] + g2[j] + g3[j];
      s23[j] = g2[j] + g3[j];
      s4[j] = g1[j] + g4v[j];
    }
    axpy(p, sdt2, s3, D);
    axpy(s23, T(2), s23, s4);
    axpy(q, sdt, s23, q);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const T m = fabs(p[j]);
      if (!(m <= m) || isinf(m)) bad = 1;  // NaN or infinite
      lmax = tmax(lmax, m);
    }
    if (bad) atomicOr(&sh.any_nonfinite, 1);
    flag = bad || (use_stop && lmax > stop_t);
    if (rec_done < a.nrec && --rec_left == 0) {  // after steps record_every, 2 record_every, ...
      rec_left = a.record_every;
      ++rec_done;
      // partial max|phi| and strict sign changes (|phi| <= eps ignored) of this
      // thread's run of nodes; combined by thread 0 after the next barrier
      T m = lmax;
      for (int o = 16; o > 0; o >>= 1) m = tmax(m, __shfl_xor_sync(full, m, o));
      if (lane == 0) sh.wmax[warp] = m;
      int f = 0, l = 0, c = 0;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (i0 + j >= n) continue;
        const double v = (double)p[j];
        const int sg = v > a.eps ? 1 : (v < -a.eps ? -1 : 0);
        if (sg == 0) continue;
        if (f == 0) f = sg;
        else if (sg != l) ++c;
        l = sg;
      }
      sh.first[tid] = f;
      sh.last[tid] = l;
      sh.changes[tid] = c;
      pending = rec_done;
    }
  }

#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = i0 + j;
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

template <typename T, int V, int TH, int MINB>
cudaError_t launch(Args a, int batch, cudaStream_t st) {
  const int threads = std::max(32, ((a.n + V - 1) / V + 31) / 32 * 32);
  if (threads > TH) return cudaErrorInvalidConfiguration;
  // the coefficient table lives for this launch only (stream-ordered memory)
  T *tab = nullptr;
  if (a.nsteps > 0) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&tab),
                                    (size_t)a.nsteps * 4 * sizeof(T), st);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((4 * a.nsteps + 255) / 256, 4096);
    radial_coef_kernel<T><<<(int)blocks, 256, 0, st>>>(tab, a.t0, a.dt, 1.0 / (a.dr * a.dr),
                                                       a.nsteps);
  }
  a.ctab = tab;
  radial_kernel<T, V, TH, MINB><<<batch, threads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (tab) cudaFreeAsync(tab, st);
  return e;
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
  // 8 nodes a thread: up to 2048 nodes a CTA of <= 256 threads, two CTAs per SM
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prec == HBE_FP64)
    e = n <= 2048 ? launch<double, 8, 256, 1>(a, batch, st) : launch<double, 8, 512, 1>(a, batch, st);
  else
    e = n <= 2048 ? launch<float, 8, 256, 2>(a, batch, st) : launch<float, 8, 512, 1>(a, batch, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return HBE_ENOMEM;
  }
  return e == cudaSuccess ? HBE_OK : HBE_ECUDA;
}
