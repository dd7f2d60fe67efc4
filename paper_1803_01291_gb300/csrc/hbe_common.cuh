// hbe_common.cuh -- types shared by the host side and the kernels of libhbe.
//
// Data layout in device memory (one per field, per precision):
//   A field of N^3 unknowns is stored "padded": each x-row has HX ghost/alignment
//   elements before and after it (HX = 16 bytes / element size, so the first
//   unknown of a row is 16-byte aligned), each z-plane has 2 ghost rows before
//   and after, and z is not padded:
//       element (x, y, z) at  (z + zoff)*plane + (y + 2)*pitch + (x + HX),
//       pitch = round_up(N + 2*HX, HX),  plane = (N + 4)*pitch,
//   zoff = 0 for a whole grid; a z-slab of a decomposed grid stores its nz
//   planes after zoff = 2 halo planes and before 2 more (Desc::zoff).
//   Zero-Dirichlet: ghosts stay 0 (the two ghost layers of Eq. BC, zeroed at
//   allocation and never written).  Periodic: the wrapped copies x in
//   {-2,-1,N,N+1} and y in {-2,-1,N,N+1} are written by the initial-data
//   kernels and, after each stage launch, by a ghost-copy launch for the
//   fields later stages read with a halo (the stage kernels store interior
//   points only).  z-ghosts come from the TMA unit: out-of-range z planes read
//   as zero (Dirichlet) or the plane index is wrapped (periodic).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hbe {

enum Field : int {
  F_P0 = 0, F_P1, F_Q0, F_Q1, F_PLO0, F_PLO1, F_QLO0, F_QLO1, F_G1, F_G2, F_G3, NUM_FIELDS
};

// TMA descriptors of one context: halo boxes (tile + 2 rows / HX columns of
// ghost on each side) and interior boxes (the tile only).  The stages 1+2
// kernel may use a taller tile than the others; its halo boxes of p and q are
// the *_P maps (the same boxes as TM_P_H* / TM_Q_H* when the tiles agree).
enum TMap : int {
  TM_P_H0 = 0, TM_P_H1, TM_Q_H0, TM_Q_H1, TM_Q_I0, TM_Q_I1, TM_PLO_I0, TM_PLO_I1,
  TM_QLO_I0, TM_QLO_I1, TM_G1_H, TM_G1_I, TM_G2_H, TM_G2_I, TM_G3_I,
  TM_P_H0_P, TM_P_H1_P, TM_Q_H0_P, TM_Q_H1_P, NUM_TMAPS
};

enum DevError : unsigned { DEV_ERR_TIMEOUT = 1u, DEV_ERR_UNIONFIND = 2u };

enum StopStatus : int { ST_RUNNING = 0, ST_STOPPED = 1, ST_NONFINITE = 2 };

constexpr long long kNoStop = 0x7fffffffffffffffLL;
constexpr int kMaxK = 64;  // steps per captured graph

// Step coefficients of the stage kernels (Sec. 2.1, S7), tabled in FP64 by
// coef_kernel for the steps of a batch.  Per step k: for each RK stage s of
// the step (stage times t, t + dt/2, t + dt/2, t + dt with t = t0 + n dt,
// n = n_base + k) and c = e^{-2 t_s} / h^2: 4/3 c, -c/12, mu^2 - 15/2 c.
// After the kMaxK steps: the dt-only constants, in the order of kCoef*.
constexpr int kCoefPerStage = 3;
constexpr int kCoefPerStep = 4 * kCoefPerStage;
enum CoefConst : int {
  kCoefSq = 0,    // [4] q weight of the stage argument P_s: 0, dt/2, dt/2, dt
  kCoefSg = 4,    // [4] G weight of P_s: 0, 0, dt^2/4, dt^2/2
  kCoefSp = 8,    // [4] G weight of the point argument Q_s: 0, dt/2, dt/2, dt
  kCoefB6 = 12,   // dt^2/6
  kCoefD6 = 13,   // dt/6
  kCoefDt = 14,   // dt
  kCoefNlam = 15, // -lambda
  kCoefConsts = 16
};
constexpr int kCoefDoubles = kMaxK * kCoefPerStep + kCoefConsts;

// Per-context state the kernels read; host keeps a mirror.  All stage kernels
// of one batch read it; only the per-batch advance kernel writes n_base,
// n_end, stop_k and status (stage-1 kernels may lower stop_k).
struct alignas(64) Desc {
  int32_t N, bc, prec, pad0;
  // z extent of the stored block: nz interior planes starting at storage plane
  // zoff (a z-slab keeps zoff = 2 halo planes on each side, filled by the halo
  // exchange); zwrap = 1 wraps z-plane indices (a periodic context stored
  // whole), else planes outside the storage read as zero.  withhold = 1 (a
  // test hook, 0 in normal use): the stages 1+2 producer of block 0 never
  // issues the first plane of its first work item, so the consumers' bounded
  // waits on a barrier nothing completes run out (HBE_ETIMEOUT)
  int32_t nz, zoff, zwrap, withhold;
  int32_t pitch_s, pitch_g;      // padded row pitch (elements) of state / G fields
  int64_t plane_s, plane_g;      // elements per padded z-plane
  double inv_h2, mu2, lambda;
  double t0, dt;
  int64_t n_base;                // steps completed before the current batch
  int64_t n_end;                 // stop stepping when n reaches this
  long long stop_k;              // first step index of the batch skipped by the stop rule
  double stop_thr;               // 0: off
  int64_t last_done;             // steps executed by the last batch (advance kernel)
  int32_t status;                // StopStatus after the last batch
  int32_t pad1;
  unsigned long long *maxabs;    // [kMaxK] max|phi| after step k of the batch (double bits)
  double *coef;                  // [kCoefDoubles] step coefficients (coef_kernel)
  // Laplacian monitor (stages 1+2 kernel with the monitor): entry n % mon_cap
  // holds max |h^2 Delta_h phi| of the state before step n as double bits
  // (atomicMax; the advance kernel zeroes the entries of the coming steps)
  unsigned long long *mon;
  int64_t mon_cap;
  const CUtensorMap *tmaps;      // [NUM_TMAPS], 64-byte aligned, in device memory
  void *f[NUM_FIELDS];
};

// One halo transfer of a z-slab decomposition: the 2 stored planes starting
// at src_plane of batch member src go to the 2 halo planes starting at
// dst_plane of member dst (whole padded planes, ghost rows and columns
// included).
struct HaloCopy {
  int32_t src, dst, src_plane, dst_plane;
};

// Work item of a stage launch: one (context, x-y tile, z-chunk) column.
// x = context index in the descriptor array, y = tile_x | tile_y << 16,
// z = first plane, w = number of planes.
using WorkItem = int4;

struct StageParams {
  Desc *descs;
  const WorkItem *items;
  const int *nitems;   // device scalar (the batch updates it between runs)
  unsigned *err;       // device error word (DevError bits)
  int k;               // step index within the batch
};

}  // namespace hbe
