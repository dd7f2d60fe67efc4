/*
 * hbe.h -- C ABI of libhbe, a GB300 (sm_103a) solver for the Higgs boson
 * equation (HBE) in de Sitter spacetime,
 *
 *     phi_tt - e^{-2t} Delta phi + 3 phi_t = mu^2 phi - lambda phi^3,          (Sec. 1, Eq. HBE)
 *     phi(x, t0) = phi0(x),  phi_t(x, t0) = phi1(x),                          (Eq. HBEinit)
 *
 * discretised as in Sec. 2.1 of Balogh, Banda & Yagdjian (arXiv:1803.01291):
 * the cube of side L centred at the origin (the paper's unit box with the
 * factor 1/L^2, Eq. higgs-boson-rescalled), a uniform grid of N^3 unknowns,
 * the 13-point fourth-order finite-difference Laplacian (Sec. 2.1), the
 * first-order system v = (phi, psi = phi_t) with right-hand side Eq. (rhs),
 * and the classic explicit fourth-order Runge-Kutta step (Sec. 2.1).
 *
 * Conventions shared by every entry point
 *   - Grid: zero-Dirichlet (Eq. BC): h = L/(N+1), node i at (i - (N-1)/2) h,
 *     phi = psi = 0 on the two ghost layers outside the box.  Periodic: h = L/N,
 *     node i at (i - N/2) h, neighbours wrap.
 *   - Host/device arrays of a field are N^3 doubles, x fastest:
 *     element (x, y, z) at index (z*N + y)*N + x.
 *   - Sign masks: N*N*W uint32 words, W = ceil(N/32); bit (x % 32) of word
 *     (z*N + y)*W + x/32 is set where the condition holds.
 *   - Time: t_n = t0 + n*dt in double precision (no running sum); the RK4
 *     stage times are t_n, t_n + dt/2, t_n + dt/2, t_n + dt (Sec. 2.1).
 *   - Every call returns an hbe_status; nothing throws or aborts.  After an
 *     error, hbe_last_error() describes it.  A context is used by one host
 *     thread at a time.  No call keeps a pointer to caller memory, except
 *     hbe_prefetch_initial and hbe_read_async, whose copies run after they
 *     return (see there: the arrays must stay valid until the matching
 *     hbe_set_initial_prefetched or hbe_read_wait).
 *   - Device memory for the fields is allocated by hbe_create (cudaMalloc)
 *     unless the caller hands a buffer of hbe_workspace_bytes() bytes to
 *     hbe_create_in, which then allocates nothing on the device for fields.
 */
#ifndef HBE_H_
#define HBE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hbe_ctx hbe_ctx;
typedef struct hbe_batch hbe_batch;

typedef enum {
  HBE_OK = 0,
  HBE_EINVAL = 1,    /* bad argument (size, pointer, parameter) */
  HBE_ENOMEM = 2,    /* device or host allocation failed */
  HBE_ECUDA = 3,     /* a CUDA call failed; see hbe_last_error */
  HBE_ESTATE = 4,    /* call out of order (e.g. step before set_initial) */
  HBE_STOPPED = 5,   /* stepping stopped early: max|phi| passed the stop threshold */
  HBE_NONFINITE = 6, /* stepping stopped early: phi became NaN or infinite */
  HBE_ETIMEOUT = 7   /* a bounded device wait expired; the context state is undefined */
} hbe_status;

typedef enum { HBE_BC_DIRICHLET0 = 0, HBE_BC_PERIODIC = 1 } hbe_bc;

/* Arithmetic of the stepping path.  t, e^{-2t}/h^2 and the stage coefficients
 * are always formed in double precision on the device.
 *   HBE_FP64       fields and arithmetic in binary64.
 *   HBE_FP32       fields and arithmetic in binary32; phi and psi carried as
 *                  compensated (hi, lo) float pairs, updated by TwoSum.
 *   HBE_BF16       as HBE_FP32, but the stage right-hand sides G1..G3 are
 *                  stored as bfloat16 (round to nearest even).
 *   HBE_FP32_PLAIN binary32 throughout, no compensation (ablation). */
typedef enum { HBE_FP64 = 0, HBE_FP32 = 1, HBE_BF16 = 2, HBE_FP32_PLAIN = 3 } hbe_prec;

typedef struct {
  double t;            /* time of the state the diagnostics describe */
  int64_t step;        /* steps taken since the last set_initial/load */
  double max_abs_phi;  /* max over the N^3 unknowns of |phi| (NaN/inf count as +inf) */
  int32_t finite;      /* 1 if every phi value is finite */
  int32_t reserved;
  int64_t n_pos;       /* 6-connected components of {phi > eps} (wrapping if periodic) */
  int64_t n_neg;       /* same for {phi < -eps} */
  int64_t bubble_count;/* max(0, n_pos + n_neg - 1): maximal connected sets across
                          which phi changes sign (the bubble definition of Sec. 1) */
} hbe_diag_t;

/* Tile configuration of the stage kernels (see hbe_variant_info). */
typedef struct {
  int32_t tile_x, tile_y;   /* x-y tile of one thread block */
  int32_t threads;          /* threads per block: 32 * (consumer_warps + 1 producer warp) */
  int32_t vec;              /* consecutive x points per lane, 1, 2 or 4 (tile_x = 32 * vec) */
  int32_t rows_per_warp;    /* tile rows per consumer warp (tile_y = consumer_warps * rows) */
  int32_t consumer_warps;
  int32_t smem_bytes[4];    /* dynamic shared memory per stage kernel */
  int32_t ring[4];          /* z-planes in the TMA ring per stage kernel */
  /* the fused stage-pair kernels (schedule 1): stages 1+2 may use a taller
   * tile with more consumer warps than the other kernels */
  int32_t pair_tile_y[2];   /* tile_y of the stages 1+2 and stages 3+4 kernels */
  int32_t pair_threads[2];
  int32_t pair_smem_bytes[2];
  int32_t pair_ring[2];
} hbe_variant_t;

/* ---- Solver context --------------------------------------------------- */

/* Bytes of device memory the fields of one context need (for hbe_create_in). */
hbe_status hbe_workspace_bytes(int N, int bc, int prec, size_t *bytes);

/* Create a solver for the N^3 problem on the box of side L with parameters
 * mu >= 0 and lambda (any sign; lambda < 0 is the focusing case, Sec. 3
 * Example blow-up).  Requires N >= 8 (periodic: N >= 8 as well), L > 0.
 * Allocates the fields on the current CUDA device.  *out receives the
 * context; it is owned by the library and released by hbe_destroy. */
hbe_status hbe_create(int N, double L, double mu, double lambda, int bc, int prec,
                      hbe_ctx **out);

/* As hbe_create, but the fields live in the caller's device buffer
 * d_workspace of at least hbe_workspace_bytes() bytes, 256-byte aligned.  The
 * buffer must stay valid until hbe_destroy; the library never frees it. */
hbe_status hbe_create_in(int N, double L, double mu, double lambda, int bc, int prec,
                         void *d_workspace, size_t bytes, hbe_ctx **out);

/* Waits for the context's work and copies, then releases everything it
 * allocated (not a caller's hbe_create_in buffer).  NULL is a no-op. */
void hbe_destroy(hbe_ctx *ctx);

/* Stream (cudaStream_t) every later call of this context enqueues on; NULL
 * is the legacy default stream. */
hbe_status hbe_set_stream(hbe_ctx *ctx, void *stream);

/* Tile variant (index into hbe_variant_info's table for this precision) and
 * z-chunk length (planes per block work item; 0 = whole column). */
hbe_status hbe_set_tuning(hbe_ctx *ctx, int variant, int zchunk);
hbe_status hbe_variant_info(int prec, int variant, hbe_variant_t *out);

/* Kernel schedule of one RK4 step (both compute the same step of Sec. 2.1):
 *   0: four launches, one per RK stage (stage s writes G_s; stage 4 applies
 *      the RK4 combine);
 *   1 (default): two launches, stages 1+2 together (G1, G2 from p, q) and
 *      stages 3+4 together with the combine (G3 stays on chip), which moves
 *      14 instead of 19 field passes per step. */
hbe_status hbe_set_schedule(hbe_ctx *ctx, int schedule);
int hbe_variant_count(int prec);

/* Initial data (Eq. HBEinit) at time t0: host arrays of N^3 doubles, copied.
 * Page-locked host arrays (cudaMallocHost / cudaHostRegister) are read by the
 * packing kernel directly over the host link; pageable arrays go through
 * device staging buffers with asynchronous copies.  Returns when the data is
 * on the device. */
hbe_status hbe_set_initial(hbe_ctx *ctx, const double *phi0, const double *phi1, double t0);
/* Same from device arrays (read on the context's stream before return). */
hbe_status hbe_set_initial_device(hbe_ctx *ctx, const double *d_phi0, const double *d_phi1,
                                  double t0);

/* Initial data (Eq. HBEinit) at time t0 as sums of the bump family of Sec. 3
 * (Eq. bump), evaluated on the device at the grid nodes in the normalisation
 *     A exp(-1 / (1 - |x - c|^2 / R^2))  for |x - c| < R,  0 outside,
 * phi0 = sum of n0 bumps (A0[i], R0[i], centre c0[3i..3i+2] = (x, y, z)),
 * phi1 = sum of n1 bumps (A1, R1, c1); n0, n1 in [0, 64]; host arrays, copied.
 * Coordinates are those of the grid convention above (box centred at 0);
 * periodic ghosts take wrapped values.  Nothing crosses the bus but the
 * parameters. */
hbe_status hbe_set_initial_bumps(hbe_ctx *ctx, int n0, const double *A0, const double *R0,
                                 const double *c0, int n1, const double *A1, const double *R1,
                                 const double *c1, double t0);

/* Stop stepping after the first step whose max|phi| exceeds threshold
 * (0 disables; a non-finite phi always stops). */
hbe_status hbe_set_stop(hbe_ctx *ctx, double threshold);

/* Advance by nsteps RK4 steps of size dt > 0 (Sec. 2.1).  Blocks until done.
 * Returns HBE_STOPPED / HBE_NONFINITE when the stop rule ended it early; the
 * state is then the one after the step that triggered it.  Changing dt
 * between calls restarts the time origin at the current t. */
hbe_status hbe_step(hbe_ctx *ctx, int64_t nsteps, double dt);

/* Enqueue nsteps steps on the context's stream without waiting; the stop
 * rule still applies on the device.  hbe_sync waits and reports status. */
hbe_status hbe_step_async(hbe_ctx *ctx, int64_t nsteps, double dt);
hbe_status hbe_sync(hbe_ctx *ctx);

/* Current state to host arrays of N^3 doubles (psi may be NULL) and time.
 * Page-locked host arrays are written by the unpacking kernel directly;
 * pageable arrays receive the data through device staging buffers. */
hbe_status hbe_read(hbe_ctx *ctx, double *phi, double *psi, double *t);
/* Same to device arrays on the context's stream (not synchronised). */
hbe_status hbe_read_device(hbe_ctx *ctx, double *d_phi, double *d_psi);

/* Streaming host I/O, for a sequence of problems solved one after another on
 * one context (the Cauchy data of Sec. 1 in, phi out) with the host-link
 * transfers overlapped with the neighbouring problems' steps.
 *
 * hbe_prefetch_initial starts copying phi0, phi1 (caller-owned host arrays of
 * N^3 doubles, [z][y][x] as for hbe_set_initial) into a device staging area of
 * the context by DMA on its copy stream and returns; page-locked arrays are
 * needed for the copy to overlap anything.  The current state is not touched,
 * so it may be called while hbe_step_async steps.  The arrays must stay
 * unchanged until hbe_set_initial_prefetched.  A second call before that
 * replaces the first.  The staging area (2 N^3 doubles) is allocated at the
 * first call and kept until hbe_destroy: HBE_ENOMEM if it does not fit.
 *
 * hbe_set_initial_prefetched(ctx, t0) makes the prefetched arrays the initial
 * data at time t0, as hbe_set_initial would; it waits for the copy and blocks.
 * HBE_ESTATE if nothing was prefetched.
 *
 * hbe_read_async waits for the steps taken (as hbe_read does), unpacks phi
 * (and psi if non-null; one of the two may be null) into a second staging
 * area on the context's stream, starts their copy to the caller's host arrays
 * (N^3 doubles each, page-locked for the copy to overlap) and returns.  Work
 * enqueued on the context afterwards (steps, new initial data) runs after the
 * unpack; the host arrays hold the values once hbe_read_wait returns.  A
 * second hbe_read_async first waits for the previous copy. */
hbe_status hbe_prefetch_initial(hbe_ctx *ctx, const double *phi0, const double *phi1);
hbe_status hbe_set_initial_prefetched(hbe_ctx *ctx, double t0);
hbe_status hbe_read_async(hbe_ctx *ctx, double *phi, double *psi);
hbe_status hbe_read_wait(hbe_ctx *ctx);
/* Profiling aid: nsteps (1..4096) RK4 steps with the step's kernels launched
 * one at a time (no graph), each bracketed by CUDA events on the context's
 * stream; ms_per_stage[i] receives the mean duration of the i-th launch of a
 * step (4 floats, caller-owned; schedule 1 fills [0] = stages 1+2 and
 * [1] = stages 3+4 and sets [2], [3] to 0).  The state advances as with
 * hbe_step.  Blocks. */
hbe_status hbe_profile_stages(hbe_ctx *ctx, int64_t nsteps, double dt, float *ms_per_stage);

/* Steps taken and current time. */
hbe_status hbe_progress(hbe_ctx *ctx, int64_t *steps, double *t);

/* Diagnostics of the current phi (Sec. 1 bubbles; Sec. 3 uses max|phi|):
 * sign masks of {phi > eps} and {phi < -eps} (host buffers of N*N*W words,
 * either may be NULL) and the component counts.  Blocks. */
hbe_status hbe_diag(hbe_ctx *ctx, double eps, hbe_diag_t *out, uint32_t *pos_mask,
                    uint32_t *neg_mask);

/* The analysis quantities of Sec. 3 on the current state (double precision):
 *   integral_phi      = h^3 sum phi: the integral of phi over the box, whose
 *                       blow-up marks the blow-up of Example 2 (Sec. 3);
 *   integral_phi3     = h^3 sum phi^3: the second bubble condition of the
 *                       corollary quoted in Example 3 asks it to stay >= 0;
 *   laplacian_monitor = e^{-2t} max |FD4 Laplacian of phi|: the quantity
 *                       P(t) of Example 4 (physical units), whose decay shows
 *                       the approach to the Duffing limit;
 *   support_points    = nodes with |phi| + |psi| > eps;
 *   condition1_violations = support nodes where (3/2 + sqrt(9/4 + mu^2)) phi +
 *                       psi >= 0, i.e. where the first bubble condition of that
 *                       corollary (read at the current time) fails.
 * The sums are added in a fixed order (bitwise reproducible).  Blocks. */
typedef struct {
  double t;
  double integral_phi;
  double integral_phi3;
  double laplacian_monitor;
  int64_t support_points;
  int64_t condition1_violations;
} hbe_analysis_t;
/* Fills *out (caller-owned) for the current state; eps >= 0 (HBE_EINVAL
 * otherwise), HBE_ESTATE without initial data. */
hbe_status hbe_analysis(hbe_ctx *ctx, double eps, hbe_analysis_t *out);

/* The Laplacian monitor P(t) = e^{-2t} max|Delta_h phi| of Sec. 3 (Example
 * long-bubble: P(t) -> 0 as the solution approaches its limit) as a
 * by-product of stepping.  With the monitor on, the stages 1+2 kernel of
 * every step n also forms max over the grid of |Delta_h phi_n| -- the FD4
 * Laplacian of the step's starting state, which is that kernel's stage-1
 * argument -- in the context's arithmetic (FP32 or FP64), and records it;
 * no extra pass over the fields.  Applies to hbe_step / hbe_step_async with
 * the fused schedule (1), not to batches.  on: 1 (allocates a history of
 * 65536 entries, 512 KiB) or 0.  Blocks. */
hbe_status hbe_set_monitor(hbe_ctx *ctx, int on);
/* P(t_n) and t_n = t0 + n dt (the current time origin) for the states before
 * steps n = first .. first + count - 1; those steps must have been taken with
 * the monitor on, and lie in the last 65472 steps (HBE_EINVAL otherwise).
 * t may be NULL.  Blocks. */
hbe_status hbe_monitor_read(hbe_ctx *ctx, int64_t first, int64_t count, double *P, double *t);

/* Raw state (both fields in storage precision, step count, t0, dt) to/from
 * a file; a load into a context of the same N, bc and precision continues
 * bit for bit. */
hbe_status hbe_save(hbe_ctx *ctx, const char *path);
hbe_status hbe_load(hbe_ctx *ctx, const char *path);

/* Text of the context's last error ("" if none; "null context" for NULL),
 * valid until the context's next call; the name of a status code ("HBE_OK",
 * ...; "unknown" for any other value), static. */
const char *hbe_last_error(const hbe_ctx *ctx);
const char *hbe_status_string(int status);

/* Number of stage-kernel launches (and, for a periodic context, ghost-copy
 * launches) this context (or batch) has enqueued; the two small bookkeeping
 * kernels of each batch of steps (step coefficients, step advance) are not
 * counted. */
int64_t hbe_launch_count(const hbe_ctx *ctx);

/* ---- Radial solutions (Sec. 2.2, Eq. radial) ---------------------------- */
/* Largest n hbe_radial_run accepts for precision prec (HBE_FP64 or HBE_FP32;
 * 0 for any other value). */
int hbe_radial_max_n(int prec);

/* Integrates a batch of radially symmetric problems, each
 *     phi_tt - e^{-2t} (phi_rr + (2/r) phi_r) + 3 phi_t = mu^2 phi - lambda phi^3
 * on 0 <= r <= R with phi_r(0) = 0 and phi(R) = 0 (the paper's Eq. radial with
 * r in (0, 1) and the factor 1/L^2 is R = L in these physical units).
 * Discretisation (Sec. 2.2): nodes r_i = i R/n, unknowns i = 0 .. n-1; the
 * fourth-order second difference of Sec. 2.1 and the fourth-order central first
 * difference in the interior; the ghosts phi(-r) = phi(r) at the origin and zero
 * from the wall on; at r = 0 the operator is 3 phi_rr(0) (L'Hospital) with the
 * even closure (-5/2 phi_0 + 8/3 phi_1 - 1/6 phi_2)/dr^2.  Classic RK4 in time,
 * stage times as for hbe_step, t_n = t0 + n dt.
 *
 * All array arguments are DEVICE pointers owned by the caller:
 *   d_mu, d_lambda       [batch] doubles: each problem's mu and lambda;
 *   d_phi0, d_phi1       [batch][n] doubles: phi and phi_t at the nodes at t0;
 *   d_phi, d_psi         [batch][n] doubles, written: phi and phi_t after the
 *                        last step taken (may not alias the inputs);
 *   d_records            [batch][nsteps / record_every][3] doubles, written
 *                        after every record_every-th step: t, max|phi|, and the
 *                        number of strict sign changes of phi along r with
 *                        |phi| <= eps ignored (each is a spherical shell where
 *                        the solution changes sign).  Needed only when
 *                        record_every > 0 and nsteps >= record_every;
 *   d_steps (int64), d_status (int32)   [batch], optional (NULL): steps taken
 *                        and 0 (all steps), 1 (max|phi| passed stop > 0) or 2
 *                        (phi not finite); a problem ends after the first such
 *                        step, the others keep going.
 * prec: HBE_FP64, or HBE_FP32 (state and arithmetic in binary32, t and the
 * stage coefficients formed in binary64).  4 <= n <= hbe_radial_max_n(prec).
 * stop = 0 disables the threshold; non-finite values always end a problem.
 * One CTA per problem integrates all steps on chip; the stage coefficients
 * e^{-2 t_s} / dr^2, the same for every problem, are tabled once per call in
 * a stream-ordered temporary of 4 entries a step (16 bytes a step in FP32,
 * 32 in FP64), freed on the stream after the solve.
 * Asynchronous on `stream` (cudaStream_t, NULL = legacy default); returns
 * HBE_EINVAL for bad arguments (nothing is launched), HBE_ENOMEM if the table
 * cannot be allocated and HBE_ECUDA if the launch fails. */
hbe_status hbe_radial_run(int batch, int n, double R, const double *d_mu, const double *d_lambda,
                          const double *d_phi0, const double *d_phi1, double t0, double dt,
                          int64_t nsteps, int prec, int record_every, double stop, double eps,
                          double *d_phi, double *d_psi, double *d_records, int64_t *d_steps,
                          int32_t *d_status, void *stream);

/* ---- Stepping without device allocation -------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory at the moment they step a problem: runtimes
 * that own all device memory through their own pool and forbid other
 * allocations, real-time loops where cudaMalloc may block or fail under
 * memory pressure, and code that must not grow the device footprint once it
 * is set up.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * The caller passes the initial fields d_phi0, d_phi1 and the result fields
 * d_phi, d_psi (device arrays of N^3 doubles, x fastest); every intermediate
 * array (padded state, stage values, kernel descriptors) lives in one fixed
 * __device__ array inside libhbe of 7.33 MB (7,333,888 bytes), which every
 * GPU that loads the library holds until the process exits.  FP64
 * arithmetic; N in [8, 48], and a larger N returns HBE_EINVAL because the
 * array holds nothing bigger.  Grid, boundary and time conventions as for
 * hbe_create / hbe_step: nsteps RK4 steps of size dt (finite, > 0) from time
 * t0; nsteps = 0 returns the initial data.  A step whose phi is not finite
 * ends the solve: the call returns HBE_NONFINITE and the outputs hold the
 * state after that step (what hbe_read gives after hbe_step reports
 * HBE_NONFINITE).  The call copies its descriptors from host memory,
 * synchronises `stream` (cudaStream_t, NULL = legacy default) and blocks
 * until done, so it must run on a stream that is not being captured into a
 * CUDA graph.  The first call on a device looks up the array's device address
 * with that device current.  All calls share the one array (each clears what
 * must start at zero), so calls that overlap on the GPU race.  Returns
 * HBE_ETIMEOUT if a kernel's bounded wait expired. */
hbe_status hbe_step_fp64_noalloc(int N, double L, double mu, double lambda, int bc,
                                 const double *d_phi0, const double *d_phi1, double t0,
                                 double dt, int64_t nsteps, double *d_phi, double *d_psi,
                                 void *stream);

/* ---- Batched stepping (continuous batching) ---------------------------- */
/* A batch advances many contexts of one precision together: every RK4 stage
 * is one persistent kernel launch over the tiles of all members, and K steps
 * are replayed as one CUDA graph.  Members join and leave between runs
 * without re-capturing the graph.  A member's per-point arithmetic is the same
 * as when it steps alone, so its results are bitwise identical.  */

/* K = steps per run (1..64).  stream as in hbe_set_stream. */
hbe_status hbe_batch_create(int prec, int K, void *stream, hbe_batch **out);
void hbe_batch_destroy(hbe_batch *b);
/* Admit ctx (same precision, state set) with nsteps more steps of size dt. */
hbe_status hbe_batch_add(hbe_batch *b, hbe_ctx *ctx, int64_t nsteps, double dt);
/* Remove a member (finished or not); its state stays readable. */
hbe_status hbe_batch_remove(hbe_batch *b, hbe_ctx *ctx);
/* One run: up to K steps for every member.  On return *n_finished holds how
 * many members reached their step count or stopped, listed in finished[]
 * (capacity max_finished); they are removed from the batch.  Equivalent to
 * hbe_batch_launch followed by hbe_batch_collect. */
hbe_status hbe_batch_run(hbe_batch *b, hbe_ctx **finished, int max_finished, int *n_finished);
/* The two halves of hbe_batch_run.  hbe_batch_launch enqueues one run on the
 * batch's stream and returns at once; hbe_batch_collect waits for it and
 * retires the members that finished, as hbe_batch_run does.  Between the two
 * the host may work on members retired earlier (read them, run diagnostics
 * on another stream); hbe_batch_add, hbe_batch_remove and a second launch
 * return HBE_ESTATE until the run is collected.  Collecting with no run in
 * flight returns HBE_OK and no members. */
hbe_status hbe_batch_launch(hbe_batch *b);
hbe_status hbe_batch_collect(hbe_batch *b, hbe_ctx **finished, int max_finished,
                             int *n_finished);
int hbe_batch_size(const hbe_batch *b);
const char *hbe_batch_last_error(const hbe_batch *b);
int64_t hbe_batch_launch_count(const hbe_batch *b);

/* ---- z-slab decomposition (virtual slabs on one GPU) ------------------- */
/* The grid split along z into k slabs that exchange 2-plane halos after each
 * fused stage pair, the partitioning a run over several GPUs would use (the
 * stencil of Sec. 2.1 reaches 2 planes, so every stage argument read with a
 * halo -- phi, psi after stages 3+4, G1, G2 after stages 1+2 -- needs 2 planes
 * of each neighbour).  Here all slabs live on the current device and the
 * halos are plain device copies into the receiving slab's own buffers; the
 * result is bitwise that of the undivided grid. */
typedef struct hbe_slabs hbe_slabs;

/* The exchange plan: nz[i] = planes of slab i (N/k, +1 for the first N % k
 * slabs); each transfer is 4 ints (source slab, destination slab, first
 * stored plane at the source, first halo plane at the destination), 2
 * planes each.  A slab stores its nz planes at stored planes 2 .. nz+1, with
 * halo planes 0, 1 below and nz+2, nz+3 above.  Periodic: slab 0 and slab k-1
 * are neighbours.  Pure host function (no CUDA call).  Returns the number of
 * transfers (2k periodic, 2k - 2 Dirichlet; copies may be NULL to count), or
 * -1 if k < 1, N < 2k or max_copies is too small. */
int hbe_slab_plan(int N, int k, int periodic, int32_t *nz, int32_t *copies, int max_copies);

/* k slabs of the problem of hbe_create (same arguments), work on `stream`
 * (cudaStream_t, NULL = legacy default).  No stop threshold: a slab that
 * turns non-finite ends the steps of all slabs with HBE_NONFINITE. */
hbe_status hbe_slabs_create(int N, double L, double mu, double lambda, int bc, int prec, int k,
                            void *stream, hbe_slabs **out);
void hbe_slabs_destroy(hbe_slabs *s);
/* Initial data from device arrays of N^3 doubles (x fastest); blocks. */
hbe_status hbe_slabs_set_initial_device(hbe_slabs *s, const double *d_phi0,
                                        const double *d_phi1, double t0);
/* nsteps RK4 steps of size dt on every slab (blocks until done). */
hbe_status hbe_slabs_step(hbe_slabs *s, int64_t nsteps, double dt);
/* The whole grid's state into device arrays of N^3 doubles (either may be
 * NULL) and the current time. */
hbe_status hbe_slabs_read_device(hbe_slabs *s, double *d_phi, double *d_psi, double *t);
const char *hbe_slabs_last_error(const hbe_slabs *s);

#ifdef __cplusplus
}
#endif
#endif /* HBE_H_ */
