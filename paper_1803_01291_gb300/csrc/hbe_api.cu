// hbe_api.cu -- the C ABI of libhbe (include/hbe.h): contexts, device memory,
// TMA descriptors, work lists, CUDA-graph stepping, diagnostics, checkpoints
// and the batched (continuous-batching) runner.
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "hbe.h"
#include "hbe_aux.h"
#include "hbe_common.cuh"
#include "hbe_variants.h"

using namespace hbe;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
std::mutex g_attr_mu;
std::set<const void *> g_attr_done;

const VariantTable &table_for(int prec) {
  switch (prec) {
    case HBE_FP64: return variants_fp64();
    case HBE_FP32: return variants_fp32();
    case HBE_BF16: return variants_bf16();
    default: return variants_fp32_plain();
  }
}

int state_size(int prec) { return prec == HBE_FP64 ? 8 : 4; }
int g_size(int prec) { return prec == HBE_FP64 ? 8 : (prec == HBE_BF16 ? 2 : 4); }
bool is_kahan(int prec) { return prec == HBE_FP32 || prec == HBE_BF16; }

CUtensorMapDataType tm_type(int esize) {
  return esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                    : (esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

constexpr int64_t kMonCap = 65536;  // monitor history: the last 65536 - kMaxK steps

}  // namespace

struct hbe_ctx {
  int N = 0, bc = 0, prec = 0;
  int nz = 0, zoff = 0;  // stored z-planes: nz interior after zoff halo planes (a z-slab: 2)
  double L = 0, mu = 0, lambda = 0, h = 0;
  int device = 0, sms = 0;
  cudaStream_t stream = nullptr;      // user stream (work is enqueued here)
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  int variant = 0, zchunk = 0;
  int hxs = 0, hxg = 0, pitch_s = 0, pitch_g = 0;
  int64_t plane_s = 0, plane_g = 0;
  size_t bytes_s = 0, bytes_g = 0, ws_bytes = 0;
  void *ws = nullptr;
  bool own_ws = false;
  void *f[NUM_FIELDS] = {};
  CUtensorMap *d_tmaps = nullptr;
  unsigned long long *d_maxabs = nullptr;
  double *d_coef = nullptr;          // step coefficients (Desc::coef)
  Desc *d_desc = nullptr;
  Desc *h_desc = nullptr;  // pinned mirror
  WorkItem *d_items = nullptr;
  int *d_nitems = nullptr;
  int *d_one = nullptr;
  int nitems = 0, items_cap = 0;
  // work list of the stages 1+2 kernel, whose tile may differ from the others'
  WorkItem *d_items_p = nullptr;
  int *d_nitems_p = nullptr;
  int nitems_p = 0, items_cap_p = 0, zchunk_p = 0;
  int grid[7] = {0, 0, 0, 0, 0, 0, 0};  // [6]: the stages 1+2 kernel with the monitor
  int schedule = 1;  // 0: four one-stage kernels per step; 1: two fused stage pairs
  bool monitor = false;                 // stages 1+2 record the Laplacian monitor
  unsigned long long *d_mon = nullptr;  // kMonCap monitor entries (Desc::mon)
  unsigned *d_err = nullptr;
  int K = 8;
  // gexec[n]: graph of n RK4 steps (n = K for the full replays, n < K for the
  // last replay of a call whose step count is not a multiple of K)
  cudaGraphExec_t gexec[kMaxK + 1] = {};
  double *d_stage = nullptr;   // 2 buffer sets x 2 fields x stage_elems doubles
  size_t stage_elems = 0;
  cudaStream_t copy_stream = nullptr;   // host <-> staging copies
  cudaEvent_t ev_ready[2] = {}, ev_free[2] = {};
  // streaming host I/O (hbe_prefetch_initial, hbe_read_async): whole-field
  // staging areas of 2 N^3 doubles each, allocated at first use
  double *d_pre = nullptr, *d_rout = nullptr;
  cudaEvent_t ev_pre = nullptr, ev_rout_ready = nullptr, ev_rout_done = nullptr;
  bool pre_pending = false;    // a prefetch not yet consumed
  bool rout_pending = false;   // a read whose copy to the host may still run
  uint32_t *d_masks = nullptr;
  int *d_labels = nullptr;
  unsigned long long *d_counts = nullptr;
  double *d_part = nullptr;  // analysis partials (5 x blocks) + result (5)
  bool has_state = false;
  bool pending = false;        // device work enqueued since the last sync
  bool desc_stale = false;     // device descriptor older than the host mirror
  bool in_batch = false;
  int64_t launches = 0;
  std::string err;
};

struct hbe_batch {
  int prec = 0, K = 8, sms = 0, device = 0;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::vector<hbe_ctx *> members;
  Desc *d_descs = nullptr, *h_descs = nullptr;
  int *d_ndesc = nullptr;
  int cap_desc = 0;
  struct List {
    WorkItem *d_items = nullptr;
    int *d_n = nullptr;
    int cap = 0;
    int grid[6] = {0, 0, 0, 0, 0, 0};
  } lists[kMaxVariants], lists_p[kMaxVariants];  // lists_p: the stages 1+2 kernel's tiles
  int nvariants = 0;
  unsigned *d_err = nullptr;
  unsigned *h_err = nullptr;    // pinned copy of d_err, read after a run
  cudaGraphExec_t gexec = nullptr;
  unsigned graph_variants = 0;  // bit v: the captured graph launches variant v's kernels
  bool dirty = true;
  bool wraps = false;  // the captured graph has the periodic ghost copies
  bool in_flight = false;       // a run is enqueued and not yet collected
  int run_members = 0;          // members of the run in flight
  cudaEvent_t ev_done = nullptr;
  // z-slab decomposition: halo transfers between members (member i = slab i)
  // after each stage pair; empty for an ordinary batch
  HaloCopy *d_halo = nullptr;
  int nhalo = 0;
  int64_t launches = 0;
  std::string err;
};

namespace {

hbe_status set_err(std::string &dst, hbe_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  dst = buf;
  return st;
}

#define CKX(dst, call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return set_err(dst, e_ == cudaErrorMemoryAllocation ? HBE_ENOMEM : HBE_ECUDA,        \
                     "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,       \
                     __LINE__);                                                              \
  } while (0)
#define CK(call) CKX(ctx->err, call)

hbe_status prepare_kernel(std::string &err, const KernelInfo &ki) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done.count(ki.fn)) return HBE_OK;
  CKX(err, cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem));
  g_attr_done.insert(ki.fn);
  return HBE_OK;
}

hbe_status persistent_grid(std::string &err, const KernelInfo &ki, int sms, int *out) {
  hbe_status st = prepare_kernel(err, ki);
  if (st != HBE_OK) return st;
  int nb = 0;
  CKX(err, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ki.fn, ki.threads, ki.smem));
  if (nb < 1) return set_err(err, HBE_ECUDA, "stage kernel does not fit on an SM");
  *out = nb * sms;
  return HBE_OK;
}

hbe_status get_encoder(std::string &err) {
  std::call_once(g_encode_once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return set_err(err, HBE_ECUDA, "cuTensorMapEncodeTiled unavailable");
  return HBE_OK;
}

// 3D map over a padded field: dims (pitch, N + 4, N), box (bx, by, 1).
hbe_status encode_map(hbe_ctx *ctx, CUtensorMap *m, void *base, int esize, int pitch, int bx,
                      int by) {
  cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)(ctx->N + 4),
                        (cuuint64_t)(ctx->nz + 2 * ctx->zoff)};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)pitch * (ctx->N + 4) * esize};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, tm_type(esize), 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_err(ctx->err, HBE_ECUDA, "cuTensorMapEncodeTiled failed (%d), box %dx%d", (int)r,
                   bx, by);
  return HBE_OK;
}

// z-chunk length minimising (waves of work items) x (planes per item, with the
// 4 planes of start-up each chunk costs) over the resident blocks.
int auto_zchunk(int N, int columns, int resident) {
  double best = 1e300;
  int best_zc = N;
  for (int nz = 1; nz <= std::max(1, N / 16); ++nz) {
    const int zc = (N + nz - 1) / nz;
    const int items = columns * ((N + zc - 1) / zc);
    const double waves = std::ceil((double)items / resident);
    const double cost = waves * (zc + 4);
    if (cost < best - 1e-9) {
      best = cost;
      best_zc = zc;
    }
  }
  return best_zc;
}

// Work items of one context for the tile of stage kernel `kidx` (0: the
// tile of every kernel but the stages 1+2 one, 4: that kernel's), ordered
// z-chunk, then y, then x (neighbouring tiles run together, so halo rows are
// still in L2 when they are read).
void build_items(const hbe_ctx *ctx, int member, int zchunk, int kidx, std::vector<WorkItem> &out) {
  const KernelInfo &ki = table_for(ctx->prec).k[ctx->variant][kidx];
  const int tx = (ctx->N + ki.tx - 1) / ki.tx, ty = (ctx->N + ki.ty - 1) / ki.ty;
  for (int z0 = 0; z0 < ctx->nz; z0 += zchunk)
    for (int j = 0; j < ty; ++j)
      for (int i = 0; i < tx; ++i)
        out.push_back(make_int4(member, i | (j << 16), z0, std::min(zchunk, ctx->nz - z0)));
}

void drop_graphs(hbe_ctx *ctx) {
  for (auto &g : ctx->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

hbe_status apply_tuning(hbe_ctx *ctx, int variant, int zchunk) {
  const VariantTable &vt = table_for(ctx->prec);
  if (variant < 0 || variant >= vt.count)
    return set_err(ctx->err, HBE_EINVAL, "variant %d out of range [0, %d)", variant, vt.count);
  if (zchunk < 0) return set_err(ctx->err, HBE_EINVAL, "zchunk must be >= 0");
  const KernelInfo *ks = vt.k[variant];
  ctx->variant = variant;
  // tensor maps for this tile shape
  const int es = state_size(ctx->prec), eg = g_size(ctx->prec);
  const int tx = ks[0].tx, ty = ks[0].ty;
  const int bxs = tx + 2 * ctx->hxs, bxg = tx + 2 * ctx->hxg, by = ty + 4;
  CUtensorMap maps[NUM_TMAPS];
  memset(maps, 0, sizeof(maps));
  hbe_status st;
  auto E = [&](int idx, int field, int esz, int pitch, int bx, int byy) {
    void *base = ctx->f[field] ? ctx->f[field] : ctx->f[F_P0];  // unused maps point at p
    return encode_map(ctx, &maps[idx], base, esz, pitch, bx, byy);
  };
  if ((st = E(TM_P_H0, F_P0, es, ctx->pitch_s, bxs, by))) return st;
  if ((st = E(TM_P_H1, F_P1, es, ctx->pitch_s, bxs, by))) return st;
  if ((st = E(TM_Q_H0, F_Q0, es, ctx->pitch_s, bxs, by))) return st;
  if ((st = E(TM_Q_H1, F_Q1, es, ctx->pitch_s, bxs, by))) return st;
  if ((st = E(TM_Q_I0, F_Q0, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_Q_I1, F_Q1, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_PLO_I0, F_PLO0, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_PLO_I1, F_PLO1, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_QLO_I0, F_QLO0, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_QLO_I1, F_QLO1, es, ctx->pitch_s, tx, ty))) return st;
  if ((st = E(TM_G1_H, F_G1, eg, ctx->pitch_g, bxg, by))) return st;
  if ((st = E(TM_G1_I, F_G1, eg, ctx->pitch_g, tx, ty))) return st;
  if ((st = E(TM_G2_H, F_G2, eg, ctx->pitch_g, bxg, by))) return st;
  if ((st = E(TM_G2_I, F_G2, eg, ctx->pitch_g, tx, ty))) return st;
  if ((st = E(TM_G3_I, F_G3, eg, ctx->pitch_g, tx, ty))) return st;
  // halo boxes of p and q for the stages 1+2 kernel's own tile
  const int txp = ks[4].tx, typ = ks[4].ty;
  if ((st = E(TM_P_H0_P, F_P0, es, ctx->pitch_s, txp + 2 * ctx->hxs, typ + 4))) return st;
  if ((st = E(TM_P_H1_P, F_P1, es, ctx->pitch_s, txp + 2 * ctx->hxs, typ + 4))) return st;
  if ((st = E(TM_Q_H0_P, F_Q0, es, ctx->pitch_s, txp + 2 * ctx->hxs, typ + 4))) return st;
  if ((st = E(TM_Q_H1_P, F_Q1, es, ctx->pitch_s, txp + 2 * ctx->hxs, typ + 4))) return st;
  CK(cudaMemcpy(ctx->d_tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice));
  // persistent grid per stage and the two work lists
  int resident = 1 << 30;
  for (int s = 0; s < 7; ++s) {
    if ((st = persistent_grid(ctx->err, ks[s], ctx->sms, &ctx->grid[s]))) return st;
    if (s != 4 && s != 6) resident = std::min(resident, ctx->grid[s]);
  }
  const int columns = ((ctx->N + tx - 1) / tx) * ((ctx->N + ty - 1) / ty);
  const int columns_p = ((ctx->N + txp - 1) / txp) * ((ctx->N + typ - 1) / typ);
  ctx->zchunk = zchunk > 0 ? std::min(zchunk, ctx->nz) : auto_zchunk(ctx->nz, columns, resident);
  ctx->zchunk_p =
      zchunk > 0 ? std::min(zchunk, ctx->nz) : auto_zchunk(ctx->nz, columns_p, ctx->grid[4]);
  for (int li = 0; li < 2; ++li) {
    std::vector<WorkItem> items;
    build_items(ctx, 0, li ? ctx->zchunk_p : ctx->zchunk, li ? 4 : 0, items);
    WorkItem *&d_items = li ? ctx->d_items_p : ctx->d_items;
    int &cap = li ? ctx->items_cap_p : ctx->items_cap;
    int &n = li ? ctx->nitems_p : ctx->nitems;
    if ((int)items.size() > cap) {
      if (d_items) cudaFree(d_items);
      d_items = nullptr;
      CK(cudaMalloc(&d_items, items.size() * sizeof(WorkItem)));
      cap = (int)items.size();
    }
    n = (int)items.size();
    CK(cudaMemcpy(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(li ? ctx->d_nitems_p : ctx->d_nitems, &n, sizeof(int), cudaMemcpyHostToDevice));
  }
  for (int s = 0; s < 7; ++s)
    ctx->grid[s] = std::min(ctx->grid[s], (s == 4 || s == 6) ? ctx->nitems_p : ctx->nitems);
  drop_graphs(ctx);
  return HBE_OK;
}

// Parameters of stage kernel s (0..5) of a context for step k of a graph replay.
StageParams ctx_params(const hbe_ctx *ctx, int s, int k) {
  return StageParams{ctx->d_desc, s == 4 ? ctx->d_items_p : ctx->d_items,
                     s == 4 ? ctx->d_nitems_p : ctx->d_nitems, ctx->d_err, k};
}

hbe_status launch_stage(std::string &err, const KernelInfo &ki, int grid, const StageParams &p,
                        cudaStream_t st) {
  StageParams prm = p;
  void *args[] = {&prm};
  CKX(err, cudaLaunchKernel(ki.fn, dim3(grid), dim3(ki.threads), args, ki.smem, st));
  return HBE_OK;
}

// Debug mode: periodic contexts start with NaN bit patterns in every field
// (HBE_DEBUG_NAN_GHOSTS set and not "0"), read at each context creation.
// Device-side address of a host buffer the GPU can read and write directly
// (page-locked memory: cudaMallocHost, cudaHostAlloc or cudaHostRegister), or
// nullptr for pageable memory.  On a Grace host such a buffer is reached over
// NVLink-C2C by ordinary loads and stores, so the pack / unpack kernels can
// move the fields without the copy engines or a staging buffer.
const void *pinned_device_ptr(const void *host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Test hook for the bounded waits (HBE_DEBUG_WITHHOLD_PLANE set and not "0",
// read at each context creation): see Desc::withhold.
bool withhold_plane() {
  const char *v = std::getenv("HBE_DEBUG_WITHHOLD_PLANE");
  return v && *v && std::strcmp(v, "0") != 0;
}

bool nan_canary(const hbe_ctx *ctx) {
  if (ctx->bc != HBE_BC_PERIODIC) return false;
  const char *v = std::getenv("HBE_DEBUG_NAN_GHOSTS");
  return v && *v && std::strcmp(v, "0") != 0;
}

// NVTX range over a host call (visible in Nsight timelines; no cost without a tool)
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// blocks of the ghost-copy launch of one context: a thread per row of a plane
// (N^2 rows; more threads in flight hide the latency of the scattered accesses)
int wrap_blocks(const hbe_ctx *ctx) {
  const long long rows = (long long)ctx->N * ctx->N;
  return (int)std::min<long long>(4096, std::max<long long>(2 * ctx->sms, (rows + 255) / 256));
}

// kernels one RK4 step launches: the stage kernels, and for a periodic context
// the ghost copy after each stage whose output is read with a halo
int launches_per_step(const hbe_ctx *ctx) {
  const int first = ctx->schedule ? 4 : 0, last = ctx->schedule ? 6 : 4;
  int n = last - first;
  if (ctx->bc == HBE_BC_PERIODIC)
    for (int s = first; s < last; ++s) n += stage_needs_wrap(s + 1) ? 1 : 0;
  return n;
}

// The graph of nk RK4 steps: step coefficients, nk x (stage kernels + ghost
// copies), advance.
hbe_status ensure_graph(hbe_ctx *ctx, int nk) {
  if (ctx->gexec[nk]) return HBE_OK;
  const VariantTable &vt = table_for(ctx->prec);
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  hbe_status st = HBE_OK;
  const int first = ctx->schedule ? 4 : 0, last = ctx->schedule ? 6 : 4;
  cudaError_t ec = launch_coef(ctx->d_desc, ctx->d_one, 1, nk, ctx->cap_stream);
  if (ec != cudaSuccess) st = set_err(ctx->err, HBE_ECUDA, "%s", cudaGetErrorString(ec));
  for (int k = 0; k < nk && st == HBE_OK; ++k)
    for (int s = first; s < last && st == HBE_OK; ++s) {
      const int kid = (s == 4 && ctx->monitor) ? 6 : s;  // stages 1+2 with the monitor
      st = launch_stage(ctx->err, vt.k[ctx->variant][kid], ctx->grid[kid], ctx_params(ctx, s, k),
                        ctx->cap_stream);
      if (st == HBE_OK && ctx->bc == HBE_BC_PERIODIC && stage_needs_wrap(s + 1)) {
        cudaError_t ew = launch_wrap(ctx->d_desc, ctx->d_one, 1, k, s + 1, wrap_blocks(ctx),
                                     ctx->cap_stream);
        if (ew != cudaSuccess) st = set_err(ctx->err, HBE_ECUDA, "%s", cudaGetErrorString(ew));
      }
    }
  cudaError_t e = launch_advance(ctx->d_desc, ctx->d_one, 1, nk, ctx->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (st != HBE_OK) return st;
  CK(e);
  CK(e2);
  e = cudaGraphInstantiate(&ctx->gexec[nk], g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return HBE_OK;
}

hbe_status ensure_stage_buffer(hbe_ctx *ctx) {
  if (ctx->d_stage) return HBE_OK;
  const size_t plane = (size_t)ctx->N * ctx->N;
  size_t planes = std::max<size_t>(1, (size_t)(4u << 20) / plane);  // <= 32 MiB of doubles
  planes = std::min<size_t>(planes, (size_t)ctx->N);
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) {
    if (!ctx->ev_ready[b]) CK(cudaEventCreateWithFlags(&ctx->ev_ready[b], cudaEventDisableTiming));
    if (!ctx->ev_free[b]) CK(cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming));
  }
  CK(cudaMalloc(&ctx->d_stage, 4 * planes * plane * sizeof(double)));
  ctx->stage_elems = planes * plane;
  return HBE_OK;
}

hbe_status sync_ctx(hbe_ctx *ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->pending) {
    CK(cudaMemcpy(ctx->h_desc, ctx->d_desc, sizeof(Desc), cudaMemcpyDeviceToHost));
    ctx->pending = false;
  }
  unsigned e = 0;
  CK(cudaMemcpy(&e, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (e & DEV_ERR_TIMEOUT)
    return set_err(ctx->err, HBE_ETIMEOUT, "a stage kernel's TMA wait timed out");
  if (e & DEV_ERR_UNIONFIND)
    return set_err(ctx->err, HBE_ETIMEOUT, "connected-component union did not converge");
  return HBE_OK;
}

hbe_status push_desc(hbe_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->d_desc, ctx->h_desc, sizeof(Desc), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->desc_stale = false;
  return HBE_OK;
}

double current_t(const hbe_ctx *ctx) {
  return ctx->h_desc->t0 + (double)ctx->h_desc->n_base * ctx->h_desc->dt;
}

hbe_status validate(std::string &err, int N, double L, double mu, double lambda, int bc, int prec) {
  if (N < 8 || N > 2048) return set_err(err, HBE_EINVAL, "N=%d outside [8, 2048]", N);
  if (!(L > 0.0) || !std::isfinite(L)) return set_err(err, HBE_EINVAL, "L must be finite and > 0");
  if (!(mu >= 0.0) || !std::isfinite(mu)) return set_err(err, HBE_EINVAL, "mu must be finite and >= 0");
  if (!std::isfinite(lambda)) return set_err(err, HBE_EINVAL, "lambda must be finite");
  if (bc != HBE_BC_DIRICHLET0 && bc != HBE_BC_PERIODIC) return set_err(err, HBE_EINVAL, "bad bc %d", bc);
  if (prec < HBE_FP64 || prec > HBE_FP32_PLAIN) return set_err(err, HBE_EINVAL, "bad precision %d", prec);
  return HBE_OK;
}

// Padded layout of a field of N x N x planes stored elements.
void layout(int N, int planes, int prec, int *hxs, int *hxg, int *ps, int *pg, int64_t *pls,
            int64_t *plg, size_t *bs, size_t *bg) {
  const int es = state_size(prec), eg = g_size(prec);
  *hxs = 16 / es;
  *hxg = 16 / eg;
  *ps = round_up(N + 2 * *hxs, *hxs);
  *pg = round_up(N + 2 * *hxg, *hxg);
  *pls = (int64_t)(N + 4) * *ps;
  *plg = (int64_t)(N + 4) * *pg;
  *bs = (size_t)(((size_t)*pls * planes * es + 255) / 256 * 256);
  *bg = (size_t)(((size_t)*plg * planes * eg + 255) / 256 * 256);
}

size_t workspace_bytes(int N, int prec, int planes) {
  int a, b, c, d;
  int64_t e, f;
  size_t bs, bg;
  layout(N, planes, prec, &a, &b, &c, &d, &e, &f, &bs, &bg);
  const int nstate = is_kahan(prec) ? 8 : 4;
  return nstate * bs + 3 * bg;
}

// Host-side fault injection for tests: HBE_FAULT="alloc:k" makes the k-th
// context creation, counted from when the variable took its current value,
// fail with HBE_ENOMEM as if the device were out of memory.
bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char *v = std::getenv("HBE_FAULT");
  const std::string cur = v ? v : "";
  std::lock_guard<std::mutex> lock(mu);
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.compare(0, 6, "alloc:") != 0) return false;
  return ++count == std::atol(cur.c_str() + 6);
}

// A context of the N^3 problem storing nz z-planes after zoff halo planes
// (nz = N, zoff = 0: the whole grid; zoff = 2: one z-slab of a decomposition).
hbe_status create_common(int N, double L, double mu, double lambda, int bc, int prec, void *ws,
                         size_t bytes, hbe_ctx **out, int nz = 0, int zoff = 0) {
  if (!out) return HBE_EINVAL;
  *out = nullptr;
  hbe_ctx *ctx = new hbe_ctx();
  hbe_status st = validate(ctx->err, N, L, mu, lambda, bc, prec);
  if (st == HBE_OK) st = get_encoder(ctx->err);
  auto bail = [&](hbe_status s) {
    hbe_destroy(ctx);
    return s;
  };
  if (st != HBE_OK) return bail(st);
  if (injected_alloc_failure()) return bail(HBE_ENOMEM);
  ctx->N = N; ctx->L = L; ctx->mu = mu; ctx->lambda = lambda; ctx->bc = bc; ctx->prec = prec;
  ctx->nz = nz > 0 ? nz : N;
  ctx->zoff = zoff;
  ctx->h = bc == HBE_BC_PERIODIC ? L / N : L / (N + 1);
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    set_err(ctx->err, HBE_ECUDA, "no CUDA device");
    return bail(HBE_ECUDA);
  }
  const int planes = ctx->nz + 2 * ctx->zoff;
  layout(N, planes, prec, &ctx->hxs, &ctx->hxg, &ctx->pitch_s, &ctx->pitch_g, &ctx->plane_s,
         &ctx->plane_g, &ctx->bytes_s, &ctx->bytes_g);
  ctx->ws_bytes = workspace_bytes(N, prec, planes);
  if (ws) {
    if (bytes < ctx->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255u)) {
      set_err(ctx->err, HBE_EINVAL, "workspace too small (%zu < %zu) or not 256-byte aligned",
              bytes, ctx->ws_bytes);
      return bail(HBE_EINVAL);
    }
    ctx->ws = ws;
  } else {
    if (cudaMalloc(&ctx->ws, ctx->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      set_err(ctx->err, HBE_ENOMEM, "cudaMalloc of %zu bytes failed", ctx->ws_bytes);
      return bail(HBE_ENOMEM);
    }
    ctx->own_ws = true;
  }
  // carve the fields
  char *p = static_cast<char *>(ctx->ws);
  const int state_fields[] = {F_P0, F_P1, F_Q0, F_Q1, F_PLO0, F_PLO1, F_QLO0, F_QLO1};
  const int nstate = is_kahan(prec) ? 8 : 4;
  for (int i = 0; i < nstate; ++i) { ctx->f[state_fields[i]] = p; p += ctx->bytes_s; }
  for (int i = 0; i < 3; ++i) { ctx->f[F_G1 + i] = p; p += ctx->bytes_g; }
#define CKB(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      set_err(ctx->err, HBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
      return bail(e_ == cudaErrorMemoryAllocation ? HBE_ENOMEM : HBE_ECUDA);        \
    }                                                                               \
  } while (0)
  // zero: the Dirichlet ghost layers (never written again).  A periodic context
  // under HBE_DEBUG_NAN_GHOSTS starts from all-ones bit patterns instead (NaN in
  // every precision), so that any ghost cell a stage reads before the ghost copy
  // has refreshed it turns the result non-finite.
  CKB(cudaMemset(ctx->ws, nan_canary(ctx) ? 0xFF : 0, ctx->ws_bytes));
  CKB(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  CKB(cudaMalloc(&ctx->d_tmaps, NUM_TMAPS * sizeof(CUtensorMap)));
  CKB(cudaMalloc(&ctx->d_maxabs, kMaxK * sizeof(unsigned long long)));
  CKB(cudaMemset(ctx->d_maxabs, 0, kMaxK * sizeof(unsigned long long)));
  CKB(cudaMalloc(&ctx->d_coef, kCoefDoubles * sizeof(double)));
  CKB(cudaMemset(ctx->d_coef, 0, kCoefDoubles * sizeof(double)));
  CKB(cudaMalloc(&ctx->d_desc, sizeof(Desc)));
  CKB(cudaMallocHost(&ctx->h_desc, sizeof(Desc)));
  CKB(cudaMalloc(&ctx->d_nitems, sizeof(int)));
  CKB(cudaMalloc(&ctx->d_nitems_p, sizeof(int)));
  CKB(cudaMalloc(&ctx->d_one, sizeof(int)));
  CKB(cudaMalloc(&ctx->d_err, sizeof(unsigned)));
  CKB(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  const int one = 1;
  CKB(cudaMemcpy(ctx->d_one, &one, sizeof(int), cudaMemcpyHostToDevice));
  Desc &d = *ctx->h_desc;
  memset(&d, 0, sizeof(Desc));
  d.N = N; d.bc = bc; d.prec = prec;
  d.nz = ctx->nz; d.zoff = ctx->zoff;
  d.zwrap = (bc == HBE_BC_PERIODIC && ctx->zoff == 0) ? 1 : 0;
  d.withhold = withhold_plane() ? 1 : 0;
  d.pitch_s = ctx->pitch_s; d.pitch_g = ctx->pitch_g;
  d.plane_s = ctx->plane_s; d.plane_g = ctx->plane_g;
  d.inv_h2 = 1.0 / (ctx->h * ctx->h);
  d.mu2 = mu * mu;
  d.lambda = lambda;
  d.t0 = 0.0; d.dt = 0.0;
  d.n_base = 0; d.n_end = 0; d.stop_k = kNoStop; d.stop_thr = 0.0;
  d.maxabs = ctx->d_maxabs;
  d.coef = ctx->d_coef;
  d.tmaps = ctx->d_tmaps;
  for (int i = 0; i < NUM_FIELDS; ++i) d.f[i] = ctx->f[i];
  if ((st = push_desc(ctx)) != HBE_OK) return bail(st);
  if ((st = apply_tuning(ctx, 0, 0)) != HBE_OK) return bail(st);
  *out = ctx;
  return HBE_OK;
#undef CKB
}

}  // namespace

// =============================================================== C ABI
extern "C" {

const char *hbe_status_string(int s) {
  static const char *names[] = {"HBE_OK", "HBE_EINVAL", "HBE_ENOMEM", "HBE_ECUDA",
                                "HBE_ESTATE", "HBE_STOPPED", "HBE_NONFINITE", "HBE_ETIMEOUT"};
  return (s >= 0 && s <= 7) ? names[s] : "unknown";
}

hbe_status hbe_workspace_bytes(int N, int bc, int prec, size_t *bytes) {
  std::string e;
  if (!bytes) return HBE_EINVAL;
  hbe_status st = validate(e, N, 1.0, 0.0, 0.0, bc, prec);
  if (st != HBE_OK) return st;
  *bytes = workspace_bytes(N, prec, N);
  return HBE_OK;
}

hbe_status hbe_create(int N, double L, double mu, double lambda, int bc, int prec, hbe_ctx **out) {
  return create_common(N, L, mu, lambda, bc, prec, nullptr, 0, out);
}

hbe_status hbe_create_in(int N, double L, double mu, double lambda, int bc, int prec,
                         void *d_workspace, size_t bytes, hbe_ctx **out) {
  if (!d_workspace) return HBE_EINVAL;
  return create_common(N, L, mu, lambda, bc, prec, d_workspace, bytes, out);
}

void hbe_destroy(hbe_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream || ctx->cap_stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  drop_graphs(ctx);
  if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
  cudaFree(ctx->d_tmaps);
  cudaFree(ctx->d_maxabs);
  cudaFree(ctx->d_coef);
  cudaFree(ctx->d_desc);
  if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
  cudaFree(ctx->d_items);
  cudaFree(ctx->d_nitems);
  cudaFree(ctx->d_items_p);
  cudaFree(ctx->d_nitems_p);
  cudaFree(ctx->d_one);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_pre);
  cudaFree(ctx->d_rout);
  for (cudaEvent_t e : {ctx->ev_pre, ctx->ev_rout_ready, ctx->ev_rout_done})
    if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (int b = 0; b < 2; ++b) {
    if (ctx->ev_ready[b]) cudaEventDestroy(ctx->ev_ready[b]);
    if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
  }
  cudaFree(ctx->d_masks);
  cudaFree(ctx->d_labels);
  cudaFree(ctx->d_counts);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_mon);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

hbe_status hbe_set_stream(hbe_ctx *ctx, void *stream) {
  if (!ctx) return HBE_EINVAL;
  if (ctx->pending) {
    hbe_status st = sync_ctx(ctx);
    if (st != HBE_OK) return st;
  }
  ctx->stream = static_cast<cudaStream_t>(stream);
  return HBE_OK;
}

int hbe_variant_count(int prec) {
  if (prec < HBE_FP64 || prec > HBE_FP32_PLAIN) return 0;
  return table_for(prec).count;
}

hbe_status hbe_variant_info(int prec, int variant, hbe_variant_t *out) {
  if (!out || prec < HBE_FP64 || prec > HBE_FP32_PLAIN) return HBE_EINVAL;
  const VariantTable &vt = table_for(prec);
  if (variant < 0 || variant >= vt.count) return HBE_EINVAL;
  const KernelInfo *k = vt.k[variant];
  out->tile_x = k[0].tx;
  out->tile_y = k[0].ty;
  out->threads = k[0].threads;
  out->vec = k[0].vec;
  out->rows_per_warp = k[0].vy;
  out->consumer_warps = k[0].nw;
  for (int s = 0; s < 4; ++s) {
    out->smem_bytes[s] = k[s].smem;
    out->ring[s] = k[s].ring;
  }
  for (int i = 0; i < 2; ++i) {
    out->pair_tile_y[i] = k[4 + i].ty;
    out->pair_threads[i] = k[4 + i].threads;
    out->pair_smem_bytes[i] = k[4 + i].smem;
    out->pair_ring[i] = k[4 + i].ring;
  }
  return HBE_OK;
}

hbe_status hbe_set_schedule(hbe_ctx *ctx, int schedule) {
  if (!ctx) return HBE_EINVAL;
  if (schedule != 0 && schedule != 1) return set_err(ctx->err, HBE_EINVAL, "schedule is 0 or 1");
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (ctx->pending) {
    hbe_status st = sync_ctx(ctx);
    if (st != HBE_OK) return st;
  }
  if (ctx->schedule != schedule) drop_graphs(ctx);
  ctx->schedule = schedule;
  return HBE_OK;
}

hbe_status hbe_set_tuning(hbe_ctx *ctx, int variant, int zchunk) {
  if (!ctx) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (ctx->pending) {
    hbe_status st = sync_ctx(ctx);
    if (st != HBE_OK) return st;
  }
  return apply_tuning(ctx, variant, zchunk);
}

static hbe_status set_initial_impl(hbe_ctx *ctx, const double *phi0, const double *phi1, double t0,
                                   bool device) {
  if (!ctx || !phi0 || !phi1) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (!std::isfinite(t0)) return set_err(ctx->err, HBE_EINVAL, "t0 must be finite");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  const int N = ctx->N;
  const int sprec = ctx->prec == HBE_FP64 ? 0 : 1;
  const bool kahan = is_kahan(ctx->prec);
  const size_t plane = (size_t)N * N;
  const double *dp0 = device ? phi0 : static_cast<const double *>(pinned_device_ptr(phi0));
  const double *dp1 = device ? phi1 : static_cast<const double *>(pinned_device_ptr(phi1));
  if (dp0 && dp1) {
    // device arrays, or page-locked host arrays read by the pack kernel itself
    CK(launch_pack(sprec, dp0, ctx->f[F_P0], kahan ? ctx->f[F_PLO0] : nullptr, N, ctx->pitch_s,
                   ctx->hxs, ctx->bc, 0, N, ctx->stream));
    CK(launch_pack(sprec, dp1, ctx->f[F_Q0], kahan ? ctx->f[F_QLO0] : nullptr, N, ctx->pitch_s,
                   ctx->hxs, ctx->bc, 0, N, ctx->stream));
    if (!device) CK(cudaStreamSynchronize(ctx->stream));
  } else {
    // chunks of planes through two staging sets: the copy of chunk i + 1
    // (copy stream) overlaps the pack of chunk i (work stream)
    if ((st = ensure_stage_buffer(ctx)) != HBE_OK) return st;
    const int zs = (int)(ctx->stage_elems / plane);
    for (int z = 0, i = 0; z < N; z += zs, ++i) {
      const int nz = std::min(zs, N - z), b = i & 1;
      double *s0 = ctx->d_stage + 2 * b * ctx->stage_elems, *s1 = s0 + ctx->stage_elems;
      if (i >= 2) CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0));
      CK(cudaMemcpyAsync(s0, phi0 + (size_t)z * plane, nz * plane * sizeof(double),
                         cudaMemcpyHostToDevice, ctx->copy_stream));
      CK(cudaMemcpyAsync(s1, phi1 + (size_t)z * plane, nz * plane * sizeof(double),
                         cudaMemcpyHostToDevice, ctx->copy_stream));
      CK(cudaEventRecord(ctx->ev_ready[b], ctx->copy_stream));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_ready[b], 0));
      CK(launch_pack(sprec, s0, ctx->f[F_P0],
                     kahan ? ctx->f[F_PLO0] : nullptr, N, ctx->pitch_s, ctx->hxs, ctx->bc, z, nz,
                     ctx->stream));
      CK(launch_pack(sprec, s1, ctx->f[F_Q0], kahan ? ctx->f[F_QLO0] : nullptr, N, ctx->pitch_s,
                     ctx->hxs, ctx->bc, z, nz, ctx->stream));
      CK(cudaEventRecord(ctx->ev_free[b], ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
  }
  Desc &d = *ctx->h_desc;
  d.t0 = t0;
  d.dt = 0.0;
  d.n_base = 0;
  d.n_end = 0;
  d.stop_k = kNoStop;
  d.status = ST_RUNNING;
  d.last_done = 0;
  if (ctx->d_mon) CK(cudaMemset(ctx->d_mon, 0, kMonCap * sizeof(unsigned long long)));
  if ((st = push_desc(ctx)) != HBE_OK) return st;
  CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  ctx->has_state = true;
  return HBE_OK;
}

hbe_status hbe_set_initial(hbe_ctx *ctx, const double *phi0, const double *phi1, double t0) {
  Range range_("hbe_set_initial");
  return set_initial_impl(ctx, phi0, phi1, t0, false);
}

hbe_status hbe_set_initial_device(hbe_ctx *ctx, const double *d_phi0, const double *d_phi1,
                                  double t0) {
  Range range_("hbe_set_initial_device");
  hbe_status st = set_initial_impl(ctx, d_phi0, d_phi1, t0, true);
  if (st == HBE_OK && ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_err(ctx->err, HBE_ECUDA, "%s", cudaGetErrorString(e));
  }
  return st;
}

hbe_status hbe_set_initial_bumps(hbe_ctx *ctx, int n0, const double *A0, const double *R0,
                                 const double *c0, int n1, const double *A1, const double *R1,
                                 const double *c1, double t0) {
  Range range_("hbe_set_initial_bumps");
  if (!ctx) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (n0 < 0 || n1 < 0 || n0 > 64 || n1 > 64)
    return set_err(ctx->err, HBE_EINVAL, "bump counts must be in [0, 64]");
  if ((n0 && (!A0 || !R0 || !c0)) || (n1 && (!A1 || !R1 || !c1)))
    return set_err(ctx->err, HBE_EINVAL, "null bump parameter array");
  if (!std::isfinite(t0)) return set_err(ctx->err, HBE_EINVAL, "t0 must be finite");
  double prm[2][64 * 5];
  for (int i = 0; i < n0; ++i) {
    if (!(R0[i] > 0.0)) return set_err(ctx->err, HBE_EINVAL, "bump radius must be > 0");
    const double v[5] = {A0[i], R0[i], c0[3 * i], c0[3 * i + 1], c0[3 * i + 2]};
    memcpy(&prm[0][5 * i], v, sizeof(v));
  }
  for (int i = 0; i < n1; ++i) {
    if (!(R1[i] > 0.0)) return set_err(ctx->err, HBE_EINVAL, "bump radius must be > 0");
    const double v[5] = {A1[i], R1[i], c1[3 * i], c1[3 * i + 1], c1[3 * i + 2]};
    memcpy(&prm[1][5 * i], v, sizeof(v));
  }
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  // the parameters ride in the G fields (free until the first step): no allocation
  if (3 * ctx->bytes_g < sizeof(prm)) return set_err(ctx->err, HBE_EINVAL, "grid too small");
  double *d_prm = static_cast<double *>(ctx->f[F_G1]);
  CK(cudaMemcpy(d_prm, prm, sizeof(prm), cudaMemcpyHostToDevice));
  const int sprec = ctx->prec == HBE_FP64 ? 0 : 1;
  const bool kahan = is_kahan(ctx->prec);
  CK(launch_bumps(sprec, ctx->f[F_P0], kahan ? ctx->f[F_PLO0] : nullptr, ctx->N, ctx->pitch_s,
                  ctx->hxs, ctx->bc, ctx->h, n0, d_prm, ctx->stream));
  CK(launch_bumps(sprec, ctx->f[F_Q0], kahan ? ctx->f[F_QLO0] : nullptr, ctx->N, ctx->pitch_s,
                  ctx->hxs, ctx->bc, ctx->h, n1, d_prm + 64 * 5, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // the stage kernels overwrite G before reading it, but the Dirichlet ghosts must be 0
  CK(cudaMemset(ctx->f[F_G1], nan_canary(ctx) ? 0xFF : 0, 3 * ctx->bytes_g));
  Desc &d = *ctx->h_desc;
  d.t0 = t0;
  d.dt = 0.0;
  d.n_base = 0;
  d.n_end = 0;
  d.stop_k = kNoStop;
  d.status = ST_RUNNING;
  d.last_done = 0;
  if (ctx->d_mon) CK(cudaMemset(ctx->d_mon, 0, kMonCap * sizeof(unsigned long long)));
  if ((st = push_desc(ctx)) != HBE_OK) return st;
  CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  ctx->has_state = true;
  return HBE_OK;
}

hbe_status hbe_set_stop(hbe_ctx *ctx, double threshold) {
  if (!ctx) return HBE_EINVAL;
  if (!(threshold >= 0.0)) return set_err(ctx->err, HBE_EINVAL, "threshold must be >= 0");
  if (ctx->pending) {
    hbe_status st = sync_ctx(ctx);
    if (st != HBE_OK) return st;
  }
  ctx->h_desc->stop_thr = threshold;
  ctx->desc_stale = true;
  return HBE_OK;
}

hbe_status hbe_step_async(hbe_ctx *ctx, int64_t nsteps, double dt) {
  Range range_("hbe_step");
  if (!ctx) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  if (nsteps < 0) return set_err(ctx->err, HBE_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(ctx->err, HBE_EINVAL, "dt must be > 0");
  if (nsteps == 0) return HBE_OK;
  hbe_status st;
  Desc &d = *ctx->h_desc;
  if (ctx->pending && dt != d.dt) {
    if ((st = sync_ctx(ctx)) != HBE_OK) return st;
  }
  if (ctx->desc_stale) {
    if ((st = push_desc(ctx)) != HBE_OK) return st;
  }
  // whole replays of K steps, then one replay of the remaining steps (its own
  // graph), so no replay launches kernels for steps that are not taken
  const int64_t full = nsteps / ctx->K;
  const int rem = (int)(nsteps % ctx->K);
  if (full > 0 && (st = ensure_graph(ctx, ctx->K)) != HBE_OK) return st;
  if (rem > 0 && (st = ensure_graph(ctx, rem)) != HBE_OK) return st;
  if (!ctx->pending) {
    // restart: clear the stop status; a new dt moves the time origin to the current t
    if (dt != d.dt) {
      const double t_now = d.dt > 0.0 ? current_t(ctx) : d.t0;
      d.t0 = t_now - (double)d.n_base * dt;
      d.dt = dt;
    }
    CK(launch_set_run(ctx->d_desc, nsteps, d.t0, d.dt, d.stop_thr, 1, ctx->stream));
  } else {
    CK(launch_set_run(ctx->d_desc, nsteps, d.t0, d.dt, d.stop_thr, 0, ctx->stream));
  }
  for (int64_t r = 0; r < full; ++r) CK(cudaGraphLaunch(ctx->gexec[ctx->K], ctx->stream));
  if (rem > 0) CK(cudaGraphLaunch(ctx->gexec[rem], ctx->stream));
  ctx->launches += nsteps * launches_per_step(ctx);
  ctx->pending = true;
  return HBE_OK;
}

hbe_status hbe_sync(hbe_ctx *ctx) {
  Range range_("hbe_sync");
  if (!ctx) return HBE_EINVAL;
  const bool was_pending = ctx->pending;
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if (was_pending) {
    if (ctx->h_desc->status == ST_STOPPED)
      return set_err(ctx->err, HBE_STOPPED, "max|phi| passed the stop threshold at step %lld",
                     (long long)ctx->h_desc->n_base);
    if (ctx->h_desc->status == ST_NONFINITE)
      return set_err(ctx->err, HBE_NONFINITE, "phi became non-finite at step %lld",
                     (long long)ctx->h_desc->n_base);
  }
  return HBE_OK;
}

hbe_status hbe_step(hbe_ctx *ctx, int64_t nsteps, double dt) {
  hbe_status st = hbe_step_async(ctx, nsteps, dt);
  if (st != HBE_OK) return st;
  return hbe_sync(ctx);
}

hbe_status hbe_profile_stages(hbe_ctx *ctx, int64_t nsteps, double dt, float *ms_per_stage) {
  Range range_("hbe_profile_stages");
  if (!ctx || !ms_per_stage) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  if (nsteps < 1 || nsteps > 4096) return set_err(ctx->err, HBE_EINVAL, "nsteps in [1, 4096]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(ctx->err, HBE_EINVAL, "dt must be > 0");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if (ctx->desc_stale && (st = push_desc(ctx)) != HBE_OK) return st;
  Desc &d = *ctx->h_desc;
  if (dt != d.dt) {
    const double t_now = d.dt > 0.0 ? current_t(ctx) : d.t0;
    d.t0 = t_now - (double)d.n_base * dt;
    d.dt = dt;
  }
  CK(launch_set_run(ctx->d_desc, nsteps, d.t0, d.dt, d.stop_thr, 1, ctx->stream));
  const int first = ctx->schedule ? 4 : 0, nl = ctx->schedule ? 2 : 4;
  // events before and after each stage kernel (a periodic context's ghost copy
  // runs after the second event and is not part of the stage's time)
  std::vector<cudaEvent_t> ev((size_t)nsteps * nl * 2, nullptr);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  const VariantTable &vt = table_for(ctx->prec);
  int64_t wraps = 0;
  for (int64_t n = 0; n < nsteps && st == HBE_OK; ++n) {
    CK(launch_coef(ctx->d_desc, ctx->d_one, 1, 1, ctx->stream));
    for (int s = 0; s < nl && st == HBE_OK; ++s) {
      CK(cudaEventRecord(ev[(n * nl + s) * 2], ctx->stream));
      st = launch_stage(ctx->err, vt.k[ctx->variant][first + s], ctx->grid[first + s],
                        ctx_params(ctx, first + s, 0), ctx->stream);
      CK(cudaEventRecord(ev[(n * nl + s) * 2 + 1], ctx->stream));
      if (st == HBE_OK && ctx->bc == HBE_BC_PERIODIC && stage_needs_wrap(first + s + 1)) {
        CK(launch_wrap(ctx->d_desc, ctx->d_one, 1, 0, first + s + 1, wrap_blocks(ctx), ctx->stream));
        ++wraps;
      }
    }
    CK(launch_advance(ctx->d_desc, ctx->d_one, 1, 1, ctx->stream));
  }
  ctx->launches += nsteps * nl + wraps;
  ctx->pending = true;
  hbe_status st2 = sync_ctx(ctx);
  double acc[4] = {0, 0, 0, 0};
  if (st == HBE_OK && st2 == HBE_OK) {
    for (int64_t n = 0; n < nsteps; ++n)
      for (int s = 0; s < nl; ++s) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[(n * nl + s) * 2], ev[(n * nl + s) * 2 + 1]);
        acc[s] += ms;
      }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (st != HBE_OK) return st;
  if (st2 != HBE_OK) return st2;
  for (int s = 0; s < 4; ++s) ms_per_stage[s] = (float)(acc[s] / (double)nsteps);
  if (d.status == ST_STOPPED) return HBE_STOPPED;
  if (d.status == ST_NONFINITE) return HBE_NONFINITE;
  return HBE_OK;
}

hbe_status hbe_progress(hbe_ctx *ctx, int64_t *steps, double *t) {
  if (!ctx) return HBE_EINVAL;
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if (steps) *steps = ctx->h_desc->n_base;
  if (t) *t = current_t(ctx);
  return HBE_OK;
}

static hbe_status read_impl(hbe_ctx *ctx, double *phi, double *psi, bool device) {
  const int N = ctx->N;
  const int sprec = ctx->prec == HBE_FP64 ? 0 : 1;
  const bool kahan = is_kahan(ctx->prec);
  const int set = (int)(ctx->h_desc->n_base & 1);
  void *hp = ctx->f[F_P0 + set], *hq = ctx->f[F_Q0 + set];
  void *lp = kahan ? ctx->f[F_PLO0 + set] : nullptr, *lq = kahan ? ctx->f[F_QLO0 + set] : nullptr;
  double *dphi = device || !phi ? phi : static_cast<double *>(const_cast<void *>(pinned_device_ptr(phi)));
  double *dpsi = device || !psi ? psi : static_cast<double *>(const_cast<void *>(pinned_device_ptr(psi)));
  if ((!phi || dphi) && (!psi || dpsi)) {
    // device arrays, or page-locked host arrays written by the unpack kernel itself
    if (phi) CK(launch_unpack(sprec, hp, lp, dphi, N, ctx->pitch_s, ctx->hxs, 0, N, ctx->stream));
    if (psi) CK(launch_unpack(sprec, hq, lq, dpsi, N, ctx->pitch_s, ctx->hxs, 0, N, ctx->stream));
    if (!device) CK(cudaStreamSynchronize(ctx->stream));
    return HBE_OK;
  }
  // chunks of planes through two staging sets: the unpack of chunk i + 1
  // (work stream) overlaps the copy of chunk i to the host (copy stream)
  hbe_status st = ensure_stage_buffer(ctx);
  if (st != HBE_OK) return st;
  const size_t plane = (size_t)N * N;
  const int zs = (int)(ctx->stage_elems / plane);
  for (int z = 0, i = 0; z < N; z += zs, ++i) {
    const int nz = std::min(zs, N - z), b = i & 1;
    double *s0 = ctx->d_stage + 2 * b * ctx->stage_elems, *s1 = s0 + ctx->stage_elems;
    if (i >= 2) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_free[b], 0));
    if (phi) CK(launch_unpack(sprec, hp, lp, s0, N, ctx->pitch_s, ctx->hxs, z, nz, ctx->stream));
    if (psi) CK(launch_unpack(sprec, hq, lq, s1, N, ctx->pitch_s, ctx->hxs, z, nz, ctx->stream));
    CK(cudaEventRecord(ctx->ev_ready[b], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_ready[b], 0));
    if (phi)
      CK(cudaMemcpyAsync(phi + (size_t)z * plane, s0, nz * plane * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->copy_stream));
    if (psi)
      CK(cudaMemcpyAsync(psi + (size_t)z * plane, s1, nz * plane * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->copy_stream));
    CK(cudaEventRecord(ctx->ev_free[b], ctx->copy_stream));
  }
  CK(cudaStreamSynchronize(ctx->copy_stream));
  return HBE_OK;
}

hbe_status hbe_read(hbe_ctx *ctx, double *phi, double *psi, double *t) {
  Range range_("hbe_read");
  if (!ctx) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if (t) *t = current_t(ctx);
  if (!phi && !psi) return HBE_OK;
  return read_impl(ctx, phi, psi, false);
}

hbe_status hbe_read_device(hbe_ctx *ctx, double *d_phi, double *d_psi) {
  Range range_("hbe_read_device");
  if (!ctx) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  return read_impl(ctx, d_phi, d_psi, true);
}

// ---------------------------------------------------------------- streaming host I/O
// The next problem's initial data crosses the host link while the current one
// steps, and a result crosses back while the next one steps: both by DMA on
// the copy stream, through whole-field staging areas, so the context's stream
// only packs and unpacks device memory.
static hbe_status ensure_async_io(hbe_ctx *ctx, double **buf) {
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t *e : {&ctx->ev_pre, &ctx->ev_rout_ready, &ctx->ev_rout_done})
    if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  if (!*buf) {
    const size_t n = (size_t)ctx->N * ctx->N * ctx->N;
    if (cudaMalloc(buf, 2 * n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      *buf = nullptr;
      return set_err(ctx->err, HBE_ENOMEM, "no device memory for a %zu-byte staging area",
                     2 * n * sizeof(double));
    }
  }
  return HBE_OK;
}

hbe_status hbe_prefetch_initial(hbe_ctx *ctx, const double *phi0, const double *phi1) {
  Range range_("hbe_prefetch_initial");
  if (!ctx || !phi0 || !phi1) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  hbe_status st = ensure_async_io(ctx, &ctx->d_pre);
  if (st != HBE_OK) return st;
  const size_t n = (size_t)ctx->N * ctx->N * ctx->N;
  CK(cudaMemcpyAsync(ctx->d_pre, phi0, n * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->copy_stream));
  CK(cudaMemcpyAsync(ctx->d_pre + n, phi1, n * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->copy_stream));
  CK(cudaEventRecord(ctx->ev_pre, ctx->copy_stream));
  ctx->pre_pending = true;
  return HBE_OK;
}

hbe_status hbe_set_initial_prefetched(hbe_ctx *ctx, double t0) {
  Range range_("hbe_set_initial_prefetched");
  if (!ctx) return HBE_EINVAL;
  if (!ctx->pre_pending) return set_err(ctx->err, HBE_ESTATE, "no prefetched initial data");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_pre, 0));
  const size_t n = (size_t)ctx->N * ctx->N * ctx->N;
  hbe_status st = set_initial_impl(ctx, ctx->d_pre, ctx->d_pre + n, t0, true);
  if (st != HBE_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->pre_pending = false;
  return HBE_OK;
}

hbe_status hbe_read_async(hbe_ctx *ctx, double *phi, double *psi) {
  Range range_("hbe_read_async");
  if (!ctx || (!phi && !psi)) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if ((st = ensure_async_io(ctx, &ctx->d_rout)) != HBE_OK) return st;
  if (ctx->rout_pending) {  // the staging area still feeds the previous read's copy
    CK(cudaEventSynchronize(ctx->ev_rout_done));
    ctx->rout_pending = false;
  }
  const size_t n = (size_t)ctx->N * ctx->N * ctx->N;
  // unpack on the context's stream (later work there is ordered after it),
  // then the copy to the host once the unpack is done
  if ((st = read_impl(ctx, phi ? ctx->d_rout : nullptr, psi ? ctx->d_rout + n : nullptr, true)) !=
      HBE_OK)
    return st;
  CK(cudaEventRecord(ctx->ev_rout_ready, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rout_ready, 0));
  if (phi)
    CK(cudaMemcpyAsync(phi, ctx->d_rout, n * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
  if (psi)
    CK(cudaMemcpyAsync(psi, ctx->d_rout + n, n * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
  CK(cudaEventRecord(ctx->ev_rout_done, ctx->copy_stream));
  ctx->rout_pending = true;
  return HBE_OK;
}

hbe_status hbe_read_wait(hbe_ctx *ctx) {
  Range range_("hbe_read_wait");
  if (!ctx) return HBE_EINVAL;
  if (ctx->rout_pending) {
    CK(cudaEventSynchronize(ctx->ev_rout_done));
    ctx->rout_pending = false;
  }
  return HBE_OK;
}

hbe_status hbe_diag(hbe_ctx *ctx, double eps, hbe_diag_t *out, uint32_t *pos_mask,
                    uint32_t *neg_mask) {
  Range range_("hbe_diag");
  if (!ctx || !out) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  if (!(eps >= 0.0)) return set_err(ctx->err, HBE_EINVAL, "eps must be >= 0");
  if ((int64_t)ctx->N * ctx->N * ctx->N >= 0x7fffffffLL)
    return set_err(ctx->err, HBE_EINVAL, "diagnostics need N^3 < 2^31");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  const int N = ctx->N;
  const size_t words = (size_t)N * N * ((N + 31) / 32);
  if (!ctx->d_masks) {
    CK(cudaMalloc(&ctx->d_masks, 2 * words * sizeof(uint32_t)));
    CK(cudaMalloc(&ctx->d_labels, (size_t)N * N * N * sizeof(int)));
    CK(cudaMalloc(&ctx->d_counts, 4 * sizeof(unsigned long long)));
  }
  const int sprec = ctx->prec == HBE_FP64 ? 0 : 1;
  const bool kahan = is_kahan(ctx->prec);
  const int set = (int)(ctx->h_desc->n_base & 1);
  CK(cudaMemsetAsync(ctx->d_counts, 0, 4 * sizeof(unsigned long long), ctx->stream));
  CK(launch_signpack(sprec, ctx->f[F_P0 + set], kahan ? ctx->f[F_PLO0 + set] : nullptr, N,
                     ctx->pitch_s, ctx->hxs, eps, ctx->d_masks, ctx->d_masks + words,
                     ctx->d_counts, ctx->stream));
  CK(launch_ccl(ctx->d_masks, N, ctx->bc, ctx->d_labels, ctx->d_counts + 1, ctx->d_err, ctx->stream));
  CK(launch_ccl(ctx->d_masks + words, N, ctx->bc, ctx->d_labels, ctx->d_counts + 2, ctx->d_err,
                ctx->stream));
  unsigned long long c[4];
  CK(cudaMemcpyAsync(c, ctx->d_counts, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
  if (pos_mask)
    CK(cudaMemcpyAsync(pos_mask, ctx->d_masks, words * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (neg_mask)
    CK(cudaMemcpyAsync(neg_mask, ctx->d_masks + words, words * sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, ctx->stream));
  if ((st = sync_ctx(ctx)) != HBE_OK) return st;
  double mx;
  memcpy(&mx, &c[0], sizeof(double));
  out->t = current_t(ctx);
  out->step = ctx->h_desc->n_base;
  out->finite = std::isfinite(mx) ? 1 : 0;
  out->max_abs_phi = mx;
  out->reserved = 0;
  out->n_pos = (int64_t)c[1];
  out->n_neg = (int64_t)c[2];
  const int64_t b = out->n_pos + out->n_neg - 1;
  out->bubble_count = b > 0 ? b : 0;
  return HBE_OK;
}

hbe_status hbe_analysis(hbe_ctx *ctx, double eps, hbe_analysis_t *out) {
  Range range_("hbe_analysis");
  if (!ctx || !out) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  if (!(eps >= 0.0)) return set_err(ctx->err, HBE_EINVAL, "eps must be >= 0");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  const int nb = analysis_blocks();
  if (!ctx->d_part) CK(cudaMalloc(&ctx->d_part, (5 * (size_t)nb + 5) * sizeof(double)));
  const int sprec = ctx->prec == HBE_FP64 ? 0 : 1;
  const bool kahan = is_kahan(ctx->prec);
  const int set = (int)(ctx->h_desc->n_base & 1);
  const double mcoef = 1.5 + std::sqrt(2.25 + ctx->mu * ctx->mu);
  CK(launch_analysis(sprec, ctx->f[F_P0 + set], kahan ? ctx->f[F_PLO0 + set] : nullptr,
                     ctx->f[F_Q0 + set], kahan ? ctx->f[F_QLO0 + set] : nullptr, ctx->N,
                     ctx->pitch_s, ctx->hxs, ctx->bc, 1.0 / (ctx->h * ctx->h), mcoef, eps,
                     ctx->d_part, ctx->d_part + 5 * (size_t)nb, ctx->stream));
  double r[5];
  CK(cudaMemcpyAsync(r, ctx->d_part + 5 * (size_t)nb, sizeof(r), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double t = current_t(ctx);
  const double h3 = ctx->h * ctx->h * ctx->h;
  out->t = t;
  out->integral_phi = r[0] * h3;
  out->integral_phi3 = r[1] * h3;
  out->laplacian_monitor = std::exp(-2.0 * t) * r[2];
  out->support_points = (int64_t)r[3];
  out->condition1_violations = (int64_t)r[4];
  return HBE_OK;
}

hbe_status hbe_set_monitor(hbe_ctx *ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  if (on && !ctx->d_mon) {
    CK(cudaMalloc(&ctx->d_mon, kMonCap * sizeof(unsigned long long)));
    CK(cudaMemset(ctx->d_mon, 0, kMonCap * sizeof(unsigned long long)));
  }
  if ((bool)on != ctx->monitor) drop_graphs(ctx);
  ctx->monitor = on != 0;
  ctx->h_desc->mon = on ? ctx->d_mon : nullptr;
  ctx->h_desc->mon_cap = kMonCap;
  return push_desc(ctx);
}

hbe_status hbe_monitor_read(hbe_ctx *ctx, int64_t first, int64_t count, double *P, double *t) {
  if (!ctx || !P || count < 0) return HBE_EINVAL;
  if (!ctx->monitor) return set_err(ctx->err, HBE_ESTATE, "the monitor is off");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  const Desc &d = *ctx->h_desc;
  if (first < 0 || first + count > d.n_base || first < d.n_base - (kMonCap - kMaxK))
    return set_err(ctx->err, HBE_EINVAL, "steps [%lld, %lld) outside the recorded [%lld, %lld)",
                   (long long)first, (long long)(first + count),
                   (long long)std::max<int64_t>(0, d.n_base - (kMonCap - kMaxK)),
                   (long long)d.n_base);
  std::vector<unsigned long long> raw((size_t)count);
  for (int64_t i = 0; i < count;) {
    const int64_t at = (first + i) % kMonCap, n = std::min(count - i, kMonCap - at);
    CK(cudaMemcpy(raw.data() + i, ctx->d_mon + at, n * sizeof(unsigned long long),
                  cudaMemcpyDeviceToHost));
    i += n;
  }
  for (int64_t i = 0; i < count; ++i) {
    double v;
    memcpy(&v, &raw[i], sizeof(v));
    const double tn = d.t0 + (double)(first + i) * d.dt;
    P[i] = std::exp(-2.0 * tn) * v / (ctx->h * ctx->h);
    if (t) t[i] = tn;
  }
  return HBE_OK;
}

namespace {
struct SaveHeader {
  char magic[8];
  int32_t N, bc, prec, pad;
  double L, mu, lambda, t0, dt, stop_thr;
  int64_t n_base;
  uint64_t field_bytes;
};
}  // namespace

hbe_status hbe_save(hbe_ctx *ctx, const char *path) {
  if (!ctx || !path) return HBE_EINVAL;
  if (!ctx->has_state) return set_err(ctx->err, HBE_ESTATE, "no initial data");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  FILE *fp = fopen(path, "wb");
  if (!fp) return set_err(ctx->err, HBE_EINVAL, "cannot open %s", path);
  SaveHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "HBESAVE1", 8);
  const Desc &d = *ctx->h_desc;
  hd.N = ctx->N; hd.bc = ctx->bc; hd.prec = ctx->prec;
  hd.L = ctx->L; hd.mu = ctx->mu; hd.lambda = ctx->lambda;
  hd.t0 = d.t0; hd.dt = d.dt; hd.stop_thr = d.stop_thr; hd.n_base = d.n_base;
  hd.field_bytes = ctx->bytes_s;
  bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1;
  const int set = (int)(d.n_base & 1);
  const int nf = is_kahan(ctx->prec) ? 4 : 2;
  const int fields[4] = {F_P0 + set, F_Q0 + set, F_PLO0 + set, F_QLO0 + set};
  std::vector<char> buf(ctx->bytes_s);
  for (int i = 0; i < nf && ok; ++i) {
    if (cudaMemcpy(buf.data(), ctx->f[fields[i]], ctx->bytes_s, cudaMemcpyDeviceToHost) != cudaSuccess) {
      fclose(fp);
      return set_err(ctx->err, HBE_ECUDA, "device read failed");
    }
    ok = fwrite(buf.data(), 1, ctx->bytes_s, fp) == ctx->bytes_s;
  }
  fclose(fp);
  return ok ? HBE_OK : set_err(ctx->err, HBE_EINVAL, "write to %s failed", path);
}

hbe_status hbe_load(hbe_ctx *ctx, const char *path) {
  if (!ctx || !path) return HBE_EINVAL;
  if (ctx->in_batch) return set_err(ctx->err, HBE_ESTATE, "context is in a batch");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return st;
  FILE *fp = fopen(path, "rb");
  if (!fp) return set_err(ctx->err, HBE_EINVAL, "cannot open %s", path);
  SaveHeader hd;
  if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, "HBESAVE1", 8) != 0 ||
      hd.N != ctx->N || hd.bc != ctx->bc || hd.prec != ctx->prec ||
      hd.field_bytes != ctx->bytes_s) {
    fclose(fp);
    return set_err(ctx->err, HBE_EINVAL, "%s is not a checkpoint of this problem shape", path);
  }
  const int set = (int)(hd.n_base & 1);
  const int nf = is_kahan(ctx->prec) ? 4 : 2;
  const int fields[4] = {F_P0 + set, F_Q0 + set, F_PLO0 + set, F_QLO0 + set};
  std::vector<char> buf(ctx->bytes_s);
  for (int i = 0; i < nf; ++i) {
    if (fread(buf.data(), 1, ctx->bytes_s, fp) != ctx->bytes_s) {
      fclose(fp);
      return set_err(ctx->err, HBE_EINVAL, "%s is truncated", path);
    }
    CK(cudaMemcpy(ctx->f[fields[i]], buf.data(), ctx->bytes_s, cudaMemcpyHostToDevice));
  }
  fclose(fp);
  Desc &d = *ctx->h_desc;
  d.t0 = hd.t0; d.dt = hd.dt; d.stop_thr = hd.stop_thr;
  d.n_base = hd.n_base; d.n_end = hd.n_base; d.stop_k = kNoStop; d.status = ST_RUNNING;
  if (ctx->d_mon) CK(cudaMemset(ctx->d_mon, 0, kMonCap * sizeof(unsigned long long)));
  if ((st = push_desc(ctx)) != HBE_OK) return st;
  ctx->has_state = true;
  return HBE_OK;
}

const char *hbe_last_error(const hbe_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t hbe_launch_count(const hbe_ctx *ctx) { return ctx ? ctx->launches : 0; }

// =============================================================== batches
hbe_status hbe_batch_create(int prec, int K, void *stream, hbe_batch **out) {
  if (!out || prec < HBE_FP64 || prec > HBE_FP32_PLAIN || K < 1 || K > kMaxK) return HBE_EINVAL;
  *out = nullptr;
  hbe_batch *b = new hbe_batch();
  b->prec = prec;
  b->K = K;
  b->stream = static_cast<cudaStream_t>(stream);
  b->nvariants = table_for(prec).count;
  std::string e;
  if (get_encoder(e) != HBE_OK || cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&b->d_err, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->d_err, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->d_ndesc, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->h_err, sizeof(unsigned)) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    hbe_batch_destroy(b);
    return HBE_ECUDA;
  }
  *out = b;
  return HBE_OK;
}

void hbe_batch_destroy(hbe_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (hbe_ctx *c : b->members) c->in_batch = false;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->d_descs);
  if (b->h_descs) cudaFreeHost(b->h_descs);
  cudaFree(b->d_ndesc);
  for (auto *ls : {b->lists, b->lists_p})
    for (int v = 0; v < kMaxVariants; ++v) {
      cudaFree(ls[v].d_items);
      cudaFree(ls[v].d_n);
    }
  cudaFree(b->d_err);
  cudaFree(b->d_halo);
  if (b->h_err) cudaFreeHost(b->h_err);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

int hbe_batch_size(const hbe_batch *b) { return b ? (int)b->members.size() : 0; }
const char *hbe_batch_last_error(const hbe_batch *b) { return b ? b->err.c_str() : "null batch"; }
int64_t hbe_batch_launch_count(const hbe_batch *b) { return b ? b->launches : 0; }

hbe_status hbe_batch_add(hbe_batch *b, hbe_ctx *ctx, int64_t nsteps, double dt) {
  if (!b || !ctx) return HBE_EINVAL;
  if (b->in_flight) return set_err(b->err, HBE_ESTATE, "a run is in flight: collect it first");
  if (ctx->prec != b->prec) return set_err(b->err, HBE_EINVAL, "precision differs from the batch");
  if (ctx->in_batch) return set_err(b->err, HBE_ESTATE, "context already in a batch");
  if (!ctx->has_state) return set_err(b->err, HBE_ESTATE, "context has no initial data");
  if (nsteps < 0 || !(dt > 0.0)) return set_err(b->err, HBE_EINVAL, "bad nsteps/dt");
  hbe_status st = sync_ctx(ctx);
  if (st != HBE_OK) return set_err(b->err, st, "%s", ctx->err.c_str());
  Desc &d = *ctx->h_desc;
  if (dt != d.dt) {
    const double t_now = d.dt > 0.0 ? current_t(ctx) : d.t0;
    d.t0 = t_now - (double)d.n_base * dt;
    d.dt = dt;
  }
  d.n_end = d.n_base + nsteps;
  d.stop_k = kNoStop;
  d.status = ST_RUNNING;
  ctx->in_batch = true;
  b->members.push_back(ctx);
  b->dirty = true;
  return HBE_OK;
}

static void leave_batch(hbe_ctx *ctx) {
  ctx->in_batch = false;
  ctx->desc_stale = true;  // the member's own descriptor copy is older than the mirror
}

hbe_status hbe_batch_remove(hbe_batch *b, hbe_ctx *ctx) {
  if (!b || !ctx) return HBE_EINVAL;
  if (b->in_flight) return set_err(b->err, HBE_ESTATE, "a run is in flight: collect it first");
  auto it = std::find(b->members.begin(), b->members.end(), ctx);
  if (it == b->members.end()) return set_err(b->err, HBE_EINVAL, "not a member");
  cudaStreamSynchronize(b->stream);
  b->members.erase(it);
  leave_batch(ctx);
  b->dirty = true;
  return HBE_OK;
}

static hbe_status batch_rebuild(hbe_batch *b) {
  const int M = (int)b->members.size();
  bool recapture = !b->gexec;
  bool periodic = false;
  unsigned used = 0;
  for (hbe_ctx *c : b->members) {
    periodic |= c->bc == HBE_BC_PERIODIC;
    used |= 1u << c->variant;
  }
  if (periodic && !b->wraps) recapture = true;
  // the graph launches the kernels of the variants that have members (kept
  // while members of other variants come and go, so joins rarely re-capture)
  if ((used & ~b->graph_variants) != 0) recapture = true;
  if (M > b->cap_desc) {
    int cap = std::max(64, b->cap_desc);
    while (cap < M) cap *= 2;
    cudaFree(b->d_descs);
    if (b->h_descs) cudaFreeHost(b->h_descs);
    b->d_descs = nullptr;
    b->h_descs = nullptr;
    CKX(b->err, cudaMalloc(&b->d_descs, cap * sizeof(Desc)));
    CKX(b->err, cudaMallocHost(&b->h_descs, cap * sizeof(Desc)));
    b->cap_desc = cap;
    recapture = true;
  }
  std::vector<WorkItem> items[2][kMaxVariants];
  for (int i = 0; i < M; ++i) {
    hbe_ctx *c = b->members[i];
    b->h_descs[i] = *c->h_desc;
    build_items(c, i, c->zchunk, 0, items[0][c->variant]);
    build_items(c, i, c->zchunk_p, 4, items[1][c->variant]);
  }
  const VariantTable &vt = table_for(b->prec);
  for (int lv = 0; lv < 2 * b->nvariants; ++lv) {
    const int li = lv / b->nvariants, v = lv % b->nvariants;
    auto &l = li ? b->lists_p[v] : b->lists[v];
    const int n = (int)items[li][v].size();
    if (n > l.cap || !l.d_n) {
      int cap = std::max(4096, l.cap);
      while (cap < n) cap *= 2;
      cudaFree(l.d_items);
      l.d_items = nullptr;
      if (!l.d_n) CKX(b->err, cudaMalloc(&l.d_n, sizeof(int)));
      CKX(b->err, cudaMalloc(&l.d_items, cap * sizeof(WorkItem)));
      l.cap = cap;
      for (int s = 0; s < 6; ++s) {
        hbe_status st = persistent_grid(b->err, vt.k[v][s], b->sms, &l.grid[s]);
        if (st != HBE_OK) return st;
      }
      recapture = true;
    }
    if (n)
      CKX(b->err, cudaMemcpyAsync(l.d_items, items[li][v].data(), n * sizeof(WorkItem),
                                  cudaMemcpyHostToDevice, b->stream));
    CKX(b->err, cudaMemcpyAsync(l.d_n, &n, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CKX(b->err, cudaStreamSynchronize(b->stream));  // n lives on this stack frame
  }
  CKX(b->err, cudaMemcpyAsync(b->d_descs, b->h_descs, M * sizeof(Desc), cudaMemcpyHostToDevice,
                              b->stream));
  CKX(b->err, cudaMemcpyAsync(b->d_ndesc, &M, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  CKX(b->err, cudaStreamSynchronize(b->stream));
  if (recapture) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaGraph_t g = nullptr;
    CKX(b->err, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    hbe_status st = HBE_OK;
    cudaError_t ec = launch_coef(b->d_descs, b->d_ndesc, b->cap_desc, b->K, b->cap_stream);
    if (ec != cudaSuccess) st = set_err(b->err, HBE_ECUDA, "%s", cudaGetErrorString(ec));
    // the batch always runs the fused stage pairs (kernels 4 and 5 of a variant)
    const unsigned gv = used;
    for (int k = 0; k < b->K && st == HBE_OK; ++k)
      for (int s = 4; s < 6 && st == HBE_OK; ++s) {
        for (int v = 0; v < b->nvariants && st == HBE_OK; ++v) {
          auto &l = s == 4 ? b->lists_p[v] : b->lists[v];
          if (!l.d_n || !(gv >> v & 1u)) continue;
          StageParams p{b->d_descs, l.d_items, l.d_n, b->d_err, k};
          st = launch_stage(b->err, vt.k[v][s], l.grid[s], p, b->cap_stream);
        }
        // ghost copies of the periodic members' outputs of this stage pair
        if (st == HBE_OK && periodic) {
          cudaError_t ew = launch_wrap(b->d_descs, b->d_ndesc, b->cap_desc, k, s + 1, 2 * b->sms,
                                       b->cap_stream);
          if (ew != cudaSuccess) st = set_err(b->err, HBE_ECUDA, "%s", cudaGetErrorString(ew));
        }
        // halo planes of the stage pair's outputs between the slabs
        if (st == HBE_OK && b->nhalo > 0) {
          cudaError_t eh = launch_halo(b->d_descs, b->d_halo, b->nhalo, k, s + 1, b->cap_stream);
          if (eh != cudaSuccess) st = set_err(b->err, HBE_ECUDA, "%s", cudaGetErrorString(eh));
        }
      }
    b->wraps = periodic;
    b->graph_variants = gv;
    cudaError_t e = launch_advance(b->d_descs, b->d_ndesc, b->cap_desc, b->K, b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != HBE_OK) return st;
    CKX(b->err, e);
    CKX(b->err, e2);
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    CKX(b->err, e);
  }
  b->dirty = false;
  return HBE_OK;
}

hbe_status hbe_batch_launch(hbe_batch *b) {
  Range range_("hbe_batch_launch");
  if (!b) return HBE_EINVAL;
  if (b->in_flight) return set_err(b->err, HBE_ESTATE, "a run is in flight: collect it first");
  if (b->members.empty()) return HBE_OK;
  if (b->dirty) {
    hbe_status st = batch_rebuild(b);
    if (st != HBE_OK) return st;
  }
  const int M = (int)b->members.size();
  CKX(b->err, cudaGraphLaunch(b->gexec, b->stream));
  int used = 0;
  for (int v = 0; v < b->nvariants; ++v) used += (b->graph_variants >> v & 1u) ? 1 : 0;
  b->launches += (int64_t)(2 * used + (b->wraps ? 2 : 0) + (b->nhalo > 0 ? 2 : 0)) * b->K;
  // the members' descriptors and the error word come back behind the run
  CKX(b->err, cudaMemcpyAsync(b->h_descs, b->d_descs, M * sizeof(Desc), cudaMemcpyDeviceToHost,
                              b->stream));
  CKX(b->err, cudaMemcpyAsync(b->h_err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              b->stream));
  CKX(b->err, cudaEventRecord(b->ev_done, b->stream));
  b->in_flight = true;
  b->run_members = M;
  return HBE_OK;
}

hbe_status hbe_batch_collect(hbe_batch *b, hbe_ctx **finished, int max_finished,
                             int *n_finished) {
  Range range_("hbe_batch_collect");
  if (!b || !n_finished) return HBE_EINVAL;
  *n_finished = 0;
  if (!b->in_flight) return HBE_OK;
  b->in_flight = false;
  CKX(b->err, cudaEventSynchronize(b->ev_done));
  if (*b->h_err) return set_err(b->err, HBE_ETIMEOUT, "a stage kernel's TMA wait timed out");
  const int M = b->run_members;
  std::vector<hbe_ctx *> keep;
  for (int i = 0; i < M; ++i) {
    hbe_ctx *c = b->members[i];
    *c->h_desc = b->h_descs[i];
    c->launches += (int64_t)(c->bc == HBE_BC_PERIODIC ? 4 : 2) * b->K;
    const Desc &d = b->h_descs[i];
    if (d.n_base >= d.n_end || d.status != ST_RUNNING) {
      leave_batch(c);
      if (*n_finished < max_finished && finished) finished[*n_finished] = c;
      ++*n_finished;
      b->dirty = true;
    } else {
      keep.push_back(c);
    }
  }
  b->members.swap(keep);
  return HBE_OK;
}

hbe_status hbe_batch_run(hbe_batch *b, hbe_ctx **finished, int max_finished, int *n_finished) {
  Range range_("hbe_batch_run");
  if (!b || !n_finished) return HBE_EINVAL;
  *n_finished = 0;
  hbe_status st = hbe_batch_launch(b);
  if (st != HBE_OK) return st;
  return hbe_batch_collect(b, finished, max_finished, n_finished);
}

// =============================================================== z-slabs
// The grid split along z into k slabs of nz_i = N/k (+1 for the first N % k)
// planes.  Slab i stores its planes after 2 halo planes and before 2 more;
// after every stage pair the 2 planes next to each slab boundary go into the
// neighbour's halo planes (the upper neighbour of the last slab and the lower
// neighbour of the first are each other when periodic; zero-Dirichlet outer
// halos stay 0, like the out-of-grid planes of an undivided grid).
int hbe_slab_plan(int N, int k, int periodic, int32_t *nz, int32_t *copies, int max_copies) {
  if (k < 1 || N < 2 * k || !nz || (periodic != 0 && periodic != 1)) return -1;
  for (int i = 0; i < k; ++i) nz[i] = N / k + (i < N % k ? 1 : 0);
  int n = 0;
  auto add = [&](int src, int dst, int sp, int dp) {
    if (copies && n < max_copies) {
      copies[4 * n] = src; copies[4 * n + 1] = dst;
      copies[4 * n + 2] = sp; copies[4 * n + 3] = dp;
    }
    ++n;
  };
  for (int i = 0; i < k; ++i) {
    const int up = i + 1 < k ? i + 1 : (periodic ? 0 : -1);
    const int down = i > 0 ? i - 1 : (periodic ? k - 1 : -1);
    // top two interior planes (stored at nz_i, nz_i + 1) -> the upper neighbour's lower halo
    if (up >= 0) add(i, up, nz[i], 0);
    // bottom two interior planes (stored at 2, 3) -> the lower neighbour's upper halo
    if (down >= 0) add(i, down, 2, nz[down] + 2);
  }
  return copies && n > max_copies ? -1 : n;
}

}  // extern "C"

struct hbe_slabs {
  int N = 0, k = 0, bc = 0, prec = 0;
  cudaStream_t stream = nullptr;
  std::vector<hbe_ctx *> parts;
  std::vector<int> nz, z0;  // planes and first global plane of each slab
  std::vector<HaloCopy> plan;
  hbe_batch *batch = nullptr;
  std::string err;
};

extern "C" {

void hbe_slabs_destroy(hbe_slabs *s) {
  if (!s) return;
  if (s->batch) hbe_batch_destroy(s->batch);
  for (hbe_ctx *c : s->parts) hbe_destroy(c);
  delete s;
}

hbe_status hbe_slabs_create(int N, double L, double mu, double lambda, int bc, int prec, int k,
                            void *stream, hbe_slabs **out) {
  if (!out) return HBE_EINVAL;
  *out = nullptr;
  hbe_slabs *s = new hbe_slabs();
  s->N = N; s->k = k; s->bc = bc; s->prec = prec;
  s->stream = static_cast<cudaStream_t>(stream);
  std::string e;
  hbe_status st = validate(e, N, L, mu, lambda, bc, prec);
  if (st != HBE_OK) { hbe_slabs_destroy(s); return st; }
  s->nz.assign(k > 0 ? k : 1, 0);
  const int nc = hbe_slab_plan(N, k, bc == HBE_BC_PERIODIC, s->nz.data(), nullptr, 0);
  if (nc < 0) { hbe_slabs_destroy(s); return HBE_EINVAL; }
  std::vector<int32_t> cp(4 * (size_t)std::max(nc, 1));
  hbe_slab_plan(N, k, bc == HBE_BC_PERIODIC, s->nz.data(), cp.data(), nc);
  for (int c = 0; c < nc; ++c)
    s->plan.push_back(HaloCopy{cp[4 * c], cp[4 * c + 1], cp[4 * c + 2], cp[4 * c + 3]});
  int g = 0;
  for (int i = 0; i < k; ++i) {
    s->z0.push_back(g);
    g += s->nz[i];
    hbe_ctx *c = nullptr;
    st = create_common(N, L, mu, lambda, bc, prec, nullptr, 0, &c, s->nz[i], 2);
    if (st != HBE_OK) { hbe_slabs_destroy(s); return st; }
    c->stream = s->stream;
    s->parts.push_back(c);
  }
  st = hbe_batch_create(prec, 8, stream, &s->batch);
  if (st != HBE_OK) { hbe_slabs_destroy(s); return st; }
  if (nc > 0) {
    if (cudaMalloc(&s->batch->d_halo, nc * sizeof(HaloCopy)) != cudaSuccess ||
        cudaMemcpy(s->batch->d_halo, s->plan.data(), nc * sizeof(HaloCopy),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      hbe_slabs_destroy(s);
      return HBE_ENOMEM;
    }
    s->batch->nhalo = nc;
  }
  *out = s;
  return HBE_OK;
}

const char *hbe_slabs_last_error(const hbe_slabs *s) { return s ? s->err.c_str() : "null slabs"; }

hbe_status hbe_slabs_set_initial_device(hbe_slabs *s, const double *d_phi0, const double *d_phi1,
                                        double t0) {
  Range range_("hbe_slabs_set_initial");
  if (!s || !d_phi0 || !d_phi1) return HBE_EINVAL;
  if (!std::isfinite(t0)) return set_err(s->err, HBE_EINVAL, "t0 must be finite");
  const size_t plane = (size_t)s->N * s->N;
  for (int i = 0; i < s->k; ++i) {
    hbe_ctx *c = s->parts[i];
    hbe_status st = sync_ctx(c);
    if (st != HBE_OK) return set_err(s->err, st, "%s", c->err.c_str());
    const int sprec = c->prec == HBE_FP64 ? 0 : 1;
    const bool kahan = is_kahan(c->prec);
    // the slab's planes of the global fields into its interior planes
    CKX(s->err, launch_pack(sprec, d_phi0 + s->z0[i] * plane, c->f[F_P0],
                            kahan ? c->f[F_PLO0] : nullptr, s->N, c->pitch_s, c->hxs, c->bc,
                            c->zoff, s->nz[i], s->stream));
    CKX(s->err, launch_pack(sprec, d_phi1 + s->z0[i] * plane, c->f[F_Q0],
                            kahan ? c->f[F_QLO0] : nullptr, s->N, c->pitch_s, c->hxs, c->bc,
                            c->zoff, s->nz[i], s->stream));
  }
  // initial halo planes of phi and psi (set 0), plain copies between the slabs
  for (const HaloCopy &h : s->plan) {
    hbe_ctx *a = s->parts[h.src], *b = s->parts[h.dst];
    const size_t pb = (size_t)a->plane_s * state_size(a->prec);
    for (int f : {F_P0, F_Q0})
      CKX(s->err, cudaMemcpyAsync(static_cast<char *>(b->f[f]) + h.dst_plane * pb,
                                  static_cast<const char *>(a->f[f]) + h.src_plane * pb, 2 * pb,
                                  cudaMemcpyDeviceToDevice, s->stream));
  }
  CKX(s->err, cudaStreamSynchronize(s->stream));
  for (hbe_ctx *c : s->parts) {
    Desc &d = *c->h_desc;
    d.t0 = t0; d.dt = 0.0; d.n_base = 0; d.n_end = 0; d.stop_k = kNoStop;
    d.status = ST_RUNNING; d.last_done = 0;
    hbe_status st = push_desc(c);
    if (st != HBE_OK) return set_err(s->err, st, "%s", c->err.c_str());
    CKX(s->err, cudaMemset(c->d_err, 0, sizeof(unsigned)));
    c->has_state = true;
  }
  return HBE_OK;
}

hbe_status hbe_slabs_step(hbe_slabs *s, int64_t nsteps, double dt) {
  Range range_("hbe_slabs_step");
  if (!s) return HBE_EINVAL;
  if (nsteps < 0) return set_err(s->err, HBE_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(s->err, HBE_EINVAL, "dt must be > 0");
  if (nsteps == 0) return HBE_OK;
  for (hbe_ctx *c : s->parts) {
    hbe_status st = hbe_batch_add(s->batch, c, nsteps, dt);
    if (st != HBE_OK) return set_err(s->err, st, "%s", s->batch->err.c_str());
  }
  // every slab takes the same steps; the halo plan indexes the members in
  // slab order, so a slab that stops early (non-finite values) ends the run
  // of all of them
  std::vector<hbe_ctx *> fin(s->k);
  hbe_status result = HBE_OK;
  while (hbe_batch_size(s->batch) > 0) {
    int nf = 0;
    hbe_status st = hbe_batch_run(s->batch, fin.data(), s->k, &nf);
    if (st != HBE_OK) return set_err(s->err, st, "%s", s->batch->err.c_str());
    for (int i = 0; i < nf && i < s->k; ++i)
      if (fin[i]->h_desc->status == ST_NONFINITE) result = HBE_NONFINITE;
    if (nf > 0 && hbe_batch_size(s->batch) > 0) {
      std::vector<hbe_ctx *> rest(s->batch->members);
      for (hbe_ctx *c : rest) hbe_batch_remove(s->batch, c);
      if (result == HBE_OK) result = HBE_NONFINITE;
    }
  }
  if (result != HBE_OK) set_err(s->err, result, "phi became non-finite");
  return result;
}

hbe_status hbe_slabs_read_device(hbe_slabs *s, double *d_phi, double *d_psi, double *t) {
  Range range_("hbe_slabs_read");
  if (!s) return HBE_EINVAL;
  const size_t plane = (size_t)s->N * s->N;
  for (int i = 0; i < s->k; ++i) {
    hbe_ctx *c = s->parts[i];
    hbe_status st = sync_ctx(c);
    if (st != HBE_OK) return set_err(s->err, st, "%s", c->err.c_str());
    const int sprec = c->prec == HBE_FP64 ? 0 : 1;
    const bool kahan = is_kahan(c->prec);
    const int set = (int)(c->h_desc->n_base & 1);
    if (d_phi)
      CKX(s->err, launch_unpack(sprec, c->f[F_P0 + set], kahan ? c->f[F_PLO0 + set] : nullptr,
                                d_phi + s->z0[i] * plane, s->N, c->pitch_s, c->hxs, c->zoff,
                                s->nz[i], s->stream));
    if (d_psi)
      CKX(s->err, launch_unpack(sprec, c->f[F_Q0 + set], kahan ? c->f[F_QLO0 + set] : nullptr,
                                d_psi + s->z0[i] * plane, s->N, c->pitch_s, c->hxs, c->zoff,
                                s->nz[i], s->stream));
  }
  CKX(s->err, cudaStreamSynchronize(s->stream));
  if (t) *t = current_t(s->parts[0]);
  return HBE_OK;
}

}  // extern "C"
