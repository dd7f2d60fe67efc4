// hbe_noalloc.cu -- an RK4 entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they want to step a problem:
// runtimes that own all device memory through their own pool and forbid
// other allocations, real-time loops where an allocation may block on the
// driver or fail under memory pressure, and code that must not add to the
// device's footprint once it is set up.  hbe_step_fp64_noalloc serves them:
// the caller passes the input and output fields (device arrays), and every
// intermediate array the stage kernels need -- the padded ping-pong state,
// the three stage right-hand sides, the kernels' descriptor, TMA descriptors,
// work list and per-step maxima -- lives in one file-scope __device__ array
// of fixed size, reserved when the library is loaded.  Every GPU that loads
// libhbe therefore holds kNoAllocScratchBytes (7,333,888 bytes, 7.33 MB, for
// N <= 48) until the process exits.
//
// The call copies its descriptors from host memory, synchronises the stream
// and reads the outcome back, so it must be made on a stream that is not
// being captured into a CUDA graph.  The array is shared by every call: each
// call clears the parts that must start at zero, and two calls that overlap
// on the GPU (different host threads, or different streams) race on it.  The
// first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hbe.h"
#include "hbe_aux.h"
#include "hbe_common.cuh"
#include "hbe_variants.h"

namespace {

using namespace hbe;

constexpr int kNoAllocMaxN = 48;
constexpr int kHX = 2;  // FP64: 16 bytes of x-ghost / alignment per side
constexpr int kMaxPitch = (kNoAllocMaxN + 2 * kHX + kHX - 1) / kHX * kHX;
constexpr size_t kFieldBytes =
    ((size_t)(kNoAllocMaxN + 4) * kMaxPitch * kNoAllocMaxN * sizeof(double) + 255) / 256 * 256;
constexpr int kFields = 7;  // p0, p1, q0, q1, G1, G2, G3
constexpr size_t kMetaBytes = 64 * 1024;
constexpr size_t kNoAllocScratchBytes = kFields * kFieldBytes + kMetaBytes;
static_assert(kNoAllocScratchBytes == 7333888, "7 fields of 1,038,336 bytes + 64 KiB");

// The scratch.  Host code must not use this name as a pointer: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// metadata layout inside the scratch, after the fields
constexpr size_t kOffDesc = kFields * kFieldBytes;               // Desc (64-byte aligned)
constexpr size_t kOffTmaps = kOffDesc + (sizeof(Desc) + 127) / 128 * 128;  // NUM_TMAPS x 128 bytes
static_assert(kOffDesc % 64 == 0 && kOffTmaps % 128 == 0 && kOffTmaps >= kOffDesc + sizeof(Desc),
              "the descriptor must not overlap the tensor maps");
static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
constexpr size_t kOffMaxabs = kOffTmaps + NUM_TMAPS * 128;       // kMaxK x 8 bytes
constexpr size_t kOffErr = kOffMaxabs + kMaxK * 8;               // unsigned
constexpr size_t kOffCounts = kOffErr + 16;                      // int nitems, int one
constexpr size_t kOffCoef = kOffCounts + 16;                     // kCoefDoubles x 8 bytes
constexpr size_t kOffItems = kOffCoef + kCoefDoubles * 8;        // work items (int4)
constexpr int kMaxItems = (int)((kMetaBytes - (kOffItems - kOffDesc)) / sizeof(WorkItem));
static_assert(kOffItems + kMaxItems * sizeof(WorkItem) <= kNoAllocScratchBytes, "layout");

struct PerDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;
};
std::mutex g_mu;
PerDevice g_dev[64];
PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;

hbe_status setup(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return HBE_EINVAL;
  if (!g_dev[dev].ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return HBE_ECUDA;
    if (!g_enc) {
      void *fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                           cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess)
        return HBE_ECUDA;
      g_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    g_dev[dev].scratch = static_cast<unsigned char *>(ptr);
    g_dev[dev].ready = true;
  }
  *out = g_dev[dev].scratch;
  return HBE_OK;
}

bool encode(CUtensorMap *m, void *base, int N, int pitch, int bx, int by) {
  cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)(N + 4), (cuuint64_t)N};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 8, (cuuint64_t)pitch * (N + 4) * 8};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

#define NA_CK(call)                                 \
  do {                                              \
    if ((call) != cudaSuccess) return HBE_ECUDA;    \
  } while (0)

}  // namespace

extern "C" hbe_status hbe_step_fp64_noalloc(int N, double L, double mu, double lambda, int bc,
                                           const double *d_phi0, const double *d_phi1, double t0,
                                           double dt, int64_t nsteps, double *d_phi,
                                           double *d_psi, void *stream) {
  if (N < 8 || N > kNoAllocMaxN) return HBE_EINVAL;  // beyond the scratch array's size
  if (!(L > 0.0) || !std::isfinite(L) || !(mu >= 0.0) || !std::isfinite(mu) ||
      !std::isfinite(lambda) || (bc != HBE_BC_DIRICHLET0 && bc != HBE_BC_PERIODIC) ||
      !d_phi0 || !d_phi1 || !d_phi || !d_psi || !(dt > 0.0) || !std::isfinite(dt) ||
      !std::isfinite(t0) || nsteps < 0)
    return HBE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  NA_CK(cudaGetDevice(&dev));
  NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  unsigned char *scr = nullptr;
  hbe_status s = setup(dev, &scr);
  if (s != HBE_OK) return s;

  const VariantTable &vt = variants_fp64();
  const KernelInfo *ks = vt.k[0];
  const int pitch = (N + 2 * kHX + kHX - 1) / kHX * kHX;
  const int64_t plane = (int64_t)(N + 4) * pitch;
  const double h = bc == HBE_BC_PERIODIC ? L / N : L / (N + 1);
  void *f[NUM_FIELDS] = {};
  const int state_fields[4] = {F_P0, F_P1, F_Q0, F_Q1};
  for (int i = 0; i < 4; ++i) f[state_fields[i]] = scr + i * kFieldBytes;
  for (int i = 0; i < 3; ++i) f[F_G1 + i] = scr + (4 + i) * kFieldBytes;
  Desc *d_desc = reinterpret_cast<Desc *>(scr + kOffDesc);
  CUtensorMap *d_tm = reinterpret_cast<CUtensorMap *>(scr + kOffTmaps);
  unsigned long long *d_maxabs = reinterpret_cast<unsigned long long *>(scr + kOffMaxabs);
  unsigned *d_err = reinterpret_cast<unsigned *>(scr + kOffErr);
  int *d_counts = reinterpret_cast<int *>(scr + kOffCounts);
  WorkItem *d_items = reinterpret_cast<WorkItem *>(scr + kOffItems);
  double *d_coef = reinterpret_cast<double *>(scr + kOffCoef);

  // tensor maps of the fields in the scratch: halo boxes for the fields read
  // with a stencil, interior boxes for the fields read at the point (the
  // compensation fields do not exist in FP64; their maps point at p unused)
  const int tx = ks[0].tx, ty = ks[0].ty, bxs = tx + 2 * kHX, by = ty + 4;
  CUtensorMap maps[NUM_TMAPS];
  memset(maps, 0, sizeof(maps));
  struct MapSpec { int map, field, bx, by; };
  const MapSpec specs[] = {
      {TM_P_H0, F_P0, bxs, by}, {TM_P_H1, F_P1, bxs, by}, {TM_Q_H0, F_Q0, bxs, by},
      {TM_Q_H1, F_Q1, bxs, by}, {TM_Q_I0, F_Q0, tx, ty},  {TM_Q_I1, F_Q1, tx, ty},
      {TM_PLO_I0, F_P0, tx, ty}, {TM_PLO_I1, F_P0, tx, ty}, {TM_QLO_I0, F_P0, tx, ty},
      {TM_QLO_I1, F_P0, tx, ty}, {TM_G1_H, F_G1, bxs, by}, {TM_G1_I, F_G1, tx, ty},
      {TM_G2_H, F_G2, bxs, by}, {TM_G2_I, F_G2, tx, ty},  {TM_G3_I, F_G3, tx, ty}};
  for (const MapSpec &m : specs)
    if (!encode(&maps[m.map], f[m.field], N, pitch, m.bx, m.by)) return HBE_ECUDA;

  // work list: whole columns, one item per x-y tile
  std::vector<WorkItem> items;
  const int ntx = (N + tx - 1) / tx, nty = (N + ty - 1) / ty;
  for (int j = 0; j < nty; ++j)
    for (int i = 0; i < ntx; ++i) items.push_back(make_int4(0, i | (j << 16), 0, N));
  if ((int)items.size() > kMaxItems) return HBE_EINVAL;
  const int counts[2] = {(int)items.size(), 1};

  Desc hd;
  memset(&hd, 0, sizeof(hd));
  hd.N = N; hd.bc = bc; hd.prec = HBE_FP64;
  hd.nz = N; hd.zoff = 0; hd.zwrap = bc == HBE_BC_PERIODIC ? 1 : 0;
  hd.pitch_s = pitch; hd.pitch_g = pitch; hd.plane_s = plane; hd.plane_g = plane;
  hd.inv_h2 = 1.0 / (h * h); hd.mu2 = mu * mu; hd.lambda = lambda;
  hd.t0 = t0; hd.dt = dt;
  hd.n_base = 0; hd.n_end = nsteps; hd.stop_k = kNoStop; hd.stop_thr = 0.0;
  hd.maxabs = d_maxabs; hd.coef = d_coef; hd.tmaps = d_tm;
  for (int i = 0; i < NUM_FIELDS; ++i) hd.f[i] = f[i];

  // the scratch keeps the last call's contents: clear what must start at 0
  // (ghost layers of every field, the per-step maxima, the error word)
  NA_CK(cudaMemsetAsync(scr, 0, kFields * kFieldBytes, st));
  NA_CK(cudaMemsetAsync(d_maxabs, 0, kMaxK * 8 + 16, st));
  NA_CK(cudaMemcpyAsync(d_tm, maps, sizeof(maps), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_desc, &hd, sizeof(hd), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem),
                        cudaMemcpyHostToDevice, st));
  NA_CK(launch_pack(0, d_phi0, f[F_P0], nullptr, N, pitch, kHX, bc, 0, N, st));
  NA_CK(launch_pack(0, d_phi1, f[F_Q0], nullptr, N, pitch, kHX, bc, 0, N, st));

  int grid[4];
  for (int s4 = 0; s4 < 4; ++s4) {
    NA_CK(cudaFuncSetAttribute(ks[s4].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               ks[s4].smem));
    int nb = 0;
    NA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ks[s4].fn, ks[s4].threads,
                                                        ks[s4].smem));
    grid[s4] = std::max(1, std::min(nb * sms, counts[0]));
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    NA_CK(launch_coef(d_desc, d_counts + 1, 1, 1, st));
    for (int s4 = 0; s4 < 4; ++s4) {
      StageParams prm{d_desc, d_items, d_counts, d_err, 0};
      void *args[] = {&prm};
      NA_CK(cudaLaunchKernel(ks[s4].fn, dim3(grid[s4]), dim3(ks[s4].threads), args, ks[s4].smem,
                             st));
      if (bc == 1 && stage_needs_wrap(s4 + 1))
        NA_CK(launch_wrap(d_desc, d_counts + 1, 1, 0, s4 + 1, 2 * sms, st));
    }
    NA_CK(launch_advance(d_desc, d_counts + 1, 1, 1, st));
  }
  // where the steps ended: a step whose phi was not finite ends the solve
  // (the advance kernel sets the status and lets no later step run), so the
  // last state is that of step n_base, in buffer set n_base & 1
  Desc out;
  unsigned err = 0;
  NA_CK(cudaMemcpyAsync(&out, d_desc, sizeof(out), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (err) return HBE_ETIMEOUT;
  const int set = (int)(out.n_base & 1);
  NA_CK(launch_unpack(0, f[F_P0 + set], nullptr, d_phi, N, pitch, kHX, 0, N, st));
  NA_CK(launch_unpack(0, f[F_Q0 + set], nullptr, d_psi, N, pitch, kHX, 0, N, st));
  NA_CK(cudaStreamSynchronize(st));
  return out.status == ST_NONFINITE ? HBE_NONFINITE : HBE_OK;
}
