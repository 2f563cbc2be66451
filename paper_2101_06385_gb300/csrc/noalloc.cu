// sp2_density_matrix_noalloc: the split-FP16 SP2 solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any routine that allocates) at the
// time they need a density matrix: callers that own a fixed memory budget and
// must not grow the process footprint mid-run (MD engines that pre-size every
// buffer at start-up), real-time loops in which an allocation, which can
// synchronise the device, would stall a step, and hosts that hand the library
// only pointers they manage themselves.  This entry
// point therefore takes all of its scratch from one file-scope device array
// of fixed size, which the module loader places in device memory when the
// library is loaded on a GPU; every GPU that loads the library keeps it until
// the process exits.
//
// Limits: N <= SP2_NOALLOC_MAX_N (1024); split-FP16 precision, identity shift
// on, epsilon 0, low-part scale 2^11 (the defaults of sp2_init), independent
// of sp2_init and of the library workspace.
//
// Set-up: the first call on a device (with that device current) looks up the
// device address of the array with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture.  Every call shares the array and
// leaves its contents behind: the counters that must start at zero are cleared
// by the first kernel of each call, and two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/sp2.h"
#include "common.cuh"
#include "kernels.h"

namespace sp2 {
void set_error_text(const char* s);  // defined with sp2_last_error

namespace noalloc {

constexpr int kMaxN = SP2_NOALLOC_MAX_N;
constexpr long long kLdH = ((kMaxN + 63) / 64) * 64;   // FP16 row stride of a split buffer
constexpr int kT2 = (kMaxN + kTcBN - 1) / kTcBN;       // 256-wide block rows
constexpr int kMaxTiles = kT2 * (kT2 + 1);             // two CTA tiles per upper super tile
constexpr int kMaxPartials = 1024;                     // per-block partials of the small kernels

// byte offsets inside the scratch array (each 256-aligned)
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kSplitBytes = (size_t)kLdH * kMaxN * 2;
constexpr size_t OFF_HI0 = 0;
constexpr size_t OFF_LO0 = OFF_HI0 + align256(kSplitBytes);
constexpr size_t OFF_HI1 = OFF_LO0 + align256(kSplitBytes);
constexpr size_t OFF_LO1 = OFF_HI1 + align256(kSplitBytes);
constexpr size_t OFF_RN = OFF_LO1 + align256(kSplitBytes);
constexpr size_t OFF_CTL = OFF_RN + align256(sizeof(double) * kMaxN);
constexpr size_t OFF_TILES = OFF_CTL + align256(sizeof(Ctl));
constexpr size_t OFF_TPART = OFF_TILES + align256(sizeof(uint32_t) * kMaxTiles);
constexpr size_t OFF_PART = OFF_TPART + align256(sizeof(double2) * kMaxTiles);
constexpr size_t OFF_SMALL = OFF_PART + align256(sizeof(double2) * kMaxPartials);
// small block: tile_off, tile_cnt, inst_done, tickets[8], err, N, H ptr, D ptr
constexpr size_t kSmallBytes = 256;
constexpr size_t kScratchBytes = OFF_SMALL + kSmallBytes;

static_assert(kScratchBytes <= (size_t)SP2_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

struct Small {
  int tile_off;
  int tile_cnt;
  unsigned inst_done;
  int err;
  unsigned tickets[8];
  int N;
  int pad;
  const float* H;
  float* D;
};
static_assert(sizeof(Small) <= kSmallBytes, "small block too large");

}  // namespace noalloc
}  // namespace sp2

// The scratch of every sp2_density_matrix_noalloc call.  Host code must not
// pass this name to a kernel (on the host it is only a stand-in symbol); it
// uses the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sp2_noalloc_scratch[SP2_NOALLOC_SCRATCH_BYTES];

namespace sp2 {
namespace noalloc {

// Per-call reset and set-up on the device: control block, tile list and the
// zero-start counters; no host-to-device copies are needed.
__global__ void init_kernel(unsigned char* base, const float* H, float* D, int N, int n_occ, double tol,
                            int max_iter) {
  Small* sm = reinterpret_cast<Small*>(base + OFF_SMALL);
  uint32_t* tiles = reinterpret_cast<uint32_t*>(base + OFF_TILES);
  const int T = (N + kTcBN - 1) / kTcBN;
  if (threadIdx.x == 0) {
    Ctl* c = reinterpret_cast<Ctl*>(base + OFF_CTL);
    memset(c, 0, sizeof(Ctl));
    c->N = N;
    c->n_occ = n_occ;
    c->max_iter = max_iter;
    c->shift = 1;
    c->tol = tol;
    c->eps = 0.0;
    c->phase = PHASE_LOOP;
    c->status = SP2_OK;
    c->next.active = 1;
    // upper 256 x 256 super tiles, row-major (T <= 4 here), two 128-row halves each
    int n = 0;
    for (int I = 0; I < T; ++I)
      for (int J = I; J < T; ++J) {
        tiles[n++] = pack_tile(0, I, J, 0);
        if (I * kTcBN + kTcBM < N) tiles[n++] = pack_tile(0, I, J, 1);
      }
    sm->tile_off = 0;
    sm->tile_cnt = n;
    sm->inst_done = 0u;
    sm->err = 0;
    for (int i = 0; i < 8; ++i) sm->tickets[i] = 0u;
    sm->N = N;
    sm->H = H;
    sm->D = D;
  }
}

struct DeviceState {
  std::atomic<bool> ready{false};
  unsigned char* scratch = nullptr;
  int num_sms = 0;
};
DeviceState g_dev[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
// serialises the one-time set-up (host threads making their first calls at once)
std::mutex g_setup;

// the text sp2_last_error() returns
void msg(const char* s) { set_error_text(s); }

bool tmap(CUtensorMap* out, const void* base, int N, long long ld, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, 1};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * N * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace noalloc
}  // namespace sp2

using namespace sp2;
using namespace sp2::noalloc;

#define NA_CK(expr)                                  \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) {                         \
      msg(cudaGetErrorString(e_));                   \
      return SP2_ERR_CUDA;                           \
    }                                                \
  } while (0)

extern "C" sp2_status sp2_density_matrix_noalloc(const float* H, int N, int N_occ, double tol, int max_iter,
                                                 float* D_out, sp2_stats* stats, void* stream) {
  msg("");
  if (!H || !D_out || H == D_out || N < 1 || N_occ < 0 || N_occ > N || !(tol >= 0.0) || !std::isfinite(tol) ||
      max_iter < 1 || max_iter > SP2_MAX_LAYERS - 3) {
    msg("sp2_density_matrix_noalloc: invalid argument");
    return SP2_ERR_INVALID_ARG;
  }
  if (N > kMaxN) {
    msg("sp2_density_matrix_noalloc: N exceeds SP2_NOALLOC_MAX_N (1024); use sp2_density_matrix");
    return SP2_ERR_INVALID_ARG;
  }
  int dev = 0;
  NA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    msg("sp2_density_matrix_noalloc: device ordinal out of range");
    return SP2_ERR_UNSUPPORTED;
  }
  DeviceState& ds = g_dev[dev];
  if (!ds.ready.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_setup);
    if (!ds.ready.load(std::memory_order_relaxed)) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_sp2_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        msg("sp2_density_matrix_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return SP2_ERR_CUDA;
      }
      int major = 0;
      NA_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
      if (major != 10) {
        msg("sp2_density_matrix_noalloc: needs an sm_103a device");
        return SP2_ERR_UNSUPPORTED;
      }
      NA_CK(cudaDeviceGetAttribute(&ds.num_sms, cudaDevAttrMultiProcessorCount, dev));
      if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        NA_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (!fn || q != cudaDriverEntryPointSuccess) {
          msg("sp2_density_matrix_noalloc: cuTensorMapEncodeTiled not available");
          return SP2_ERR_UNSUPPORTED;
        }
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
      }
      ds.scratch = static_cast<unsigned char*>(p);
      ds.ready.store(true, std::memory_order_release);
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (stats) {
    // the stats read-back copies to the host and synchronises the stream,
    // which a stream under capture does not allow
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NA_CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      msg("sp2_density_matrix_noalloc: stats must be NULL on a stream that is being captured");
      return SP2_ERR_INVALID_ARG;
    }
  }
  unsigned char* base = ds.scratch;
  __half* hi[2] = {reinterpret_cast<__half*>(base + OFF_HI0), reinterpret_cast<__half*>(base + OFF_HI1)};
  __half* lo[2] = {reinterpret_cast<__half*>(base + OFF_LO0), reinterpret_cast<__half*>(base + OFF_LO1)};
  double* rn = reinterpret_cast<double*>(base + OFF_RN);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + OFF_CTL);
  uint32_t* tiles = reinterpret_cast<uint32_t*>(base + OFF_TILES);
  double2* tpart = reinterpret_cast<double2*>(base + OFF_TPART);
  double2* part = reinterpret_cast<double2*>(base + OFF_PART);
  Small* sm = reinterpret_cast<Small*>(base + OFF_SMALL);

  const long long ld_h = ((N + 63) / 64) * 64, slot_h = ld_h * N;
  const int T = (N + kTcBN - 1) / kTcBN;
  int ntiles = 0;
  for (int I = 0; I < T; ++I)
    for (int J = I; J < T; ++J) ntiles += (I * kTcBN + kTcBM < N) ? 2 : 1;
  const float lo_scale = 2048.f, lo_unscale = 1.f / 2048.f;

  init_kernel<<<1, 32, 0, st>>>(base, H, D_out, N, N_occ, tol, max_iter);
  NA_CK(cudaGetLastError());
  const int ggrid = (N + 7) / 8 < 4 * ds.num_sms ? (N + 7) / 8 : 4 * ds.num_sms;
  const int igrid = N < 8 * ds.num_sms ? N : 8 * ds.num_sms;
  const int rgrid = (N + 7) / 8 < 2 * ds.num_sms ? (N + 7) / 8 : 2 * ds.num_sms;
  NA_CK(launch_gershgorin(H, N, N, (long long)N * N, 1, part, &sm->tickets[0], ctl, nullptr, ggrid, st));
  NA_CK(launch_input_layer(reinterpret_cast<const float* const*>(&sm->H), &sm->N, N, D_out, N, (long long)N * N,
                           hi[0], lo[0], nullptr, ld_h, slot_h, N, (int)ld_h, lo_scale, ctl, nullptr, part, &sm->tickets[0], 1,
                           1, 1, igrid, st));
  NA_CK(launch_rownorm(D_out, N, (long long)N * N, &sm->N, 1, N, rn, N, ctl, part, &sm->tickets[0], rgrid, st));

  CUtensorMap m[2][4];
  for (int b = 0; b < 2; ++b) {
    if (!tmap(&m[b][0], hi[b], N, ld_h, kTcBM) || !tmap(&m[b][1], lo[b], N, ld_h, kTcBM) ||
        !tmap(&m[b][2], hi[b], N, ld_h, kTcBN) || !tmap(&m[b][3], lo[b], N, ld_h, kTcBN)) {
      msg("sp2_density_matrix_noalloc: cuTensorMapEncodeTiled failed");
      return SP2_ERR_CUDA;
    }
  }
  SqArgs A;
  memset(&A, 0, sizeof(A));
  A.Yin = D_out;
  A.Yout = D_out;
  A.ld_y = N;
  A.slot_y = (long long)N * N;
  A.ld_h = ld_h;
  A.slot_h = slot_h;
  A.Dptr = reinterpret_cast<float* const*>(&sm->D);
  A.Ns = &sm->N;
  A.tiles = tiles;
  A.ntiles = ntiles;
  A.tile_off = &sm->tile_off;
  A.tile_cnt = &sm->tile_cnt;
  A.ctl = ctl;
  A.lp = nullptr;
  A.tile_part = tpart;
  A.inst_done = &sm->inst_done;
  A.traces_out = nullptr;
  A.rn = rn;
  A.ld_rn = N;
  A.lo_scale = lo_scale;
  A.lo_unscale = lo_unscale;
  A.err = &sm->err;
  const int grid = ntiles < ds.num_sms ? ntiles : ds.num_sms;
  for (int k = 0; k < max_iter + 2; ++k) {
    const int cur = k & 1;
    A.hi_out = hi[cur ^ 1];
    A.lo_out = lo[cur ^ 1];
    NA_CK(launch_syrk_tc(A, m[cur], true, grid, st));
    NA_CK(launch_rownorm(D_out, N, (long long)N * N, &sm->N, 1, N, rn, N, ctl, part, &sm->tickets[0], rgrid, st));
  }
  if (!stats) return SP2_OK;

  // read back the control block (pageable host memory: a copy, no allocation)
  static thread_local Ctl hc;
  int herr = 0;
  NA_CK(cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaMemcpyAsync(&herr, &sm->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  memset(stats, 0, sizeof(*stats));
  stats->iterations = hc.n;
  stats->converged_by = hc.converged_by;
  stats->status_device = hc.status;
  stats->n_occ = hc.n_occ;
  stats->e_min = hc.e_min;
  stats->e_max = hc.e_max;
  stats->idemp_err = (hc.n >= 1 && hc.n <= kMaxL) ? hc.iderr[hc.n] : 0.0;
  stats->trace = hc.trace_final;
  stats->alpha = hc.alpha;
  stats->flops_alg = (hc.phase == PHASE_DONE ? hc.n + 2 : hc.n) * 3.0 * (double)N * N * N;
  stats->launches = max_iter + 2;
  for (int k = 0; k < kMaxL; ++k) {
    stats->sigma[k] = (k + 1 <= hc.n) ? (int8_t)hc.sigma[k + 1] : 0;
    stats->iderr[k] = (k + 1 <= hc.n) ? hc.iderr[k + 1] : 0.0;
  }
  if (herr != 0) {
    msg("sp2_density_matrix_noalloc: a bounded device wait timed out");
    return SP2_ERR_DEVICE_TIMEOUT;
  }
  if (hc.status < 0) {
    msg(hc.status == SP2_ERR_NONFINITE ? "non-finite spectral bounds (NaN or Inf in H)"
                                       : "degenerate spectrum: e_max - e_min <= 0 with 0 < N_occ < N");
    return (sp2_status)hc.status;
  }
  if (hc.phase != PHASE_DONE) {
    msg("sp2_density_matrix_noalloc: solve did not finish");
    return SP2_ERR_CUDA;
  }
  return hc.converged_by == SP2_STOP_MAXITER ? SP2_NOT_CONVERGED : SP2_OK;
}
