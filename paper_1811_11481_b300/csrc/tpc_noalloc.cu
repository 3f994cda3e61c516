// Refit entry point that allocates no device memory (tpc_refit_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a refit:
// code running while a CUDA stream is being captured into a graph (cudaMalloc
// is not a stream operation and breaks the capture), real-time loops that
// must not take the device-wide synchronisation an allocation can imply, and
// plug-ins living inside a host framework whose caching allocator already
// owns the device memory budget. For them this entry point takes every input
// and output from the caller and keeps its own working memory in a fixed
// file-scope device array: every GPU that loads the library reserves it
// (TPC_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "tpc_impl.h"
#include "tpc_refit_core.cuh"

namespace {

using namespace tpc;

// Scratch: per assigned cluster a packed (row, flags) word and the rejection
// pass of the three-pass refit.
constexpr int64_t kMaxAssigned = TPC_NOALLOC_MAX_ASSIGNED;
constexpr size_t kMetaBytes = sizeof(uint32_t) * (size_t)kMaxAssigned;
constexpr size_t kRowXBytes = 1024;  // pad-row positions (TPC_MAX_ROWS floats)
constexpr size_t kScratchBytes = kRowXBytes + kMetaBytes + (size_t)kMaxAssigned;
static_assert(sizeof(float) * TPC_MAX_ROWS <= kRowXBytes, "row table");
static_assert(kScratchBytes == TPC_NOALLOC_SCRATCH_BYTES, "scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, resolved once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_of_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// The pad-row positions travel by value in the launch (no host memory is
// read by a copy) into the scratch array.
struct RowX {
  float v[TPC_MAX_ROWS];
};
__global__ void k_na_rowx(RowX in, int n_rows, float* out) {
  int r = threadIdx.x;
  if (r < n_rows) out[r] = in.v[r];
}

__global__ void k_na_meta(int64_t n_assigned, const uint8_t* row, const uint8_t* flags,
                          int n_rows, uint32_t* meta) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_assigned) return;
  uint32_t r = row[j];
  if (r >= (uint32_t)n_rows) r = 0xffu;  // marks the cluster invalid for the refit
  uint32_t f = flags ? flags[j] : 0u;
  meta[j] = r | (f << 8);
}

// One thread per track, contiguous layout, no checkpoints.
__global__ void k_na_refit(Geo g, RefitCfg p, int64_t n_tracks, int64_t n_assigned,
                           const uint32_t* track_start, const float* yc, const float* zc,
                           const uint32_t* meta, uint8_t* rej, float* o_params, float* o_cov,
                           float* o_chi2, int32_t* o_ndf, int32_t* o_status) {
  int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= n_tracks) return;
  uint32_t a = track_start[T], b = track_start[T + 1];
  bool bad = b < a || (int64_t)b > n_assigned;
  for (uint32_t j = a; !bad && j < b; ++j) bad = (meta[j] & 0xffu) == 0xffu;
  if (bad) {
    if (o_status) o_status[T] = 3;
    if (o_chi2) o_chi2[T] = 0.0f;
    if (o_ndf) o_ndf[T] = 0;
    return;
  }
  int n = (int)(b - a);
  TrackIn in{track_start, yc, zc, meta};
  Lay ly = contiguous_layout(a, n);
  // the packed words carry no sector: one frame per track
  RefitOut o = refit_track<false>(g, p, in, ly, n, rej, nullptr, nullptr, false);
  if (o.status != 0) {
    o.chi2 = 0.0f;
    o.ndf = 0;
  }
  if (o_status) o_status[T] = o.status;
  if (o_params)
    for (int i = 0; i < 5; ++i) o_params[T * 5 + i] = o.st[i];
  if (o_cov)
    for (int i = 0; i < 15; ++i) o_cov[T * 15 + i] = o.C[i];
  if (o_chi2) o_chi2[T] = o.chi2;
  if (o_ndf) o_ndf[T] = o.ndf;
}

}  // namespace

extern "C" tpc_status tpc_refit_noalloc(const tpc_geometry* geo, const tpc_params* params,
                                        void* stream, int64_t n_tracks, int64_t n_assigned,
                                        const uint32_t* track_start, const float* yc,
                                        const float* zc, const uint8_t* row,
                                        const uint8_t* flags, float* params_out, float* cov_out,
                                        float* chi2_out, int32_t* ndf_out,
                                        int32_t* status_out) {
  if (!geometry_valid(geo)) return TPC_ERR_ARG;
  // the uniform-field helix refit only: a full field is refused rather than
  // ignored (tpc_refit of a context transports in it)
  if (geo->field) return TPC_ERR_ARG;
  if (n_tracks < 0 || n_assigned < 0) return TPC_ERR_ARG;
  if (n_assigned > kMaxAssigned) return TPC_ERR_CAPACITY;
  if (n_tracks == 0) return TPC_OK;
  if (!track_start || (n_assigned > 0 && (!yc || !zc || !row))) return TPC_ERR_ARG;
  unsigned char* scratch = nullptr;
  if (scratch_of_current_device(&scratch) != cudaSuccess) return TPC_ERR_CUDA;
  tpc_params pc;
  if (params) pc = *params;
  else tpc_default_params(&pc);
  Geo g{};
  RowX rx;
  for (int r = 0; r < TPC_MAX_ROWS; ++r) rx.v[r] = r < geo->n_rows ? geo->row_x[r] : 0.0f;
  g.rx = reinterpret_cast<const float*>(scratch);
  g.n_rows = geo->n_rows;
  g.tan_half = geo->tan_half;
  g.L = geo->drift_length;
  g.bz = geo->bz;
  g.kB = (float)2.99792458e-3 * geo->bz;
  RefitCfg cfg{};
  cfg.kB = g.kB;
  cfg.s_max = pc.s_max;
  cfg.sigma = pc.sigma;
  cfg.flag_scale[0] = pc.split_scale;
  cfg.flag_scale[1] = pc.single_row_scale;
  cfg.flag_scale[2] = pc.single_time_scale;
  cfg.flag_scale[3] = pc.edge_scale;
  cfg.flag_scale[4] = pc.shared_scale;
  cfg.chi2_out = pc.chi2_out;
  cfg.refit_inflate = pc.refit_inflate;
  cfg.min_acc_reject = pc.min_acc_reject;
  for (int i = 0; i < 5; ++i) cfg.c0r[i] = pc.c0r[i];
  set_frame_rotations(cfg);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* meta = reinterpret_cast<uint32_t*>(scratch + kRowXBytes);
  uint8_t* rej = scratch + kRowXBytes + kMetaBytes;
  k_na_rowx<<<1, TPC_MAX_ROWS, 0, s>>>(rx, g.n_rows, reinterpret_cast<float*>(scratch));
  if (n_assigned > 0)
    k_na_meta<<<(int)((n_assigned + 255) / 256), 256, 0, s>>>(n_assigned, row, flags, g.n_rows,
                                                              meta);
  k_na_refit<<<(int)((n_tracks + 127) / 128), 128, 0, s>>>(
      g, cfg, n_tracks, n_assigned, track_start, yc, zc, meta, rej, params_out, cov_out, chi2_out,
      ndf_out, status_out);
  return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
