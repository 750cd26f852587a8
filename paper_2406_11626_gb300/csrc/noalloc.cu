// Constraint monitors for callers that cannot allocate device memory.
//
// ccz4_constraints needs a grid, whose buffers (including the per-block
// partial sums of its reduction) come from cudaMalloc. Some callers cannot
// allocate: a host framework that owns every byte of device memory and
// forbids other allocations, or a time loop that must not allocate once it
// runs. For them, ccz4_constraints_noalloc evaluates the same monitors from
// halo tiles the caller already holds, and keeps its only scratch -- the
// per-block partial sums -- in the fixed device array below, which every
// GPU that loads this library holds until the process exits.
#include <mutex>

#include "ccz4_internal.cuh"

namespace ccz4 {
int constraint_blocks(long long n_points);
}

using namespace ccz4;

namespace {

// 16384 blocks of 256 points: up to 4,194,304 interior points per call;
// 16384 x 5 doubles = 640 KiB of device memory.
constexpr int kMaxBlocks = 16384;
constexpr long long kMaxPoints = (long long)kMaxBlocks * 256;
// largest patch edge whose p^3 fits within kMaxPoints (161^3 = 4,173,281)
constexpr int kMaxEdge = 161;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxBlocks * 5];

// Device address of g_partials on each device. In host code the name
// g_partials is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current. The
// address is kept for the life of the process: after a reset of the device
// (cudaDeviceReset) the module may load elsewhere, so a process that resets
// a device must not call this entry point again on it.
double *g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

ccz4_status partials_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d beyond the %d devices this entry point supports", dev, kMaxDevices);
    return CCZ4_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the reduction scratch failed: %s", cudaGetErrorString(e));
      return CCZ4_ERR_CUDA;
    }
    g_partials_addr[dev] = (double *)p;
  }
  *out = g_partials_addr[dev];
  return CCZ4_OK;
}

}  // namespace

extern "C" ccz4_status ccz4_constraints_noalloc(const double *tiles, int p, int n_patches, double dx,
                                                double *dev_H, double *dev_M, double *dev_out, void *stream) {
  if (!tiles || !dev_out || p < 1 || n_patches < 1 || !(dx > 0.0)) {
    set_error("constraints_noalloc: tiles and dev_out must be given, p >= 1, n_patches >= 1, dx > 0");
    return CCZ4_ERR_INVALID;
  }
  // bound p before any product is formed, so that no size can overflow
  if (p > kMaxEdge || (long long)n_patches > kMaxPoints / ((long long)p * p * p)) {
    set_error("constraints_noalloc: %d patches of %d^3 points exceed the maximum of %lld points (fixed scratch "
              "of %d blocks)", n_patches, p, kMaxPoints, kMaxBlocks);
    return CCZ4_ERR_INVALID;
  }
  const long long n_points = (long long)n_patches * p * p * p;
  double *partials = nullptr;
  ccz4_status st = partials_address(&partials);
  if (st != CCZ4_OK) return st;
  GridView v = {};
  v.p = p;
  v.T = p + 2 * HALO;
  v.n_patches = n_patches;
  v.n_points = n_points;
  v.T3 = (long long)v.T * v.T * v.T;
  v.dx = dx;
  v.n_levels = 1;
  v.n_leaf_points = n_points;
  v.ldx[0] = dx;
  for (int l = 1; l < MAX_LEVELS; ++l) v.ldx[l] = v.ldx[l - 1] / 3.0;
  const int blocks = constraint_blocks(n_points);
  cudaError_t e = launch_constraints(v, tiles, dev_H, dev_M, partials, blocks, dev_out, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error("constraints_noalloc launch failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  return CCZ4_OK;
}
