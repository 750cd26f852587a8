// One launch per RK stage (CCZ4_LAUNCH_FUSED): a cooperative kernel whose
// blocks first fill the halo'd tiles of all patches (one patch per block at
// a time, the fill of halo.cu), wait for one another at a grid-wide barrier,
// then evolve the interior points (32-point items per warp, strided over the
// grid) and the Sommerfeld ghost cells. This is the paper's enclave
// batching taken to a whole stage: every patch of every level in one task.
// Compiled for 9^3 patches (the stage kernel's instance for that edge) and
// the RK stages; the restriction after a step stays its own launch.
//
// The mixed derivatives are written by the fill phase of the same launch, so
// they are read back with coherent loads (not the read-only path); the tiles
// already are (streaming loads), and the grid barrier orders them.
#define CCZ4_MIX_LOAD __ldcg
#include <cooperative_groups.h>

#include "halo_fill.cuh"
#include "stage_kernels.cuh"

namespace ccz4 {
namespace {

constexpr int FUSED_THREADS = 128;
constexpr int FUSED_PF = 9;

template <int MODE, class R, bool MESH>
__global__ void __launch_bounds__(FUSED_THREADS, (StageBlocks<R, 0>::value))
    fused_stage_kernel(GridView g, Phys<R> P, LevelCoef<R> LC, LevelScale ls, ccz4_params Pg,
                       const double *__restrict__ in, const double *__restrict__ ini, double *tile, double *mix,
                       StageArgs a) {
  extern __shared__ double smem[];
  constexpr bool F32W = std::is_same<R, float>::value;
  for (int n = blockIdx.x; n < g.n_patches; n += gridDim.x) {
    fill_patch<MESH, F32W, FUSED_THREADS, 8, FUSED_PF>(g, in, tile, mix, ls, n, smem);
    __syncthreads();  // the next patch's source table overwrites this one's shared memory
  }
  cooperative_groups::this_grid().sync();
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (FUSED_THREADS / 32);
  for (long long item = (long long)blockIdx.x * (FUSED_THREADS / 32) + threadIdx.x / 32; item * 32 < g.n_points;
       item += warps) {
    const long long i = item * 32 + lane;
    if (i < g.n_points) stage_point<MODE, R, MESH, FUSED_PF>(g, P, LC, tile, mix, a, i);
  }
  const long long total = g.n_ghost * NV;
  for (long long q = (long long)blockIdx.x * FUSED_THREADS + threadIdx.x; q < total;
       q += (long long)gridDim.x * FUSED_THREADS)
    ghost_point<MODE>(g, Pg, in, ini, a, q % g.n_ghost, (int)(q / g.n_ghost));
}

template <int MODE, class R, bool MESH>
const void *fused_fn() {
  return (const void *)fused_stage_kernel<MODE, R, MESH>;
}

// Every instance, for the shared-memory attribute and the occupancy query.
const void *fused_any(int mode, bool mixed, bool mesh) {
#define CCZ4_FUSED_CASE(M)                                                                       \
  case M:                                                                                        \
    return mixed ? (mesh ? fused_fn<M, float, true>() : fused_fn<M, float, false>())             \
                 : (mesh ? fused_fn<M, double, true>() : fused_fn<M, double, false>());
  switch (mode) {
    CCZ4_FUSED_CASE(0)
    CCZ4_FUSED_CASE(1)
    CCZ4_FUSED_CASE(2)
    CCZ4_FUSED_CASE(3)
  }
#undef CCZ4_FUSED_CASE
  return nullptr;
}

template <int MODE, class R, bool MESH>
cudaError_t launch_fused_as(const GridView &g, const ccz4_params &P, double *tile, double *mix, const double *in,
                            const double *ini, const StageArgs &a, cudaStream_t s) {
  const void *fn = fused_fn<MODE, R, MESH>();
  const size_t smem = fill_smem_bytes(FUSED_PF);
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, FUSED_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  LevelCoef<R> LC;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    const StencilCoef<double> C = coefs(g.ldx[l], P);
    LC.C[l] = C;
    LC.CR[l] = StencilCoef<R>{R(C.c1), R(C.c2), R(C.c3), R(C.cko)};
  }
  GridView gv = g;
  Phys<R> ph = make_phys<R>(P);
  LevelScale ls = level_scale(g);
  ccz4_params Pg = P;
  StageArgs av = a;
  void *args[] = {&gv, &ph, &LC, &ls, &Pg, (void *)&in, (void *)&ini, &tile, &mix, &av};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: the grid barrier may wait for every one
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3((unsigned)(sms * occ));
  cfg.blockDim = dim3(FUSED_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

template <int MODE>
cudaError_t launch_fused_mode(const GridView &g, const ccz4_params &P, double *tile, double *mix, const double *in,
                              const double *ini, const StageArgs &a, cudaStream_t s) {
  const bool mixed = P.precision == CCZ4_PREC_MIXED, mesh = g.src != nullptr;
  if (mixed)
    return mesh ? launch_fused_as<MODE, float, true>(g, P, tile, mix, in, ini, a, s)
                : launch_fused_as<MODE, float, false>(g, P, tile, mix, in, ini, a, s);
  return mesh ? launch_fused_as<MODE, double, true>(g, P, tile, mix, in, ini, a, s)
              : launch_fused_as<MODE, double, false>(g, P, tile, mix, in, ini, a, s);
}

}  // namespace

cudaError_t prepare_fused() {
  const int bytes = (int)fill_smem_bytes(FUSED_PF);
  for (int m = 0; m < 4; ++m)
    for (int x = 0; x < 2; ++x)
      for (int h = 0; h < 2; ++h) {
        cudaError_t e = cudaFuncSetAttribute(fused_any(m, x, h), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

cudaError_t launch_fused_stage(const GridView &g, const ccz4_params &P, int stage, double dt, double *tile,
                               double *mix, const double *in, const double *ini, const double *U, double *acc,
                               double *out, cudaStream_t s) {
  if (g.p != FUSED_PF || stage < 0 || stage > 3) return cudaErrorInvalidValue;
  const StageArgs a{U, acc, out, dt};
  switch (stage) {
    case 0: return launch_fused_mode<0>(g, P, tile, mix, in, ini, a, s);
    case 1: return launch_fused_mode<1>(g, P, tile, mix, in, ini, a, s);
    case 2: return launch_fused_mode<2>(g, P, tile, mix, in, ini, a, s);
    default: return launch_fused_mode<3>(g, P, tile, mix, in, ini, a, s);
  }
}

}  // namespace ccz4
