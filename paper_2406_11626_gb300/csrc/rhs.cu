// Stage kernels of a single uniform level, and the dispatch of the stage
// launches between single levels and refined meshes.
#include "stage_kernels.cuh"

namespace ccz4 {

namespace {
// The static geometry of each Sommerfeld ghost cell: its face is the one of
// its highest outside axis; the neighbour one cell inward along that axis,
// the factor (r / x_d) sign / dx of the one-sided normal derivative and
// 1 / r at the cell centre.
__global__ void __launch_bounds__(128) ghost_setup_kernel(GridView g, GhostGeo *out) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= g.n_ghost) return;
  const int c[3] = {__ldg(g.gcoord + 3 * id), __ldg(g.gcoord + 3 * id + 1), __ldg(g.gcoord + 3 * id + 2)};
  int d = 0, side = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (c[q] < 0) {
      d = q;
      side = -1;
    }
    if (c[q] >= g.N[q]) {
      d = q;
      side = 1;
    }
  }
  const int nb[3] = {c[0] - (d == 0 ? side : 0), c[1] - (d == 1 ? side : 0), c[2] - (d == 2 ? side : 0)};
  const long long sn = locate(g, nb[0], nb[1], nb[2]);
  GhostGeo r{-1, 0.0, 0.0};
  if (sn >= 0 && side != 0) {
    double xs[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) xs[q] = g.origin[q] + (c[q] + 0.5) * g.dx;
    const double rr = sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
    const double xd = d == 0 ? xs[0] : d == 1 ? xs[1] : xs[2];
    r.sn = sn;
    r.ir = 1.0 / rr;
    r.geo = rr / xd * (side > 0 ? 1.0 : -1.0) / g.dx;
  }
  out[id] = r;
}
}  // namespace

cudaError_t launch_ghost_setup(const GridView &g, GhostGeo *out, cudaStream_t s) {
  if (g.n_ghost <= 0) return cudaSuccess;
  ghost_setup_kernel<<<(unsigned)((g.n_ghost + 127) / 128), 128, 0, s>>>(g, out);
  return cudaGetLastError();
}

cudaError_t launch_stage_uniform(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                                 const double *mix, const double *in, const double *ini, const StageArgs &a,
                                 cudaStream_t s) {
  return launch_stage<false>(g, P, stage, tile, mix, in, ini, a, s);
}

static cudaError_t dispatch(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                            const double *mix, const double *in, const double *ini, const StageArgs &a,
                            cudaStream_t s) {
  if (g.src) return launch_stage_mesh(g, P, stage, tile, mix, in, ini, a, s);
  return launch_stage_uniform(g, P, stage, tile, mix, in, ini, a, s);
}

cudaError_t launch_rhs(const GridView &g, const ccz4_params &P, const double *tile, const double *mix,
                       const double *in, const double *ini, double *out, cudaStream_t s) {
  StageArgs a{nullptr, nullptr, out, 0.0};
  return dispatch(g, P, -1, tile, mix, in, ini, a, s);
}

cudaError_t launch_rk_stage(const GridView &g, const ccz4_params &P, int stage, double dt,
                            const double *tile, const double *mix, const double *in, const double *ini,
                            const double *U, double *acc, double *out, cudaStream_t s) {
  if (stage < 0 || stage > 3) return cudaErrorInvalidValue;
  StageArgs a{U, acc, out, dt};
  return dispatch(g, P, stage, tile, mix, in, ini, a, s);
}

}  // namespace ccz4
