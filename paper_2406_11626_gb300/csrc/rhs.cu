// Stage kernels of a single uniform level, and the dispatch of the stage
// launches between single levels and refined meshes.
#include "stage_kernels.cuh"

namespace ccz4 {

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
