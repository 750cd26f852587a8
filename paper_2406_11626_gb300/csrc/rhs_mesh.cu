// Stage kernels of refined meshes: each thread takes the stencil
// coefficients of its patch's level.
#include "stage_kernels.cuh"

namespace ccz4 {

cudaError_t launch_stage_mesh(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                              const double *mix, const double *in, const double *ini, const StageArgs &a,
                              cudaStream_t s) {
  return launch_stage<true>(g, P, stage, tile, mix, in, ini, a, s);
}

}  // namespace ccz4
