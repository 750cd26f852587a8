// Stage kernels of a single level in the launch shapes other than the
// default (one resident block more or fewer per SM), for the autotuner;
// a translation unit of their own so they compile in parallel.
#include "stage_kernels.cuh"

namespace ccz4 {

cudaError_t launch_shaped_uniform(const GridView &g, int stage, const Phys<double> &ph, const LevelCoef<double> &LC,
                                  const double *tile, const double *mix, const StageArgs &a, cudaStream_t s) {
  return launch_shaped<double, false>(g, stage, ph, LC, tile, mix, a, s);
}

cudaError_t launch_shaped_uniform(const GridView &g, int stage, const Phys<float> &ph, const LevelCoef<float> &LC,
                                  const double *tile, const double *mix, const StageArgs &a, cudaStream_t s) {
  return launch_shaped<float, false>(g, stage, ph, LC, tile, mix, a, s);
}

cudaError_t prepare_shaped_uniform() { return prepare_split<false>(); }

}  // namespace ccz4
