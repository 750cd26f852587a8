// The stage kernel of the 58-variable formulations compiled for 9^3
// patches (tile strides and index divisions as compile-time constants), in a
// translation unit of its own so that it compiles beside fo.cu.
#include "fo_stage.cuh"

namespace ccz4 {

cudaError_t launch_fo_interior_p9(int mode, bool red, bool aux, const GridView &g, const ccz4_params &P,
                                  const double *tile, const FoStageArgs &a, cudaStream_t s) {
  // the combinations fo.cu launches: first order (red, aux) in every mode; the reconstructed second
  // order without red terms, with the auxiliary equations for the plain right-hand side only
  if (red && aux) {
    switch (mode) {
      case -1: return launch_fo_interior_pf<-1, true, true, 9>(g, P, tile, a, s);
      case 0: return launch_fo_interior_pf<0, true, true, 9>(g, P, tile, a, s);
      case 1: return launch_fo_interior_pf<1, true, true, 9>(g, P, tile, a, s);
      case 2: return launch_fo_interior_pf<2, true, true, 9>(g, P, tile, a, s);
      case 3: return launch_fo_interior_pf<3, true, true, 9>(g, P, tile, a, s);
    }
  } else if (!red && aux && mode == -1) {
    return launch_fo_interior_pf<-1, false, true, 9>(g, P, tile, a, s);
  } else if (!red && !aux) {
    switch (mode) {
      case 0: return launch_fo_interior_pf<0, false, false, 9>(g, P, tile, a, s);
      case 1: return launch_fo_interior_pf<1, false, false, 9>(g, P, tile, a, s);
      case 2: return launch_fo_interior_pf<2, false, false, 9>(g, P, tile, a, s);
      case 3: return launch_fo_interior_pf<3, false, false, 9>(g, P, tile, a, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ccz4
