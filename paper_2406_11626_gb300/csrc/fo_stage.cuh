// The stage kernel of the 58-variable formulations (ccz4_fo_*), shared by
// fo.cu (the general instance) and fo_p9.cu (the instance compiled for 9^3
// patches), so that the two compile in parallel.
#ifndef CCZ4_FO_STAGE_CUH
#define CCZ4_FO_STAGE_CUH

#include "fo_algebra.cuh"

#ifndef CCZ4_FO_MIN_BLOCKS
#define CCZ4_FO_MIN_BLOCKS 4
#endif

namespace ccz4 {

struct FoStageArgs {
  const double *U;  // U_n
  double *acc;      // RK accumulator
  double *out;      // plain right-hand side (MODE < 0), next stage state, or U_{n+1}
  double dt;
};

namespace {

// Receives d_t of each variable of one interior point and applies the stage
// update at once; the last stage holds g~ and A~ back for the enforcement.
template <int MODE>
struct FoSink {
  long long S, i;
  const FoStageArgs &a;
  double ug[6], uA[6];
  __device__ __forceinline__ void operator()(int v, double k) {
    const long long o = v * S + i;
    if (MODE < 0) {
      a.out[o] = k;
      return;
    }
    double acc = MODE == 0 ? 0.0 : a.acc[o];
    const double un = rk_combine<(MODE < 0 ? 0 : MODE), double>(a.U[o], acc, k, a.dt);
    if (MODE < 3) a.acc[o] = acc;
    if (MODE == 3 && v >= GXX && v <= GZZ) {
      ug[v - GXX] = un;
      return;
    }
    if (MODE == 3 && v >= AXX && v <= AZZ) {
      uA[v - AXX] = un;
      return;
    }
    a.out[o] = un;
  }
  __device__ __forceinline__ void finish() {
    if (MODE != 3) return;
    enforce_point<double>(ug, uA);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      a.out[(GXX + c) * S + i] = ug[c];
      a.out[(AXX + c) * S + i] = uA[c];
    }
  }
};

// PF > 0: the patch edge is PF (the grid's p must equal it), so the tile
// strides and the index divisions are compile-time constants.
template <int PF = 0>
__device__ __forceinline__ Nbhd fo_nbhd(const GridView &g, const double *tile, long long i) {
  const int p = PF > 0 ? PF : g.p, T = PF > 0 ? PF + 2 * HALO : g.T;
  const long long T3 = PF > 0 ? (long long)T * T * T : g.T3;
  const int p3 = p * p * p;
  const int n = (int)i / p3;
  const int r = (int)(i - (long long)n * p3);
  const int z = r / (p * p), y = (r / p) % p, x = r % p;
  Nbhd N;
  N.c = tile + n * T3 + ((long long)(z + HALO) * T + (y + HALO)) * T + (x + HALO);
  N.fs = (long long)g.n_patches * T3;
  N.st[0] = 1;
  N.st[1] = T;
  N.st[2] = T * T;
  N.mix = nullptr;
  N.ms = 0;
  N.mixf = nullptr;
  N.msf = 0;
  return N;
}

// One thread per interior point: the 58-variable right-hand side (RED: with
// the red terms; AUX: the auxiliary variables' equations too) and the stage
// update of what it evolves.
template <int MODE, bool RED, bool AUX, int PF = 0>
__global__ void __launch_bounds__(128, CCZ4_FO_MIN_BLOCKS) fo_interior_kernel(GridView g, FoPhys F,
                                                                             StencilCoef<double> C,
                                                                             const double *__restrict__ tile,
                                                                             FoStageArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_points) return;
  const Nbhd N = fo_nbhd<PF>(g, tile, i);
  FoSink<MODE> sink{g.S, i, a};
  fo_rhs_point<RED, AUX>(F, N, C, sink);
  sink.finish();
}

inline StencilCoef<double> fo_coefs(double dx, double eps) {
  StencilCoef<double> C;
  C.c1 = 1.0 / (12.0 * dx);
  C.c2 = 1.0 / (12.0 * dx * dx);
  C.c3 = 1.0 / (144.0 * dx * dx);
  C.cko = eps / (64.0 * dx);
  return C;
}

// Launches the stage kernel of one (MODE, RED, AUX) on every interior point.
template <int MODE, bool RED, bool AUX, int PF>
cudaError_t launch_fo_interior_pf(const GridView &g, const ccz4_params &P, const double *tile, const FoStageArgs &a,
                                  cudaStream_t s) {
  if (g.n_points == 0) return cudaSuccess;
  FoPhys F{make_phys<double>(P), P.mu};
  fo_interior_kernel<MODE, RED, AUX, PF><<<(unsigned)((g.n_points + 127) / 128), 128, 0, s>>>(
      g, F, fo_coefs(g.dx, P.ko_eps), tile, a);
  return cudaGetLastError();
}

}  // namespace

// The instance for 9^3 patches (fo_p9.cu): mode -1..3, red, aux as the template arguments above.
cudaError_t launch_fo_interior_p9(int mode, bool red, bool aux, const GridView &g, const ccz4_params &P,
                                  const double *tile, const FoStageArgs &a, cudaStream_t s);

}  // namespace ccz4

#endif
