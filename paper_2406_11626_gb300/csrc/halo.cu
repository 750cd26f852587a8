// Halo fill: glue every patch and the data around it into a (p+6)^3 tile
// (Sec. "Spatial Discretisation", Fig. patch-face-reconstruction). One
// thread per tile point resolves the global point once (neighbour patch,
// periodic wrap, clamped copy or Sommerfeld ghost cell) and moves the 25
// field values; consecutive threads write consecutive tile addresses.
#include "ccz4_internal.cuh"

namespace ccz4 {
namespace {

__global__ void __launch_bounds__(256) fill_halos_kernel(GridView g, const double *__restrict__ src,
                                                         double *__restrict__ tile) {
  const long long total = (long long)g.n_patches * g.T3;
  const long long fs = total;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t / g.T3);
    const int r = (int)(t - (long long)n * g.T3);
    const int T = g.T;
    const int lz = r / (T * T), ly = (r / T) % T, lx = r % T;
    const int gx = __ldg(g.ijk + 3 * n) * g.p + lx - HALO;
    const int gy = __ldg(g.ijk + 3 * n + 1) * g.p + ly - HALO;
    const int gz = __ldg(g.ijk + 3 * n + 2) * g.p + lz - HALO;
    const long long s = locate(g, gx, gy, gz);
    if (s < 0) continue;
#pragma unroll 5
    for (int v = 0; v < NV; ++v) tile[v * fs + t] = __ldg(src + v * g.S + s);
  }
}

}  // namespace

cudaError_t launch_fill_halos(const GridView &g, const double *src, double *tile, cudaStream_t s) {
  const long long total = (long long)g.n_patches * g.T3;
  if (total == 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  fill_halos_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, src, tile);
  return cudaGetLastError();
}

}  // namespace ccz4
