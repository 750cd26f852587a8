// Halo fill: glue every patch and the data around it into a (p+6)^3 tile
// (Sec. "Spatial Discretisation", Fig. patch-face-reconstruction), and take
// the mixed second derivatives of the fields that need them while the tile
// sits in shared memory.
//
// One CTA per patch. It resolves the source of every tile point once
// (neighbour patch, periodic wrap, clamped copy or Sommerfeld ghost cell;
// on a refined mesh it reads the host-built table instead) into an index
// table, then for each of the 25 fields gathers the field's tile into
// shared memory and writes it out with coalesced stores. On a refined mesh
// the coarse-to-fine interpolations of the halo are evaluated separably per
// field (the patch's distinct x-interpolations, then the distinct
// y-interpolations of their pairs, then one z-interpolation per halo point,
// in shared memory), or point by point for all fields at once where the
// host planned no separable tables. For g~,
// alpha, beta and phi it also forms the mixed derivatives d_x d_y, d_x d_z,
// d_y d_z as the first-derivative stencil applied to first derivatives
// shared through shared memory: d_y Q is taken once on the patch widened by
// two points along x and reused by the five neighbours that need it, which
// costs about half the FP64 operations of evaluating each point's 16-point
// tensor-product stencil on its own. The result is the same FD4 mixed
// derivative (the tensor product of two first-derivative stencils).
// For the mixed-precision stage kernel (F32W) the tiles of every field but
// alpha and phi are written as split FP32 pairs (split_pair), and the
// shared-memory tile of such a field holds the same pairs, from which the
// inner first derivatives of g~ and beta are taken in FP32.
#include "halo_fill.cuh"

namespace ccz4 {
namespace {

template <bool MESH, bool F32W, int SHAPE, int PF = 0>
__global__ void __launch_bounds__(FILL_SHAPE_THREADS[SHAPE], 1024 / FILL_SHAPE_THREADS[SHAPE])
    fill_halos_kernel(GridView g, const double *__restrict__ src, double *__restrict__ tile,
                      double *__restrict__ mix, LevelScale ls) {
  extern __shared__ double smem[];
  fill_patch<MESH, F32W, FILL_SHAPE_THREADS[SHAPE], FILL_SHAPE_BATCH[SHAPE], PF>(g, src, tile, mix, ls,
                                                                                 blockIdx.x, smem);
}

}  // namespace

// Raises the kernel's dynamic shared-memory limit for patch edge p (once per
// grid, outside any stream capture).
template <int SHAPE>
cudaError_t prepare_shape(int bytes) {
  const void *kernels[8] = {(const void *)fill_halos_kernel<false, false, SHAPE>,
                            (const void *)fill_halos_kernel<false, true, SHAPE>,
                            (const void *)fill_halos_kernel<true, false, SHAPE>,
                            (const void *)fill_halos_kernel<true, true, SHAPE>,
                            (const void *)fill_halos_kernel<false, false, SHAPE, 9>,
                            (const void *)fill_halos_kernel<false, true, SHAPE, 9>,
                            (const void *)fill_halos_kernel<true, false, SHAPE, 9>,
                            (const void *)fill_halos_kernel<true, true, SHAPE, 9>};
  for (const void *k : kernels) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t prepare_fill_halos(int p) {
  const int bytes = (int)fill_smem_bytes(MAX_P > p ? MAX_P : p);
  cudaError_t e = prepare_shape<0>(bytes);
  if (e == cudaSuccess) e = prepare_shape<1>(bytes);
  if (e == cudaSuccess) e = prepare_shape<2>(bytes);
  if (e == cudaSuccess) e = prepare_shape<3>(bytes);
  return e;
}

template <int SHAPE, int PF>
void launch_fill_edge(const GridView &g, const double *src, double *tile, double *mix, cudaStream_t s,
                      bool fp32_weights, size_t bytes, const LevelScale &ls) {
  const dim3 grid(g.n_patches), block(FILL_SHAPE_THREADS[SHAPE]);
  if (g.src && fp32_weights)
    fill_halos_kernel<true, true, SHAPE, PF><<<grid, block, bytes, s>>>(g, src, tile, mix, ls);
  else if (g.src)
    fill_halos_kernel<true, false, SHAPE, PF><<<grid, block, bytes, s>>>(g, src, tile, mix, ls);
  else if (fp32_weights)
    fill_halos_kernel<false, true, SHAPE, PF><<<grid, block, bytes, s>>>(g, src, tile, mix, ls);
  else
    fill_halos_kernel<false, false, SHAPE, PF><<<grid, block, bytes, s>>>(g, src, tile, mix, ls);
}

// p = 9 (the paper's patch edge) takes the fill compiled for that edge.
template <int SHAPE>
void launch_fill_shape(const GridView &g, const double *src, double *tile, double *mix, cudaStream_t s,
                       bool fp32_weights, size_t bytes, const LevelScale &ls) {
  if (g.p == 9)
    launch_fill_edge<SHAPE, 9>(g, src, tile, mix, s, fp32_weights, bytes, ls);
  else
    launch_fill_edge<SHAPE, 0>(g, src, tile, mix, s, fp32_weights, bytes, ls);
}

cudaError_t launch_fill_halos(const GridView &g, const double *src, double *tile, double *mix, cudaStream_t s,
                              bool fp32_weights) {
  if (g.n_patches == 0) return cudaSuccess;
  const size_t bytes = fill_smem_bytes(g.p);
  const LevelScale ls = level_scale(g);
  switch (g.fill_shape) {
    case 1: launch_fill_shape<1>(g, src, tile, mix, s, fp32_weights, bytes, ls); break;
    case 2: launch_fill_shape<2>(g, src, tile, mix, s, fp32_weights, bytes, ls); break;
    case 3: launch_fill_shape<3>(g, src, tile, mix, s, fp32_weights, bytes, ls); break;
    default: launch_fill_shape<0>(g, src, tile, mix, s, fp32_weights, bytes, ls); break;
  }
  return cudaGetLastError();
}

}  // namespace ccz4
