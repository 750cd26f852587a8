// Internal definitions shared by the CUDA translation units of the CCZ4
// library: the device view of a grid, point lookup across patches and the
// boundary, and host-side error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ccz4.h"

namespace ccz4 {

constexpr int NV = CCZ4_NV;
constexpr int HALO = CCZ4_HALO;

// Device-side status bits (OR-ed by kernels, read at synchronising calls).
constexpr unsigned STATUS_BOUNDS = 1u;

// Field indices in the order of the C ABI.
enum : int {
  GXX = 0, GXY, GXZ, GYY, GYZ, GZZ, ALPHA, BETAX, BETAY, BETAZ, PHI,
  AXX, AXY, AXZ, AYY, AYZ, AZZ, KTR, THETA, GHX, GHY, GHZ, BBX, BBY, BBZ
};

// First slot in the mixed-derivative buffer of field v (three slots: d_x d_y,
// d_x d_z, d_y d_z), or -1 for fields without second derivatives.
__host__ __device__ __forceinline__ constexpr int mix_slot(int v) {
  return (v >= GXX && v <= GZZ) ? 3 * (v - GXX)
         : v == ALPHA          ? 18
         : (v >= BETAX && v <= BETAZ) ? 21 + 3 * (v - BETAX)
         : v == PHI            ? 30
                               : -1;
}

constexpr int MAX_LEVELS = CCZ4_MAX_LEVELS;

// One interpolated halo point of a refined mesh: the source indices of the
// 2x2x2 coarse corners, (z, y, x) with x fastest, the remainders
// r = rx | ry << 2 | rz << 4 that select the weights along each axis, and
// the point's index t in its patch's tile. The entries of a patch are
// contiguous (patch after patch).
struct InterpEntry {
  int src[8];
  int r;
  int t;
};

// Static geometry of an evolved Sommerfeld ghost cell: the index of its
// neighbour one cell inward along the normal of its face (-1: none), the
// factor (r / x_d) sign / dx of the normal derivative and 1 / r.
struct GhostGeo {
  long long sn;
  double geo, ir;
};

// Separable form of a patch's interpolations (the same values, rounded the
// same way): the distinct x-interpolations of the patch (value
// rx ? (1-w) q(s0) + w q(s1) : q(s0), w = rx/3), then the distinct
// y-interpolations of pairs of x results (packed: xa | xb << 14 | ry << 28,
// indices into the patch's x results), then one z-interpolation per
// interpolated tile point (packed: ya | yb << 14 | rz << 28, indices into
// the y results, and the tile point). A patch whose x and y results do not
// fit in its tile's shared memory has no jobs and is interpolated entry by
// entry.
struct XJob {
  int s0, s1, rx;
};
constexpr int JOB_BITS = 14;  // local indices < 2^14 > (18 + 6)^3
struct ZJob {
  int yab;  // ya | yb << 14 | rz << 28
  int t;
};

// The mixed path keeps the mixed derivatives it uses in FP32 -- those of
// g~ (slots 0..17) and beta (slots 21..29) -- as FP32 in the first 27 float
// slots of the mixed-derivative buffer: FP32 slot of slot s, or -1 for the
// FP64-only slots of alpha and phi.
__host__ __device__ __forceinline__ constexpr int mix_fslot(int s) {
  return s < 18 ? s : (s >= 21 && s < 30 ? s - 3 : -1);
}
constexpr int NMIXF = 27;

// Plain-data view of a grid, passed by value to every kernel.
struct GridView {
  int p, T;                    // points per patch edge; tile edge p + 2*HALO
  int np[3], N[3];             // patches and points per axis
  int n_patches;
  int bc;
  long long n_points;          // n_patches * p^3
  long long n_ghost;           // Sommerfeld ghost cells (0 otherwise)
  long long S;                 // field stride of state-shaped buffers
  long long T3;                // T^3
  double origin[3], dx;
  const int *ijk;              // [n_patches][3]
  const int *owner;            // [np2][np1][np0] -> patch id
  const int *gcoord;           // [n_ghost][3] global coordinates of the ghost cells
  const GhostGeo *ghost_geo;   // [n_ghost] their static geometry
  unsigned *status;            // device status word
  // refined meshes only (src == nullptr on a single level)
  int n_levels;
  long long n_leaf_points;     // points of patches without children
  const int *src;              // [n_patches][T3] tile sources: >= 0 index, <= -2 entry -(s+2)
  const InterpEntry *interp;   // interpolated tile points
  const int *ibeg;             // [n_patches + 1] first entry of each patch in interp
  const XJob *xjob;            // separable interpolation (see XJob): x jobs, patch after patch
  const int *yjob;             //   y jobs
  const ZJob *zjob;            //   z jobs, one per entry of interp
  const int *xbeg, *ybeg;      //   [n_patches + 1] first x / y job of each patch
  const int *plev;             // [n_patches] level of each patch
  const unsigned char *leaf;   // [n_patches] 1 if the patch has no children
  double ldx[MAX_LEVELS];      // spacing of each level (ldx[0] = dx)
  unsigned long long *queue;   // work counter of the queue launch of the stage kernel, or nullptr (flat)
  int stage_shape;             // launch shape of the flat stage kernel (CCZ4_STAGE_SHAPE_*)
  int fill_shape;              // launch shape of the halo fill (CCZ4_FILL_SHAPE_*)
};

// Level of patch n (0 on a single level).
__device__ __forceinline__ int patch_level(const GridView &g, int n) {
  return g.plev ? __ldg(g.plev + n) : 0;
}

__host__ __device__ __forceinline__ int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__host__ __device__ __forceinline__ int clampi(int a, int lo, int hi) {
  return a < lo ? lo : (a > hi ? hi : a);
}

// Rank of an outside cell (x, y, z) within the ghost shell of width HALO,
// cells counted in lexicographic (z, y, x) order. Closed form: whole planes
// (z outside) contribute Mx*My cells, planes with z inside contribute
// Mx*My - Nx*Ny; within a plane with z inside, rows with y outside
// contribute Mx cells and rows with y inside 2*HALO cells.
__host__ __device__ __forceinline__ long long ghost_rank(const GridView &g, int x, int y, int z) {
  const long long Mx = g.N[0] + 2 * HALO, My = g.N[1] + 2 * HALO;
  const int zz = z + HALO, yy = y + HALO, xx = x + HALO;
  const long long full_planes = (zz < HALO ? zz : HALO) + (zz > g.N[2] + HALO ? zz - (g.N[2] + HALO) : 0);
  const long long inner_planes = clampi(zz - HALO, 0, g.N[2]);
  long long r = full_planes * Mx * My + inner_planes * (Mx * My - (long long)g.N[0] * g.N[1]);
  if (z < 0 || z >= g.N[2]) return r + (long long)yy * Mx + xx;
  const long long full_rows = (yy < HALO ? yy : HALO) + (yy > g.N[1] + HALO ? yy - (g.N[1] + HALO) : 0);
  const long long inner_rows = clampi(yy - HALO, 0, g.N[1]);
  r += full_rows * Mx + inner_rows * (2 * HALO);
  if (y < 0 || y >= g.N[1]) return r + xx;
  return r + (x < 0 ? xx : HALO + (x - g.N[0]));
}

// Index, within a field of a state-shaped buffer, of the value at global
// point (x, y, z), which may lie up to HALO points outside the domain.
// Returns -1 if the point cannot be resolved (sets the bounds status bit).
__device__ __forceinline__ long long locate(const GridView &g, int x, int y, int z) {
  const bool inside = x >= 0 && x < g.N[0] && y >= 0 && y < g.N[1] && z >= 0 && z < g.N[2];
  if (!inside) {
    if (g.bc == CCZ4_BC_PERIODIC) {
      x = wrap(x, g.N[0]); y = wrap(y, g.N[1]); z = wrap(z, g.N[2]);
    } else if (g.bc == CCZ4_BC_COPY) {
      x = clampi(x, 0, g.N[0] - 1); y = clampi(y, 0, g.N[1] - 1); z = clampi(z, 0, g.N[2] - 1);
    } else {
      if (x < -HALO || x >= g.N[0] + HALO || y < -HALO || y >= g.N[1] + HALO ||
          z < -HALO || z >= g.N[2] + HALO) {
        atomicOr(g.status, STATUS_BOUNDS);
        return -1;
      }
      return g.n_points + ghost_rank(g, x, y, z);
    }
  }
  const int p = g.p;
  const int px = x / p, py = y / p, pz = z / p;
  const int n = __ldg(g.owner + ((long long)pz * g.np[1] + py) * g.np[0] + px);
  return (long long)n * p * p * p + ((long long)(z - pz * p) * p + (y - py * p)) * p + (x - px * p);
}

}  // namespace ccz4

// Host-side helpers implemented in ccz4_capi.cu.
namespace ccz4 {
void set_error(const char *fmt, ...);
}

struct ccz4_grid {
  ccz4::GridView v;
  int device;
  double *buf[8];            // U, Y0, Y1, ACC, RHS, INI, TILE, MIX
  long long buf_len[8];      // doubles
  int *d_ijk, *d_owner, *d_gcoord;
  unsigned *d_status;
  double *red_partial;       // per-block partial sums of the constraint reduction
  int red_blocks;
  double *red_out;           // device [5]
  double *host_out;          // pinned [5]
  cudaStream_t cap_stream;   // private stream for graph capture (created on first use)
  cudaGraphExec_t step_exec; // one captured RK4 step, or NULL
  ccz4_params step_P;        // parameters and dt baked into step_exec
  double step_dt;
  // refined meshes: tile sources, interpolation entries, levels, leaf flags
  // and, per level l >= 1, the parents on level l-1 with their 27 children
  int *d_src;
  ccz4::InterpEntry *d_interp;
  int *d_ibeg;
  ccz4::XJob *d_xjob;
  int *d_yjob;
  ccz4::ZJob *d_zjob;
  int *d_xbeg, *d_ybeg;
  int *d_plev;
  unsigned char *d_leaf;
  int *d_rpar[CCZ4_MAX_LEVELS], *d_rkid[CCZ4_MAX_LEVELS];
  int n_rpar[CCZ4_MAX_LEVELS];
  unsigned long long *d_queue;  // work counter of the queue launch (allocated on first use)
  ccz4::GhostGeo *d_ghost_geo;  // [n_ghost] static geometry of the Sommerfeld ghost cells
  ccz4_alloc_fn alloc;          // allocator of buf[] (NULL: cudaMalloc), kept for their release
  ccz4_dealloc_fn dealloc;
  void *alloc_ctx;
  int fused;                    // CCZ4_LAUNCH_FUSED: one cooperative launch per RK stage (p = 9)
};

// Kernel launchers (one translation unit each).
namespace ccz4 {
// Fills the static geometry of the Sommerfeld ghost cells (rhs.cu).
cudaError_t launch_ghost_setup(const GridView &g, GhostGeo *out, cudaStream_t s);
// fp32_weights: mixed derivatives with FP32 weights (for the mixed-precision stage kernel)
cudaError_t launch_fill_halos(const GridView &g, const double *src, double *tile, double *mix, cudaStream_t s,
                              bool fp32_weights = false);
cudaError_t prepare_fill_halos(int p);
// One cooperative launch per RK stage (rhs_fused.cu): the halo fill of every
// patch, a grid-wide barrier, the interior points and the Sommerfeld ghost
// cells; p = 9 only. prepare_fused raises its shared-memory limit (once per
// grid, outside any stream capture).
cudaError_t prepare_fused();
cudaError_t launch_fused_stage(const GridView &g, const ccz4_params &P, int stage, double dt, double *tile,
                               double *mix, const double *in, const double *ini, const double *U, double *acc,
                               double *out, cudaStream_t s);
// psi_4 at every interior point from the halo'd tiles: Re into out[0 .. n_points), Im into out[S ..),
// the tetrad centred at centre (psi4.cu)
cudaError_t launch_psi4(const GridView &g, const double *tile, const double centre[3], double *out, cudaStream_t s);
// number of mixed second derivatives kept per point (d_xy, d_xz, d_yz of g~, alpha, beta, phi)
constexpr int NMIX = 33;
// largest patch edge whose halo'd tile of one field fits in the fill kernel's shared memory
constexpr int MAX_P = 18;
cudaError_t launch_rhs(const GridView &g, const ccz4_params &P, const double *tile, const double *mix,
                       const double *in, const double *ini, double *out, cudaStream_t s);
cudaError_t launch_rk_stage(const GridView &g, const ccz4_params &P, int stage, double dt,
                            const double *tile, const double *mix, const double *in, const double *ini,
                            const double *U, double *acc, double *out, cudaStream_t s);
cudaError_t launch_enforce(const GridView &g, double *U, cudaStream_t s);
// restriction of level l onto the n_par parents par[] of level l-1 (children kid[n_par][27])
cudaError_t launch_restrict(const GridView &g, const int *par, const int *kid, int n_par, double *U,
                            cudaStream_t s);
cudaError_t launch_constraints(const GridView &g, const double *tile, double *H, double *M,
                               double *partial, int blocks, double *out5, cudaStream_t s);
}  // namespace ccz4
