// Puncture initial data on the GPU (include/ccz4_id.h): Bowen-York
// curvature and the Brill-Lindquist part of the conformal factor per cell,
// and the red-black nonlinear Gauss-Seidel solve of the Hamiltonian
// constraint for the regular correction u.
//
// A half-sweep updates the cells of one colour; their 7-point neighbours
// all have the other colour, so the update order within a colour does not
// matter and one thread per cell reproduces the serial sweep. The grid is
// small (96^3 cells are 7 MB per field) and stays in L2 across sweeps, so a
// sweep costs about two kernel launches; the solve replays a CUDA graph of
// `check` sweeps between residual checks.
//
// Nested boxes: a solver may take fixed ghost values from a coarser solver
// (its parent), interpolated once at its ghost-cell centres; a chain of
// boxes around the punctures then resolves u at the spacing of the finest
// box, each box's boundary data coming from the box around it.
#include <string.h>

#include "../../include/ccz4_id.h"
#include "ccz4_algebra.cuh"
#include "ccz4_internal.cuh"

struct ccz4_idsolver {
  int n;
  double L, h;
  double *u, *aa, *psi;
  double *partial;      // per-block maxima of the residual
  int blocks;
  double *dev_max;      // device [1]
  double *host_max;     // pinned [1]
  cudaStream_t cap;     // private stream for the graph capture
  cudaGraphExec_t exec; // `exec_check` sweeps, or NULL
  int exec_check;
  double omega;         // relaxation factor
  double *gwt;          // [n_shell][6] 1/r ghost weights of the boundary-shell cells
  double *gb;           // [6][n][n] fixed ghost values of a nested box, or NULL: the 1/r fall-off
};

namespace {

constexpr int ID_THREADS = 256;

struct PunctureSet {
  int n;
  double m[CCZ4_ID_MAX_PUNCTURES];
  double c[CCZ4_ID_MAX_PUNCTURES][3];
  double P[CCZ4_ID_MAX_PUNCTURES][3];
  double S[CCZ4_ID_MAX_PUNCTURES][3];
};

__device__ __forceinline__ double cell_coord(double L, double h, int i) { return -L + (i + 0.5) * h; }

// Index into the [6][n][n] fixed ghost values of the ghost at index o
// (-1 or n) along axis d of cell I: face 2 d (low side) or 2 d + 1, then the
// two other cell indices, the lower axis fastest.
__device__ __forceinline__ long long ghost_slot(int n, const int I[3], int d, int o) {
  const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
  return ((long long)(2 * d + (o >= n)) * n + I[b]) * n + I[a];
}

// 1/d for positive or negative normal d of moderate size: an FP32
// reciprocal (conversions by integer bit operations) refined by two
// Newton-Raphson steps r <- r + r (1 - d r) in FP64, i.e. four FMAs on the
// narrow FP64 pipe instead of a division; the result is within a few ulps.
__device__ __forceinline__ double recip(double d) {
  double r = ccz4::f2d_bits(__frcp_rn(ccz4::d2f_bits(d)));
  r = fma(r, fma(-d, r, 1.0), r);
  return fma(r, fma(-d, r, 1.0), r);
}

__global__ void __launch_bounds__(ID_THREADS) setup_kernel(int n, double L, double h, PunctureSet B,
                                                            double *aa, double *psi) {
  // n <= 1024: every cell index fits 32-bit arithmetic (no 64-bit division)
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n * n * n) return;
  const int i = c % n, j = (c / n) % n, k = c / (n * n);
  const double X[3] = {cell_coord(L, h, i), cell_coord(L, h, j), cell_coord(L, h, k)};
  double A[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  double s = 1.0;
  for (int p = 0; p < B.n; ++p) {
    double d[3], nv[3];
    for (int q = 0; q < 3; ++q) d[q] = X[q] - B.c[p][q];
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int q = 0; q < 3; ++q) nv[q] = d[q] / r;
    const double Pn = B.P[p][0] * nv[0] + B.P[p][1] * nv[1] + B.P[p][2] * nv[2];
    // w = S x n: the spin term is 3/r^3 (w_i n_j + w_j n_i)
    const double w[3] = {B.S[p][1] * nv[2] - B.S[p][2] * nv[1], B.S[p][2] * nv[0] - B.S[p][0] * nv[2],
                         B.S[p][0] * nv[1] - B.S[p][1] * nv[0]};
    const double cp = 1.5 / (r * r), cs = 3.0 / (r * r * r);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double dab = a == b ? 1.0 : 0.0;
        A[a][b] += cp * (B.P[p][a] * nv[b] + B.P[p][b] * nv[a] - (dab - nv[a] * nv[b]) * Pn) +
                   cs * (w[a] * nv[b] + w[b] * nv[a]);
      }
    s += B.m[p] / (2.0 * r);
  }
  double q = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) q += A[a][b] * A[a][b];
  aa[c] = q;
  psi[c] = s;
}

// Weight r_cell / r_ghost of the 1/r fall-off ghost at index o along axis d
// of the cell at X (radius rc).
__device__ __forceinline__ double ghost_weight(double L, double h, const double X[3], double rc, int d, int o) {
  double g[3] = {X[0], X[1], X[2]};
  g[d] = cell_coord(L, h, o);
  return rc / sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
}

// Laplacian neighbour sum of a cell on the boundary of the grid, where
// one or more neighbours are ghosts: fixed values (gb), else 1/r ghosts
// whose weights r_cell / r_ghost go to *ghost_w. Kept out of line so that the interior cells
// (94 % of a 96^3 grid) do not pay for its coordinates, roots and
// divisions.
__device__ __noinline__ double boundary_sum(int n, double L, double h, const double *u, const double *gb, int i,
                                            int j, int k, double uc, double *ghost_w) {
  const long long c = ((long long)k * n + j) * n + i;
  const int I[3] = {i, j, k};
  const long long st[3] = {1, n, (long long)n * n};
  const double X[3] = {cell_coord(L, h, i), cell_coord(L, h, j), cell_coord(L, h, k)};
  const double rc = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  double s = 0.0, gw = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int side = -1; side <= 1; side += 2) {
      const int o = I[d] + side;
      if (o >= 0 && o < n) {
        s += u[c + side * st[d]];
      } else if (gb) {
        s += gb[ghost_slot(n, I, d, o)];
      } else {
        const double w = ghost_weight(L, h, X, rc, d, o);
        s += uc * w;
        gw += w;
      }
    }
  *ghost_w = gw;
  return s;
}

// Laplacian neighbour sum of cell (i, j, k) with the 1/r ghosts; returns
// the sum and sets *ghost_w to the ghosts' weights (0 inside).
__device__ __forceinline__ double neighbour_sum(int n, double L, double h, const double *u, const double *gb, int i,
                                                int j, int k, double uc, double *ghost_w) {
  if (i > 0 && i < n - 1 && j > 0 && j < n - 1 && k > 0 && k < n - 1) {
    const long long c = ((long long)k * n + j) * n + i;
    const long long nn = (long long)n * n;
    *ghost_w = 0.0;
    return ((u[c - 1] + u[c + 1]) + (u[c - n] + u[c + n])) + (u[c - nn] + u[c + nn]);
  }
  return boundary_sum(n, L, h, u, gb, i, j, k, uc, ghost_w);
}

// Threads of one half-sweep: the interior cells of the colour first, then
// every cell of the boundary shell (those of the other colour return). The
// split keeps the boundary path off the warps of interior cells (with rows
// of n/2 cells of a colour nearly every warp would otherwise hold a
// boundary cell).
__host__ __device__ inline int sweep_interior_threads(int n) {
  const int m = n - 2;
  return m > 0 ? ((m + 1) / 2) * m * m : 0;
}
__host__ __device__ inline int shell_cells(int n) {
  const int m = n - 2 > 0 ? n - 2 : 0;
  return n * n * n - m * m * m;
}
__host__ __device__ inline int sweep_threads(int n) { return sweep_interior_threads(n) + shell_cells(n); }

// Cell (i, j, k) of boundary-shell index b < shell_cells(n): the planes
// k = 0 and k = n-1, then per interior k the rows j = 0 and j = n-1, then
// the cells i = 0 and i = n-1 of the interior rows.
__device__ __forceinline__ void shell_cell(int n, int b, int &i, int &j, int &k) {
  const int n2 = n * n, m = n - 2;
  if (b < 2 * n2) {
    k = b < n2 ? 0 : n - 1;
    j = (b % n2) / n;
    i = b % n;
    return;
  }
  const int per = 2 * n + 2 * m, b2 = b - 2 * n2;
  k = 1 + b2 / per;
  const int r = b2 % per;
  if (r < 2 * n) {
    j = r < n ? 0 : n - 1;
    i = r % n;
  } else {
    j = 1 + (r - 2 * n) / 2;
    i = ((r - 2 * n) & 1) ? n - 1 : 0;
  }
}

// Ghost weights of the shell cells, w[6 b + 2 d + (side > 0)] for the
// neighbour on axis d and side -1 / +1 (0 where that neighbour is a cell):
// they depend on the grid only, so the sweeps read them instead of taking
// roots and divisions.
__global__ void __launch_bounds__(ID_THREADS) ghost_table_kernel(int n, double L, double h, double *w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= shell_cells(n)) return;
  int i, j, k;
  shell_cell(n, b, i, j, k);
  const int I[3] = {i, j, k};
  const double X[3] = {cell_coord(L, h, i), cell_coord(L, h, j), cell_coord(L, h, k)};
  const double rc = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      const int o = I[d] + (side ? 1 : -1);
      w[6 * b + 2 * d + side] = (o >= 0 && o < n) ? 0.0 : ghost_weight(L, h, X, rc, d, o);
    }
}

// One half-sweep: the cells with i + j + k + color even take one Newton
// step of the discrete Hamiltonian constraint, over-relaxed by omega.
__global__ void __launch_bounds__(ID_THREADS) sweep_kernel(int n, double ih2, int color, double omega,
                                                            const double *__restrict__ aa,
                                                            const double *__restrict__ psi,
                                                            const double *__restrict__ gwt,
                                                            const double *__restrict__ gb, double *u) {
  // 32-bit index arithmetic (n <= 1024)
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_int = sweep_interior_threads(n);
  const long long nn = (long long)n * n;
  double uc, s, gw;
  long long c;
  if (q < n_int) {
    const int m = n - 2, half = (m + 1) / 2;
    const int i2 = q % half;
    const int j = (q / half) % m + 1;
    const int k = q / (half * m) + 1;
    const int i = 1 + 2 * i2 + ((1 + j + k + color) & 1);
    if (i >= n - 1) return;
    c = ((long long)k * n + j) * n + i;
    uc = u[c];
    s = ((u[c - 1] + u[c + 1]) + (u[c - n] + u[c + n])) + (u[c - nn] + u[c + nn]);
    gw = 0.0;
  } else {
    const int b = q - n_int;
    if (b >= shell_cells(n)) return;
    int i, j, k;
    shell_cell(n, b, i, j, k);
    if ((i + j + k + color) & 1) return;
    c = ((long long)k * n + j) * n + i;
    uc = u[c];
    // the same terms in the same order as boundary_sum, the ghost weights
    // from the table
    const int I[3] = {i, j, k};
    const long long st[3] = {1, n, nn};
    s = 0.0;
    gw = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int o = I[d] + (side ? 1 : -1);
        if (o >= 0 && o < n) {
          s += u[c + (side ? st[d] : -st[d])];
        } else if (gb) {  // a nested box: a fixed ghost, no derivative
          s += __ldg(gb + ghost_slot(n, I, d, o));
        } else {
          const double w = __ldg(gwt + 6 * b + 2 * d + side);
          s += uc * w;
          gw += w;
        }
      }
  }
  const double a = __ldg(aa + c);
  const double iq = recip(__ldg(psi + c) + uc);
  const double iq2 = iq * iq, iq4 = iq2 * iq2;
  const double F = (s - 6.0 * uc) * ih2 + 0.125 * a * (iq4 * iq2 * iq);
  const double dF = (gw - 6.0) * ih2 - 0.875 * a * (iq4 * iq4);
  u[c] = uc - omega * (F * recip(dF));
}

__global__ void __launch_bounds__(ID_THREADS) residual_kernel(int n, double L, double h, double ih2,
                                                               const double *__restrict__ aa,
                                                               const double *__restrict__ psi,
                                                               const double *__restrict__ u,
                                                               const double *__restrict__ gb, double *res,
                                                               double *partial) {
  __shared__ double sh[ID_THREADS];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < n * n * n) {
    const int i = c % n, j = (c / n) % n, k = c / (n * n);
    const double uc = u[c];
    double gw;
    const double s = neighbour_sum(n, L, h, u, gb, i, j, k, uc, &gw);
    const double iq = recip(psi[c] + uc);
    const double iq2 = iq * iq, iq4 = iq2 * iq2;
    const double F = (s - 6.0 * uc) * ih2 + 0.125 * aa[c] * (iq4 * iq2 * iq);
    if (res) res[c] = F;
    v = fabs(F);
    if (!(v == v)) v = INFINITY;  // a NaN residual never passes a tolerance
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = ID_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(ID_THREADS) max_kernel(const double *partial, int blocks, double *out) {
  __shared__ double sh[ID_THREADS];
  double v = 0.0;
  for (int b = threadIdx.x; b < blocks; b += ID_THREADS) v = fmax(v, partial[b]);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = ID_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Lagrange weights of the cubic through nodes 0..3 (unit spacing) at t.
__device__ __forceinline__ void cubic_w(double t, double w[4]) {
  const double t0 = t, t1 = t - 1.0, t2 = t - 2.0, t3 = t - 3.0;
  w[0] = -(t1 * t2 * t3) / 6.0;
  w[1] = (t0 * t2 * t3) / 2.0;
  w[2] = -(t0 * t1 * t3) / 2.0;
  w[3] = (t0 * t1 * t2) / 6.0;
}

__device__ __forceinline__ void cubic_stencil(int n, double L, double h, double x, int *k0, double *t) {
  const double s = (x + L) / h - 0.5;
  int k = (int)floor(s) - 1;
  k = k < 0 ? 0 : (k > n - 4 ? n - 4 : k);
  *k0 = k;
  *t = s - k;
}

// u of a solver grid at X by tricubic interpolation (see ccz4_id_assemble).
__device__ double interp_u(int n, double L, double h, const double *__restrict__ u, const double X[3]) {
  int k[3];
  double w[3][4];
  for (int d = 0; d < 3; ++d) {
    double t;
    cubic_stencil(n, L, h, X[d], &k[d], &t);
    cubic_w(t, w[d]);
  }
  double uz = 0.0;
  for (int c = 0; c < 4; ++c) {
    double uy = 0.0;
    for (int b = 0; b < 4; ++b) {
      const double *row = u + ((long long)(k[2] + c) * n + (k[1] + b)) * n + k[0];
      const double ux = w[0][0] * row[0] + w[0][1] * row[1] + w[0][2] * row[2] + w[0][3] * row[3];
      uy += w[1][b] * ux;
    }
    uz += w[2][c] * uy;
  }
  return uz;
}

// A nested box's fixed ghost values: the parent's u (np^3 cells of
// [-Lp, Lp]^3) at the centres of the box's ghost cells, in the [6][n][n]
// order of ghost_slot.
__global__ void __launch_bounds__(ID_THREADS) box_ghost_kernel(int n, double L, double h, int np, double Lp,
                                                                double hp, const double *__restrict__ up,
                                                                double *gb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 6 * n * n) return;
  const int f = q / (n * n), ib = (q / n) % n, ia = q % n;
  const int d = f / 2, a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
  int I[3];
  I[d] = (f & 1) ? n : -1;
  I[a] = ia;
  I[b] = ib;
  const double X[3] = {cell_coord(L, h, I[0]), cell_coord(L, h, I[1]), cell_coord(L, h, I[2])};
  gb[q] = interp_u(np, Lp, hp, up, X);
}

// A nested box's first guess: the parent's u at the box's cell centres.
__global__ void __launch_bounds__(ID_THREADS) box_cells_kernel(int n, double L, double h, int np, double Lp,
                                                                double hp, const double *__restrict__ up,
                                                                double *u) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n * n * n) return;
  const double X[3] = {cell_coord(L, h, c % n), cell_coord(L, h, (c / n) % n), cell_coord(L, h, c / (n * n))};
  u[c] = interp_u(np, Lp, hp, up, X);
}

// State of the data at one point (see ccz4_id_assemble); with lim > 0 only
// the points with every |X_d| < lim are written.
__global__ void __launch_bounds__(ID_THREADS) assemble_kernel(ccz4::GridView g, int n, double L, double h,
                                                               PunctureSet B, const double *__restrict__ u,
                                                               double lim, double *state) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.n_points + g.n_ghost) return;
  double X[3];
  if (e < g.n_points) {
    const int p = g.p;
    const long long p3 = (long long)p * p * p;
    const int pn = (int)e / (int)p3;  // state indices are below 2^31
    const int q = (int)(e - pn * p3);
    const int loc[3] = {q % p, (q / p) % p, q / (p * p)};
    const double dx = g.ldx[g.plev ? __ldg(g.plev + pn) : 0];
    for (int d = 0; d < 3; ++d) X[d] = g.origin[d] + ((double)__ldg(g.ijk + 3 * pn + d) * p + loc[d] + 0.5) * dx;
  } else {
    const long long id = e - g.n_points;
    for (int d = 0; d < 3; ++d) X[d] = g.origin[d] + (__ldg(g.gcoord + 3 * id + d) + 0.5) * g.dx;
  }
  if (lim > 0.0 && !(fabs(X[0]) < lim && fabs(X[1]) < lim && fabs(X[2]) < lim)) return;
  const double uz = interp_u(n, L, h, u, X);
  // curvature, Brill-Lindquist factor
  double A[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  double sbl = 0.0;
  for (int p = 0; p < B.n; ++p) {
    double dd[3], nv[3];
    for (int q = 0; q < 3; ++q) dd[q] = X[q] - B.c[p][q];
    const double r = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    for (int q = 0; q < 3; ++q) nv[q] = dd[q] / r;
    const double Pn = B.P[p][0] * nv[0] + B.P[p][1] * nv[1] + B.P[p][2] * nv[2];
    const double wv[3] = {B.S[p][1] * nv[2] - B.S[p][2] * nv[1], B.S[p][2] * nv[0] - B.S[p][0] * nv[2],
                          B.S[p][0] * nv[1] - B.S[p][1] * nv[0]};
    const double cp = 1.5 / (r * r), cs = 3.0 / (r * r * r);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double dab = a == b ? 1.0 : 0.0;
        A[a][b] += cp * (B.P[p][a] * nv[b] + B.P[p][b] * nv[a] - (dab - nv[a] * nv[b]) * Pn) +
                   cs * (wv[a] * nv[b] + wv[b] * nv[a]);
      }
    sbl += B.m[p] / (2.0 * r);
  }
  const double psi = 1.0 + sbl + uz;
  const double ip = 1.0 / psi, ip2 = ip * ip, ip6 = ip2 * ip2 * ip2;
  const long long S = g.S;
  for (int v = 0; v < ccz4::NV; ++v) state[v * S + e] = 0.0;
  state[ccz4::GXX * S + e] = 1.0;
  state[ccz4::GYY * S + e] = 1.0;
  state[ccz4::GZZ * S + e] = 1.0;
  state[ccz4::ALPHA * S + e] = 0.5 * ((1.0 - sbl) / (1.0 + sbl) + 1.0);
  state[ccz4::PHI * S + e] = ip2;
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int c = 0; c < 6; ++c) state[(ccz4::AXX + c) * S + e] = ip6 * A[ia[c]][ib[c]];
}

cudaError_t launch_sweeps(const ccz4_idsolver *s, int n_sweeps, cudaStream_t st) {
  const int n = s->n;
  const unsigned grid = (unsigned)((sweep_threads(n) + ID_THREADS - 1) / ID_THREADS);
  const double ih2 = 1.0 / (s->h * s->h);
  for (int k = 0; k < n_sweeps; ++k)
    for (int color = 0; color < 2; ++color) {
      sweep_kernel<<<grid, ID_THREADS, 0, st>>>(n, ih2, color, s->omega, s->aa, s->psi, s->gwt, s->gb, s->u);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace

using namespace ccz4;

#define ID_TRY(call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                           \
      return CCZ4_ERR_CUDA;                                                                \
    }                                                                                      \
  } while (0)

static void id_release(ccz4_idsolver *s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->cap) cudaStreamDestroy(s->cap);
  cudaFree(s->u);
  cudaFree(s->aa);
  cudaFree(s->psi);
  cudaFree(s->partial);
  cudaFree(s->dev_max);
  cudaFree(s->gwt);
  cudaFree(s->gb);
  cudaFreeHost(s->host_max);
  free(s);
}

extern "C" ccz4_status ccz4_id_create(int n, double L, ccz4_idsolver **out) {
  if (!out || n < 2 || n > 1024 || !(L > 0.0)) {
    set_error("id_create: need out, 2 <= n <= 1024 and L > 0 (n=%d L=%g)", n, L);
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  ccz4_idsolver *s = (ccz4_idsolver *)calloc(1, sizeof(ccz4_idsolver));
  if (!s) {
    set_error("host allocation failed");
    return CCZ4_ERR_NOMEM;
  }
  s->n = n;
  s->L = L;
  s->h = 2.0 * L / n;
  s->omega = 1.0;
  const size_t cells = (size_t)n * n * n;
  s->blocks = (int)((cells + ID_THREADS - 1) / ID_THREADS);
  bool ok = cudaMalloc(&s->u, sizeof(double) * cells) == cudaSuccess &&
            cudaMalloc(&s->aa, sizeof(double) * cells) == cudaSuccess &&
            cudaMalloc(&s->psi, sizeof(double) * cells) == cudaSuccess &&
            cudaMalloc(&s->partial, sizeof(double) * (size_t)s->blocks) == cudaSuccess &&
            cudaMalloc(&s->dev_max, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->gwt, sizeof(double) * 6 * (size_t)shell_cells(n)) == cudaSuccess &&
            cudaMallocHost(&s->host_max, sizeof(double)) == cudaSuccess;
  if (!ok) {
    set_error("id_create: device allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
    id_release(s);
    return CCZ4_ERR_NOMEM;
  }
  cudaMemset(s->u, 0, sizeof(double) * cells);
  cudaMemset(s->aa, 0, sizeof(double) * cells);
  cudaMemset(s->psi, 0, sizeof(double) * cells);
  ghost_table_kernel<<<(shell_cells(n) + ID_THREADS - 1) / ID_THREADS, ID_THREADS>>>(n, L, s->h, s->gwt);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("id_create: %s", cudaGetErrorString(e));
    id_release(s);
    return CCZ4_ERR_CUDA;
  }
  *out = s;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_free(ccz4_idsolver *s) {
  if (!s) return CCZ4_OK;
  cudaDeviceSynchronize();
  id_release(s);
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_set_punctures(ccz4_idsolver *s, const ccz4_punctures *B, void *stream) {
  if (!s || !B || B->n < 1 || B->n > CCZ4_ID_MAX_PUNCTURES) {
    set_error("id_set_punctures: need a solver and 1..%d punctures", CCZ4_ID_MAX_PUNCTURES);
    return CCZ4_ERR_INVALID;
  }
  PunctureSet P;
  memset(&P, 0, sizeof(P));
  P.n = B->n;
  for (int p = 0; p < B->n; ++p) {
    P.m[p] = B->m[p];
    for (int d = 0; d < 3; ++d) {
      P.c[p][d] = B->c[p][d];
      P.P[p][d] = B->P[p][d];
      P.S[p][d] = B->S[p][d];
    }
  }
  const long long cells = (long long)s->n * s->n * s->n;
  setup_kernel<<<(unsigned)((cells + ID_THREADS - 1) / ID_THREADS), ID_THREADS, 0, (cudaStream_t)stream>>>(
      s->n, s->L, s->h, P, s->aa, s->psi);
  ID_TRY(cudaGetLastError());
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_u_ptr(ccz4_idsolver *s, double **dev_u) {
  if (!s || !dev_u) {
    set_error("id_u_ptr: NULL argument");
    return CCZ4_ERR_INVALID;
  }
  *dev_u = s->u;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_set_relaxation(ccz4_idsolver *s, double omega) {
  if (!s || !(omega > 0.0 && omega < 2.0)) {
    set_error("id_set_relaxation: need a solver and 0 < omega < 2");
    return CCZ4_ERR_INVALID;
  }
  if (omega != s->omega && s->exec) {
    cudaGraphExecDestroy(s->exec);  // the captured sweeps carry the old factor
    s->exec = nullptr;
  }
  s->omega = omega;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_sweeps(ccz4_idsolver *s, int n_sweeps, void *stream) {
  if (!s || n_sweeps < 0) {
    set_error("id_sweeps: need a solver and n_sweeps >= 0");
    return CCZ4_ERR_INVALID;
  }
  ID_TRY(launch_sweeps(s, n_sweeps, (cudaStream_t)stream));
  return CCZ4_OK;
}

static ccz4_status residual(ccz4_idsolver *s, double *max_res, double *res_dev, cudaStream_t st) {
  const double ih2 = 1.0 / (s->h * s->h);
  residual_kernel<<<s->blocks, ID_THREADS, 0, st>>>(s->n, s->L, s->h, ih2, s->aa, s->psi, s->u, s->gb, res_dev,
                                                     s->partial);
  ID_TRY(cudaGetLastError());
  max_kernel<<<1, ID_THREADS, 0, st>>>(s->partial, s->blocks, s->dev_max);
  ID_TRY(cudaGetLastError());
  ID_TRY(cudaMemcpyAsync(s->host_max, s->dev_max, sizeof(double), cudaMemcpyDeviceToHost, st));
  ID_TRY(cudaStreamSynchronize(st));
  *max_res = *s->host_max;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_residual(ccz4_idsolver *s, double *max_res, double *res_dev, void *stream) {
  if (!s || !max_res) {
    set_error("id_residual: NULL argument");
    return CCZ4_ERR_INVALID;
  }
  return residual(s, max_res, res_dev, (cudaStream_t)stream);
}

static ccz4_status capture_sweeps(ccz4_idsolver *s, int check) {
  if (s->exec) {
    cudaGraphExecDestroy(s->exec);
    s->exec = nullptr;
  }
  if (!s->cap) ID_TRY(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  ID_TRY(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_sweeps(s, check, s->cap);
  cudaError_t e2 = cudaStreamEndCapture(s->cap, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    set_error("id_solve: sweep capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return CCZ4_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&s->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    s->exec = nullptr;
    set_error("id_solve: graph instantiation failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  s->exec_check = check;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_solve(ccz4_idsolver *s, double tol, int max_sweeps, int check, int *sweeps,
                                     double *final_res, void *stream) {
  if (!s || !(tol > 0.0) || max_sweeps < 0 || check < 1) {
    set_error("id_solve: need a solver, tol > 0, max_sweeps >= 0 and check >= 1");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!s->exec || s->exec_check != check) {
    ID_TRY(cudaStreamSynchronize(st));
    ccz4_status r = capture_sweeps(s, check);
    if (r != CCZ4_OK) return r;
  }
  double res = 0.0;
  ccz4_status r = residual(s, &res, nullptr, st);
  if (r != CCZ4_OK) return r;
  int done = 0;
  while (!(res < tol) && done < max_sweeps) {
    ID_TRY(cudaGraphLaunch(s->exec, st));
    done += check;
    r = residual(s, &res, nullptr, st);
    if (r != CCZ4_OK) return r;
  }
  if (sweeps) *sweeps = res < tol ? done : -1;
  if (final_res) *final_res = res;
  return CCZ4_OK;
}

static ccz4_status assemble(ccz4_idsolver *s, const ccz4_punctures *B, ccz4_grid *g, int buf, double lim,
                           void *stream, const char *who) {
  if (!s || !B || !g || B->n < 1 || B->n > CCZ4_ID_MAX_PUNCTURES || s->n < 4 || buf < CCZ4_BUF_U ||
      buf > CCZ4_BUF_INI || !g->buf[buf]) {
    set_error("%s: need a solver (n >= 4), 1..%d punctures, a grid and one of its state buffers", who,
              CCZ4_ID_MAX_PUNCTURES);
    return CCZ4_ERR_INVALID;
  }
  PunctureSet P;
  memset(&P, 0, sizeof(P));
  P.n = B->n;
  for (int p = 0; p < B->n; ++p) {
    P.m[p] = B->m[p];
    for (int d = 0; d < 3; ++d) {
      P.c[p][d] = B->c[p][d];
      P.P[p][d] = B->P[p][d];
      P.S[p][d] = B->S[p][d];
    }
  }
  const long long total = g->v.n_points + g->v.n_ghost;
  if (total == 0) return CCZ4_OK;
  assemble_kernel<<<(unsigned)((total + ID_THREADS - 1) / ID_THREADS), ID_THREADS, 0, (cudaStream_t)stream>>>(
      g->v, s->n, s->L, s->h, P, s->u, lim, g->buf[buf]);
  ID_TRY(cudaGetLastError());
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_id_assemble(ccz4_idsolver *s, const ccz4_punctures *B, ccz4_grid *g, int buf,
                                        void *stream) {
  return assemble(s, B, g, buf, 0.0, stream, "id_assemble");
}

extern "C" ccz4_status ccz4_id_assemble_box(ccz4_idsolver *s, const ccz4_punctures *B, ccz4_grid *g, int buf,
                                            void *stream) {
  if (!s) {
    set_error("id_assemble_box: NULL solver");
    return CCZ4_ERR_INVALID;
  }
  return assemble(s, B, g, buf, s->L - 1.5 * s->h, stream, "id_assemble_box");
}

extern "C" ccz4_status ccz4_id_set_parent(ccz4_idsolver *s, const ccz4_idsolver *parent, int init_u,
                                          void *stream) {
  if (!s || s == parent) {
    set_error("id_set_parent: need a solver other than the parent");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (s->exec) {  // the captured sweeps carry the old boundary rule
    ID_TRY(cudaStreamSynchronize(st));
    cudaGraphExecDestroy(s->exec);
    s->exec = nullptr;
  }
  const int n = s->n;
  if (!parent) {
    if (s->gb) {
      ID_TRY(cudaStreamSynchronize(st));
      cudaFree(s->gb);
      s->gb = nullptr;
    }
    return CCZ4_OK;
  }
  if (parent->n < 4 || !(s->L + 0.5 * s->h <= parent->L)) {
    set_error("id_set_parent: the box [-%g, %g]^3 and its ghost cells must lie inside the parent's [-%g, %g]^3 "
              "(parent n >= 4)", s->L, s->L, parent->L, parent->L);
    return CCZ4_ERR_INVALID;
  }
  if (!s->gb && cudaMalloc(&s->gb, sizeof(double) * 6 * (size_t)n * n) != cudaSuccess) {
    s->gb = nullptr;
    set_error("id_set_parent: device allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
    return CCZ4_ERR_NOMEM;
  }
  box_ghost_kernel<<<(6 * n * n + ID_THREADS - 1) / ID_THREADS, ID_THREADS, 0, st>>>(
      n, s->L, s->h, parent->n, parent->L, parent->h, parent->u, s->gb);
  ID_TRY(cudaGetLastError());
  if (init_u) {
    box_cells_kernel<<<s->blocks, ID_THREADS, 0, st>>>(n, s->L, s->h, parent->n, parent->L, parent->h, parent->u,
                                                        s->u);
    ID_TRY(cudaGetLastError());
  }
  return CCZ4_OK;
}
