// Constraint monitors (Eqs. hamilton_constraints and momentum_constraints)
// with a deterministic two-stage reduction, and the standalone algebraic
// enforcement kernel.
//
// The Ricci tensor of the monitor is the modified Ricci tensor of Eq.
// NR_foccz4_modified_ricci with Z = 0: Gamma-hat replaced by the contracted
// Christoffel symbol G~^k of the metric, whose derivative is taken through
// the closing relations (d_k g~^ij = -2 D_k^ij and the derivative of the
// Christoffel symbols), i.e. from first and second derivatives of g~.
#include "ccz4_algebra.cuh"

namespace ccz4 {
namespace {

constexpr int RED_THREADS = 256;

__device__ void constraints_point(const Nbhd &N, const StencilCoef<double> &C, double &H, double M[3]) {
  double g[6], A[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    g[c] = N.at(GXX + c, 0);
    A[c] = N.at(AXX + c, 0);
  }
  const double ph = N.at(PHI, 0), Kt = N.at(KTR, 0);
  double dg[3][6], dA[3][6], dP[3], dK[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dg[k][c] = fd1<double>(N, GXX + c, s, C.c1);
      dA[k][c] = fd1<double>(N, AXX + c, s, C.c1);
    }
    dP[k] = fd1<double>(N, PHI, s, C.c1);
    dK[k] = fd1<double>(N, KTR, s, C.c1);
  }
  double ig[6];
  ig[0] = g[3] * g[5] - g[4] * g[4];
  ig[1] = g[2] * g[4] - g[1] * g[5];
  ig[2] = g[1] * g[4] - g[2] * g[3];
  ig[3] = g[0] * g[5] - g[2] * g[2];
  ig[4] = g[1] * g[2] - g[0] * g[4];
  ig[5] = g[0] * g[3] - g[1] * g[1];
  const double idet = 1.0 / (g[0] * ig[0] + g[1] * ig[1] + g[2] * ig[2]);
#pragma unroll
  for (int c = 0; c < 6; ++c) ig[c] *= idet;
  const double w6[6] = {1.0, 2.0, 2.0, 1.0, 2.0, 1.0};
  double Gd[3][6], Gu[3][6], Gc[3], Gl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        Gd[k][S6(i, j)] = 0.5 * (dg[i][S6(j, k)] + dg[j][S6(i, k)] - dg[k][S6(i, j)]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      Gu[k][c] = ig[S6(k, 0)] * Gd[0][c] + ig[S6(k, 1)] * Gd[1][c] + ig[S6(k, 2)] * Gd[2][c];
    double s = 0.0, t = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      s = fma(w6[c] * ig[c], Gu[k][c], s);
      t = fma(w6[c] * ig[c], Gd[k][c], t);
    }
    Gc[k] = s;  // G~^k
    Gl[k] = t;  // G~_k = g~^ml G~_kml
  }
  // second derivatives of g~: dd[c][kl]
  double dd[6][6];
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) dd[c][S6(k, l)] = fdkl<double>(N, GXX + c, k, l, C);
  // dIg[j][ml] = g~^ma g~^lb d_j g~_ab  (= -d_j g~^ml)
  double dIg[3][6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double t[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        t[m][b] = ig[S6(m, 0)] * dg[j][S6(0, b)] + ig[S6(m, 1)] * dg[j][S6(1, b)] + ig[S6(m, 2)] * dg[j][S6(2, b)];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int l = m; l < 3; ++l)
        dIg[j][S6(m, l)] = t[m][0] * ig[S6(0, l)] + t[m][1] * ig[S6(1, l)] + t[m][2] * ig[S6(2, l)];
  }
  // d_j G~_n = -dIg[j]:G~_n.. + g~^ml (d_j d_m g~_ln - 1/2 d_j d_n g~_ml)
  // d_j G~^k = -dIg[j][kn] G~_n + g~^kn d_j G~_n
  double dGt[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double dGl[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 6; ++c) s = fma(-w6[c] * dIg[j][c], Gd[n][c], s);
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          s = fma(ig[S6(m, l)], dd[S6(l, n)][S6(j, m)] - 0.5 * dd[S6(m, l)][S6(j, n)], s);
      dGl[n] = s;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
#pragma unroll
      for (int n = 0; n < 3; ++n) s += -dIg[j][S6(k, n)] * Gl[n] + ig[S6(k, n)] * dGl[n];
      dGt[j][k] = s;
    }
  }
  const double iph = 1.0 / ph;
  double Pu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) Pu[k] = ig[S6(k, 0)] * dP[0] + ig[S6(k, 1)] * dP[1] + ig[S6(k, 2)] * dP[2];
  const double PP = Pu[0] * dP[0] + Pu[1] * dP[1] + Pu[2] * dP[2];
  double cdph[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      cdph[c] = fdkl<double>(N, PHI, i, j, C) - (Gu[0][c] * dP[0] + Gu[1][c] * dP[1] + Gu[2][c] * dP[2]);
    }
  double trcdph = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) trcdph = fma(w6[c] * ig[c], cdph[c], trcdph);
  double Cm[3][3][3], Em[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Cm[k][i][m] = ig[S6(0, m)] * Gu[k][S6(0, i)] + ig[S6(1, m)] * Gu[k][S6(1, i)] + ig[S6(2, m)] * Gu[k][S6(2, i)];
        Em[k][i][m] = ig[S6(0, m)] * Gd[k][S6(0, i)] + ig[S6(1, m)] * Gd[k][S6(1, i)] + ig[S6(2, m)] * Gd[k][S6(2, i)];
      }
  double R = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      double lap = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) lap = fma(w6[q] * ig[q], dd[c][q], lap);
      double t = -0.5 * lap;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        t += 0.5 * (g[S6(k, i)] * dGt[j][k] + g[S6(k, j)] * dGt[i][k] + Gc[k] * dg[k][c]);
      double x1 = 0.0, x2 = 0.0, q3 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          x1 = fma(Cm[k][i][m], Gd[j][S6(k, m)], x1);
          x2 = fma(Cm[k][j][m], Gd[i][S6(k, m)], x2);
          q3 = fma(Gu[k][S6(i, m)], Em[k][j][m], q3);
        }
      t += x1 + x2 + q3 + iph * (cdph[c] + g[c] * trcdph) - 2.0 * iph * iph * g[c] * PP;
      R = fma(w6[c] * ig[c], t, R);
    }
  R *= ph * ph;
  double Am[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m)
      Am[i][m] = A[S6(i, 0)] * ig[S6(0, m)] + A[S6(i, 1)] * ig[S6(1, m)] + A[S6(i, 2)] * ig[S6(2, m)];
  double AA = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m) AA = fma(Am[i][m], Am[m][i], AA);
  H = R + (2.0 / 3.0) * Kt * Kt - AA;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) s = fma(ig[S6(k, l)], dA[k][S6(l, i)], s);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
      for (int l = 0; l < 3; ++l) s = fma(-Gu[m][S6(l, i)], Am[m][l], s);
      s = fma(-Gc[m], A[S6(i, m)], s);
      s = fma(-3.0 * iph * A[S6(i, m)], Pu[m], s);
    }
    M[i] = s - (2.0 / 3.0) * dK[i];
  }
}

struct ConsCoef {
  StencilCoef<double> C[MAX_LEVELS];
};

__global__ void __launch_bounds__(RED_THREADS) constraints_kernel(GridView g, ConsCoef LC,
                                                                  const double *__restrict__ tile,
                                                                  double *H, double *M, double *partial) {
  __shared__ double sh[5][RED_THREADS];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < g.n_points) {
    const int p = g.p, T = g.T;
    const int p3 = p * p * p;  // 32-bit division: every state index is below 2^31
    const int n = (int)i / p3;
    const int r = (int)i - n * p3;
    const int z = r / (p * p), y = (r / p) % p, x = r % p;
    Nbhd N;
    N.c = tile + n * g.T3 + ((long long)(z + HALO) * T + (y + HALO)) * T + (x + HALO);
    N.fs = (long long)g.n_patches * g.T3;
    N.st[0] = 1;
    N.st[1] = T;
    N.st[2] = T * T;
    N.mix = nullptr;
    N.ms = 0;
    N.mixf = nullptr;
    N.msf = 0;
    double h, m[3];
    constraints_point(N, LC.C[patch_level(g, n)], h, m);
    if (H) H[i] = h;
    if (M) {
      M[i] = m[0];
      M[g.n_points + i] = m[1];
      M[2 * g.n_points + i] = m[2];
    }
    const double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    // the norms count leaf patches only (a covered point is not counted twice)
    const bool counted = !g.leaf || __ldg(g.leaf + n);
    if (counted && isfinite(h) && isfinite(m2)) {
      v[0] = h * h;
      v[1] = m2;
      v[2] = fabs(h);
      v[3] = sqrt(m2);
    } else if (counted) {
      v[4] = 1.0;
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
      sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

// One block folds the per-block partials in a fixed order.
__global__ void __launch_bounds__(RED_THREADS) reduce_partials(const double *partial, int blocks,
                                                               double n_points, double *out) {
  __shared__ double sh[5][RED_THREADS];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += RED_THREADS) {
    v[0] += partial[b * 5 + 0];
    v[1] += partial[b * 5 + 1];
    v[2] = fmax(v[2], partial[b * 5 + 2]);
    v[3] = fmax(v[3], partial[b * 5 + 3]);
    v[4] += partial[b * 5 + 4];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
      sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(sh[0][0] / n_points);
    out[1] = sqrt(sh[1][0] / n_points);
    out[2] = sh[2][0];
    out[3] = sh[3][0];
    out[4] = sh[4][0];
  }
}

// Centres and radius of the regions left out of the constraint norms.
struct Excl {
  int n;
  double c[CCZ4_MAX_EXCLUDED][3];
  double r2;
};

// Per-block partial sums of H^2 and |M|^2, maxima of |H| and |M| and the
// count over the interior points of leaf patches outside every ball.
__global__ void __launch_bounds__(RED_THREADS) excluded_kernel(GridView g, Excl E, const double *__restrict__ H,
                                                               const double *__restrict__ M, double *partial) {
  __shared__ double sh[5][RED_THREADS];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (i < g.n_points) {
    const int p = g.p;
    const int p3 = p * p * p;
    const int n = (int)i / p3;
    const int r = (int)i - n * p3;
    const int z = r / (p * p), y = (r / p) % p, x = r % p;
    const double h = g.ldx[patch_level(g, n)];
    const double pos[3] = {g.origin[0] + (__ldg(g.ijk + 3 * n) * p + x + 0.5) * h,
                           g.origin[1] + (__ldg(g.ijk + 3 * n + 1) * p + y + 0.5) * h,
                           g.origin[2] + (__ldg(g.ijk + 3 * n + 2) * p + z + 0.5) * h};
    bool near = false;
    for (int c = 0; c < E.n; ++c) {
      const double d0 = pos[0] - E.c[c][0], d1 = pos[1] - E.c[c][1], d2 = pos[2] - E.c[c][2];
      near = near || d0 * d0 + d1 * d1 + d2 * d2 < E.r2;
    }
    const bool counted = (!g.leaf || __ldg(g.leaf + n)) && !near;
    const double hv = H[i];
    const double m2 = M[i] * M[i] + M[g.n_points + i] * M[g.n_points + i] + M[2 * g.n_points + i] * M[2 * g.n_points + i];
    if (counted && isfinite(hv) && isfinite(m2)) {
      v[0] = hv * hv;
      v[1] = m2;
      v[2] = fabs(hv);
      v[3] = sqrt(m2);
      v[4] = 1.0;
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
      sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

// Folds the partials in a fixed order; the norms divide by the point count.
__global__ void __launch_bounds__(RED_THREADS) reduce_excluded(const double *partial, int blocks, double *out) {
  __shared__ double sh[5][RED_THREADS];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += RED_THREADS) {
    v[0] += partial[b * 5 + 0];
    v[1] += partial[b * 5 + 1];
    v[2] = fmax(v[2], partial[b * 5 + 2]);
    v[3] = fmax(v[3], partial[b * 5 + 3]);
    v[4] += partial[b * 5 + 4];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
      sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cnt = sh[4][0];
    out[0] = cnt > 0.0 ? sqrt(sh[0][0] / cnt) : 0.0;
    out[1] = cnt > 0.0 ? sqrt(sh[1][0] / cnt) : 0.0;
    out[2] = sh[2][0];
    out[3] = sh[3][0];
    out[4] = cnt;
  }
}

__global__ void __launch_bounds__(256) enforce_kernel(GridView g, double *U) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_points) return;
  double gm[6], A[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    gm[c] = U[(GXX + c) * g.S + i];
    A[c] = U[(AXX + c) * g.S + i];
  }
  enforce_point<double>(gm, A);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    U[(GXX + c) * g.S + i] = gm[c];
    U[(AXX + c) * g.S + i] = A[c];
  }
}

}  // namespace

int constraint_blocks(long long n_points) { return (int)((n_points + RED_THREADS - 1) / RED_THREADS); }

cudaError_t launch_constraints(const GridView &g, const double *tile, double *H, double *M, double *partial,
                               int blocks, double *out5, cudaStream_t s) {
  ConsCoef LC;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    const double dx = g.ldx[l];
    LC.C[l].c1 = 1.0 / (12.0 * dx);
    LC.C[l].c2 = 1.0 / (12.0 * dx * dx);
    LC.C[l].c3 = 1.0 / (144.0 * dx * dx);
    LC.C[l].cko = 0.0;
  }
  if (blocks > 0) {
    constraints_kernel<<<blocks, RED_THREADS, 0, s>>>(g, LC, tile, H, M, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  reduce_partials<<<1, RED_THREADS, 0, s>>>(partial, blocks, (double)g.n_leaf_points, out5);
  return cudaGetLastError();
}

cudaError_t launch_constraints_excluded(const GridView &g, const double *H, const double *M, int n_centres,
                                        const double *centres, double radius, double *partial, int blocks,
                                        double *out5, cudaStream_t s) {
  Excl E;
  E.n = n_centres;
  for (int c = 0; c < n_centres; ++c)
    for (int d = 0; d < 3; ++d) E.c[c][d] = centres[3 * c + d];
  E.r2 = radius * radius;
  if (blocks > 0) {
    excluded_kernel<<<blocks, RED_THREADS, 0, s>>>(g, E, H, M, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  reduce_excluded<<<1, RED_THREADS, 0, s>>>(partial, blocks, out5);
  return cudaGetLastError();
}

cudaError_t launch_enforce(const GridView &g, double *U, cudaStream_t s) {
  if (g.n_points == 0) return cudaSuccess;
  enforce_kernel<<<(unsigned)((g.n_points + 255) / 256), 256, 0, s>>>(g, U);
  return cudaGetLastError();
}

}  // namespace ccz4
