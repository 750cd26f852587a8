/*
 * Bowen-York puncture initial data (oracle; see bowen_york.h for the
 * equations and the discretisation). Plain loops, FP64, no FMA contraction.
 */
#include "bowen_york.h"

#include <math.h>
#include <stdlib.h>

static const int SY[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

/* Levi-Civita symbol */
static double eps3(int i, int j, int k) {
  if (i == j || j == k || i == k) return 0.0;
  return ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1)) ? 1.0
                                                                                                         : -1.0;
}

void og_by_abar(const og_punctures *B, double x, double y, double z, double A[6]) {
  double M[3][3] = {{0.0}};
  for (int p = 0; p < B->n; ++p) {
    double d[3] = {x - B->c[p][0], y - B->c[p][1], z - B->c[p][2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double nv[3] = {d[0] / r, d[1] / r, d[2] / r};
    double Pn = B->P[p][0] * nv[0] + B->P[p][1] * nv[1] + B->P[p][2] * nv[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double dij = i == j ? 1.0 : 0.0;
        /* momentum part */
        double a = 3.0 / (2.0 * r * r) *
                   (B->P[p][i] * nv[j] + B->P[p][j] * nv[i] - (dij - nv[i] * nv[j]) * Pn);
        /* spin part: eps_kil S_l n_k n_j + eps_kjl S_l n_k n_i */
        double s = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            s += eps3(k, i, l) * B->S[p][l] * nv[k] * nv[j] + eps3(k, j, l) * B->S[p][l] * nv[k] * nv[i];
        M[i][j] += a + 3.0 / (r * r * r) * s;
      }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) A[SY[i][j]] = M[i][j];
}

double og_by_aa(const og_punctures *B, double x, double y, double z) {
  double A[6];
  og_by_abar(B, x, y, z, A);
  double s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += A[SY[i][j]] * A[SY[i][j]];
  return s;
}

double og_by_psi_bl(const og_punctures *B, double x, double y, double z) {
  double s = 1.0;
  for (int p = 0; p < B->n; ++p) {
    double d[3] = {x - B->c[p][0], y - B->c[p][1], z - B->c[p][2]};
    s += B->m[p] / (2.0 * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  }
  return s;
}

void og_by_points(const og_punctures *B, long m, const double *x, const double *y, const double *z, double *A,
                  double *aa, double *psi) {
  for (long q = 0; q < m; ++q) {
    if (A) og_by_abar(B, x[q], y[q], z[q], A + 6 * q);
    if (aa) aa[q] = og_by_aa(B, x[q], y[q], z[q]);
    if (psi) psi[q] = og_by_psi_bl(B, x[q], y[q], z[q]);
  }
}

typedef struct {
  int n;
  double L, h;
  double *aa, *psi; /* per cell: Abar.Abar and psi_BL */
  const double *gb; /* fixed ghost values [6][n][n] (a nested box), or NULL: the 1/r fall-off */
} grid_t;

static double coord(const grid_t *g, int i) { return -g->L + (i + 0.5) * g->h; }

static void grid_init(grid_t *g, const og_punctures *B, int n, double L) {
  g->n = n;
  g->L = L;
  g->h = 2.0 * L / n;
  g->gb = NULL;
  long N = (long)n * n * n;
  g->aa = (double *)malloc(sizeof(double) * (size_t)N);
  g->psi = (double *)malloc(sizeof(double) * (size_t)N);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = ((long)k * n + j) * n + i;
        double x = coord(g, i), y = coord(g, j), z = coord(g, k);
        g->aa[c] = og_by_aa(B, x, y, z);
        g->psi[c] = og_by_psi_bl(B, x, y, z);
      }
}

static void grid_free(grid_t *g) {
  free(g->aa);
  free(g->psi);
}

/* Index into a [6][n][n] ghost array of the ghost cell (i, j, k), one cell
   outside the grid along one axis d: face 2 d (low side) or 2 d + 1 (high
   side), then the two other cell indices, the lower axis fastest. */
static long ghost_index(int n, int i, int j, int k) {
  int I[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) {
    if (I[d] < 0 || I[d] >= n) {
      int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
      return ((long)(2 * d + (I[d] >= n)) * n + I[b]) * n + I[a];
    }
  }
  return -1;
}

/* u at cell (i, j, k), which may be one ghost cell outside along one axis:
   the given ghost value of a nested box, else the 1/r fall-off rule
   u_ghost = u_cell * r_cell / r_ghost. */
static double u_at(const grid_t *g, const double *u, int i, int j, int k) {
  int n = g->n;
  int ci = i < 0 ? 0 : (i >= n ? n - 1 : i);
  int cj = j < 0 ? 0 : (j >= n ? n - 1 : j);
  int ck = k < 0 ? 0 : (k >= n ? n - 1 : k);
  double v = u[((long)ck * n + cj) * n + ci];
  if (ci == i && cj == j && ck == k) return v;
  if (g->gb) return g->gb[ghost_index(n, i, j, k)];
  double xc = coord(g, ci), yc = coord(g, cj), zc = coord(g, ck);
  double xg = coord(g, i), yg = coord(g, j), zg = coord(g, k);
  double rc = sqrt(xc * xc + yc * yc + zc * zc), rg = sqrt(xg * xg + yg * yg + zg * zg);
  return v * rc / rg;
}

static double laplacian(const grid_t *g, const double *u, int i, int j, int k) {
  double s = u_at(g, u, i - 1, j, k) + u_at(g, u, i + 1, j, k) + u_at(g, u, i, j - 1, k) +
             u_at(g, u, i, j + 1, k) + u_at(g, u, i, j, k - 1) + u_at(g, u, i, j, k + 1);
  return (s - 6.0 * u_at(g, u, i, j, k)) / (g->h * g->h);
}

double og_by_residual(const og_punctures *B, int n, double L, const double *u, double *res) {
  return og_by_residual_box(B, n, L, u, NULL, res);
}

double og_by_residual_box(const og_punctures *B, int n, double L, const double *u, const double *gb,
                          double *res) {
  grid_t g;
  grid_init(&g, B, n, L);
  g.gb = gb;
  double mx = 0.0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = ((long)k * n + j) * n + i;
        double F = laplacian(&g, u, i, j, k) + 0.125 * g.aa[c] * pow(g.psi[c] + u[c], -7.0);
        if (res) res[c] = F;
        if (fabs(F) > mx) mx = fabs(F);
      }
  grid_free(&g);
  return mx;
}

static void sweeps(const grid_t *g, double *u, int n_sweeps, double omega) {
  int n = g->n;
  double ih2 = 1.0 / (g->h * g->h);
  for (int s = 0; s < n_sweeps; ++s)
    for (int color = 0; color < 2; ++color)
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            if (((i + j + k) & 1) != color) continue;
            long c = ((long)k * n + j) * n + i;
            double q = g->psi[c] + u[c];
            double F = laplacian(g, u, i, j, k) + 0.125 * g->aa[c] * pow(q, -7.0);
            /* derivative of F with respect to u at this cell (the fall-off
               ghosts of a boundary cell depend on it too: r_cell / r_ghost
               each; fixed ghosts do not) */
            double diag = -6.0;
            int idx[3] = {i, j, k};
            for (int d = 0; d < 3 && !g->gb; ++d) {
              for (int side = -1; side <= 1; side += 2) {
                int o[3] = {i, j, k};
                o[d] += side;
                if (o[d] < 0 || o[d] >= n) {
                  double xc = coord(g, idx[0]), yc = coord(g, idx[1]), zc = coord(g, idx[2]);
                  double xg = coord(g, o[0]), yg = coord(g, o[1]), zg = coord(g, o[2]);
                  diag += sqrt(xc * xc + yc * yc + zc * zc) / sqrt(xg * xg + yg * yg + zg * zg);
                }
              }
            }
            double dF = diag * ih2 - 0.875 * g->aa[c] * pow(q, -8.0);
            u[c] = u[c] - omega * (F / dF);
          }
}

void og_by_sweeps(const og_punctures *B, int n, double L, double *u, int n_sweeps, double omega) {
  og_by_sweeps_box(B, n, L, u, NULL, n_sweeps, omega);
}

void og_by_sweeps_box(const og_punctures *B, int n, double L, double *u, const double *gb, int n_sweeps,
                      double omega) {
  grid_t g;
  grid_init(&g, B, n, L);
  g.gb = gb;
  sweeps(&g, u, n_sweeps, omega);
  grid_free(&g);
}

int og_by_solve(const og_punctures *B, int n, double L, double *u, double tol, int max_sweeps, int check,
                double omega, double *final_res) {
  return og_by_solve_box(B, n, L, u, NULL, tol, max_sweeps, check, omega, final_res);
}

int og_by_solve_box(const og_punctures *B, int n, double L, double *u, const double *gb, double tol,
                    int max_sweeps, int check, double omega, double *final_res) {
  grid_t g;
  grid_init(&g, B, n, L);
  g.gb = gb;
  if (check < 1) check = 1;
  int done = 0;
  double r = og_by_residual_box(B, n, L, u, gb, NULL);
  while (r >= tol && done < max_sweeps) {
    sweeps(&g, u, check, omega);
    done += check;
    r = og_by_residual_box(B, n, L, u, gb, NULL);
  }
  grid_free(&g);
  if (final_res) *final_res = r;
  return r < tol ? done : -1;
}

/* Lagrange weights of the cubic through nodes k0..k0+3 (unit spacing) at
   offset t from node k0. */
static void cubic_weights(double t, double w[4]) {
  for (int a = 0; a < 4; ++a) {
    double num = 1.0, den = 1.0;
    for (int b = 0; b < 4; ++b) {
      if (b == a) continue;
      num *= t - b;
      den *= (double)(a - b);
    }
    w[a] = num / den;
  }
}

/* first stencil node and offset of coordinate x on n cells of [-L, L] */
static void stencil(int n, double L, double x, int *k0, double *t) {
  double h = 2.0 * L / n;
  double s = (x + L) / h - 0.5; /* position in cell-centre units */
  int k = (int)floor(s) - 1;
  if (k < 0) k = 0;
  if (k > n - 4) k = n - 4;
  *k0 = k;
  *t = s - k;
}

void og_by_interp(int n, double L, const double *u, long m, const double *x, const double *y, const double *z,
                  double *out) {
  for (long q = 0; q < m; ++q) {
    int kx, ky, kz;
    double tx, ty, tz, wx[4], wy[4], wz[4];
    stencil(n, L, x[q], &kx, &tx);
    stencil(n, L, y[q], &ky, &ty);
    stencil(n, L, z[q], &kz, &tz);
    cubic_weights(tx, wx);
    cubic_weights(ty, wy);
    cubic_weights(tz, wz);
    double sz = 0.0;
    for (int c = 0; c < 4; ++c) {
      double sy = 0.0;
      for (int b = 0; b < 4; ++b) {
        double sx = 0.0;
        for (int a = 0; a < 4; ++a) sx += wx[a] * u[((long)(kz + c) * n + (ky + b)) * n + (kx + a)];
        sy += wy[b] * sx;
      }
      sz += wz[c] * sy;
    }
    out[q] = sz;
  }
}

void og_by_state(const og_punctures *B, int n, double L, const double *u, long m, const double *x,
                 const double *y, const double *z, double *Q) {
  enum { NV = 25, GXX = 0, GYY = 3, GZZ = 5, ALPHA = 6, PHI = 10, AXX = 11 };
  double *uu = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  og_by_interp(n, L, u, m, x, y, z, uu);
  for (long q = 0; q < m; ++q) {
    for (int v = 0; v < NV; ++v) Q[(long)v * m + q] = 0.0;
    double A[6];
    og_by_abar(B, x[q], y[q], z[q], A);
    double psi = og_by_psi_bl(B, x[q], y[q], z[q]) + uu[q];
    double s = og_by_psi_bl(B, x[q], y[q], z[q]) - 1.0;
    Q[(long)GXX * m + q] = 1.0;
    Q[(long)GYY * m + q] = 1.0;
    Q[(long)GZZ * m + q] = 1.0;
    Q[(long)ALPHA * m + q] = 0.5 * ((1.0 - s) / (1.0 + s) + 1.0);
    Q[(long)PHI * m + q] = 1.0 / (psi * psi);
    double p6 = pow(psi, -6.0);
    for (int c = 0; c < 6; ++c) Q[(long)(AXX + c) * m + q] = p6 * A[c];
  }
  free(uu);
}

void og_by_box_ghosts(int n, double L, int np, double Lp, const double *up, double *gb) {
  double h = 2.0 * L / n;
  long m = 6L * n * n;
  double *x = (double *)malloc(sizeof(double) * (size_t)m);
  double *y = (double *)malloc(sizeof(double) * (size_t)m);
  double *z = (double *)malloc(sizeof(double) * (size_t)m);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side)
      for (int ib = 0; ib < n; ++ib)
        for (int ia = 0; ia < n; ++ia) {
          /* the ghost cell: index -1 or n along d, (ia, ib) along the two other axes */
          int I[3];
          int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
          I[d] = side ? n : -1;
          I[a] = ia;
          I[b] = ib;
          long q = ((long)(2 * d + side) * n + ib) * n + ia;
          x[q] = -L + (I[0] + 0.5) * h;
          y[q] = -L + (I[1] + 0.5) * h;
          z[q] = -L + (I[2] + 0.5) * h;
        }
  og_by_interp(np, Lp, up, m, x, y, z, gb);
  free(x);
  free(y);
  free(z);
}

void og_by_cells_from(int n, double L, int np, double Lp, const double *up, double *u) {
  double h = 2.0 * L / n;
  long m = (long)n * n * n;
  double *x = (double *)malloc(sizeof(double) * (size_t)m);
  double *y = (double *)malloc(sizeof(double) * (size_t)m);
  double *z = (double *)malloc(sizeof(double) * (size_t)m);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = ((long)k * n + j) * n + i;
        x[c] = -L + (i + 0.5) * h;
        y[c] = -L + (j + 0.5) * h;
        z[c] = -L + (k + 0.5) * h;
      }
  og_by_interp(np, Lp, up, m, x, y, z, u);
  free(x);
  free(y);
  free(z);
}
