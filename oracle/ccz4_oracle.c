/*
 * CCZ4 oracle: plain, slow, FP64 CPU restatement of the fourth-order
 * finite-difference (FD4) CCZ4 method of the ExaGRyPE paper
 * (arXiv 2406.11626).
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
 * CPU-baseline leg of bench.py are its only users. It shares no code with the
 * CUDA path. Build with -O2 -ffp-contract=off (no FMA contraction), so that
 * every operation below is one correctly rounded IEEE double operation.
 *
 * What it computes, step by step, with the passage each step follows:
 *   - patch grid and halo of width K = 3 (Sec. "Spatial Discretisation":
 *     p^3 patches with K halo layers, cell-centred sample points);
 *   - halo fill: periodic wrap (Sec. "Gauge Wave": periodic domain), Neumann
 *     copy filled layer by layer outward (Sec. "Boundary Treatment"), and
 *     Sommerfeld ghost cells that are evolved in time (Eqs.
 *     SommerfeldBC_v1 and exa_sommerfeld_inter);
 *   - FD4 first derivatives (Eq. exa_fd4_central_difference), FD4 second
 *     derivatives (pure: the five-point fourth-order stencil; mixed: the
 *     tensor product of two first-derivative stencils, Sec. "Finite
 *     Differences" speaks of a tensor-product approach) and Kreiss-Oliger
 *     dissipation of order N = 3 summed over the three directions
 *     (Eq. exa_fd4_ko);
 *   - the second-order CCZ4 right-hand side: the nine primary evolution
 *     equations of the appendix "Spacetime foliation" with the red terms
 *     removed, closed by the listed relations and the modified Ricci tensor
 *     of Eq. NR_foccz4_modified_ricci;
 *   - classic RK4 time stepping (Sec. "Finite Differences": Runge-Kutta up to
 *     order four) and the algebraic constraint enforcement after each step
 *     (Sec. "Evolution equations": det g~ = 1 by rescaling, tr A~ = 0 by
 *     trace removal);
 *   - the Hamiltonian and momentum constraints (Eqs. hamilton_constraints and
 *     momentum_constraints), with the Ricci tensor through the Riemann
 *     relation of the appendix, and their L2 norm (Sec. "Gauge Wave").
 * Readings of the paper where it is silent or ambiguous are listed in the
 * header comments of the functions that take them.
 */
#include "ccz4_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum {
  GXX, GXY, GXZ, GYY, GYZ, GZZ, ALPHA, BETAX, BETAY, BETAZ, PHI,
  AXX, AXY, AXZ, AYY, AYZ, AZZ, KTR, THETA, GHX, GHY, GHZ, BBX, BBY, BBZ
};

/* index of the symmetric pair (i, j) in the six stored components */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

struct og_grid {
  int p, T;           /* points per patch edge; tile edge p + 2K */
  int np[3], N[3];    /* patches and points per axis */
  int n_patches, bc;
  int *ijk;           /* [n][3] patch coordinates */
  int *owner;         /* [np2][np1][np0] -> patch id */
  double origin[3], dx;
  long n_ghost;
  int *gcoord;        /* [n_ghost][3] global coordinates (x, y, z) */
  long *gid;          /* dense map over [-K, N+K)^3 -> ghost id, or -1 */
  int Mx[3];          /* N + 2K */
  /* static mesh refinement (appendix "refinement transition"): level 0 is
     the grid above; each level l >= 1 holds complete sets of 3x3x3 children
     of level l-1 patches, with spacing dx / 3^l */
  int n_levels;
  int *lev;                      /* [n] level of each patch */
  int *nchild;                   /* [n] children of each patch (0 or 27) */
  double dxl[OG_MAX_LEVELS];     /* spacing of each level */
  int llo[OG_MAX_LEVELS][3];     /* levels >= 1: bounding box of the patch slots */
  int lext[OG_MAX_LEVELS][3];
  int *lowner[OG_MAX_LEVELS];    /* levels >= 1: dense bounding box -> patch id, or -1 */
};

/* ------------------------------------------------------------------------ */
/* grid                                                                     */
/* ------------------------------------------------------------------------ */

/* Builds the grid of level 0 (patches with level[n] == 0, or all of them
   when level is NULL) and, for a refined mesh, the levels above it. */
static og_grid *grid_build(int p, int np0, int np1, int np2, int n_patches, const int *level,
                           const int *ijk, double ox, double oy, double oz, double dx, int bc) {
  if (p < 1 || np0 < 1 || np1 < 1 || np2 < 1 || !(dx > 0.0) || n_patches < 1 || ijk == NULL) return NULL;
  if (bc != OG_BC_PERIODIC && bc != OG_BC_COPY && bc != OG_BC_SOMMERFELD) return NULL;
  og_grid *g = (og_grid *)calloc(1, sizeof(og_grid));
  g->p = p;
  g->T = p + 2 * OG_HALO;
  g->np[0] = np0; g->np[1] = np1; g->np[2] = np2;
  for (int d = 0; d < 3; ++d) {
    g->N[d] = g->np[d] * p;
    g->Mx[d] = g->N[d] + 2 * OG_HALO;
  }
  g->n_patches = n_patches;
  g->bc = bc;
  g->origin[0] = ox; g->origin[1] = oy; g->origin[2] = oz;
  g->dx = dx;
  g->ijk = (int *)malloc(sizeof(int) * 3 * (size_t)n_patches);
  memcpy(g->ijk, ijk, sizeof(int) * 3 * (size_t)n_patches);
  g->lev = (int *)calloc((size_t)n_patches, sizeof(int));
  g->nchild = (int *)calloc((size_t)n_patches, sizeof(int));
  g->n_levels = 1;
  if (level) {
    for (int n = 0; n < n_patches; ++n) {
      if (level[n] < 0 || level[n] >= OG_MAX_LEVELS) { og_grid_free(g); return NULL; }
      g->lev[n] = level[n];
      if (level[n] + 1 > g->n_levels) g->n_levels = level[n] + 1;
    }
  }
  for (int l = 0; l < g->n_levels; ++l) g->dxl[l] = l == 0 ? dx : g->dxl[l - 1] / 3.0;
  /* level 0 covers every slot exactly once */
  long n0 = (long)np0 * np1 * np2, count0 = 0;
  g->owner = (int *)malloc(sizeof(int) * (size_t)n0);
  for (long i = 0; i < n0; ++i) g->owner[i] = -1;
  for (int n = 0; n < n_patches; ++n) {
    if (g->lev[n] != 0) continue;
    int a = ijk[3 * n], b = ijk[3 * n + 1], c = ijk[3 * n + 2];
    if (a < 0 || a >= np0 || b < 0 || b >= np1 || c < 0 || c >= np2) { og_grid_free(g); return NULL; }
    long cell = ((long)c * np1 + b) * np0 + a;
    if (g->owner[cell] != -1) { og_grid_free(g); return NULL; }
    g->owner[cell] = n;
    ++count0;
  }
  if (count0 != n0) { og_grid_free(g); return NULL; }
  /* levels >= 1: slot maps over their bounding boxes */
  for (int l = 1; l < g->n_levels; ++l) {
    int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1}, any = 0;
    for (int n = 0; n < n_patches; ++n) {
      if (g->lev[n] != l) continue;
      for (int d = 0; d < 3; ++d) {
        int v = ijk[3 * n + d];
        if (!any || v < lo[d]) lo[d] = v;
        if (!any || v > hi[d]) hi[d] = v;
      }
      any = 1;
    }
    if (!any) { og_grid_free(g); return NULL; }
    long size = 1;
    for (int d = 0; d < 3; ++d) {
      g->llo[l][d] = lo[d];
      g->lext[l][d] = hi[d] - lo[d] + 1;
      size *= g->lext[l][d];
    }
    g->lowner[l] = (int *)malloc(sizeof(int) * (size_t)size);
    for (long i = 0; i < size; ++i) g->lowner[l][i] = -1;
    for (int n = 0; n < n_patches; ++n) {
      if (g->lev[n] != l) continue;
      long k = 0;
      for (int d = 2; d >= 0; --d) k = k * g->lext[l][d] + (ijk[3 * n + d] - lo[d]);
      if (g->lowner[l][k] != -1) { og_grid_free(g); return NULL; }
      g->lowner[l][k] = n;
    }
  }
  /* every refined patch is the child of a patch one level down, and a
     parent has either no children or all 27 */
  for (int n = 0; n < n_patches; ++n) {
    int l = g->lev[n];
    if (l == 0) continue;
    int a = ijk[3 * n] / 3, b = ijk[3 * n + 1] / 3, c = ijk[3 * n + 2] / 3;
    int par = -1;
    for (int m = 0; m < n_patches; ++m)
      if (g->lev[m] == l - 1 && ijk[3 * m] == a && ijk[3 * m + 1] == b && ijk[3 * m + 2] == c) par = m;
    if (par < 0 || ijk[3 * n] < 0 || ijk[3 * n + 1] < 0 || ijk[3 * n + 2] < 0) { og_grid_free(g); return NULL; }
    g->nchild[par] += 1;
  }
  for (int n = 0; n < n_patches; ++n)
    if (g->nchild[n] != 0 && g->nchild[n] != 27) { og_grid_free(g); return NULL; }
  /* ghost shell (level 0): every cell within K of the domain and outside
     it, enumerated in lexicographic (z, y, x) order */
  long total = (long)g->Mx[0] * g->Mx[1] * g->Mx[2];
  g->gid = (long *)malloc(sizeof(long) * (size_t)total);
  long count = 0;
  for (int z = -OG_HALO; z < g->N[2] + OG_HALO; ++z)
    for (int y = -OG_HALO; y < g->N[1] + OG_HALO; ++y)
      for (int x = -OG_HALO; x < g->N[0] + OG_HALO; ++x) {
        long k = ((long)(z + OG_HALO) * g->Mx[1] + (y + OG_HALO)) * g->Mx[0] + (x + OG_HALO);
        int inside = x >= 0 && x < g->N[0] && y >= 0 && y < g->N[1] && z >= 0 && z < g->N[2];
        g->gid[k] = (bc == OG_BC_SOMMERFELD && !inside) ? count++ : -1;
      }
  g->n_ghost = count;
  g->gcoord = (int *)malloc(sizeof(int) * 3 * (size_t)(count > 0 ? count : 1));
  for (int z = -OG_HALO; z < g->N[2] + OG_HALO; ++z)
    for (int y = -OG_HALO; y < g->N[1] + OG_HALO; ++y)
      for (int x = -OG_HALO; x < g->N[0] + OG_HALO; ++x) {
        long k = ((long)(z + OG_HALO) * g->Mx[1] + (y + OG_HALO)) * g->Mx[0] + (x + OG_HALO);
        long id = g->gid[k];
        if (id >= 0) { g->gcoord[3 * id] = x; g->gcoord[3 * id + 1] = y; g->gcoord[3 * id + 2] = z; }
      }
  return g;
}

static int check_nesting(const og_grid *g);

og_grid *og_grid_new(int p, int np0, int np1, int np2, int n_patches, const int *ijk,
                     double ox, double oy, double oz, double dx, int bc) {
  if ((long)n_patches != (long)np0 * np1 * np2) return NULL;
  return grid_build(p, np0, np1, np2, n_patches, NULL, ijk, ox, oy, oz, dx, bc);
}

og_grid *og_mesh_new(int p, int np0, int np1, int np2, int n_patches, const int *level,
                     const int *ijk, double ox, double oy, double oz, double dx, int bc) {
  og_grid *g = grid_build(p, np0, np1, np2, n_patches, level, ijk, ox, oy, oz, dx, bc);
  if (g && check_nesting(g)) {
    og_grid_free(g);
    return NULL;
  }
  return g;
}

int og_n_levels(const og_grid *g) { return g->n_levels; }

void og_grid_free(og_grid *g) {
  if (!g) return;
  for (int l = 0; l < OG_MAX_LEVELS; ++l) free(g->lowner[l]);
  free(g->ijk); free(g->owner); free(g->gid); free(g->gcoord); free(g->lev); free(g->nchild); free(g);
}

long og_n_ghost(const og_grid *g) { return g->n_ghost; }

void og_ghost_coords(const og_grid *g, int *out) {
  memcpy(out, g->gcoord, sizeof(int) * 3 * (size_t)g->n_ghost);
}

static long n_interior(const og_grid *g) { return (long)g->n_patches * g->p * g->p * g->p; }

/* Where the value at global point (x, y, z) lives. Returns 0 for an interior
   point (linear index into U), 1 for a ghost-shell point (index into G).
   Periodic: wrap. Copy: the paper fills the K ghost layers outward one at a
   time with Q_out = Q_in, so every ghost layer equals the last interior
   layer; with that rule applied face by face, edge and corner ghosts equal
   the nearest interior point, i.e. the clamped coordinate. Sommerfeld: the
   ghost cell itself (its value is evolved state). */
static int locate(const og_grid *g, int x, int y, int z, long *idx) {
  int c[3] = {x, y, z};
  int inside = 1;
  for (int d = 0; d < 3; ++d) if (c[d] < 0 || c[d] >= g->N[d]) inside = 0;
  if (!inside) {
    if (g->bc == OG_BC_PERIODIC) {
      for (int d = 0; d < 3; ++d) c[d] = ((c[d] % g->N[d]) + g->N[d]) % g->N[d];
    } else if (g->bc == OG_BC_COPY) {
      for (int d = 0; d < 3; ++d) c[d] = c[d] < 0 ? 0 : (c[d] >= g->N[d] ? g->N[d] - 1 : c[d]);
    } else {
      long k = ((long)(z + OG_HALO) * g->Mx[1] + (y + OG_HALO)) * g->Mx[0] + (x + OG_HALO);
      *idx = g->gid[k];
      return 1;
    }
  }
  int pa = c[0] / g->p, pb = c[1] / g->p, pc = c[2] / g->p;
  int lx = c[0] % g->p, ly = c[1] % g->p, lz = c[2] % g->p;
  int n = g->owner[((long)pc * g->np[1] + pb) * g->np[0] + pa];
  *idx = (long)n * g->p * g->p * g->p + ((long)lz * g->p + ly) * g->p + lx;
  return 0;
}

/* Patch of level l >= 1 holding global level-l point (x, y, z), or -1. */
static int level_owner(const og_grid *g, int l, int x, int y, int z) {
  int c[3] = {x, y, z};
  long k = 0;
  for (int d = 2; d >= 0; --d) {
    if (c[d] < 0) return -1;
    int s = c[d] / g->p - g->llo[l][d];
    if (s < 0 || s >= g->lext[l][d]) return -1;
    k = k * g->lext[l][d] + s;
  }
  return g->lowner[l][k];
}

/* locate() on level l: 0 interior point, 1 ghost-shell point (level 0), 2
   not covered by level l (the value comes from level l-1). */
static int locate_l(const og_grid *g, int l, int x, int y, int z, long *idx) {
  if (l == 0) return locate(g, x, y, z, idx);
  int n = level_owner(g, l, x, y, z);
  if (n < 0) return 2;
  int p = g->p;
  int lx = x - g->ijk[3 * n] * p, ly = y - g->ijk[3 * n + 1] * p, lz = z - g->ijk[3 * n + 2] * p;
  *idx = (long)n * p * p * p + ((long)lz * p + ly) * p + lx;
  return 0;
}

/* Whether level l holds (x, y, z) as an interior point of one of its
   patches (for level 0: inside the domain, no boundary rule applied). */
static int level_has(const og_grid *g, int l, int x, int y, int z, long *idx) {
  if (l == 0 && (x < 0 || x >= g->N[0] || y < 0 || y >= g->N[1] || z < 0 || z >= g->N[2])) return 0;
  return locate_l(g, l, x, y, z, idx) == 0;
}

/* Interior value of level l at (x, y, z); NaN where level l has no patch. */
static double level_value(const og_grid *g, const double *U, int v, int l, int x, int y, int z) {
  long idx;
  if (!level_has(g, l, x, y, z, &idx)) return NAN;
  return U[(long)v * n_interior(g) + idx];
}

/* Coarse-to-fine interpolation (appendix "refinement transition"): the
   tensor product of three one-dimensional linear maps between cell centres,
   applied along x, then y, then z. Fine cell i of level l has its centre at
   coarse coordinate (i - 1)/3 of level l-1 (coarse centres at the integers),
   so it lies between coarse cells c = floor((i-1)/3) and c+1, at remainder
   r = i - 1 - 3c, with weights PW[r]: the rows (1), (2/3, 1/3) and
   (1/3, 2/3) of the printed matrices P^par and P^perp. A weight of one
   takes the single coarse value. */
static const double PW[3][2] = {{1.0, 0.0}, {2.0 / 3.0, 1.0 / 3.0}, {1.0 / 3.0, 2.0 / 3.0}};

static void coarse_cell(int i, int *c, int *r) {
  int q = i - 1;
  int f = q >= 0 ? q / 3 : -((2 - q) / 3);
  *c = f;
  *r = q - 3 * f;
}

static double interpolate(const og_grid *g, const double *U, int v, int l, int x, int y, int z) {
  int c0[3], r[3];
  coarse_cell(x, &c0[0], &r[0]);
  coarse_cell(y, &c0[1], &r[1]);
  coarse_cell(z, &c0[2], &r[2]);
  int nb = r[1] ? 2 : 1, nc = r[2] ? 2 : 1;
  double t[2][2], s[2];
  for (int c = 0; c < nc; ++c)
    for (int b = 0; b < nb; ++b) {
      double q0 = level_value(g, U, v, l - 1, c0[0], c0[1] + b, c0[2] + c);
      if (r[0]) {
        double q1 = level_value(g, U, v, l - 1, c0[0] + 1, c0[1] + b, c0[2] + c);
        t[c][b] = PW[r[0]][0] * q0 + PW[r[0]][1] * q1;
      } else {
        t[c][b] = q0;
      }
    }
  for (int c = 0; c < nc; ++c) s[c] = r[1] ? PW[r[1]][0] * t[c][0] + PW[r[1]][1] * t[c][1] : t[c][0];
  return r[2] ? PW[r[2]][0] * s[0] + PW[r[2]][1] * s[1] : s[0];
}

static double value_at_l(const og_grid *g, const double *U, const double *G, int v, int l, int x, int y,
                         int z) {
  long idx;
  int k = locate_l(g, l, x, y, z, &idx);
  if (k == 0) return U[(long)v * n_interior(g) + idx];
  if (k == 1) return G[(long)v * g->n_ghost + idx];
  return interpolate(g, U, v, l, x, y, z);
}

static double value_at(const og_grid *g, const double *U, const double *G, int v, int x, int y, int z) {
  return value_at_l(g, U, G, v, 0, x, y, z);
}

/* Every tile point that a refined level does not cover must interpolate
   from interior points of the level below (proper nesting). Returns 1 if
   some point cannot. */
static int check_nesting(const og_grid *g) {
  int T = g->T, p = g->p;
  for (int n = 0; n < g->n_patches; ++n) {
    int l = g->lev[n];
    if (l == 0) continue;
    int bx = g->ijk[3 * n] * p, by = g->ijk[3 * n + 1] * p, bz = g->ijk[3 * n + 2] * p;
    for (int lz = 0; lz < T; ++lz)
      for (int ly = 0; ly < T; ++ly)
        for (int lx = 0; lx < T; ++lx) {
          int x = bx + lx - OG_HALO, y = by + ly - OG_HALO, z = bz + lz - OG_HALO;
          long idx;
          if (locate_l(g, l, x, y, z, &idx) != 2) continue;
          int c0[3], r[3];
          coarse_cell(x, &c0[0], &r[0]);
          coarse_cell(y, &c0[1], &r[1]);
          coarse_cell(z, &c0[2], &r[2]);
          for (int c = 0; c <= (r[2] ? 1 : 0); ++c)
            for (int b = 0; b <= (r[1] ? 1 : 0); ++b)
              for (int a = 0; a <= (r[0] ? 1 : 0); ++a)
                if (!level_has(g, l - 1, c0[0] + a, c0[1] + b, c0[2] + c, &idx)) return 1;
        }
  }
  return 0;
}

/* Halo'd tile of patch n in the oracle's working layout: point-major, the
   25 fields of a point contiguous. */
static void build_tile(const og_grid *g, int n, const double *U, const double *G, double *tile) {
  int T = g->T, p = g->p, l = g->lev[n];
  int bx = g->ijk[3 * n] * p, by = g->ijk[3 * n + 1] * p, bz = g->ijk[3 * n + 2] * p;
  for (int lz = 0; lz < T; ++lz)
    for (int ly = 0; ly < T; ++ly)
      for (int lx = 0; lx < T; ++lx) {
        long t = ((long)lz * T + ly) * T + lx;
        for (int v = 0; v < OG_NV; ++v)
          tile[t * OG_NV + v] =
              value_at_l(g, U, G, v, l, bx + lx - OG_HALO, by + ly - OG_HALO, bz + lz - OG_HALO);
      }
}

int og_fill_tiles(const og_grid *g, const double *U, const double *G, double *tiles) {
  int T = g->T;
  long T3 = (long)T * T * T;
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * OG_NV);
  for (int n = 0; n < g->n_patches; ++n) {
    build_tile(g, n, U, G, tile);
    for (int v = 0; v < OG_NV; ++v)
      for (long t = 0; t < T3; ++t)
        tiles[((long)v * g->n_patches + n) * T3 + t] = tile[t * OG_NV + v];
  }
  free(tile);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* FD4 stencils (Eqs. exa_fd4_central_difference and exa_fd4_ko)            */
/* ------------------------------------------------------------------------ */

/* weights of the first-derivative stencil at offsets -2, -1, +1, +2 (times
   1/(12 dx)): 8 (Q+ - Q-) - (Q++ - Q--) */
static const int OFF4[4] = {-2, -1, 1, 2};
static const double W1[4] = {1.0, -8.0, 8.0, -1.0};

typedef struct {
  const double *tile;
  long c;          /* centre point in the tile */
  long st[3];      /* strides of x, y, z in points */
} tview;

static double tq(const tview *tv, long off, int v) { return tv->tile[(tv->c + off) * OG_NV + v]; }

static double fd1(const tview *tv, int v, int k, double dx) {
  long s = tv->st[k];
  return (8.0 * (tq(tv, s, v) - tq(tv, -s, v)) - (tq(tv, 2 * s, v) - tq(tv, -2 * s, v))) / (12.0 * dx);
}

/* pure second derivative: the five-point fourth-order stencil
   (-Q++ + 16 Q+ - 30 Q + 16 Q- - Q--) / (12 dx^2) */
static double fd2pure(const tview *tv, int v, int k, double dx) {
  long s = tv->st[k];
  return (-tq(tv, 2 * s, v) + 16.0 * tq(tv, s, v) - 30.0 * tq(tv, 0, v) + 16.0 * tq(tv, -s, v) -
          tq(tv, -2 * s, v)) / (12.0 * dx * dx);
}

/* mixed second derivative: first-derivative stencil along k applied to the
   first-derivative stencil along l */
static double fd2mixed(const tview *tv, int v, int k, int l, double dx) {
  double acc = 0.0;
  for (int a = 0; a < 4; ++a) {
    double inner = 0.0;
    for (int b = 0; b < 4; ++b) inner += W1[b] * tq(tv, OFF4[a] * tv->st[k] + OFF4[b] * tv->st[l], v);
    acc += W1[a] * inner;
  }
  return acc / (144.0 * dx * dx);
}

/* Kreiss-Oliger dissipation of order N = 3, summed over the three directions:
   eps/(64 dx) (Q--- - 6 Q-- + 15 Q- - 20 Q + 15 Q+ - 6 Q++ + Q+++) */
static double ko_sum(const tview *tv, int v, double eps, double dx) {
  double acc = 0.0;
  for (int k = 0; k < 3; ++k) {
    long s = tv->st[k];
    double d = tq(tv, -3 * s, v) - 6.0 * tq(tv, -2 * s, v) + 15.0 * tq(tv, -s, v) - 20.0 * tq(tv, 0, v) +
               15.0 * tq(tv, s, v) - 6.0 * tq(tv, 2 * s, v) + tq(tv, 3 * s, v);
    acc += eps / (64.0 * dx) * d;
  }
  return acc;
}

static void point_derivs(const tview *tv, double dx, double d1[OG_NV][3], double d2[OG_NV][3][3]) {
  for (int v = 0; v < OG_NV; ++v) {
    for (int k = 0; k < 3; ++k) d1[v][k] = fd1(tv, v, k, dx);
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l)
        d2[v][k][l] = (k == l) ? fd2pure(tv, v, k, dx) : fd2mixed(tv, v, k, l, dx);
  }
}

/* ------------------------------------------------------------------------ */
/* pointwise geometry shared by the right-hand side and the constraints     */
/* ------------------------------------------------------------------------ */

typedef struct {
  double g[3][3], ig[3][3], det;    /* conformal metric, inverse, determinant */
  double dg[3][3][3];               /* dg[k][i][j] = d_k g~_ij */
  double D[3][3][3];                /* D_kij = 1/2 d_k g~_ij */
  double Gam[3][3][3];              /* Gam[k][i][j] = conformal Christoffel G~^k_ij */
  double GamL[3][3][3];             /* GamL[k][i][j] = G~_kij = g~_kl G~^l_ij */
  double Gc[3];                     /* G~^i = g~^jk G~^i_jk */
  double ph, P[3], ddph[3][3];      /* phi, P_i = d_i phi, d_i d_j phi */
  double PGam[3][3][3];             /* physical Christoffel Gamma^k_ij */
} geom;

static void metric_inverse(const double g[3][3], double ig[3][3], double *det) {
  double d = g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
             g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
             g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
  ig[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / d;
  ig[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / d;
  ig[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / d;
  ig[1][0] = (g[1][2] * g[2][0] - g[1][0] * g[2][2]) / d;
  ig[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / d;
  ig[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / d;
  ig[2][0] = (g[1][0] * g[2][1] - g[1][1] * g[2][0]) / d;
  ig[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / d;
  ig[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / d;
  *det = d;
}

static void build_geom(const double q[OG_NV], const double d1[OG_NV][3], const double d2[OG_NV][3][3], geom *G) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G->g[i][j] = q[GXX + SYM[i][j]];
  metric_inverse(G->g, G->ig, &G->det);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        G->dg[k][i][j] = d1[GXX + SYM[i][j]][k];
        G->D[k][i][j] = 0.5 * G->dg[k][i][j];
      }
  /* G~^k_ij = g~^kl (D_ijl + D_jil - D_lij) */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += G->ig[k][l] * (G->D[i][j][l] + G->D[j][i][l] - G->D[l][i][j]);
        G->Gam[k][i][j] = s;
      }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += G->g[k][l] * G->Gam[l][i][j];
        G->GamL[k][i][j] = s;
      }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G->ig[j][k] * G->Gam[i][j][k];
    G->Gc[i] = s;
  }
  G->ph = q[PHI];
  for (int i = 0; i < 3; ++i) {
    G->P[i] = d1[PHI][i];
    for (int j = 0; j < 3; ++j) G->ddph[i][j] = d2[PHI][i][j];
  }
  /* Gamma^k_ij = G~^k_ij - (1/phi) g~^kl (g~_jl P_i + g~_il P_j - g~_ij P_l) */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l)
          s += G->ig[k][l] * (G->g[j][l] * G->P[i] + G->g[i][l] * G->P[j] - G->g[i][j] * G->P[l]);
        G->PGam[k][i][j] = G->Gam[k][i][j] - s / G->ph;
      }
}

/* ------------------------------------------------------------------------ */
/* the second-order CCZ4 right-hand side at one point                       */
/* ------------------------------------------------------------------------ */

/* The nine primary evolution equations of the appendix, red terms removed
   (the paper keeps them only in the first-order formulation). Auxiliary
   quantities are the FD4 derivatives of the primaries: A_i = d_i alpha,
   B_k^i = d_k beta^i, D_kij = 1/2 d_k g~_ij, P_i = d_i phi, and their
   derivatives are the FD4 second derivatives.
   Readings taken here:
   - K0 is a parameter (default 0); the slicing function is g(alpha) = 1
     (harmonic) or 2/alpha (1+log);
   - tr A~ = g~^ij A~_ij (conformal metric);
   - G~^i in the Gamma-hat equation and in Z_i is the contracted Christoffel
     symbol of the conformal metric computed from its derivatives;
   - nabla~_i nabla~_j phi = d_i d_j phi - G~^k_ij d_k phi;
   - the trace-free part is taken with the physical metric, which for a
     covariant pair equals X_ij - 1/3 g~_ij g~^kl X_kl;
   - zero shift sets the right-hand sides of beta^i and b^i to zero; the
     Gamma-driver uses d_t Gamma-hat^i of this same point (before the
     dissipation term is added) in the b^i equation. */
static void ccz4_point_rhs(const og_params *P, const double q[OG_NV], const double d1[OG_NV][3],
                           const double d2[OG_NV][3][3], double rhs[OG_NV]) {
  geom G;
  build_geom(q, d1, d2, &G);
  double (*g)[3] = G.g, (*ig)[3] = G.ig;
  const double al = q[ALPHA], ph = q[PHI], Kt = q[KTR], Th = q[THETA];
  double be[3], dal[3], ddal[3][3], dbe[3][3], ddbe[3][3][3], At[3][3], dAt[3][3][3];
  double dKt[3], dTh[3], Gh[3], dGh[3][3], bb[3], dbb[3][3];
  for (int i = 0; i < 3; ++i) {
    be[i] = q[BETAX + i];
    Gh[i] = q[GHX + i];
    bb[i] = q[BBX + i];
    dal[i] = d1[ALPHA][i];
    dKt[i] = d1[KTR][i];
    dTh[i] = d1[THETA][i];
    for (int j = 0; j < 3; ++j) {
      ddal[i][j] = d2[ALPHA][i][j];
      At[i][j] = q[AXX + SYM[i][j]];
    }
  }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) {
      dbe[k][i] = d1[BETAX + i][k];   /* B_k^i */
      dGh[k][i] = d1[GHX + i][k];     /* d_k Gamma-hat^i */
      dbb[k][i] = d1[BBX + i][k];     /* d_k b^i */
      for (int l = 0; l < 3; ++l) ddbe[k][l][i] = d2[BETAX + i][k][l];
      for (int j = 0; j < 3; ++j) dAt[k][i][j] = d1[AXX + SYM[i][j]][k];
    }

  /* Z_i = 1/2 g~_ij (Gh^j - G~^j); Z^i = 1/2 phi^2 (Gh^i - G~^i) */
  double Zcov[3], Zup[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += g[i][j] * (Gh[j] - G.Gc[j]);
    Zcov[i] = 0.5 * s;
    Zup[i] = 0.5 * ph * ph * (Gh[i] - G.Gc[i]);
  }
  /* nabla~_i nabla~_j phi */
  double cdph[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += G.Gam[k][i][j] * G.P[k];
      cdph[i][j] = G.ddph[i][j] - s;
    }
  double trcdph = 0.0, PP = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      trcdph += ig[k][l] * cdph[k][l];
      PP += ig[k][l] * G.P[k] * G.P[l];
    }
  /* R_ij + 2 nabla_(i Z_j), Eq. NR_foccz4_modified_ricci */
  double RZ[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t1 = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) t1 += ig[k][l] * d2[GXX + SYM[i][j]][k][l];
      double t2 = 0.0, t3 = 0.0;
      for (int k = 0; k < 3; ++k) {
        t2 += 0.5 * (g[k][i] * dGh[j][k] + g[k][j] * dGh[i][k]);
        t3 += Gh[k] * G.dg[k][i][j];
      }
      double t4 = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m)
          for (int k = 0; k < 3; ++k)
            t4 += ig[l][m] * (G.Gam[k][l][i] * G.GamL[j][k][m] + G.Gam[k][l][j] * G.GamL[i][k][m] +
                              G.Gam[k][i][m] * G.GamL[k][l][j]);
      double t7 = 0.0;
      for (int k = 0; k < 3; ++k) t7 += Zup[k] * (g[i][k] * G.P[j] + g[j][k] * G.P[i] - g[i][j] * G.P[k]);
      RZ[i][j] = -0.5 * t1 + t2 + 0.5 * t3 + t4 + (cdph[i][j] + g[i][j] * trcdph) / ph -
                 2.0 / (ph * ph) * g[i][j] * PP + 2.0 / (ph * ph * ph) * t7;
    }
  /* nabla_i nabla_j alpha = d_i d_j alpha - Gamma^k_ij A_k (physical) */
  double DDal[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += G.PGam[k][i][j] * dal[k];
      DDal[i][j] = ddal[i][j] - s;
    }
  /* R + 2 nabla_k Z^k = phi^2 g~^ij (R_ij + 2 nabla_(i Z_j)); nabla^i nabla_i alpha */
  double RpZ = 0.0, lapal = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      RpZ += ig[i][j] * RZ[i][j];
      lapal += ig[i][j] * DDal[i][j];
    }
  RpZ *= ph * ph;
  lapal *= ph * ph;
  /* traces and raised A~ */
  double trA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trA += ig[i][j] * At[i][j];
  double Aup[3][3], AgA[3][3], AA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0, u = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          s += ig[i][k] * ig[j][l] * At[k][l];
          u += At[i][k] * ig[k][l] * At[l][j];
        }
      Aup[i][j] = s;
      AgA[i][j] = u;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += At[i][j] * Aup[i][j];
  double trB = dbe[0][0] + dbe[1][1] + dbe[2][2];
  double gfun = (P->slicing == OG_SLICING_ONE_PLUS_LOG) ? 2.0 / al : 1.0;

  /* d_t g~_ij */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double adv = 0.0, lie = 0.0;
      for (int k = 0; k < 3; ++k) {
        adv += be[k] * 2.0 * G.D[k][i][j];
        lie += g[k][i] * dbe[j][k] + g[k][j] * dbe[i][k];
      }
      rhs[GXX + SYM[i][j]] = adv + lie - 2.0 / 3.0 * g[i][j] * trB -
                             2.0 * al * (At[i][j] - 1.0 / 3.0 * g[i][j] * trA) -
                             (1.0 / P->tau) * (G.det - 1.0) * g[i][j];
    }
  /* d_t alpha */
  {
    double adv = 0.0;
    for (int k = 0; k < 3; ++k) adv += be[k] * dal[k];
    rhs[ALPHA] = adv - al * al * gfun * (Kt - P->K0 - 2.0 * P->c * Th);
  }
  /* d_t phi */
  {
    double adv = 0.0;
    for (int k = 0; k < 3; ++k) adv += be[k] * G.P[k];
    rhs[PHI] = adv + 1.0 / 3.0 * ph * (al * Kt - trB);
  }
  /* d_t A~_ij */
  {
    double Mx[3][3], trM = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Mx[i][j] = -DDal[i][j] + al * RZ[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) trM += ig[i][j] * Mx[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        double adv = 0.0, lie = 0.0;
        for (int k = 0; k < 3; ++k) {
          adv += be[k] * dAt[k][i][j];
          lie += At[k][i] * dbe[j][k] + At[k][j] * dbe[i][k];
        }
        rhs[AXX + SYM[i][j]] = adv + ph * ph * (Mx[i][j] - 1.0 / 3.0 * g[i][j] * trM) + lie -
                               2.0 / 3.0 * At[i][j] * trB + al * At[i][j] * (Kt - 2.0 * Th * P->c) -
                               2.0 * al * AgA[i][j];
      }
  }
  /* d_t K */
  {
    double adv = 0.0;
    for (int k = 0; k < 3; ++k) adv += be[k] * dKt[k];
    rhs[KTR] = adv - lapal + al * RpZ + al * Kt * (Kt - 2.0 * Th * P->c) -
               3.0 * al * P->kappa1 * (1.0 + P->kappa2) * Th;
  }
  /* d_t Theta */
  {
    double adv = 0.0, ZA = 0.0;
    for (int k = 0; k < 3; ++k) {
      adv += be[k] * dTh[k];
      ZA += Zup[k] * dal[k];
    }
    rhs[THETA] = adv + 0.5 * al * P->e * P->e * RpZ +
                 0.5 * al * P->e * P->e * (2.0 / 3.0 * Kt * Kt - AA) - al * Th * Kt * P->c - ZA -
                 al * P->kappa1 * (2.0 + P->kappa2) * Th;
  }
  /* d_t Gamma-hat^i */
  double rGh[3], advGh[3];
  for (int i = 0; i < 3; ++i) {
    double adv = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0, t5 = 0.0, t6 = 0.0, t7 = 0.0, t8 = 0.0;
    for (int k = 0; k < 3; ++k) {
      adv += be[k] * dGh[k][i];
      t1 += 2.0 * al * ig[k][i] * dTh[k];
      for (int l = 0; l < 3; ++l) {
        t2 += ig[k][l] * ddbe[k][l][i];
        t3 += P->s / 3.0 * ig[i][k] * ddbe[k][l][l];
      }
      t4 += -4.0 / 3.0 * al * ig[i][k] * dKt[k];
      t5 += -G.Gc[k] * dbe[k][i];
    }
    double GA = 0.0, AP = 0.0, thz = 0.0, AA1 = 0.0, kz = 0.0, k3 = 0.0;
    for (int j = 0; j < 3; ++j) {
      for (int k = 0; k < 3; ++k) {
        GA += G.Gam[i][j][k] * Aup[j][k];
        k3 += ig[j][k] * Zcov[j] * dbe[k][i];
      }
      AP += Aup[i][j] * G.P[j] / ph;
      thz += ig[j][i] * (Th * dal[j] / al + 2.0 / 3.0 * Kt * Zcov[j]);
      AA1 += Aup[i][j] * dal[j];
      kz += ig[i][j] * Zcov[j];
    }
    t6 = 2.0 / 3.0 * G.Gc[i] * trB + 2.0 * al * (GA - 3.0 * AP) - 2.0 * al * thz - 2.0 * AA1;
    t7 = -2.0 * al * P->kappa1 * kz;
    t8 = 2.0 * P->kappa3 * (2.0 / 3.0 * kz * trB - k3);
    advGh[i] = adv;
    rGh[i] = adv + t1 + t2 + t3 + t4 + t5 + t6 + t7 + t8;
    rhs[GHX + i] = rGh[i];
  }
  /* gauge: d_t beta^i, d_t b^i */
  for (int i = 0; i < 3; ++i) {
    if (P->shift == OG_SHIFT_GAMMA_DRIVER) {
      double advb = 0.0, advbb = 0.0;
      for (int k = 0; k < 3; ++k) {
        advb += be[k] * dbe[k][i];
        advbb += be[k] * dbb[k][i];
      }
      rhs[BETAX + i] = advb + P->f * bb[i];
      rhs[BBX + i] = advbb + (rGh[i] - advGh[i]) - P->eta * bb[i];
    } else {
      rhs[BETAX + i] = 0.0;
      rhs[BBX + i] = 0.0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sommerfeld ghost cells                                                   */
/* ------------------------------------------------------------------------ */

/* Right-hand side of the evolved ghost cell id: the paper's radiative
   condition d_t Q + c (r / x_d) d_d Q = -(c / r)(Q - Q_ini), with d_d Q the
   one-sided difference between the ghost cell and its neighbour one layer
   towards the domain (Eq. exa_sommerfeld_inter), r and x_d taken at the ghost
   cell. Reading for edges and corners: the paper fills layers face by face;
   a ghost cell that is outside in several directions belongs to the face
   filled last, in the order x, then y, then z, i.e. to its highest outside
   axis. */
static void ghost_rhs(const og_grid *g, const og_params *P, const double *U, const double *G,
                      const double *Gini, long id, double out[OG_NV]) {
  int c[3] = {g->gcoord[3 * id], g->gcoord[3 * id + 1], g->gcoord[3 * id + 2]};
  int d = -1, side = 0;
  for (int a = 0; a < 3; ++a) {
    if (c[a] < 0) { d = a; side = -1; }
    if (c[a] >= g->N[a]) { d = a; side = +1; }
  }
  int nb[3] = {c[0], c[1], c[2]};
  nb[d] -= side;
  double xs[3];
  for (int a = 0; a < 3; ++a) xs[a] = g->origin[a] + (c[a] + 0.5) * g->dx;
  double r = sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
  for (int v = 0; v < OG_NV; ++v) {
    double qg = G[(long)v * g->n_ghost + id];
    double qn = value_at(g, U, G, v, nb[0], nb[1], nb[2]);
    /* derivative along +x_d from the two points */
    double dQ = side > 0 ? (qg - qn) / g->dx : (qn - qg) / g->dx;
    double cv = P->somm_speed[v];
    out[v] = -cv * (r / xs[d]) * dQ - cv / r * (qg - Gini[(long)v * g->n_ghost + id]);
  }
}

/* ------------------------------------------------------------------------ */
/* full right-hand side, RK4, enforcement                                   */
/* ------------------------------------------------------------------------ */

static void patch_rhs(const og_grid *g, const og_params *P, int n, const double *tile, double *rU) {
  int p = g->p, T = g->T;
  double dx = g->dxl[g->lev[n]];
  long pts = n_interior(g);
  double d1[OG_NV][3], d2[OG_NV][3][3];
  for (int z = 0; z < p; ++z)
    for (int y = 0; y < p; ++y)
      for (int x = 0; x < p; ++x) {
        tview tv;
        tv.tile = tile;
        tv.c = ((long)(z + OG_HALO) * T + (y + OG_HALO)) * T + (x + OG_HALO);
        tv.st[0] = 1; tv.st[1] = T; tv.st[2] = (long)T * T;
        double q[OG_NV], r[OG_NV];
        for (int v = 0; v < OG_NV; ++v) q[v] = tq(&tv, 0, v);
        point_derivs(&tv, dx, d1, d2);
        ccz4_point_rhs(P, q, d1, d2, r);
        long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
        for (int v = 0; v < OG_NV; ++v) rU[(long)v * pts + li] = r[v] + ko_sum(&tv, v, P->ko_eps, dx);
      }
}

int og_rhs(const og_grid *g, const og_params *P, const double *U, const double *G,
           const double *Gini, double *rU, double *rG) {
  long T3 = (long)g->T * g->T * g->T;
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * OG_NV);
  for (int n = 0; n < g->n_patches; ++n) {
    build_tile(g, n, U, G, tile);
    patch_rhs(g, P, n, tile, rU);
  }
  free(tile);
  for (long id = 0; id < g->n_ghost; ++id) {
    double r[OG_NV];
    ghost_rhs(g, P, U, G, Gini, id, r);
    for (int v = 0; v < OG_NV; ++v) rG[(long)v * g->n_ghost + id] = r[v];
  }
  return 0;
}

/* Right-hand side of the ghost shell alone (the interior is not evaluated). */
int og_ghost_rhs(const og_grid *g, const og_params *P, const double *U, const double *G,
                 const double *Gini, double *rG) {
  for (long id = 0; id < g->n_ghost; ++id) {
    double r[OG_NV];
    ghost_rhs(g, P, U, G, Gini, id, r);
    for (int v = 0; v < OG_NV; ++v) rG[(long)v * g->n_ghost + id] = r[v];
  }
  return 0;
}

/* Algebraic constraints: det g~ = 1 by rescaling every component with
   det^(-1/3), then tr A~ = 0 by removing g~_ij / 3 times the trace taken with
   the rescaled metric. */
int og_enforce(const og_grid *g, double *U) {
  long pts = n_interior(g);
  for (long i = 0; i < pts; ++i) {
    double m[3][3], im[3][3], det, A[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        m[a][b] = U[(long)(GXX + SYM[a][b]) * pts + i];
        A[a][b] = U[(long)(AXX + SYM[a][b]) * pts + i];
      }
    metric_inverse(m, im, &det);
    double sc = 1.0 / cbrt(det);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m[a][b] *= sc;
    metric_inverse(m, im, &det);
    double tr = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) tr += im[a][b] * A[a][b];
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) {
        U[(long)(GXX + SYM[a][b]) * pts + i] = m[a][b];
        U[(long)(AXX + SYM[a][b]) * pts + i] = A[a][b] - 1.0 / 3.0 * m[a][b] * tr;
      }
  }
  return 0;
}

/* Restriction (appendix "refinement transition", R^par of the average
   scheme along every axis): each coarse point under a refined patch takes
   the mean of the 3x3x3 fine cells that tile it, as the tensor product of
   three one-dimensional averages with weights 1/3 (x, then y, then z).
   Levels are restricted from the finest down, so level 0 sees the finest
   data. */
int og_restrict(const og_grid *g, double *U) {
  const long pts = n_interior(g);
  const int p = g->p;
  const double third = 1.0 / 3.0;
  for (int l = g->n_levels - 1; l >= 1; --l)
    for (int n = 0; n < g->n_patches; ++n) {
      if (g->lev[n] != l - 1 || g->nchild[n] == 0) continue;
      for (int k = 0; k < p; ++k)
        for (int j = 0; j < p; ++j)
          for (int i = 0; i < p; ++i) {
            int X = 3 * (g->ijk[3 * n] * p + i), Y = 3 * (g->ijk[3 * n + 1] * p + j),
                Z = 3 * (g->ijk[3 * n + 2] * p + k);
            long ci = (long)n * p * p * p + ((long)k * p + j) * p + i;
            for (int v = 0; v < OG_NV; ++v) {
              double sy[3];
              for (int c = 0; c < 3; ++c) {
                double sx[3];
                for (int b = 0; b < 3; ++b) {
                  double f0 = level_value(g, U, v, l, X, Y + b, Z + c);
                  double f1 = level_value(g, U, v, l, X + 1, Y + b, Z + c);
                  double f2 = level_value(g, U, v, l, X + 2, Y + b, Z + c);
                  sx[b] = third * f0 + third * f1 + third * f2;
                }
                sy[c] = third * sx[0] + third * sx[1] + third * sx[2];
              }
              U[(long)v * pts + ci] = third * sy[0] + third * sy[1] + third * sy[2];
            }
          }
    }
  return 0;
}

/* Classic RK4 (weights 1/6, 1/3, 1/3, 1/6; nodes 0, 1/2, 1/2, 1) over the
   interior points and the evolved Sommerfeld ghost cells, then the algebraic
   enforcement on the interior points and, on a refined mesh, the
   restriction. All levels take the same step dt. */
int og_rk4_step(const og_grid *g, const og_params *P, double dt, double *U, double *G,
                const double *Gini) {
  long nu = n_interior(g) * OG_NV, ng = g->n_ghost * OG_NV;
  double *k[4], *kg[4];
  for (int s = 0; s < 4; ++s) {
    k[s] = (double *)malloc(sizeof(double) * (size_t)nu);
    kg[s] = (double *)malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1));
  }
  double *Y = (double *)malloc(sizeof(double) * (size_t)nu);
  double *YG = (double *)malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1));
  const double cnode[4] = {0.0, 0.5, 0.5, 1.0};
  for (int s = 0; s < 4; ++s) {
    if (s == 0) {
      memcpy(Y, U, sizeof(double) * (size_t)nu);
      if (ng) memcpy(YG, G, sizeof(double) * (size_t)ng);
    } else {
      for (long i = 0; i < nu; ++i) Y[i] = U[i] + cnode[s] * dt * k[s - 1][i];
      for (long i = 0; i < ng; ++i) YG[i] = G[i] + cnode[s] * dt * kg[s - 1][i];
    }
    og_rhs(g, P, Y, YG, Gini, k[s], kg[s]);
  }
  for (long i = 0; i < nu; ++i) U[i] = U[i] + dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
  for (long i = 0; i < ng; ++i) G[i] = G[i] + dt / 6.0 * (kg[0][i] + 2.0 * kg[1][i] + 2.0 * kg[2][i] + kg[3][i]);
  og_enforce(g, U);
  if (g->n_levels > 1) og_restrict(g, U);
  for (int s = 0; s < 4; ++s) { free(k[s]); free(kg[s]); }
  free(Y); free(YG);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* constraints                                                              */
/* ------------------------------------------------------------------------ */

/* Hamiltonian constraint H = R + 2/3 K^2 - A~_ij A~^ij and momentum
   constraint M_i = g~^kl (d_k A~_li - 2 G~^m_l(i A~_k)m - 3 A~_ik P_l / phi)
   - 2/3 d_i K (vacuum). R is the physical Ricci scalar, taken from the
   Riemann relation of the appendix with the physical Christoffel symbols
   and their derivatives (Z does not enter). M is computed with a lower
   index, as printed on the right-hand side. */
static void point_constraints(const double q[OG_NV], const double d1[OG_NV][3],
                              const double d2[OG_NV][3][3], double out[4]) {
  geom G;
  build_geom(q, d1, d2, &G);
  double (*g)[3] = G.g, (*ig)[3] = G.ig;
  const double ph = G.ph;
  /* D_k^{ml} = g~^ma g~^lb D_kab */
  double Dup[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m)
      for (int l = 0; l < 3; ++l) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) s += ig[m][a] * ig[l][b] * G.D[k][a][b];
        Dup[k][m][l] = s;
      }
  /* dD[k][i][j][l] = d_k D_ijl = 1/2 d_k d_i g~_jl */
  double dD[3][3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) dD[k][i][j][l] = 0.5 * d2[GXX + SYM[j][l]][k][i];
  /* d_k Gamma^m_ij, the appendix's closing relation for the physical
     Christoffel symbols */
  double dPG[3][3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
          for (int l = 0; l < 3; ++l) {
            s += -2.0 * Dup[k][m][l] * (G.D[i][j][l] + G.D[j][i][l] - G.D[l][i][j]);
            s += ig[m][l] * (dD[k][i][j][l] + dD[k][j][i][l] - dD[k][l][i][j]);
            s += 2.0 / ph * Dup[k][m][l] * (g[j][l] * G.P[i] + g[i][l] * G.P[j] - g[i][j] * G.P[l]);
            s += -2.0 / ph * ig[m][l] * (G.D[k][j][l] * G.P[i] + G.D[k][i][l] * G.P[j] - G.D[k][i][j] * G.P[l]);
            s += -1.0 / ph * ig[m][l] * (g[j][l] * G.ddph[k][i] + g[i][l] * G.ddph[k][j] - g[i][j] * G.ddph[k][l]);
            s += 1.0 / (ph * ph) * ig[m][l] *
                 (g[j][l] * G.P[i] * G.P[k] + g[i][l] * G.P[j] * G.P[k] - g[i][j] * G.P[k] * G.P[l]);
          }
          dPG[k][m][i][j] = s;
        }
  /* R_ij = R^m_imj with R^m_ikj = d_k Gamma^m_ij - d_j Gamma^m_ik
     + Gamma^l_ij Gamma^m_lk - Gamma^l_ik Gamma^m_lj */
  double R = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double Rij = 0.0;
      for (int m = 0; m < 3; ++m) {
        Rij += dPG[m][m][i][j] - dPG[j][m][i][m];
        for (int l = 0; l < 3; ++l)
          Rij += G.PGam[l][i][j] * G.PGam[m][l][m] - G.PGam[l][i][m] * G.PGam[m][l][j];
      }
      R += ph * ph * ig[i][j] * Rij;   /* gamma^ij = phi^2 g~^ij */
    }
  double At[3][3], Aup[3][3], AA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) At[i][j] = q[AXX + SYM[i][j]];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += ig[i][k] * ig[j][l] * At[k][l];
      Aup[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += At[i][j] * Aup[i][j];
  const double Kt = q[KTR];
  out[0] = R + 2.0 / 3.0 * Kt * Kt - AA;
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        double dA = d1[AXX + SYM[l][i]][k];
        double cs = 0.0;
        for (int m = 0; m < 3; ++m) cs += G.Gam[m][l][i] * At[k][m] + G.Gam[m][l][k] * At[i][m];
        s += ig[k][l] * (dA - cs - 3.0 * At[i][k] * G.P[l] / ph);
      }
    out[1 + i] = s - 2.0 / 3.0 * d1[KTR][i];
  }
}

/* L2 norms over all interior points of the leaf patches (Sec. "Gauge Wave":
   L2 = sqrt(sum H^2 / n), n the number of grid points; on a refined mesh
   the points a finer level covers are not counted again). H and M are
   written for every patch. out[0] = L2 of H,
   out[1] = L2 of |M| (|M|^2 = sum_i M_i^2), out[2] = max |H|,
   out[3] = max |M|, out[4] = number of non-finite H or M values. */
int og_constraints(const og_grid *g, const double *U, const double *G, double *H, double *M,
                   double out[5]) {
  int p = g->p, T = g->T;
  long pts = n_interior(g), T3 = (long)T * T * T;
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * OG_NV);
  double d1[OG_NV][3], d2[OG_NV][3][3];
  double sH = 0.0, sM = 0.0, mH = 0.0, mM = 0.0, bad = 0.0;
  long n_leaf_pts = 0;
  for (int n = 0; n < g->n_patches; ++n) {
    const double dx = g->dxl[g->lev[n]];
    const int leaf = g->nchild[n] == 0;
    if (leaf) n_leaf_pts += (long)p * p * p;
    build_tile(g, n, U, G, tile);
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          tview tv;
          tv.tile = tile;
          tv.c = ((long)(z + OG_HALO) * T + (y + OG_HALO)) * T + (x + OG_HALO);
          tv.st[0] = 1; tv.st[1] = T; tv.st[2] = (long)T * T;
          double q[OG_NV], c4[4];
          for (int v = 0; v < OG_NV; ++v) q[v] = tq(&tv, 0, v);
          point_derivs(&tv, dx, d1, d2);
          point_constraints(q, d1, d2, c4);
          long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
          if (H) H[li] = c4[0];
          if (M)
            for (int i = 0; i < 3; ++i) M[(long)i * pts + li] = c4[1 + i];
          if (!leaf) continue;
          double m2 = c4[1] * c4[1] + c4[2] * c4[2] + c4[3] * c4[3];
          if (!isfinite(c4[0]) || !isfinite(m2)) { bad += 1.0; continue; }
          sH += c4[0] * c4[0];
          sM += m2;
          if (fabs(c4[0]) > mH) mH = fabs(c4[0]);
          if (sqrt(m2) > mM) mM = sqrt(m2);
        }
  }
  free(tile);
  out[0] = sqrt(sH / (double)n_leaf_pts);
  out[1] = sqrt(sM / (double)n_leaf_pts);
  out[2] = mH;
  out[3] = mM;
  out[4] = bad;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sampled points (for checks at sizes where a full oracle pass is too slow) */
/* ------------------------------------------------------------------------ */

/* Small halo'd neighbourhood (7^3 points) of interior point pt, in the same
   working layout as a tile. */
static void build_neigh(const og_grid *g, const double *U, const double *G, long pt, double *nb) {
  int p = g->p;
  long p3 = (long)p * p * p;
  int n = (int)(pt / p3), l = g->lev[n];
  long r = pt % p3;
  int lz = (int)(r / (p * p)), ly = (int)((r / p) % p), lx = (int)(r % p);
  int gx = g->ijk[3 * n] * p + lx, gy = g->ijk[3 * n + 1] * p + ly, gz = g->ijk[3 * n + 2] * p + lz;
  const int W = 2 * OG_HALO + 1;
  for (int c = 0; c < W; ++c)
    for (int b = 0; b < W; ++b)
      for (int a = 0; a < W; ++a)
        for (int v = 0; v < OG_NV; ++v)
          nb[(((long)c * W + b) * W + a) * OG_NV + v] =
              value_at_l(g, U, G, v, l, gx + a - OG_HALO, gy + b - OG_HALO, gz + c - OG_HALO);
}

static double point_dx(const og_grid *g, long pt) {
  long p3 = (long)g->p * g->p * g->p;
  return g->dxl[g->lev[pt / p3]];
}

static int sample_view(const og_grid *g, const double *U, const double *G, long pt, double *nb, tview *tv) {
  if (pt < 0 || pt >= n_interior(g)) return 1;
  const int W = 2 * OG_HALO + 1;
  build_neigh(g, U, G, pt, nb);
  tv->tile = nb;
  tv->c = ((long)OG_HALO * W + OG_HALO) * W + OG_HALO;
  tv->st[0] = 1; tv->st[1] = W; tv->st[2] = (long)W * W;
  return 0;
}

int og_rhs_points(const og_grid *g, const og_params *P, const double *U, const double *G,
                  long n, const long *pts, double *out) {
  double nb[7 * 7 * 7 * OG_NV];
  double d1[OG_NV][3], d2[OG_NV][3][3];
  for (long s = 0; s < n; ++s) {
    tview tv;
    if (sample_view(g, U, G, pts[s], nb, &tv)) return 1;
    double q[OG_NV], r[OG_NV];
    for (int v = 0; v < OG_NV; ++v) q[v] = tq(&tv, 0, v);
    const double dx = point_dx(g, pts[s]);
    point_derivs(&tv, dx, d1, d2);
    ccz4_point_rhs(P, q, d1, d2, r);
    for (int v = 0; v < OG_NV; ++v) out[s * OG_NV + v] = r[v] + ko_sum(&tv, v, P->ko_eps, dx);
  }
  return 0;
}

int og_constraints_points(const og_grid *g, const double *U, const double *G, long n,
                          const long *pts, double *out) {
  double nb[7 * 7 * 7 * OG_NV];
  double d1[OG_NV][3], d2[OG_NV][3][3];
  for (long s = 0; s < n; ++s) {
    tview tv;
    if (sample_view(g, U, G, pts[s], nb, &tv)) return 1;
    double q[OG_NV];
    for (int v = 0; v < OG_NV; ++v) q[v] = tq(&tv, 0, v);
    point_derivs(&tv, point_dx(g, pts[s]), d1, d2);
    point_constraints(q, d1, d2, out + 4 * s);
  }
  return 0;
}

int og_point_derivs(const og_grid *g, const double *U, const double *G, long pt, double ko_eps,
                    double *d1o, double *d2o, double *koo) {
  double nb[7 * 7 * 7 * OG_NV];
  double d1[OG_NV][3], d2[OG_NV][3][3];
  tview tv;
  if (sample_view(g, U, G, pt, nb, &tv)) return 1;
  const double dx = point_dx(g, pt);
  point_derivs(&tv, dx, d1, d2);
  for (int v = 0; v < OG_NV; ++v) {
    for (int k = 0; k < 3; ++k) {
      d1o[v * 3 + k] = d1[v][k];
      for (int l = 0; l < 3; ++l) d2o[(v * 3 + k) * 3 + l] = d2[v][k][l];
    }
    koo[v] = ko_sum(&tv, v, ko_eps, dx);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* particle tracers (Sec. "Particle Tracers as Data Probes")                */
/* ------------------------------------------------------------------------ */

/* Data projection of the 25 fields onto the point x by trilinear
   interpolation from the 2^3 closest sample points (Sec. "Particle Tracers
   as Data Probes"). Readings: the sample points are the cell centres of the
   finest level that holds all eight as interior points of its patches;
   where no refined level does, level 0 with its boundary rule (periodic
   wrap, clamped copy, or the cells of the Sommerfeld ghost shell). The
   weights along an axis are (1 - t, t), t the offset of x from the lower
   sample point in units of the level's spacing; the value is the sum over
   the eight corners (z outermost, x innermost) of (w_x w_y) w_z q. Returns 1
   where x lies beyond what level 0 resolves (outside the Sommerfeld ghost
   shell, or not a finite coordinate). */
static int tracer_sample(const og_grid *g, const double *U, const double *G, const double x[3],
                         double out[OG_NV]) {
  for (int l = g->n_levels - 1; l >= 0; --l) {
    const double h = g->dxl[l];
    int i0[3];
    double t[3];
    int finite = 1;
    for (int d = 0; d < 3; ++d) {
      double s = (x[d] - g->origin[d]) / h - 0.5;
      if (!(fabs(s) < 1.0e9)) finite = 0;
      double f = finite ? floor(s) : 0.0;
      i0[d] = (int)f;
      t[d] = s - f;
    }
    if (!finite) return 1;
    long idx[8];
    int kind[8], ok = 1;
    for (int c = 0; c < 2 && ok; ++c)
      for (int b = 0; b < 2 && ok; ++b)
        for (int a = 0; a < 2 && ok; ++a) {
          int k = (c * 2 + b) * 2 + a, px = i0[0] + a, py = i0[1] + b, pz = i0[2] + c;
          if (l > 0) {
            kind[k] = 0;
            if (!level_has(g, l, px, py, pz, &idx[k])) ok = 0;
          } else {
            if (g->bc == OG_BC_SOMMERFELD &&
                (px < -OG_HALO || px >= g->N[0] + OG_HALO || py < -OG_HALO || py >= g->N[1] + OG_HALO ||
                 pz < -OG_HALO || pz >= g->N[2] + OG_HALO))
              return 1;
            kind[k] = locate(g, px, py, pz, &idx[k]);
          }
        }
    if (!ok) continue;
    double wx[2] = {1.0 - t[0], t[0]}, wy[2] = {1.0 - t[1], t[1]}, wz[2] = {1.0 - t[2], t[2]};
    for (int v = 0; v < OG_NV; ++v) {
      double acc = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            int k = (c * 2 + b) * 2 + a;
            double q = kind[k] == 0 ? U[(long)v * n_interior(g) + idx[k]] : G[(long)v * g->n_ghost + idx[k]];
            double w = (wx[a] * wy[b]) * wz[c];
            acc = acc + w * q;
          }
      out[v] = acc;
    }
    return 0;
  }
  return 1;
}

/* One step of n tracers: each records the projected fields at its position
   (values[s][25], if values is not NULL) and, if vel_field >= 0, moves by
   the explicit Euler step x <- x + (dt * vel_scale) v of the paper's tracer
   section, v the projected fields vel_field .. vel_field + 2 (puncture
   trackers: the shift with vel_scale = -1, Sec. "Particle tracers" on the
   opposite shift as the velocity). A tracer that cannot be projected is left
   where it is, with NaN values. Returns the number of such tracers. */
long og_tracers_step(const og_grid *g, const double *U, const double *G, long n, double *pos, double dt,
                     int vel_field, double vel_scale, double *values) {
  long bad = 0;
  for (long s = 0; s < n; ++s) {
    double val[OG_NV];
    if (tracer_sample(g, U, G, pos + 3 * s, val)) {
      ++bad;
      if (values)
        for (int v = 0; v < OG_NV; ++v) values[s * OG_NV + v] = NAN;
      continue;
    }
    if (values)
      for (int v = 0; v < OG_NV; ++v) values[s * OG_NV + v] = val[v];
    if (vel_field >= 0 && vel_field + 2 < OG_NV)
      for (int d = 0; d < 3; ++d) pos[3 * s + d] = pos[3 * s + d] + (dt * vel_scale) * val[vel_field + d];
  }
  return bad;
}

/* ======================================================================== */
/* first-order formulation (FO) and second-order with reconstruction        */
/* ======================================================================== */

/* The 58 variables of Eq. first-order-variables: the 25 primaries in their
   usual order, then the auxiliary variables of Eq. auxiliary-variables:
   A_k = d_k alpha (25..27), B_k^i = d_k beta^i (28 + 3k + i),
   D_kij = 1/2 d_k g~_ij (37 + 6k + pair(i, j)), P_k = d_k phi (55..57). */
enum { FO_A = 25, FO_B = 28, FO_D = 37, FO_P = 55 };

/* Right-hand side of the 58 variables at one point from their values q and
   their FD4 first derivatives d1[v][k] = d_k q_v (Alg. fd4-fo: only first
   derivatives are taken). The nine primary equations of the appendix
   "Spacetime foliation" are written with the auxiliary variables in place
   of the derivatives of alpha, beta, g~ and phi: first derivatives become
   A, B, D, P, and second derivatives the symmetrised first derivatives of
   those (d_i d_j alpha -> d_(i A_j), d_k d_l beta^i -> d_(k B_l)^i,
   d_k d_l g~_ij -> d_k D_lij + d_l D_kij, d_i d_j phi -> d_(i P_j)), which
   is how the relations below the equations close the system (Christoffel
   symbols from D, nabla nabla alpha = d_(i A_j) - Gamma^k_ij A_k, the
   modified Ricci tensor of Eq. NR_foccz4_modified_ricci). The four
   auxiliary equations are Eqs. NR_foccz4_A_k, NR_foccz4_B^i_j, the D_kij
   equation and NR_foccz4_P_i. red != 0 keeps the red terms (the first-order
   formulation); red == 0 removes them (the second-order formulation, whose
   auxiliary variables are reconstructed instead of evolved).
   Readings: those of the second-order right-hand side (ccz4_point_rhs),
   and: g'(alpha) = -2/alpha^2 for 1+log, 0 for harmonic slicing; K0 is a
   constant (d_k K0 = 0); zero shift sets the right-hand sides of beta^i,
   b^i and B_k^i to zero (beta is then static, so B = d beta is too);
   D_k^nm = g~^na g~^mb D_kab. */
static void fo_point_rhs(const og_params *P, int red, const double q[OG_NV_FO], const double d1[OG_NV_FO][3],
                         double rhs[OG_NV_FO]) {
  double g[3][3], ig[3][3], det;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g[i][j] = q[GXX + SYM[i][j]];
  metric_inverse(g, ig, &det);
  const double al = q[ALPHA], ph = q[PHI], Kt = q[KTR], Th = q[THETA];
  double be[3], Gh[3], bb[3], Av[3], Pv[3], B[3][3], D[3][3][3], At[3][3];
  for (int i = 0; i < 3; ++i) {
    be[i] = q[BETAX + i];
    Gh[i] = q[GHX + i];
    bb[i] = q[BBX + i];
    Av[i] = q[FO_A + i];
    Pv[i] = q[FO_P + i];
    for (int j = 0; j < 3; ++j) {
      B[i][j] = q[FO_B + 3 * i + j];                  /* B[k][i] = B_k^i */
      At[i][j] = q[AXX + SYM[i][j]];
    }
  }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) D[k][i][j] = q[FO_D + 6 * k + SYM[i][j]];
  /* first derivatives of the evolved variables */
  double dA[3][3], dP[3][3], dB[3][3][3], dD[3][3][3][3], dAt[3][3][3], dK[3], dTh[3], dGh[3][3], dbb[3][3];
  for (int k = 0; k < 3; ++k) {
    dK[k] = d1[KTR][k];
    dTh[k] = d1[THETA][k];
    for (int i = 0; i < 3; ++i) {
      dA[k][i] = d1[FO_A + i][k];                     /* d_k A_i */
      dP[k][i] = d1[FO_P + i][k];                     /* d_k P_i */
      dGh[k][i] = d1[GHX + i][k];                     /* d_k Gamma-hat^i */
      dbb[k][i] = d1[BBX + i][k];                     /* d_k b^i */
      for (int l = 0; l < 3; ++l) dB[k][l][i] = d1[FO_B + 3 * l + i][k];   /* d_k B_l^i */
      for (int j = 0; j < 3; ++j) {
        dAt[k][i][j] = d1[AXX + SYM[i][j]][k];        /* d_k A~_ij */
        for (int m = 0; m < 3; ++m) dD[m][k][i][j] = d1[FO_D + 6 * k + SYM[i][j]][m];   /* d_m D_kij */
      }
    }
  }
  /* symmetrised stand-ins of the second derivatives */
  double ddal[3][3], ddph[3][3], ddbe[3][3][3], ddg[3][3][3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ddal[i][j] = 0.5 * (dA[i][j] + dA[j][i]);
      ddph[i][j] = 0.5 * (dP[i][j] + dP[j][i]);
      for (int l = 0; l < 3; ++l) ddbe[i][j][l] = 0.5 * (dB[i][j][l] + dB[j][i][l]);   /* d_(i B_j)^l */
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ddg[i][j][a][b] = dD[i][j][a][b] + dD[j][i][a][b];   /* d_i d_j g~_ab */
    }
  /* Christoffel symbols from D: G~^k_ij = g~^kl (D_ijl + D_jil - D_lij) */
  double Gam[3][3][3], GamL[3][3][3], Gc[3], PGam[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += ig[k][l] * (D[i][j][l] + D[j][i][l] - D[l][i][j]);
        Gam[k][i][j] = s;
      }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += g[k][l] * Gam[l][i][j];
        GamL[k][i][j] = s;
      }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += ig[j][k] * Gam[i][j][k];
    Gc[i] = s;
  }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += ig[k][l] * (g[j][l] * Pv[i] + g[i][l] * Pv[j] - g[i][j] * Pv[l]);
        PGam[k][i][j] = Gam[k][i][j] - s / ph;
      }
  /* D_k^nm = g~^na g~^mb D_kab, and its contraction with A~ */
  double DuA[3];   /* D_k^nm A~_nm */
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int n = 0; n < 3; ++n)
      for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) s += ig[n][a] * ig[m][b] * D[k][a][b] * At[n][m];
    DuA[k] = s;
  }
  double gdAt[3];  /* g~^nm d_k A~_nm */
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int n = 0; n < 3; ++n)
      for (int m = 0; m < 3; ++m) s += ig[n][m] * dAt[k][n][m];
    gdAt[k] = s;
  }
  /* Z_i = 1/2 g~_ij (Gh^j - G~^j); Z^i = 1/2 phi^2 (Gh^i - G~^i) */
  double Zcov[3], Zup[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += g[i][j] * (Gh[j] - Gc[j]);
    Zcov[i] = 0.5 * s;
    Zup[i] = 0.5 * ph * ph * (Gh[i] - Gc[i]);
  }
  /* nabla~_i nabla~_j phi = d_(i P_j) - G~^k_ij P_k */
  double cdph[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Gam[k][i][j] * Pv[k];
      cdph[i][j] = ddph[i][j] - s;
    }
  double trcdph = 0.0, PP = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      trcdph += ig[k][l] * cdph[k][l];
      PP += ig[k][l] * Pv[k] * Pv[l];
    }
  /* R_ij + 2 nabla_(i Z_j), Eq. NR_foccz4_modified_ricci with D, P and d D, d P */
  double RZ[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t1 = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) t1 += ig[k][l] * ddg[k][l][i][j];
      double t2 = 0.0, t3 = 0.0;
      for (int k = 0; k < 3; ++k) {
        t2 += 0.5 * (g[k][i] * dGh[j][k] + g[k][j] * dGh[i][k]);
        t3 += Gh[k] * 2.0 * D[k][i][j];
      }
      double t4 = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m)
          for (int k = 0; k < 3; ++k)
            t4 += ig[l][m] * (Gam[k][l][i] * GamL[j][k][m] + Gam[k][l][j] * GamL[i][k][m] +
                              Gam[k][i][m] * GamL[k][l][j]);
      double t7 = 0.0;
      for (int k = 0; k < 3; ++k) t7 += Zup[k] * (g[i][k] * Pv[j] + g[j][k] * Pv[i] - g[i][j] * Pv[k]);
      RZ[i][j] = -0.5 * t1 + t2 + 0.5 * t3 + t4 + (cdph[i][j] + g[i][j] * trcdph) / ph -
                 2.0 / (ph * ph) * g[i][j] * PP + 2.0 / (ph * ph * ph) * t7;
    }
  /* nabla_i nabla_j alpha = d_(i A_j) - Gamma^k_ij A_k */
  double DDal[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += PGam[k][i][j] * Av[k];
      DDal[i][j] = ddal[i][j] - s;
    }
  double RpZ = 0.0, lapal = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      RpZ += ig[i][j] * RZ[i][j];
      lapal += ig[i][j] * DDal[i][j];
    }
  RpZ *= ph * ph;
  lapal *= ph * ph;
  double trA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trA += ig[i][j] * At[i][j];
  double Aup[3][3], AgA[3][3], AA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0, u = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          s += ig[i][k] * ig[j][l] * At[k][l];
          u += At[i][k] * ig[k][l] * At[l][j];
        }
      Aup[i][j] = s;
      AgA[i][j] = u;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AA += At[i][j] * Aup[i][j];
  const double trB = B[0][0] + B[1][1] + B[2][2];
  const double onelog = P->slicing == OG_SLICING_ONE_PLUS_LOG;
  const double gfun = onelog ? 2.0 / al : 1.0;
  const double gprime = onelog ? -2.0 / (al * al) : 0.0;
  const double lapse_src = Kt - P->K0 - 2.0 * P->c * Th;

  /* d_t g~_ij */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double adv = 0.0, lie = 0.0;
      for (int k = 0; k < 3; ++k) {
        adv += be[k] * 2.0 * D[k][i][j];
        lie += g[k][i] * B[j][k] + g[k][j] * B[i][k];
      }
      rhs[GXX + SYM[i][j]] = adv + lie - 2.0 / 3.0 * g[i][j] * trB - 2.0 * al * (At[i][j] - 1.0 / 3.0 * g[i][j] * trA) -
                             (1.0 / P->tau) * (det - 1.0) * g[i][j];
    }
  /* d_t alpha, d_t phi */
  {
    double advA = 0.0, advP = 0.0;
    for (int k = 0; k < 3; ++k) {
      advA += be[k] * Av[k];
      advP += be[k] * Pv[k];
    }
    rhs[ALPHA] = advA - al * al * gfun * lapse_src;
    rhs[PHI] = advP + 1.0 / 3.0 * ph * (al * Kt - trB);
  }
  /* d_t A~_ij */
  {
    double Mx[3][3], trM = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Mx[i][j] = -DDal[i][j] + al * RZ[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) trM += ig[i][j] * Mx[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        double adv = 0.0, lie = 0.0;
        for (int k = 0; k < 3; ++k) {
          adv += be[k] * dAt[k][i][j];
          lie += At[k][i] * B[j][k] + At[k][j] * B[i][k];
        }
        rhs[AXX + SYM[i][j]] = adv + ph * ph * (Mx[i][j] - 1.0 / 3.0 * g[i][j] * trM) + lie -
                               2.0 / 3.0 * At[i][j] * trB + al * At[i][j] * (Kt - 2.0 * Th * P->c) -
                               2.0 * al * AgA[i][j];
      }
  }
  /* d_t K, d_t Theta */
  {
    double advK = 0.0, advT = 0.0, ZA = 0.0;
    for (int k = 0; k < 3; ++k) {
      advK += be[k] * dK[k];
      advT += be[k] * dTh[k];
      ZA += Zup[k] * Av[k];
    }
    rhs[KTR] = advK - lapal + al * RpZ + al * Kt * (Kt - 2.0 * Th * P->c) - 3.0 * al * P->kappa1 * (1.0 + P->kappa2) * Th;
    rhs[THETA] = advT + 0.5 * al * P->e * P->e * RpZ + 0.5 * al * P->e * P->e * (2.0 / 3.0 * Kt * Kt - AA) -
                 al * Th * Kt * P->c - ZA - al * P->kappa1 * (2.0 + P->kappa2) * Th;
  }
  /* d_t Gamma-hat^i (red: + 2 alpha g~^ik g~^nm d_k A~_nm - 4 alpha g~^ik D_k^nm A~_nm) */
  double rGh[3], advGh[3];
  for (int i = 0; i < 3; ++i) {
    double adv = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0, t5 = 0.0, tr = 0.0;
    for (int k = 0; k < 3; ++k) {
      adv += be[k] * dGh[k][i];
      t1 += 2.0 * al * ig[k][i] * dTh[k];
      for (int l = 0; l < 3; ++l) {
        t2 += ig[k][l] * ddbe[k][l][i];
        t3 += P->s / 3.0 * ig[i][k] * ddbe[k][l][l];
      }
      t4 += -4.0 / 3.0 * al * ig[i][k] * dK[k];
      t5 += -Gc[k] * B[k][i];
      tr += 2.0 * al * ig[i][k] * gdAt[k] - 4.0 * al * ig[i][k] * DuA[k];
    }
    double GA = 0.0, AP = 0.0, thz = 0.0, AA1 = 0.0, kz = 0.0, k3 = 0.0;
    for (int j = 0; j < 3; ++j) {
      for (int k = 0; k < 3; ++k) {
        GA += Gam[i][j][k] * Aup[j][k];
        k3 += ig[j][k] * Zcov[j] * B[k][i];
      }
      AP += Aup[i][j] * Pv[j] / ph;
      thz += ig[j][i] * (Th * Av[j] / al + 2.0 / 3.0 * Kt * Zcov[j]);
      AA1 += Aup[i][j] * Av[j];
      kz += ig[i][j] * Zcov[j];
    }
    double t6 = 2.0 / 3.0 * Gc[i] * trB + 2.0 * al * (GA - 3.0 * AP) - 2.0 * al * thz - 2.0 * AA1;
    double t7 = -2.0 * al * P->kappa1 * kz;
    double t8 = 2.0 * P->kappa3 * (2.0 / 3.0 * kz * trB - k3);
    advGh[i] = adv;
    rGh[i] = adv + t1 + t2 + t3 + t4 + t5 + t6 + t7 + t8 + (red ? tr : 0.0);
    rhs[GHX + i] = rGh[i];
  }
  /* gauge: d_t beta^i, d_t b^i */
  const int driver = P->shift == OG_SHIFT_GAMMA_DRIVER;
  for (int i = 0; i < 3; ++i) {
    if (driver) {
      double advb = 0.0, advbb = 0.0;
      for (int k = 0; k < 3; ++k) {
        advb += be[k] * B[k][i];
        advbb += be[k] * dbb[k][i];
      }
      rhs[BETAX + i] = advb + P->f * bb[i];
      rhs[BBX + i] = advbb + (rGh[i] - advGh[i]) - P->eta * bb[i];
    } else {
      rhs[BETAX + i] = 0.0;
      rhs[BBX + i] = 0.0;
    }
  }
  /* Eq. NR_foccz4_A_k (red: - alpha g g~^nm d_k A~_nm + 2 alpha g D_k^nm A~_nm) */
  for (int k = 0; k < 3; ++k) {
    double adv = 0.0, BA = 0.0;
    for (int l = 0; l < 3; ++l) {
      adv += be[l] * dA[l][k];
      BA += B[k][l] * Av[l];
    }
    double r = adv - al * al * gfun * (dK[k] - 2.0 * P->c * dTh[k]) + BA -
               (2.0 * al * gfun + al * al * gprime) * lapse_src * Av[k];
    if (red) r += -al * gfun * gdAt[k] + 2.0 * al * gfun * DuA[k];
    rhs[FO_A + k] = r;
  }
  /* Eq. NR_foccz4_B^i_j (red: the mu terms) */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) {
      if (!driver) {
        rhs[FO_B + 3 * k + i] = 0.0;
        continue;
      }
      double adv = 0.0, BB = 0.0;
      for (int l = 0; l < 3; ++l) {
        adv += be[l] * dB[l][k][i];
        BB += B[k][l] * B[l][i];
      }
      double r = adv + P->f * dbb[k][i] + BB;
      if (red) {
        double m1 = 0.0, m2 = 0.0;
        for (int j = 0; j < 3; ++j) {
          m1 += ig[i][j] / ph * (dP[k][j] - dP[j][k]);
          for (int n = 0; n < 3; ++n)
            for (int l = 0; l < 3; ++l) m2 += ig[i][j] * ig[n][l] * (dD[k][l][j][n] - dD[l][k][j][n]);
        }
        r += -al * al * P->mu * m1 + al * al * P->mu * m2;
      }
      rhs[FO_B + 3 * k + i] = r;
    }
  /* the D_kij equation (red: + alpha/3 g~_ij g~^nm d_k A~_nm - 2 alpha/3 g~_ij D_k^nm A~_nm) */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        double adv = 0.0, sh = 0.0, trdB = 0.0, BD = 0.0;
        for (int l = 0; l < 3; ++l) {
          adv += be[l] * dD[l][k][i][j];
          sh += -0.5 * g[l][i] * ddbe[k][j][l] - 0.5 * g[l][j] * ddbe[k][i][l];
          trdB += ddbe[k][l][l];
          BD += B[k][l] * D[l][i][j] + B[j][l] * D[k][l][i] + B[i][l] * D[k][l][j];
        }
        sh += 1.0 / 3.0 * g[i][j] * trdB;
        double r = adv - P->s * sh - al * dAt[k][i][j] + BD - 2.0 / 3.0 * trB * D[k][i][j] -
                   Av[k] * (At[i][j] - 1.0 / 3.0 * g[i][j] * trA);
        if (red) r += al / 3.0 * g[i][j] * gdAt[k] - 2.0 * al / 3.0 * g[i][j] * DuA[k];
        rhs[FO_D + 6 * k + SYM[i][j]] = r;
      }
  /* Eq. NR_foccz4_P_i (red: + 1/3 alpha phi g~^nm d_k A~_nm - 2/3 alpha phi D_k^nm A~_nm) */
  for (int k = 0; k < 3; ++k) {
    double adv = 0.0, BP = 0.0, trdB = 0.0;
    for (int l = 0; l < 3; ++l) {
      adv += be[l] * dP[l][k];
      BP += B[k][l] * Pv[l];
      trdB += ddbe[k][l][l];
    }
    double r = adv + 1.0 / 3.0 * ph * (al * dK[k] - trdB) + BP + 1.0 / 3.0 * (al * Kt - trB) * Pv[k] +
               1.0 / 3.0 * ph * Kt * Av[k];
    if (red) r += 1.0 / 3.0 * al * ph * gdAt[k] - 2.0 / 3.0 * al * ph * DuA[k];
    rhs[FO_P + k] = r;
  }
}

/* Halo'd tile of patch n for the first nv fields of U and G (point-major,
   nv values per point). */
static void build_tile_nv(const og_grid *g, int n, const double *U, const double *G, double *tile, int nv) {
  int T = g->T, p = g->p, l = g->lev[n];
  int bx = g->ijk[3 * n] * p, by = g->ijk[3 * n + 1] * p, bz = g->ijk[3 * n + 2] * p;
  for (int lz = 0; lz < T; ++lz)
    for (int ly = 0; ly < T; ++ly)
      for (int lx = 0; lx < T; ++lx) {
        long t = ((long)lz * T + ly) * T + lx;
        for (int v = 0; v < nv; ++v)
          tile[t * nv + v] = value_at_l(g, U, G, v, l, bx + lx - OG_HALO, by + ly - OG_HALO, bz + lz - OG_HALO);
      }
}

/* The FD4 first derivative (Eq. exa_fd4_central_difference) and the
   Kreiss-Oliger sum (Eq. exa_fd4_ko) on a point-major tile of nv fields. */
static double tqn(const double *tile, long c, int nv, long off, int v) { return tile[(c + off) * nv + v]; }

static double fd1n(const double *tile, long c, const long st[3], int nv, int v, int k, double dx) {
  long s = st[k];
  return (8.0 * (tqn(tile, c, nv, s, v) - tqn(tile, c, nv, -s, v)) -
          (tqn(tile, c, nv, 2 * s, v) - tqn(tile, c, nv, -2 * s, v))) / (12.0 * dx);
}

static double ko_sumn(const double *tile, long c, const long st[3], int nv, int v, double eps, double dx) {
  double acc = 0.0;
  for (int k = 0; k < 3; ++k) {
    long s = st[k];
    double d = tqn(tile, c, nv, -3 * s, v) - 6.0 * tqn(tile, c, nv, -2 * s, v) + 15.0 * tqn(tile, c, nv, -s, v) -
               20.0 * tqn(tile, c, nv, 0, v) + 15.0 * tqn(tile, c, nv, s, v) - 6.0 * tqn(tile, c, nv, 2 * s, v) +
               tqn(tile, c, nv, 3 * s, v);
    acc += eps / (64.0 * dx) * d;
  }
  return acc;
}

/* Sommerfeld ghost cell id of the 58-variable state: the radiative
   condition of ghost_rhs for every variable, with speed somm_speed[v] for
   the primaries and 1 for the auxiliary variables. */
static void fo_ghost_rhs(const og_grid *g, const og_params *P, const double *U, const double *G, const double *Gini,
                         long id, double out[OG_NV_FO]) {
  int c[3] = {g->gcoord[3 * id], g->gcoord[3 * id + 1], g->gcoord[3 * id + 2]};
  int d = -1, side = 0;
  for (int a = 0; a < 3; ++a) {
    if (c[a] < 0) { d = a; side = -1; }
    if (c[a] >= g->N[a]) { d = a; side = +1; }
  }
  int nb[3] = {c[0], c[1], c[2]};
  nb[d] -= side;
  double xs[3];
  for (int a = 0; a < 3; ++a) xs[a] = g->origin[a] + (c[a] + 0.5) * g->dx;
  double r = sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
  for (int v = 0; v < OG_NV_FO; ++v) {
    double qg = G[(long)v * g->n_ghost + id];
    double qn = value_at(g, U, G, v, nb[0], nb[1], nb[2]);
    double dQ = side > 0 ? (qg - qn) / g->dx : (qn - qg) / g->dx;
    double cv = v < OG_NV ? P->somm_speed[v] : 1.0;
    out[v] = -cv * (r / xs[d]) * dQ - cv / r * (qg - Gini[(long)v * g->n_ghost + id]);
  }
}

/* Right-hand side of the 58 variables (Alg. fd4-fo): for every interior
   point the FD4 first derivatives of all 58, fo_point_rhs, plus the
   Kreiss-Oliger dissipation of every variable; the Sommerfeld ghost cells
   by their radiative condition. red selects the first-order formulation
   (with the red terms) or the reconstructed second-order one (without). */
int og_fo_rhs(const og_grid *g, const og_params *P, int red, const double *U, const double *G, const double *Gini,
              double *rU, double *rG) {
  const int T = g->T, p = g->p, nv = OG_NV_FO;
  const long T3 = (long)T * T * T, pts = n_interior(g);
  const long st[3] = {1, T, (long)T * T};
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * nv);
  double d1[OG_NV_FO][3];
  double q[OG_NV_FO], r[OG_NV_FO];
  for (int n = 0; n < g->n_patches; ++n) {
    build_tile_nv(g, n, U, G, tile, nv);
    const double dx = g->dxl[g->lev[n]];
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          const long c = ((long)(z + OG_HALO) * T + (y + OG_HALO)) * T + (x + OG_HALO);
          for (int v = 0; v < nv; ++v) {
            q[v] = tqn(tile, c, nv, 0, v);
            for (int k = 0; k < 3; ++k) d1[v][k] = fd1n(tile, c, st, nv, v, k, dx);
          }
          fo_point_rhs(P, red, q, (const double(*)[3])d1, r);
          const long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
          for (int v = 0; v < nv; ++v) rU[(long)v * pts + li] = r[v] + ko_sumn(tile, c, st, nv, v, P->ko_eps, dx);
        }
  }
  free(tile);
  for (long id = 0; id < g->n_ghost; ++id) {
    double rg[OG_NV_FO];
    fo_ghost_rhs(g, P, U, G, Gini, id, rg);
    for (int v = 0; v < nv; ++v) rG[(long)v * g->n_ghost + id] = rg[v];
  }
  return 0;
}

/* The reconstruction of Alg. fd4-so: the auxiliary variables of every
   interior point become the FD4 first derivatives of the primaries
   (A_k = d_k alpha, B_k^i = d_k beta^i, D_kij = 1/2 d_k g~_ij,
   P_k = d_k phi, Eq. auxiliary-variables); the ghost cells keep theirs. */
int og_fo_reconstruct(const og_grid *g, double *U, const double *G) {
  const int T = g->T, p = g->p, nv = OG_NV;
  const long T3 = (long)T * T * T, pts = n_interior(g);
  const long st[3] = {1, T, (long)T * T};
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * nv);
  double *aux = (double *)malloc(sizeof(double) * (size_t)(OG_NV_FO - OG_NV) * (size_t)pts);
  for (int n = 0; n < g->n_patches; ++n) {
    build_tile_nv(g, n, U, G, tile, nv);
    const double dx = g->dxl[g->lev[n]];
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          const long c = ((long)(z + OG_HALO) * T + (y + OG_HALO)) * T + (x + OG_HALO);
          const long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
          for (int k = 0; k < 3; ++k) {
            aux[(long)(FO_A - OG_NV + k) * pts + li] = fd1n(tile, c, st, nv, ALPHA, k, dx);
            aux[(long)(FO_P - OG_NV + k) * pts + li] = fd1n(tile, c, st, nv, PHI, k, dx);
            for (int i = 0; i < 3; ++i)
              aux[(long)(FO_B - OG_NV + 3 * k + i) * pts + li] = fd1n(tile, c, st, nv, BETAX + i, k, dx);
            for (int s = 0; s < 6; ++s)
              aux[(long)(FO_D - OG_NV + 6 * k + s) * pts + li] = 0.5 * fd1n(tile, c, st, nv, GXX + s, k, dx);
          }
        }
  }
  memcpy(U + (long)OG_NV * pts, aux, sizeof(double) * (size_t)(OG_NV_FO - OG_NV) * (size_t)pts);
  free(aux);
  free(tile);
  return 0;
}

/* One classic RK4 step of the 58-variable state (the tableau of
   og_rk4_step) over the interior points and the Sommerfeld ghost cells,
   then the algebraic enforcement of the primaries (Sec. "Evolution
   equations"; the auxiliary variables are left as they are).
   variant 0: the first-order formulation, every variable evolved with the
   red terms (Alg. fd4-fo).
   variant 1: the second-order formulation with reconstruction (Alg.
   fd4-so): before the right-hand side of every stage the auxiliary
   variables of the interior points are reconstructed from that stage's
   primaries, the red terms are removed, the interior auxiliary variables
   are not evolved, and after the step they are reconstructed from the new
   primaries. The ghost cells of the auxiliary variables follow their
   radiative condition in both variants. */
int og_fo_rk4_step(const og_grid *g, const og_params *P, int variant, double dt, double *U, double *G,
                   const double *Gini) {
  const long pts = n_interior(g), nu = pts * OG_NV_FO, ng = g->n_ghost * OG_NV_FO;
  double *k[4], *kg[4];
  for (int s = 0; s < 4; ++s) {
    k[s] = (double *)malloc(sizeof(double) * (size_t)nu);
    kg[s] = (double *)malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1));
  }
  double *Y = (double *)malloc(sizeof(double) * (size_t)nu);
  double *YG = (double *)malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1));
  const double cnode[4] = {0.0, 0.5, 0.5, 1.0};
  for (int s = 0; s < 4; ++s) {
    if (s == 0) {
      memcpy(Y, U, sizeof(double) * (size_t)nu);
      if (ng) memcpy(YG, G, sizeof(double) * (size_t)ng);
    } else {
      for (long i = 0; i < nu; ++i) Y[i] = U[i] + cnode[s] * dt * k[s - 1][i];
      for (long i = 0; i < ng; ++i) YG[i] = G[i] + cnode[s] * dt * kg[s - 1][i];
    }
    if (variant == 1) og_fo_reconstruct(g, Y, YG);
    og_fo_rhs(g, P, variant == 0, Y, YG, Gini, k[s], kg[s]);
    if (variant == 1) memset(k[s] + (long)OG_NV * pts, 0, sizeof(double) * (size_t)(nu - (long)OG_NV * pts));
  }
  for (long i = 0; i < nu; ++i) U[i] = U[i] + dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
  for (long i = 0; i < ng; ++i) G[i] = G[i] + dt / 6.0 * (kg[0][i] + 2.0 * kg[1][i] + 2.0 * kg[2][i] + kg[3][i]);
  og_enforce(g, U);
  if (variant == 1) og_fo_reconstruct(g, U, G);
  for (int s = 0; s < 4; ++s) { free(k[s]); free(kg[s]); }
  free(Y); free(YG);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* constraint norms away from the punctures                                 */
/* ------------------------------------------------------------------------ */

/* The L2 norms of Sec. "Gauge Wave" (sqrt of the mean of H^2 and of |M|^2)
   over the interior points of leaf patches whose cell centre lies at a
   distance of at least `radius` from every one of the n_c centres[3 n_c],
   from the per-point H[pts] and M[3][pts] of og_constraints (the norm that
   leaves out the region r < 1 around the punctures). out = L2 of H, L2 of
   |M|, max |H|, max |M| over those points, and their count; points with a
   non-finite H or M are left out. */
int og_constraints_excluding(const og_grid *g, const double *H, const double *M, int n_c, const double *centres,
                             double radius, double out[5]) {
  const int p = g->p;
  const long pts = n_interior(g);
  double sH = 0.0, sM = 0.0, mH = 0.0, mM = 0.0, count = 0.0;
  for (int n = 0; n < g->n_patches; ++n) {
    if (g->nchild[n] != 0) continue;
    const double h = g->dxl[g->lev[n]];
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          const double pos[3] = {g->origin[0] + (g->ijk[3 * n] * p + x + 0.5) * h,
                                 g->origin[1] + (g->ijk[3 * n + 1] * p + y + 0.5) * h,
                                 g->origin[2] + (g->ijk[3 * n + 2] * p + z + 0.5) * h};
          int near = 0;
          for (int c = 0; c < n_c; ++c) {
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) r2 += (pos[d] - centres[3 * c + d]) * (pos[d] - centres[3 * c + d]);
            if (r2 < radius * radius) near = 1;
          }
          if (near) continue;
          const long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
          const double hv = H[li];
          const double m2 = M[li] * M[li] + M[pts + li] * M[pts + li] + M[2 * pts + li] * M[2 * pts + li];
          if (!isfinite(hv) || !isfinite(m2)) continue;
          sH += hv * hv;
          sM += m2;
          if (fabs(hv) > mH) mH = fabs(hv);
          if (sqrt(m2) > mM) mM = sqrt(m2);
          count += 1.0;
        }
  }
  out[0] = count > 0.0 ? sqrt(sH / count) : 0.0;
  out[1] = count > 0.0 ? sqrt(sM / count) : 0.0;
  out[2] = mH;
  out[3] = mM;
  out[4] = count;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* psi_4 (appendix "psi_4 in ExaGRyPE")                                       */
/* ------------------------------------------------------------------------ */

static double levi(int i, int j, int k) {
  return (double)((i - j) * (j - k) * (k - i)) / 2.0;
}

/* psi_4 = (E_ij - i B_ij) mbar^i mbar^j (Eq. eq_NR_psi_code_implementation)
   at one point from its state q, derivatives d1, d2 and position X relative
   to the tetrad's centre. Written from the appendix:
   - E_ij = (R_ij - K^m_i K_jm + K_ij (K - Theta) + D_(i Z_j))^TF
     (Eq. eq_NR_psi4_E_ij, vacuum), R_ij the physical Ricci tensor of the
     metric, K_ij = (A~_ij + g~_ij K / 3) / phi^2 the physical extrinsic
     curvature, Z_i = 1/2 g~_ij (Gamma-hat^j - G~^j) as in the evolution;
   - B_ij = 1/2 (eps_mni D^m K_j^n + eps_mnj D^m K_i^n)^TF
     (Eq. eq_NR_psi4_B_ij), eps the Levi-Civita tensor of the physical metric;
   - TF the trace-free part with the physical metric;
   - the tetrad: v = (-y, x, 0), u = (x, y, z), w^i = gamma^ij eps_jkl v^k u^l,
     orthonormalised in that order by Gram-Schmidt with the physical metric;
     mbar = (w - i v) / sqrt 2 (Eq. eq_NR_psi4_m_conj).
   out[0] = Re psi_4, out[1] = Im psi_4. */
static void point_psi4(const double q[OG_NV], const double d1[OG_NV][3], const double d2[OG_NV][3][3],
                       const double X[3], double out[2]) {
  geom G;
  build_geom(q, d1, d2, &G);
  double (*g)[3] = G.g, (*ig)[3] = G.ig;
  const double ph = G.ph;
  /* physical metric and inverse */
  double gam[3][3], igam[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      gam[i][j] = g[i][j] / (ph * ph);
      igam[i][j] = ph * ph * ig[i][j];
    }
  const double sdet = sqrt(G.det) / (ph * ph * ph); /* sqrt(det gamma) */
  /* D_k^{ml} = g~^ma g~^lb D_kab (= -1/2 d_k g~^ml) */
  double Dup[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m)
      for (int l = 0; l < 3; ++l) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) s += ig[m][a] * ig[l][b] * G.D[k][a][b];
        Dup[k][m][l] = s;
      }
  double dD[3][3][3][3]; /* d_k D_ijl */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) dD[k][i][j][l] = 0.5 * d2[GXX + SYM[j][l]][k][i];
  /* physical Ricci tensor from the derivatives of the physical Christoffel
     symbols (the same route as the constraint monitor) */
  double dPG[3][3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
          for (int l = 0; l < 3; ++l) {
            s += -2.0 * Dup[k][m][l] * (G.D[i][j][l] + G.D[j][i][l] - G.D[l][i][j]);
            s += ig[m][l] * (dD[k][i][j][l] + dD[k][j][i][l] - dD[k][l][i][j]);
            s += 2.0 / ph * Dup[k][m][l] * (g[j][l] * G.P[i] + g[i][l] * G.P[j] - g[i][j] * G.P[l]);
            s += -2.0 / ph * ig[m][l] * (G.D[k][j][l] * G.P[i] + G.D[k][i][l] * G.P[j] - G.D[k][i][j] * G.P[l]);
            s += -1.0 / ph * ig[m][l] * (g[j][l] * G.ddph[k][i] + g[i][l] * G.ddph[k][j] - g[i][j] * G.ddph[k][l]);
            s += 1.0 / (ph * ph) * ig[m][l] *
                 (g[j][l] * G.P[i] * G.P[k] + g[i][l] * G.P[j] * G.P[k] - g[i][j] * G.P[k] * G.P[l]);
          }
          dPG[k][m][i][j] = s;
        }
  double Ric[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double r = 0.0;
      for (int m = 0; m < 3; ++m) {
        r += dPG[m][m][i][j] - dPG[j][m][i][m];
        for (int l = 0; l < 3; ++l) r += G.PGam[l][i][j] * G.PGam[m][l][m] - G.PGam[l][i][m] * G.PGam[m][l][j];
      }
      Ric[i][j] = r;
    }
  /* Z_i and its covariant derivative: d_k G~^j from d_k of g~^lm G~^j_lm */
  double dGt[3][3]; /* dGt[k][j] = d_k G~^j */
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          double dGjlm = 0.0; /* d_k G~^j_lm */
          for (int n = 0; n < 3; ++n) {
            dGjlm += -2.0 * Dup[k][j][n] * (G.D[l][m][n] + G.D[m][l][n] - G.D[n][l][m]);
            dGjlm += ig[j][n] * (dD[k][l][m][n] + dD[k][m][l][n] - dD[k][n][l][m]);
          }
          s += -2.0 * Dup[k][l][m] * G.Gam[j][l][m] + ig[l][m] * dGjlm;
        }
      dGt[k][j] = s;
    }
  double Gh[3], Zc[3], dZ[3][3];
  for (int i = 0; i < 3; ++i) Gh[i] = q[GHX + i];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += 0.5 * g[i][j] * (Gh[j] - G.Gc[j]);
    Zc[i] = s;
  }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int j = 0; j < 3; ++j)
        s += 0.5 * (G.dg[k][i][j] * (Gh[j] - G.Gc[j]) + g[i][j] * (d1[GHX + j][k] - dGt[k][j]));
      dZ[k][i] = s; /* d_k Z_i */
    }
  double DZ[3][3]; /* D_(i Z_j) */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.5 * (dZ[i][j] + dZ[j][i]);
      for (int k = 0; k < 3; ++k) s -= G.PGam[k][i][j] * Zc[k];
      DZ[i][j] = s;
    }
  /* extrinsic curvature: K_ij (physical, covariant) and K^n_j (mixed) */
  const double Kt = q[KTR], Th = q[THETA];
  double At[3][3], Kd[3][3], Km[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) At[i][j] = q[AXX + SYM[i][j]];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Kd[i][j] = (At[i][j] + g[i][j] * Kt / 3.0) / (ph * ph);
  for (int n = 0; n < 3; ++n)
    for (int j = 0; j < 3; ++j) {
      double s = (n == j) ? Kt / 3.0 : 0.0;
      for (int k = 0; k < 3; ++k) s += ig[n][k] * At[k][j];
      Km[n][j] = s;
    }
  /* E_ij before the trace-free part */
  double E[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double kk = 0.0; /* K^m_i K_jm = K_im K^m_j */
      for (int m = 0; m < 3; ++m) kk += Kd[i][m] * Km[m][j];
      E[i][j] = Ric[i][j] - kk + Kd[i][j] * (Kt - Th) + DZ[i][j];
    }
  /* D_l K^n_j = d_l K^n_j + Gamma^n_lp K^p_j - Gamma^p_lj K^n_p */
  double DK[3][3][3];
  for (int l = 0; l < 3; ++l)
    for (int n = 0; n < 3; ++n)
      for (int j = 0; j < 3; ++j) {
        double s = (n == j) ? d1[KTR][l] / 3.0 : 0.0;
        for (int k = 0; k < 3; ++k) s += -2.0 * Dup[l][n][k] * At[k][j] + ig[n][k] * d1[AXX + SYM[k][j]][l];
        for (int p = 0; p < 3; ++p) s += G.PGam[n][l][p] * Km[p][j] - G.PGam[p][l][j] * Km[n][p];
        DK[l][n][j] = s;
      }
  /* D^m K^n_j = gamma^ml D_l K^n_j */
  double DuK[3][3][3];
  for (int m = 0; m < 3; ++m)
    for (int n = 0; n < 3; ++n)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += igam[m][l] * DK[l][n][j];
        DuK[m][n][j] = s;
      }
  double B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n)
          s += sdet * (levi(m, n, i) * DuK[m][n][j] + levi(m, n, j) * DuK[m][n][i]);
      B[i][j] = 0.5 * s;
    }
  /* trace-free parts with the physical metric */
  double trE = 0.0, trB = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      trE += igam[i][j] * E[i][j];
      trB += igam[i][j] * B[i][j];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      E[i][j] -= gam[i][j] * trE / 3.0;
      B[i][j] -= gam[i][j] * trB / 3.0;
    }
  /* the tetrad's spatial vectors */
  double v[3] = {-X[1], X[0], 0.0}, u[3] = {X[0], X[1], X[2]}, w[3];
#define DOTG(a, b) (gam[0][0] * a[0] * b[0] + gam[1][1] * a[1] * b[1] + gam[2][2] * a[2] * b[2] + \
                    gam[0][1] * (a[0] * b[1] + a[1] * b[0]) + gam[0][2] * (a[0] * b[2] + a[2] * b[0]) + \
                    gam[1][2] * (a[1] * b[2] + a[2] * b[1]))
  double nv = sqrt(DOTG(v, v));
  for (int i = 0; i < 3; ++i) v[i] /= nv;
  double vu = DOTG(v, u);
  for (int i = 0; i < 3; ++i) u[i] -= vu * v[i];
  double nu = sqrt(DOTG(u, u));
  for (int i = 0; i < 3; ++i) u[i] /= nu;
  double wl[3]; /* eps_jkl v^k u^l */
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) s += sdet * levi(j, k, l) * v[k] * u[l];
    wl[j] = s;
  }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += igam[i][j] * wl[j];
    w[i] = s;
  }
  double vw = DOTG(v, w), uw = DOTG(u, w);
  for (int i = 0; i < 3; ++i) w[i] -= vw * v[i] + uw * u[i];
  double nw = sqrt(DOTG(w, w));
  for (int i = 0; i < 3; ++i) w[i] /= nw;
#undef DOTG
  /* (E - i B)_ij mbar^i mbar^j with mbar = (w - i v) / sqrt 2 */
  double Eww = 0.0, Evv = 0.0, Ewv = 0.0, Bww = 0.0, Bvv = 0.0, Bwv = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Eww += E[i][j] * w[i] * w[j];
      Evv += E[i][j] * v[i] * v[j];
      Ewv += E[i][j] * w[i] * v[j];
      Bww += B[i][j] * w[i] * w[j];
      Bvv += B[i][j] * v[i] * v[j];
      Bwv += B[i][j] * w[i] * v[j];
    }
  out[0] = 0.5 * (Eww - Evv) - Bwv;
  out[1] = -Ewv - 0.5 * (Bww - Bvv);
}

int og_psi4(const og_grid *g, const double *U, const double *G, const double centre[3], double *out) {
  int p = g->p, T = g->T;
  long pts = n_interior(g), T3 = (long)T * T * T;
  double *tile = (double *)malloc(sizeof(double) * (size_t)T3 * OG_NV);
  double d1[OG_NV][3], d2[OG_NV][3][3];
  for (int n = 0; n < g->n_patches; ++n) {
    const double dx = g->dxl[g->lev[n]];
    build_tile(g, n, U, G, tile);
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          tview tv;
          tv.tile = tile;
          tv.c = ((long)(z + OG_HALO) * T + (y + OG_HALO)) * T + (x + OG_HALO);
          tv.st[0] = 1; tv.st[1] = T; tv.st[2] = (long)T * T;
          double q[OG_NV], X[3], r[2];
          for (int v = 0; v < OG_NV; ++v) q[v] = tq(&tv, 0, v);
          point_derivs(&tv, dx, d1, d2);
          const int loc[3] = {x, y, z};
          for (int d = 0; d < 3; ++d)
            X[d] = g->origin[d] + ((double)g->ijk[3 * n + d] * p + loc[d] + 0.5) * dx - centre[d];
          point_psi4(q, d1, d2, X, r);
          long li = (long)n * p * p * p + ((long)z * p + y) * p + x;
          out[li] = r[0];
          out[pts + li] = r[1];
        }
  }
  free(tile);
  return 0;
}
