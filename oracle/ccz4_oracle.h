/*
 * CCZ4 oracle: plain, slow, FP64 CPU restatement of the fourth-order
 * finite-difference CCZ4 method of the ExaGRyPE paper (arXiv 2406.11626).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check of the
 * package entry point and the CPU-baseline leg of bench.py may load this
 * library. The CUDA path never calls it, includes it or links it: the two
 * share no code, and no product code path falls back to it.
 *
 * Layout of the arrays this API exchanges (the "canonical" layout; the
 * oracle's internal working layout is its own):
 *   U     [25][n_patches][p][p][p]   interior points, x fastest, fields in the
 *                                    order listed below, patches in the
 *                                    order of the ijk array
 *   G     [25][n_ghost]              ghost-shell points (Sommerfeld only),
 *                                    ghost cells in lexicographic order of
 *                                    their global (z, y, x) coordinates
 *   tiles [25][n_patches][p+6]^3     each patch with its halo of width 3
 *
 * Field order (the primary variables of the second-order formulation, Eq.
 * second-order-variables, 25 of them):
 *   0..5 conformal metric g~ (xx,xy,xz,yy,yz,zz), 6 lapse alpha,
 *   7..9 shift beta^i, 10 conformal factor phi, 11..16 A~ (xx..zz), 17 K,
 *   18 Theta, 19..21 Gamma-hat^i, 22..24 b^i.
 */
#ifndef CCZ4_ORACLE_H
#define CCZ4_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OG_NV 25
#define OG_NV_FO 58
#define OG_HALO 3
#define OG_MAX_LEVELS 8

enum { OG_BC_PERIODIC = 0, OG_BC_COPY = 1, OG_BC_SOMMERFELD = 2 };
enum { OG_SLICING_HARMONIC = 0, OG_SLICING_ONE_PLUS_LOG = 1 };
enum { OG_SHIFT_ZERO = 0, OG_SHIFT_GAMMA_DRIVER = 1 };

typedef struct {
  double kappa1, kappa2, kappa3, e, c, tau, mu, f, eta, s, K0, ko_eps;
  int slicing; /* OG_SLICING_* */
  int shift;   /* OG_SHIFT_* */
  double somm_speed[OG_NV];
} og_params;

typedef struct og_grid og_grid;

og_grid *og_grid_new(int p, int np0, int np1, int np2, int n_patches, const int *ijk,
                     double ox, double oy, double oz, double dx, int bc);
/* Statically refined mesh (appendix "refinement transition"): patches with
   level[n] == 0 cover the np0 x np1 x np2 slots of the base grid (spacing
   dx); a patch of level l >= 1 has spacing dx / 3^l (divided by 3.0 once
   per level) and slot coordinates ijk in units of its own level, and is one
   of the 27 children (slot / 3) of a level l-1 patch that has all 27. Halo
   points a refined level does not cover are interpolated from the level
   below, which must hold them as interior points. NULL if the description
   breaks any of these rules. */
og_grid *og_mesh_new(int p, int np0, int np1, int np2, int n_patches, const int *level,
                     const int *ijk, double ox, double oy, double oz, double dx, int bc);
int og_n_levels(const og_grid *g);
/* In place: coarse points under refined patches <- mean of their 27 fine cells. */
int og_restrict(const og_grid *g, double *U);
void og_grid_free(og_grid *g);
long og_n_ghost(const og_grid *g);
void og_ghost_coords(const og_grid *g, int *out /* [n_ghost][3] (x,y,z) */);

int og_fill_tiles(const og_grid *g, const double *U, const double *G, double *tiles);
int og_rhs(const og_grid *g, const og_params *P, const double *U, const double *G,
           const double *Gini, double *rU, double *rG);
int og_ghost_rhs(const og_grid *g, const og_params *P, const double *U, const double *G,
                 const double *Gini, double *rG);
int og_rk4_step(const og_grid *g, const og_params *P, double dt, double *U, double *G,
                const double *Gini);
int og_enforce(const og_grid *g, double *U);
int og_constraints(const og_grid *g, const double *U, const double *G, double *H,
                   double *M, double out[5]);
int og_rhs_points(const og_grid *g, const og_params *P, const double *U, const double *G,
                  long n, const long *pts, double *out /* [n][25] */);
int og_constraints_points(const og_grid *g, const double *U, const double *G, long n,
                          const long *pts, double *out /* [n][4] = H, M_x, M_y, M_z */);
int og_point_derivs(const og_grid *g, const double *U, const double *G, long pt,
                    double ko_eps, double *d1 /* [25][3] */, double *d2 /* [25][3][3] */,
                    double *ko /* [25] */);

/* L2 norms of H and |M| over the interior points of leaf patches at a
   distance >= radius from every one of the n_c centres (from og_constraints'
   per-point H and M): out = L2 H, L2 |M|, max |H|, max |M|, point count. */
int og_constraints_excluding(const og_grid *g, const double *H, const double *M, int n_c, const double *centres,
                             double radius, double out[5]);

/* psi_4 at every interior point (appendix "psi_4 in ExaGRyPE": Eqs.
   eq_NR_psi4_E_ij, eq_NR_psi4_B_ij, eq_NR_psi4_m_conj,
   eq_NR_psi_code_implementation), the tetrad built from each point's
   position relative to centre[3]: out[0][n_points] = Re psi_4,
   out[1][n_points] = Im psi_4. Derivatives as in og_constraints. */
int og_psi4(const og_grid *g, const double *U, const double *G, const double centre[3], double *out);

/* First-order formulation (Eq. first-order-variables): arrays of 58
   fields, the 25 primaries followed by A_k (25..27), B_k^i (28 + 3k + i),
   D_kij (37 + 6k + pair(i,j)) and P_k (55..57), in the layouts above with
   58 in place of 25. og_fo_rhs: red = 1 the first-order right-hand side
   with the red terms, 0 without them. og_fo_reconstruct: the auxiliary
   variables of the interior points from FD4 derivatives of the primaries.
   og_fo_rk4_step: variant 0 first-order, 1 second-order with the
   reconstruction of Alg. fd4-so. */
int og_fo_rhs(const og_grid *g, const og_params *P, int red, const double *U, const double *G,
              const double *Gini, double *rU, double *rG);
int og_fo_reconstruct(const og_grid *g, double *U, const double *G);
int og_fo_rk4_step(const og_grid *g, const og_params *P, int variant, double dt, double *U, double *G,
                   const double *Gini);

/* Particle tracers: trilinear projection of the fields at each of n
   positions pos[n][3] (values[n][25], may be NULL) and, for vel_field >= 0,
   one explicit Euler move by dt * vel_scale times the projected fields
   vel_field .. vel_field + 2. Returns the number of tracers that could not
   be projected (left in place, NaN values). */
long og_tracers_step(const og_grid *g, const double *U, const double *G, long n, double *pos, double dt,
                     int vel_field, double vel_scale, double *values);

#ifdef __cplusplus
}
#endif
#endif
