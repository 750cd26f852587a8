/*
 * Bowen-York puncture initial data: plain FP64 CPU restatement (oracle).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: only the test
 * suite, the smoke check and the CPU legs of bench.py load it; the CUDA
 * path never does.
 *
 * The paper initialises black holes with Bowen-York data (Sec. "Initial
 * conditions": maximal slicing K = 0, conformal flatness, extrinsic
 * curvature in closed form from the punctures' momenta and spins) and the
 * moving-puncture approach, where an elliptic equation gives the conformal
 * factor; it does not print that equation. Written out from the puncture
 * literature it cites:
 *
 *   physical metric  g_ij = psi^4 delta_ij,  K_ij = psi^-2 Abar_ij,
 *   Abar_ij = sum_n 3/(2 r^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
 *           + 3/r^3 [eps_kil S_l n_k n_j + eps_kjl S_l n_k n_i]
 *   (r, n: distance and unit vector from puncture n), and the Hamiltonian
 *   constraint  Lap psi + 1/8 psi^-7 Abar_ij Abar^ij = 0  with the puncture
 *   split  psi = 1 + sum_n m_n / (2 r_n) + u,  u regular, u -> 0 at infinity:
 *
 *       Lap u + 1/8 Abar_ij Abar^ij (psi_BL + u)^-7 = 0.
 *
 * Discretisation (a reading; the paper prints none): cell-centred n^3
 * cells on [-L, L]^3, h = 2L/n, x_i = -L + (i + 1/2) h; the 7-point
 * Laplacian; one ghost cell per face from the 1/r fall-off (Robin) rule
 * u_ghost = u_cell * r_cell / r_ghost (r from the origin). The solver is
 * red-black nonlinear Gauss-Seidel with one Newton step per point; the
 * residual is max |Lap_h u + 1/8 AA (psi_BL + u)^-7| over the cells.
 *
 * Arrays u, res: [n][n][n] with x fastest.
 */
#ifndef BOWEN_YORK_ORACLE_H
#define BOWEN_YORK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OG_BY_MAX_PUNCTURES 4

typedef struct {
  int n;                               /* number of punctures, 1..4 */
  double m[OG_BY_MAX_PUNCTURES];       /* bare masses */
  double c[OG_BY_MAX_PUNCTURES][3];    /* positions */
  double P[OG_BY_MAX_PUNCTURES][3];    /* linear momenta */
  double S[OG_BY_MAX_PUNCTURES][3];    /* spins */
} og_punctures;

/* Abar_ij at (x, y, z): A[6] = xx, xy, xz, yy, yz, zz. */
void og_by_abar(const og_punctures *B, double x, double y, double z, double A[6]);
/* Abar_ij Abar^ij (indices moved with delta). */
double og_by_aa(const og_punctures *B, double x, double y, double z);
/* psi_BL = 1 + sum m_n / (2 r_n). */
double og_by_psi_bl(const og_punctures *B, double x, double y, double z);

/* Array form of the three above over m points: A[m][6], aa[m], psi[m]. */
void og_by_points(const og_punctures *B, long m, const double *x, const double *y, const double *z, double *A,
                  double *aa, double *psi);

/* Residual of the discrete equation at every cell; returns max |res|. */
double og_by_residual(const og_punctures *B, int n, double L, const double *u, double *res);
/* n_sweeps red-black Newton-Gauss-Seidel sweeps (red: i+j+k even, first),
   each point update scaled by the relaxation factor omega (1: plain
   Gauss-Seidel; 1 < omega < 2: successive over-relaxation). */
void og_by_sweeps(const og_punctures *B, int n, double L, double *u, int n_sweeps, double omega);
/* Sweeps until the max residual is below tol, checked every `check`
   sweeps; returns the number of sweeps done (or -1 if max_sweeps is hit).
   *final_res receives the last residual. */
int og_by_solve(const og_punctures *B, int n, double L, double *u, double tol, int max_sweeps, int check,
                double omega, double *final_res);

/* Nested boxes (a reading; the paper prints none): a finer solve on n^3
   cells of a box [-L, L]^3 inside a coarser (parent) solve on np^3 cells
   of [-Lp, Lp]^3 takes fixed (Dirichlet) ghost values, the parent's u
   interpolated (og_by_interp) at the centres of its ghost cells; a fixed
   ghost adds nothing to the Newton derivative. Ghost arrays are
   gb[6][n][n]: face 2 d (the ghosts at index -1 along axis d) or 2 d + 1
   (index n), then the two other cell indices, the lower axis fastest. */
void og_by_box_ghosts(int n, double L, int np, double Lp, const double *up, double *gb);
/* The parent's u interpolated at the n^3 cell centres of the box (a first
   guess). */
void og_by_cells_from(int n, double L, int np, double Lp, const double *up, double *u);
/* og_by_residual, og_by_sweeps and og_by_solve of a box with fixed ghosts
   gb (NULL: the 1/r fall-off rule, as the functions above). */
double og_by_residual_box(const og_punctures *B, int n, double L, const double *u, const double *gb,
                          double *res);
void og_by_sweeps_box(const og_punctures *B, int n, double L, double *u, const double *gb, int n_sweeps,
                      double omega);
int og_by_solve_box(const og_punctures *B, int n, double L, double *u, const double *gb, double tol,
                    int max_sweeps, int check, double omega, double *final_res);

/* Tricubic Lagrange interpolation of u (n^3 cells of [-L, L]^3) at m
   points: along each axis the four cell centres around the point (the
   stencil is shifted inwards at the faces), weights of the cubic through
   them, applied along x, then y, then z. Points outside the cell-centre
   range extrapolate from the outermost stencil. */
void og_by_interp(int n, double L, const double *u, long m, const double *x, const double *y, const double *z,
                  double *out);
/* The 25 CCZ4 fields of the data at m points (Q[25][m], field order of the
   CCZ4 oracle): g~ = delta, alpha = the averaged lapse
   (1 - s)/(1 + s)/2 + 1/2 with s = sum m_n/(2 r_n), beta = b = 0,
   phi = psi^-2 with psi = psi_BL + u (u interpolated as above),
   A~_ij = psi^-6 Abar_ij, K = Theta = 0, Gamma-hat = 0. */
void og_by_state(const og_punctures *B, int n, double L, const double *u, long m, const double *x,
                 const double *y, const double *z, double *Q);

#ifdef __cplusplus
}
#endif
#endif
