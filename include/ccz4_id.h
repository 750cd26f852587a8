/*
 * ccz4_id.h -- C ABI of the puncture initial-data solve (GB300 path).
 *
 * The paper initialises black holes with Bowen-York data (Sec. "Initial
 * conditions": maximal slicing K = 0, conformal flatness, extrinsic
 * curvature in closed form from the punctures' momenta P and spins S) and
 * the moving-puncture approach, which solves an elliptic equation for the
 * conformal factor; it names that equation without printing it. Written
 * out from the puncture literature:
 *
 *   g_ij = psi^4 delta_ij,  K_ij = psi^-2 Abar_ij,
 *   Abar_ij = sum_n 3/(2 r^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
 *           + 3/r^3 [eps_kil S_l n_k n_j + eps_kjl S_l n_k n_i],
 *   psi = psi_BL + u,  psi_BL = 1 + sum_n m_n / (2 r_n),
 *   Lap u + 1/8 Abar_ij Abar^ij (psi_BL + u)^-7 = 0,  u -> 0 at infinity.
 *
 * Discretisation: cell-centred n^3 cells on [-L, L]^3, h = 2L/n,
 * x_i = -L + (i + 1/2) h; the 7-point Laplacian; one ghost cell per face
 * from the 1/r fall-off rule u_ghost = u_cell * r_cell / r_ghost (r from the
 * origin). Solver: red-black nonlinear Gauss-Seidel, one Newton step per
 * cell (red = i+j+k even first; the derivative includes the boundary
 * ghosts' dependence on their cell), optionally over-relaxed. The
 * residual F is evaluated in FP64; the reciprocals of the update are an
 * FP32 estimate refined by two Newton-Raphson steps in FP64 (within a few
 * ulps of a division). Residual: max over the cells of
 * |Lap_h u + 1/8 AA (psi_BL + u)^-7|. The grid u is [n][n][n], x fastest.
 *
 * The CCZ4 state of the data (phi = psi^-2, A~_ij = psi^-6 Abar_ij,
 * g~ = delta, K = Theta = 0, Gamma-hat = 0) is assembled by the caller.
 *
 * Conventions as in ccz4.h: streams as void*, asynchronous unless stated,
 * error codes never abort, ccz4_last_error() gives the message.
 */
#ifndef CCZ4_ID_H
#define CCZ4_ID_H

#include "ccz4.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CCZ4_ID_MAX_PUNCTURES 4

typedef struct {
  int n;                                /* number of punctures, 1..4 */
  double m[CCZ4_ID_MAX_PUNCTURES];      /* bare masses */
  double c[CCZ4_ID_MAX_PUNCTURES][3];   /* positions (no cell centre may coincide with one) */
  double P[CCZ4_ID_MAX_PUNCTURES][3];   /* linear momenta */
  double S[CCZ4_ID_MAX_PUNCTURES][3];   /* spins */
} ccz4_punctures;

typedef struct ccz4_idsolver ccz4_idsolver;

/* Allocates a solver for n^3 cells (2 <= n <= 1024) on [-L, L]^3 on the
   current device; u starts at zero. */
ccz4_status ccz4_id_create(int n, double L, ccz4_idsolver **out);
ccz4_status ccz4_id_free(ccz4_idsolver *s);

/* Sets the punctures: computes Abar.Abar and psi_BL at every cell on the
   device. Does not touch u. */
ccz4_status ccz4_id_set_punctures(ccz4_idsolver *s, const ccz4_punctures *B, void *stream);

/* Device address of u ([n][n][n] doubles, owned by the solver): write an
   initial guess there, read the solution from there. */
ccz4_status ccz4_id_u_ptr(ccz4_idsolver *s, double **dev_u);

/* Relaxation factor omega of the point update u <- u - omega F / F'
   (1, the default: plain Newton-Gauss-Seidel; 1 < omega < 2: successive
   over-relaxation, far fewer sweeps). 0 < omega < 2, else CCZ4_ERR_INVALID. */
ccz4_status ccz4_id_set_relaxation(ccz4_idsolver *s, double omega);

/* n_sweeps red-black sweeps (two launches each). */
ccz4_status ccz4_id_sweeps(ccz4_idsolver *s, int n_sweeps, void *stream);

/* Max residual of the current u (synchronises the stream); res_dev, if
   not NULL, receives the residual of every cell ([n][n][n] doubles). */
ccz4_status ccz4_id_residual(ccz4_idsolver *s, double *max_res, double *res_dev, void *stream);

/* Sweeps from the current u until the max residual is below tol, checking
   every `check` sweeps (a CUDA graph of `check` sweeps is captured once per
   value of check); stops after max_sweeps. *sweeps receives the sweeps
   done, or -1 if tol was not reached; *final_res the last residual.
   Synchronises. */
ccz4_status ccz4_id_solve(ccz4_idsolver *s, double tol, int max_sweeps, int check, int *sweeps,
                          double *final_res, void *stream);

/* Writes the CCZ4 state of the data at every interior point (all levels of
   a mesh) and every Sommerfeld ghost cell of grid g into its state buffer
   `buf`: g~ = delta; alpha = ((1 - s)/(1 + s) + 1)/2 with
   s = sum m_n/(2 r_n), the averaged lapse of the paper's binary setup;
   beta = b = 0; phi = psi^-2 with psi = psi_BL + u, u interpolated from the
   solver grid by tricubic Lagrange interpolation (along each axis the four
   cell centres around the point, shifted inwards at the faces; x, then y,
   then z); A~_ij = psi^-6 Abar_ij; K = Theta = 0; Gamma-hat = 0. Points of g
   should lie inside [-L, L]^3 (outside, the outermost stencil
   extrapolates). Asynchronous. */
ccz4_status ccz4_id_assemble(ccz4_idsolver *s, const ccz4_punctures *B, ccz4_grid *g, int buf, void *stream);

/* Nested boxes (a reading: the paper solves for the conformal factor on
   its mesh without printing how; a coarse global solve fed to levels 20x
   finer under-resolves u near the punctures). Makes s a box inside the
   solver `parent`: from now on the ghost cells of s hold fixed values, the
   parent's current u interpolated (tricubic, as ccz4_id_assemble) at their
   centres, and a fixed ghost adds nothing to the Newton derivative. The
   values are taken now (later changes of the parent's u do not reach s).
   init_u != 0 also sets u of s to the parent's u interpolated at its cell
   centres (a first guess). Both solvers need their punctures set; the box
   [-L, L]^3 of s, ghost cells included (L + h/2 <= L_parent), must lie
   inside the parent's, else CCZ4_ERR_INVALID. parent NULL restores the 1/r
   fall-off rule. The ghost array (6 n^2 doubles) is allocated on the first
   call and owned by s. Asynchronous; synchronises the stream if a
   captured solve graph must be dropped. */
ccz4_status ccz4_id_set_parent(ccz4_idsolver *s, const ccz4_idsolver *parent, int init_u, void *stream);

/* As ccz4_id_assemble, but writes only the points (interior and ghost) of
   g whose every coordinate satisfies |x_d| < L - 3h/2, where the tricubic
   stencil is centred; other points keep their values. Assembling the
   outermost solver with ccz4_id_assemble and then each nested box, coarse
   to fine, with this call gives every point its data from the finest box
   that covers it. Asynchronous. */
ccz4_status ccz4_id_assemble_box(ccz4_idsolver *s, const ccz4_punctures *B, ccz4_grid *g, int buf, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CCZ4_ID_H */
