/*
 * ccz4.h -- C ABI of the GB300 CCZ4 finite-difference hot path.
 *
 * The library evolves the second-order CCZ4 formulation of the Einstein
 * equations (ExaGRyPE paper, arXiv 2406.11626, appendix "Spacetime
 * foliation": the nine primary evolution equations with the red terms
 * removed) on p^3 Cartesian patches with a halo of width 3 -- one uniform
 * level, or a statically refined mesh of ratio-3 levels -- discretised by fourth-order central finite differences with
 * Kreiss-Oliger dissipation (appendix "Formulation for the kernel FD4
 * Solver") and classic RK4 in time (Sec. "Finite Differences"). Beside it:
 * the first-order formulation and the second order with reconstructed
 * auxiliary variables over 58 variables (ccz4_fo_*), particle tracers and
 * puncture trackers (ccz4_tracers_*), and the constraint monitors. All work
 * runs in CUDA kernels on the current device; there is no CPU fallback.
 *
 * Conventions for every call
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream). Every call is asynchronous on that stream unless its
 *    comment says it synchronises.
 *  - Errors: a call returns CCZ4_OK or an error code and never aborts or
 *    traps. Argument errors are caught on the host before any launch
 *    (CCZ4_ERR_INVALID). Device-side faults of the data (for example a
 *    non-finite constraint value) are reported by the synchronising calls.
 *    ccz4_last_error() returns a message for the last failing call of the
 *    calling thread.
 *  - Ownership: a ccz4_grid owns every device buffer it allocates; host
 *    arrays passed in are read (or written) during the call only and stay
 *    owned by the caller.
 *  - Fields (25, the primary variables of Eq. second-order-variables), in
 *    this order: conformal metric g~_xx, g~_xy, g~_xz, g~_yy, g~_yz, g~_zz;
 *    lapse alpha; shift beta^x, beta^y, beta^z; conformal factor phi;
 *    A~_xx, A~_xy, A~_xz, A~_yy, A~_yz, A~_zz; K; Theta; Gamma-hat^x,y,z;
 *    b^x, b^y, b^z.
 *  - Points: cell-centred, x = origin + (i + 1/2) dx (Sec. "Finite
 *    Differences": samples at the centres of the patch volumes).
 *  - Device state layout ("SoA"): a state buffer holds 25 fields of
 *    `field_stride` doubles each. Within a field, the interior points come
 *    first, patch after patch in the order of the descriptor's ijk array,
 *    each patch as [z][y][x] with x fastest (n_points = n_patches * p^3);
 *    then, for Sommerfeld boundaries, the n_ghost evolved ghost cells: every
 *    cell within 3 points of the domain and outside it, in lexicographic
 *    (z, y, x) order of its global integer coordinates. Host arrays use the
 *    same order without padding: U[25][n_points] and G[25][n_ghost].
 *  - Halo tiles (CCZ4_BUF_TILE): [25][n_patches][(p+6)^3], each patch with
 *    its width-3 halo, [z][y][x] with x fastest, local index l = patch
 *    point index + 3. 8 bytes per entry: the FP64 value, except after a
 *    mixed-precision fill (ccz4_fill_halos_for), where every field but
 *    alpha and phi holds the split pair {hi, lo} of the value as two FP32
 *    numbers (hi first): hi = the value rounded to FP32, lo = the value
 *    minus hi rounded to FP32.
 */
#ifndef CCZ4_H
#define CCZ4_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCZ4_NV 25
#define CCZ4_HALO 3

typedef enum {
  CCZ4_OK = 0,
  CCZ4_ERR_INVALID = 1,   /* bad argument; nothing was launched */
  CCZ4_ERR_NOMEM = 2,     /* a device or host allocation failed */
  CCZ4_ERR_CUDA = 3,      /* a CUDA call failed (message in ccz4_last_error) */
  CCZ4_ERR_NONFINITE = 4, /* non-finite values found by ccz4_constraints */
  CCZ4_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
  CCZ4_ERR_BOUNDS = 6     /* a kernel met an index outside its buffers */
} ccz4_status;

/* Boundary kinds (Sec. "Boundary Treatment"). PERIODIC wraps the domain.
   COPY is the homogeneous Neumann condition Q_out = Q_in filled layer by
   layer outward, so every ghost point equals the nearest interior point.
   SOMMERFELD keeps the ghost cells as evolved state and advances them with
   the radiative condition of Eq. SommerfeldBC_v1, discretised as in Eq.
   exa_sommerfeld_inter (a ghost cell outside in several directions belongs
   to its highest outside axis, z before y before x). */
enum { CCZ4_BC_PERIODIC = 0, CCZ4_BC_COPY = 1, CCZ4_BC_SOMMERFELD = 2 };

/* Slicing function g(alpha) of Eq. NR_foccz4_lapse_gauge: 1 (harmonic) or
   2/alpha ("1+log"). */
enum { CCZ4_SLICING_HARMONIC = 0, CCZ4_SLICING_ONE_PLUS_LOG = 1 };

/* Shift condition: zero (static) shift, or the Gamma-driver of Eqs.
   NR_foccz4_shift_gauge and NR_foccz4_b^i. */
enum { CCZ4_SHIFT_ZERO = 0, CCZ4_SHIFT_GAMMA_DRIVER = 1 };

/* Arithmetic of the pointwise CCZ4 algebra. FP64: everything in double.
   MIXED: state, RK accumulation, finite differences and the terms with
   1/phi in double; the rest of the pointwise algebra in single. */
enum { CCZ4_PREC_FP64 = 0, CCZ4_PREC_MIXED = 1 };

/* Device buffers of a grid. U: the state U_n. Y0, Y1: RK stage states.
   ACC: RK accumulator. RHS: output of ccz4_rhs. INI: Q_ini of the
   Sommerfeld condition (ghost part only is used). TILE: halo tiles. The
   state-shaped buffers (U, Y0, Y1, ACC, RHS, INI) share one layout.
   MIX: [33][n_points] mixed second derivatives written by ccz4_fill_halos
   with the tiles: for g~_xx..g~_zz (slots 0..17), alpha (18..20),
   beta^x..beta^z (21..29) and phi (30..32), three slots each in the order
   d_x d_y, d_x d_z, d_y d_z. */
enum {
  CCZ4_BUF_U = 0, CCZ4_BUF_Y0 = 1, CCZ4_BUF_Y1 = 2, CCZ4_BUF_ACC = 3,
  CCZ4_BUF_RHS = 4, CCZ4_BUF_INI = 5, CCZ4_BUF_TILE = 6, CCZ4_BUF_MIX = 7
};

typedef struct {
  int p;              /* points per patch edge, 1..18 (the halo'd tile of one
                         field, (p+6)^3 doubles, is staged in shared memory) */
  int np[3];          /* patch slots per axis; the domain has np[d]*p points along d */
  int n_patches;      /* must equal np[0]*np[1]*np[2]: the patches cover the domain */
  const int *ijk;     /* host [n_patches][3] integer patch coordinates, each slot once */
  double origin[3];   /* lower corner of the domain */
  double dx;          /* grid spacing, > 0, the same along every axis */
  int bc;             /* CCZ4_BC_* for the whole outer boundary */
} ccz4_grid_desc;

/* Physical and numerical parameters (appendix "Spacetime foliation":
   kappa1, kappa2, kappa3, e, c, tau, mu, f, eta, s, K0; Eq. exa_fd4_ko:
   the dissipation strength epsilon). mu enters only the first-order
   formulation (ccz4_fo_*). somm_speed is the wave speed c of the
   Sommerfeld condition per field. */
typedef struct {
  double kappa1, kappa2, kappa3, e, c, tau, mu, f, eta, s, K0, ko_eps;
  int slicing;        /* CCZ4_SLICING_* */
  int shift;          /* CCZ4_SHIFT_* */
  double somm_speed[CCZ4_NV];
  int precision;      /* CCZ4_PREC_* */
} ccz4_params;

typedef struct ccz4_grid ccz4_grid;

/* Creates a grid on the current device and allocates its buffers (Sec.
   "Spatial Discretisation": p^3 patches with K = 3 halo layers). The
   descriptor and its ijk array are copied. Buffers start zeroed. On error
   *out is set to NULL. */
ccz4_status ccz4_alloc_patches(const ccz4_grid_desc *desc, ccz4_grid **out);

/* Device-memory allocator for the large buffers of grids created from now
   on (the CCZ4_BUF_* state buffers, the halo tiles and the mixed
   derivatives of ccz4_alloc_patches and ccz4_alloc_mesh), so that a host
   framework's caching allocator can supply them: alloc(ctx, bytes, stream)
   returns a device pointer (aligned to 256 bytes, like cudaMalloc) or NULL
   on failure; dealloc(ctx, ptr, bytes, stream) releases one. stream is
   NULL (the legacy default stream): the library synchronises the device
   before it releases a grid. A grid keeps the allocator it was created with
   until it is released. Both NULL restores cudaMalloc / cudaFree; one NULL
   is CCZ4_ERR_INVALID. Process-wide; not to be called while another thread
   creates a grid. Small tables and scratch keep cudaMalloc. */
typedef void *(*ccz4_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*ccz4_dealloc_fn)(void *ctx, void *ptr, size_t bytes, void *stream);
ccz4_status ccz4_set_allocator(ccz4_alloc_fn alloc, ccz4_dealloc_fn dealloc, void *ctx);

/* Releases every buffer of the grid (synchronises the device). NULL is a no-op. */
ccz4_status ccz4_free_patches(ccz4_grid *g);

/* Sizes: interior points (n_patches * p^3), ghost cells (0 unless
   Sommerfeld) and the field stride of the state buffers, in doubles. */
ccz4_status ccz4_grid_info(const ccz4_grid *g, long long *n_points, long long *n_ghost,
                           long long *field_stride);

/* Device address of buffer `buf` (CCZ4_BUF_*) and its size in doubles.
   The grid keeps ownership. */
ccz4_status ccz4_field_ptr(ccz4_grid *g, int buf, double **dev, long long *n_doubles);

/* Copies host arrays U[25][n_points] and (Sommerfeld only, may be NULL
   otherwise) G[25][n_ghost] into a state-shaped buffer, or back. Both
   synchronise the stream before returning (the host arrays may be reused
   at once). Host arrays in pinned memory that the device can address are
   moved by a copy kernel over the CPU-GPU link, any other host memory by
   the copy engine; the environment variable CCZ4_HOST_COPY=dma selects the
   copy engine always. */
ccz4_status ccz4_upload(ccz4_grid *g, int buf, const double *U, const double *G, void *stream);
ccz4_status ccz4_download(ccz4_grid *g, int buf, double *U, double *G, void *stream);

/* Halo fill (Sec. "Spatial Discretisation", Fig. patch-face-reconstruction:
   each patch is glued with the data of its neighbours into a
   (p+2K)^3 tile). Writes CCZ4_BUF_TILE from the state-shaped buffer `buf`:
   interior points from their owning patch, points outside the domain by
   the boundary kind (periodic wrap, copy of the nearest interior point,
   or the Sommerfeld ghost cell). Faces, edges and corners are all filled.
   While a field's tile is at hand it also writes the FD4 mixed second
   derivatives of g~, alpha, beta and phi (the tensor product of two
   first-derivative stencils) into CCZ4_BUF_MIX. */
ccz4_status ccz4_fill_halos(ccz4_grid *g, int buf, void *stream);

/* The halo fill as the stage kernel for parameters P needs it. For
   P->precision == CCZ4_PREC_MIXED the tiles of every field but alpha and
   phi hold split FP32 pairs (see the TILE layout above), on which the
   mixed stage kernel takes its stencil differences with the accuracy of
   FP64 differences. The mixed derivatives that the mixed stage kernel uses
   in FP32 -- those of g~ and beta -- take their inner differences on the
   same pairs and everything else in FP32, and are stored as FP32 in the
   first 27 x n_points floats of CCZ4_BUF_MIX (g~'s 18 slots, then beta's
   9); those of alpha and phi stay FP64 in their slots (and their tiles
   FP64). Otherwise the buffers equal ccz4_fill_halos'. A mixed-precision
   ccz4_rk_stage must follow this fill (ccz4_rhs, ccz4_step and
   ccz4_step_graph fill this way). */
ccz4_status ccz4_fill_halos_for(ccz4_grid *g, int buf, const ccz4_params *P, void *stream);

/* Right-hand side d_t Q of the second-order CCZ4 system (appendix
   "Spacetime foliation", Eqs. NR_foccz4_gamma_ij ... NR_foccz4_b^i, closed
   by the listed relations and Eq. NR_foccz4_modified_ricci) plus the
   Kreiss-Oliger term of Eq. exa_fd4_ko summed over x, y, z, at every
   interior point, and the Sommerfeld right-hand side at every ghost cell.
   Fills the halos of `in_buf` first (the TILE buffer is overwritten) and
   writes `out_buf`. in_buf and out_buf must differ. */
ccz4_status ccz4_rhs(ccz4_grid *g, const ccz4_params *P, int in_buf, int out_buf, void *stream);

/* One stage s = 0..3 of classic RK4 (weights 1/6, 1/3, 1/3, 1/6; nodes
   0, 1/2, 1/2, 1), the paper's compute kernel applied to every patch. The
   halo fill is a separate step (the paper merges patch and halo before the
   kernel runs): CCZ4_BUF_TILE and CCZ4_BUF_MIX must hold the halo'd stage
   input and its mixed derivatives, i.e.
   ccz4_fill_halos must have been called on the buffer that
   ccz4_stage_buffers names as the input of stage s (U, Y0, Y1, Y0 for
   s = 0, 1, 2, 3). The kernel evaluates the right-hand side k_s and applies
   the update in the same pass:
     s = 0: ACC = k0,        Y0 = U + dt/2 k0
     s = 1: ACC += 2 k1,     Y1 = U + dt/2 k1
     s = 2: ACC += 2 k2,     Y0 = U + dt k2
     s = 3: U = U + dt/6 (ACC + k3), then the algebraic constraints are
            enforced at every interior point (Sec. "Evolution equations":
            g~ rescaled to unit determinant, then the trace of A~ removed).
   Sommerfeld ghost cells are advanced by the same stage formulas. The four
   stages in order, each after its halo fill, make one time step of size dt. */
ccz4_status ccz4_rk_stage(ccz4_grid *g, const ccz4_params *P, int stage, double dt, void *stream);

/* Input and output buffers (CCZ4_BUF_*) of RK stage s = 0..3. */
ccz4_status ccz4_stage_buffers(int stage, int *in_buf, int *out_buf);

/* n_steps full RK4 steps on U: for each stage, ccz4_fill_halos of the
   stage input followed by ccz4_rk_stage. */
ccz4_status ccz4_step(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps, void *stream);

/* n_steps RK4 steps on U, like ccz4_step, replayed from a CUDA graph of one
   step. The graph is captured on a private stream the first time, and again
   whenever the parameters or dt differ from the captured ones; capturing
   synchronises `stream` first. The graph then runs on `stream`. Results are
   bit-identical to ccz4_step. */
ccz4_status ccz4_step_graph(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps, void *stream);

/* End-to-end call from host memory: uploads U (and G) into CCZ4_BUF_U,
   runs n_steps RK4 steps, downloads the result into U_out (and G_out),
   and synchronises. In and out arrays may alias. */
ccz4_status ccz4_evolve_host(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps,
                             const double *U_in, const double *G_in, double *U_out,
                             double *G_out, void *stream);

/* Algebraic constraint enforcement alone, in place on a state buffer
   (interior points). */
ccz4_status ccz4_enforce(ccz4_grid *g, int buf, void *stream);

/* Constraint monitors of the state in `buf` (Eqs. hamilton_constraints and
   momentum_constraints, vacuum): fills its halos, evaluates H and the
   covariant M_i at every interior point, writes them to dev_H[n_points] and
   dev_M[3][n_points] when those device pointers are not NULL, and reduces
   (Sec. "Gauge Wave": L2 = sqrt(sum H^2 / n) over the n interior points):
     out[0] = L2 of H, out[1] = L2 of |M| with |M|^2 = sum_i M_i^2,
     out[2] = max |H|, out[3] = max |M|, out[4] = number of points where H
     or M is not finite (those points are left out of the sums).
   The reduction runs in a fixed order, so repeated calls give identical
   results. Synchronises the stream; returns CCZ4_ERR_NONFINITE when
   out[4] > 0 (out is still filled). */
ccz4_status ccz4_constraints(ccz4_grid *g, int buf, double out[5], double *dev_H, double *dev_M,
                             void *stream);

/* The constraint norms away from the punctures (Sec. "Gauge Wave" for the
   L2 norm; the puncture region r < 1 of Sec. "Single black hole" left
   out): from the per-point H [n_points] and M [3][n_points] on the device,
   as ccz4_constraints writes them for this grid, the L2 norms of H and |M|
   (sqrt of the mean of the squares), max |H| and max |M| over the interior
   points of leaf patches whose cell centre lies at a distance of at least
   `radius` from every one of the n_centres centres (host [n_centres][3],
   at most CCZ4_MAX_EXCLUDED), and in out[4] the number of those points.
   Points with a non-finite H or M are left out. The reduction runs in a
   fixed order (repeated calls agree bit for bit). Synchronises the stream.
   CCZ4_ERR_INVALID for missing arrays, too many centres or a negative
   radius. */
#define CCZ4_MAX_EXCLUDED 8
ccz4_status ccz4_constraints_excluding(ccz4_grid *g, const double *dev_H, const double *dev_M, int n_centres,
                                       const double *centres, double radius, double out[5], void *stream);

/* psi_4 (appendix "psi_4 in ExaGRyPE"; Sec. "Gravitational waves" for
   its use): the Newman-Penrose scalar psi_4 = (E_ij - i B_ij) mbar^i mbar^j
   (Eq. eq_NR_psi_code_implementation) at every interior point of every
   level, from the state in buffer in_buf, with
     E_ij = (R_ij - K^m_i K_jm + K_ij (K - Theta) + D_(i Z_j))^TF and
     B_ij = 1/2 (eps_mni D^m K_j^n + eps_mnj D^m K_i^n)^TF
   (Eqs. eq_NR_psi4_E_ij, eq_NR_psi4_B_ij, vacuum), R_ij the physical Ricci
   tensor, K_ij = (A~_ij + g~_ij K / 3) / phi^2, Z_i = 1/2 g~_ij
   (Gamma-hat^j - G~^j), eps the Levi-Civita tensor and TF the trace-free
   part, both of the physical metric g~_ij / phi^2; mbar = (w - i v) / sqrt 2
   with v, u, w the Gram-Schmidt orthonormalisation (physical metric, in
   that order) of (-y, x, 0), (x, y, z) and gamma^ij eps_jkl v^k u^l, the
   coordinates taken relative to centre[3] (host). FD4 stencils as in the
   stage kernel, FP64. Writes Re psi_4 into field 0 and Im psi_4 into field
   1 of state buffer out_buf at every interior point; its other fields and
   its ghost cells keep their values (static tracers, vel_field = -1, then
   sample psi_4 anywhere, e.g. on an extraction sphere). Overwrites
   CCZ4_BUF_TILE and CCZ4_BUF_MIX (the halo fill of in_buf). in_buf and
   out_buf must be different state buffers (CCZ4_ERR_INVALID otherwise).
   Asynchronous. */
ccz4_status ccz4_psi4(ccz4_grid *g, int in_buf, int out_buf, const double centre[3], void *stream);

/* Where lattice points live in a state buffer: for each of n points given
   by their global lattice indices (x, y, z) (single uniform level; point
   (x, y, z) is the cell centre origin + (x + 1/2, y + 1/2, z + 1/2) dx),
   index[q] receives the position of the point's value within a field of a
   state buffer: field v of buffer b at (field_ptr of b) + v * field_stride
   + index[q]. Points outside the domain resolve as the halo fill resolves
   them (Sec. "Spatial Discretisation": periodic grids wrap, copy grids
   clamp, Sommerfeld grids map the HALO = 3 layers outside the domain to
   their ghost cells). A point that resolves to nothing (beyond a
   Sommerfeld grid's ghost shell) gets -1; the call then fills every other
   entry and returns CCZ4_ERR_BOUNDS, raised by the same device-side bounds
   check that guards the halo fill, with a status word of its own (the
   grid's own status, which ccz4_constraints reports, is not touched).
     xyz    host [n][3] ints; index host [n]; 0 <= n <= 2^20.
   A refined mesh or invalid arguments: CCZ4_ERR_INVALID. Allocates and
   frees device memory for the points; synchronises the stream. */
ccz4_status ccz4_point_index(ccz4_grid *g, int n, const int *xyz, long long *index, void *stream);

/* Constraint monitors for callers that cannot allocate device memory (a
   host framework that owns all device memory and forbids other
   allocations, or a time loop that must not allocate once running). The
   paper has no counterpart; this is a service of this library.
   Computes what ccz4_constraints computes for a grid of one uniform level,
   but from halo tiles the caller already holds, and allocates nothing: it
   calls no cudaMalloc, cudaFree or allocating library routine.
   Single level only: every patch is differenced with the one spacing dx
   and counted in the norms. The tile buffer of a refined mesh
   (ccz4_alloc_mesh) has the same layout but patches of several spacings
   and covered coarse points; given it, this call returns wrong norms
   without an error, so use ccz4_constraints for meshes.
     tiles    device, [25][n_patches][(p+6)^3] halo tiles in the layout of
              CCZ4_BUF_TILE (for instance that buffer after ccz4_fill_halos)
     dev_H    device [n_points] or NULL; dev_M device [3][n_points] or NULL
     dev_out  device [5]: L2 of H, L2 of |M|, max |H|, max |M|, count of
              non-finite points (not copied to the host; no synchronisation)
   n_points = n_patches * p^3 must not exceed 4,194,304: the per-block
   partial sums of the reduction live in one fixed device array of
   640 KiB that every GPU loading this library holds until the process
   exits. p above 161 is rejected before any size is formed. The first
   call on a device looks up that array's address on the current device
   and keeps it for the life of the process; make that first call before
   any stream capture, and do not call this entry point again on a device
   that the process has reset (cudaDeviceReset).
   Every call shares the array and leaves its partial sums in it (each
   call overwrites all the entries it reads), so calls that overlap on
   the GPU race: serialise them, e.g. on one stream. Sizes beyond the
   maximum return CCZ4_ERR_INVALID with a message. */
ccz4_status ccz4_constraints_noalloc(const double *tiles, int p, int n_patches, double dx,
                                     double *dev_H, double *dev_M, double *dev_out, void *stream);

/* Arithmetic of one interior point-stage of the fused stage kernel for the
   given parameters and precision: the right-hand side, the dissipation, the
   RK4 update (the mean over the four stages) and a quarter of the
   enforcement, counted on the host by running the kernel's own templates
   with operation-counting scalars (add, sub, mul = 1 flop; FMA = 2;
   division = 1). Needs no GPU. out[0] = FP64 flops, out[1] = FP32 flops,
   out[2] = FP64 divisions and roots, out[3] = precision conversions,
   out[4] = FP64 FMAs, out[5] = FP64 adds and multiplies. These are the
   algorithmic flops behind the roofline of the stage kernel. */
ccz4_status ccz4_flops_per_point_stage(const ccz4_params *P, double out[6]);

/* ---- statically refined meshes (appendix "refinement transition") ----

   A mesh has ratio-3 levels of p^3 patches. Level 0 covers the np[0] x
   np[1] x np[2] slots of the base grid (spacing dx, boundary kind bc, the
   Sommerfeld ghost shell if any); a level-l patch (l >= 1) has spacing
   dx / 3^l (dx divided by 3.0 once per level), slot coordinates ijk in
   units of its own level, and is one of the 27 children (slot / 3 along
   each axis) of a level l-1 patch, which then has all 27. Every level
   overlaps the coarser ones: the coarse points under a refined patch are
   evolved too and are replaced after every RK4 step (ccz4_restrict).

   Halo points that a refined level does not cover are interpolated from
   the level below at the same stage: the tensor product of three linear
   maps between cell centres, applied along x, then y, then z, each with
   the weights of the printed matrices P^par / P^perp (fine cell i lies on
   coarse cells c = floor((i-1)/3) and c+1 with weights (1), (2/3, 1/3) or
   (1/3, 2/3) for (i-1) mod 3 = 0, 1, 2). Those coarse points must be
   interior points of the level below, inside the domain (proper nesting);
   refined levels therefore keep away from the domain boundary.

   The mesh is a ccz4_grid: every call above works on it. Buffers keep the
   same layout with the patches in descriptor order (all levels in one
   state vector), the stage kernels apply each level's spacing, all levels
   share the time step, ccz4_step / ccz4_step_graph / ccz4_evolve_host
   restrict after each step, and the constraint norms of ccz4_constraints
   run over the points of leaf patches only (H and M are written for every
   point). */
#define CCZ4_MAX_LEVELS 8

typedef struct {
  int p;              /* points per patch edge, 1..18 */
  int np[3];          /* level-0 patch slots per axis */
  int n_patches;      /* patches of all levels */
  const int *level;   /* host [n_patches] level of each patch, 0..CCZ4_MAX_LEVELS-1 */
  const int *ijk;     /* host [n_patches][3] slot coordinates in units of the patch's level */
  double origin[3];   /* lower corner of the domain */
  double dx;          /* level-0 spacing */
  int bc;             /* CCZ4_BC_* of the level-0 outer boundary */
} ccz4_mesh_desc;

/* Creates a mesh on the current device (see above). Validates the
   descriptor on the host first: CCZ4_ERR_INVALID with a message for a
   level out of range, a level-0 slot missing or listed twice, a refined
   patch without its parent or with an incomplete set of siblings, or a
   halo point whose interpolation sources are not interior points of the
   level below. The halo fill evaluates each patch's coarse-to-fine
   interpolations separably (the distinct x-interpolations of the patch,
   then the distinct y-interpolations of their pairs, then one
   z-interpolation per halo point, all in shared memory; the same products
   and sums, so the same values); with the environment variable
   CCZ4_MESH_INTERP_BY_ENTRY=1 set when the mesh is created it evaluates
   them point by point instead. */
ccz4_status ccz4_alloc_mesh(const ccz4_mesh_desc *desc, ccz4_grid **out);

/* Number of levels and of points of leaf patches (the norm's point count). */
ccz4_status ccz4_mesh_info(const ccz4_grid *g, int *n_levels, long long *n_leaf_points);

/* Restriction (printed R^par of the average scheme along every axis): in
   state buffer `buf`, every point of a patch that has children <- the mean
   of the 3x3x3 fine cells that tile it, as three one-dimensional averages
   with weight 1/3 (x, then y, then z), finest level first. A no-op on a
   single level. Asynchronous. */
ccz4_status ccz4_restrict(ccz4_grid *g, int buf, void *stream);

/* Host-only plan of a mesh (needs no GPU): validates the descriptor like
   ccz4_alloc_mesh and returns the source of every halo'd tile point.
   n_interp receives the number of interpolated tile points. If src is not
   NULL it receives [n_patches][(p+6)^3] entries: >= 0 the index of the
   value within a field of a state buffer (interior points, then the
   Sommerfeld ghost cells), <= -2 the interpolation entry -(s+2). If interp
   is not NULL it receives [n_interp][9] ints: the eight source indices of
   the coarse corners, in the order (z, y, x) with x fastest (corners with
   weight zero repeat a used index), then the remainders rx | ry << 2 |
   rz << 4. */
ccz4_status ccz4_mesh_plan(const ccz4_mesh_desc *desc, long long *n_interp, int *src, int *interp);

/* Launch of the fused stage kernel (a tuning choice; results are
   identical): CCZ4_LAUNCH_FLAT (default), one warp per 32 consecutive
   interior points of all levels; CCZ4_LAUNCH_QUEUE, a persistent launch
   sized to the resident blocks whose warps take 32-point items from a
   device work counter (reset by a memset node before each stage) until the
   points of every level are done; CCZ4_LAUNCH_FUSED, for grids of 9^3
   patches only (CCZ4_ERR_INVALID otherwise), runs each RK stage of
   ccz4_step and ccz4_step_graph as one cooperative launch sized to the
   resident blocks: the halo fill of every patch, a grid-wide barrier, the
   interior points of all levels and the Sommerfeld ghost cells (the
   restriction of a mesh stays a launch of its own; ccz4_rk_stage,
   ccz4_fill_halos and the tuning shapes keep the separate kernels).
   Drops a captured step graph. */
enum { CCZ4_LAUNCH_FLAT = 0, CCZ4_LAUNCH_QUEUE = 1, CCZ4_LAUNCH_FUSED = 2 };
ccz4_status ccz4_set_launch(ccz4_grid *g, int mode);

/* ---- the first-order formulation and the second order with reconstruction ----
   (Sec. "First- and Second-order Formulations", Eq. first-order-variables;
   appendix "Spacetime foliation": the nine primary equations with the red
   terms, Eqs. NR_foccz4_A_k, NR_foccz4_B^i_j, the D_kij equation and
   NR_foccz4_P_i; Sec. "Explicit gradient reconstruction", Alg. fd4-fo and
   Alg. fd4-so.) A ccz4_fo holds a 58-variable state on the geometry of a
   single-level grid: the 25 primaries in the order above, then
   A_k = d_k alpha (25..27), B_k^i = d_k beta^i (28 + 3k + i),
   D_kij = 1/2 d_k g~_ij (37 + 6k + pair(i, j), pairs xx, xy, xz, yy, yz,
   zz) and P_k = d_k phi (55..57). Only first derivatives are taken (FD4),
   and Kreiss-Oliger dissipation is applied to all 58.
     CCZ4_FO_FIRST_ORDER: every variable is evolved, with the red terms and
       the mu terms of the B equation.
     CCZ4_FO_SO_RECONSTRUCT: the paper's second-order formulation written
       over the same 58 variables: the red terms are removed, only the
       primaries (and the Sommerfeld ghost cells of every variable) are
       evolved, and before the right-hand side of every RK stage, and after
       every step, the auxiliary variables of the interior points are
       reconstructed as FD4 first derivatives of the primaries (the extra
       sweep of Alg. fd4-so).
   The Sommerfeld ghost cells of every variable follow the radiative
   condition of the boundary (speed somm_speed[v] for the primaries, 1 for
   the auxiliary variables). After each step the primaries are enforced
   (det g~ = 1, tr A~ = 0) as in ccz4_step. FP64 only (P->precision is
   ignored). Buffers: CCZ4_BUF_U, Y0, Y1, ACC, RHS and (Sommerfeld) INI,
   each [58][field stride] in the grid's layout; the stages use them as
   ccz4_stage_buffers says.
   ccz4_fo_alloc: CCZ4_ERR_INVALID for a refined mesh or an unknown
   variant; CCZ4_ERR_NOMEM if the device memory runs out (about
   58 x 8 bytes x (6 state buffers + 4.6 tile copies) per point).
   ccz4_fo_upload / ccz4_fo_download: host U [58][n_points] (the grid's
   point order) and G [58][n_ghost]; synchronous.
   ccz4_fo_rhs: the right-hand side of all 58 (with the red terms only in
   the first-order variant) of in_buf into out_buf; asynchronous.
   ccz4_fo_reconstruct: the interior auxiliary variables of buf from FD4
   derivatives of its primaries; asynchronous.
   ccz4_fo_rk_stage / ccz4_fo_step: RK4 stages / steps, asynchronous. */
enum { CCZ4_FO_FIRST_ORDER = 0, CCZ4_FO_SO_RECONSTRUCT = 1 };
typedef struct ccz4_fo ccz4_fo;
ccz4_status ccz4_fo_alloc(ccz4_grid *g, int variant, ccz4_fo **out);
ccz4_status ccz4_fo_free(ccz4_fo *f);
ccz4_status ccz4_fo_upload(ccz4_fo *f, int buf, const double *U, const double *G, void *stream);
ccz4_status ccz4_fo_download(ccz4_fo *f, int buf, double *U, double *G, void *stream);
ccz4_status ccz4_fo_rhs(ccz4_fo *f, const ccz4_params *P, int in_buf, int out_buf, void *stream);
ccz4_status ccz4_fo_reconstruct(ccz4_fo *f, int buf, void *stream);
ccz4_status ccz4_fo_rk_stage(ccz4_fo *f, const ccz4_params *P, int stage, double dt, void *stream);
ccz4_status ccz4_fo_step(ccz4_fo *f, const ccz4_params *P, double dt, int n_steps, void *stream);

/* ---- particle tracers and puncture trackers ----
   (Sec. "Particle Tracers as Data Probes"; Sec. "Particle tracers" for
   puncture trackers.) A set of n tracers on a grid. Each step records the
   25 fields at every tracer's position by trilinear interpolation from the
   2^3 closest sample points (cell centres): those of the finest level that
   holds all eight as interior points of its patches, or, where no refined
   level does, those of level 0 with its boundary rule (periodic wrap,
   clamped copy, or the Sommerfeld ghost cells). Weights (1 - t, t) per
   axis, t the offset from the lower sample point in units of the level's
   spacing; the value is the sum over the corners (z outermost, x innermost)
   of (w_x w_y) w_z q, every product and sum rounded on its own.
   With a velocity (vel_field >= 0) the step then moves each tracer by the
   explicit Euler step x <- x + (dt vel_scale) v, v the projected fields
   vel_field .. vel_field + 2. A puncture tracker is a tracer dropped at a
   black hole with the shift as velocity and vel_scale = -1 (the paper's
   opposite shift); vel_field = -1 gives static probes.

   ccz4_tracers_new: pos is host [n][3] (x, y, z), copied; the grid must
   outlive the tracers. Synchronous (builds the slot tables of the refined
   levels on the device). CCZ4_ERR_INVALID for n < 1 or vel_field outside
   [-1, 22].
   ccz4_tracers_step: one step on state buffer buf (CCZ4_BUF_U .. INI);
   asynchronous on stream, one small kernel (capturable in a graph). A
   tracer the grid cannot resolve (outside the Sommerfeld ghost shell, or
   a non-finite coordinate) is left in place with NaN values and flagged.
   ccz4_tracers_read: copies positions (host [n][3]) and the last step's
   values (host [n][25]) when not NULL, synchronising the stream; returns
   CCZ4_ERR_BOUNDS with a message if the last step flagged any tracer.
   ccz4_tracers_free: releases the tracers. */
typedef struct ccz4_tracers ccz4_tracers;
ccz4_status ccz4_tracers_new(ccz4_grid *g, int n, const double *pos, int vel_field, double vel_scale,
                             ccz4_tracers **out);
ccz4_status ccz4_tracers_step(ccz4_tracers *t, int buf, double dt, void *stream);
ccz4_status ccz4_tracers_read(ccz4_tracers *t, double *pos, double *values, void *stream);
ccz4_status ccz4_tracers_free(ccz4_tracers *t);

/* Launch shapes (a tuning choice; results are identical, but for SPLIT in
   the mixed precision, whose FP32 algebra may round a few intermediate
   values differently, within 1e-8 of a field's largest value): the flat stage
   kernel asks the default number of resident 128-thread blocks per SM
   (CCZ4_STAGE_SHAPE_DEFAULT: 4 in FP64, 3 in the mixed precision), one
   more (MORE_BLOCKS, fewer registers per thread) or one fewer
   (FEWER_BLOCKS, more registers), or, for the mixed precision (FP64 keeps
   its default), two phases in one launch (SPLIT: every thread first takes
   all the stencil values of its point into its own shared-memory slots,
   then evaluates the algebra and the update from them); the halo fill runs 256 threads per
   patch with 8 independent loads per thread in its gather (DEFAULT), 512
   threads (WIDE), 16 loads (DEEP) or 128 threads (NARROW). Drops a
   captured step graph. CCZ4_ERR_INVALID for an unknown shape. */
enum { CCZ4_STAGE_SHAPE_DEFAULT = 0, CCZ4_STAGE_SHAPE_MORE_BLOCKS = 1, CCZ4_STAGE_SHAPE_FEWER_BLOCKS = 2,
       CCZ4_STAGE_SHAPE_SPLIT = 3 };
enum { CCZ4_FILL_SHAPE_DEFAULT = 0, CCZ4_FILL_SHAPE_WIDE = 1, CCZ4_FILL_SHAPE_DEEP = 2, CCZ4_FILL_SHAPE_NARROW = 3 };
ccz4_status ccz4_set_tuning(ccz4_grid *g, int stage_shape, int fill_shape);

/* Message of the last failing call on this thread ("" if none). */
const char *ccz4_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CCZ4_H */
