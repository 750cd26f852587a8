/*
 * ccz4_mlp.h -- C ABI of the learned warm start of the puncture
 * initial-data solve (GB300 path, FP32).
 *
 * A multilayer perceptron maps (x, y, z, m1, m2, d, P, S) -- a cell of the
 * initial-data grid and the parameters of a binary: bare masses m1, m2,
 * separation d along x (punctures at -d/2 and +d/2), momenta (0, -+P, 0),
 * spins (0, 0, S) each -- to the correction u of the conformal factor
 * (ccz4_id.h). Its output seeds the plain relaxation solve, which stays the
 * arbiter of the residual.
 *
 * Network: n_in inputs -> depth hidden layers of `width` units with SiLU,
 * silu(z) = z / (1 + exp(-z)) -> one linear output. Parameters: one flat
 * FP32 vector, layer after layer, each its weight matrix (out x in, row
 * major) then its bias. Loss: mean over the batch of (y - t)^2. Update:
 * Adam, m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * theta <- theta - lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
 * Gradients are summed in a fixed order (deterministic).
 *
 * Feature map (fixed): (x/L, y/L, z/L, (m1-0.5)/0.2, (m2-0.5)/0.2,
 * (d-7)/5, (P-0.1)/0.1, (S-0.15)/0.15); target t = CCZ4_MLP_U_SCALE * u.
 *
 * All arrays are device memory; FP32 unless stated. Conventions as in
 * ccz4.h (streams as void*, asynchronous unless stated, error codes).
 */
#ifndef CCZ4_MLP_H
#define CCZ4_MLP_H

#include "ccz4.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CCZ4_MLP_N_FEATURES 8
#define CCZ4_MLP_U_SCALE 10.0f

typedef struct ccz4_mlp ccz4_mlp;

/* n_in 1..64, width 1..128, depth 1..8 hidden layers; max_batch rows per
   call (workspace). Parameters start at zero: write them through
   ccz4_mlp_params. */
ccz4_status ccz4_mlp_create(int n_in, int width, int depth, int max_batch, ccz4_mlp **out);
ccz4_status ccz4_mlp_free(ccz4_mlp *m);
/* Flat parameter / gradient vectors (owned by the network) and their length. */
ccz4_status ccz4_mlp_params(ccz4_mlp *m, float **dev, long long *n);
ccz4_status ccz4_mlp_grads(ccz4_mlp *m, float **dev, long long *n);

/* y[batch] = network(x[batch][n_in]). */
ccz4_status ccz4_mlp_forward(ccz4_mlp *m, const float *x, int batch, float *y, void *stream);
/* Forward and back-propagation: *loss (device float) = mean (y - t)^2 and
   the gradient vector = d loss / d theta. */
ccz4_status ccz4_mlp_loss_grad(ccz4_mlp *m, const float *x, const float *t, int batch, float *loss,
                               void *stream);
/* One Adam step with the current gradients (the step count k is kept by
   the network and starts at 1). */
ccz4_status ccz4_mlp_adam(ccz4_mlp *m, float lr, float b1, float b2, float eps, void *stream);

/* Features of every cell of the n^3 initial-data grid on [-L, L]^3 for
   binary parameters p5 = (m1, m2, d, P, S): x[n^3][8], cells x fastest. */
ccz4_status ccz4_mlp_features_grid(int n, double L, const double p5[5], float *x, void *stream);
/* Training rows: for row r, idx[r] = s * n^3 + c picks cell c of stored
   solution s; x[r][8] gets its features (parameters p5[s][5], FP32) and
   t[r] = CCZ4_MLP_U_SCALE * u_store[idx[r]] (u_store FP32). */
ccz4_status ccz4_mlp_features_sample(int n, double L, const float *p5, const float *u_store,
                                     const long long *idx, int batch, float *x, float *t, void *stream);
/* u[c] (double) = y[c] / CCZ4_MLP_U_SCALE for c < count: the network's guess
   as the initial u of the solve. */
ccz4_status ccz4_mlp_output_to_u(const float *y, long long count, double *u, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CCZ4_MLP_H */
