// Learned warm start of the initial-data solve (include/ccz4_mlp.h): the
// perceptron's forward pass, back-propagation and Adam update, in FP32, and
// the kernels that turn solver cells into network inputs and network
// outputs into a solver guess.
//
// Every layer is one tiled SIMT GEMM: a 64-row x 128-column output tile per
// 256-thread block, 4 x 8 outputs per thread, operands staged through shared
// memory 32 columns of K at a time. The same kernel serves the forward pass
// (out = A W^T + b, SiLU fused, pre-activations kept) and the input gradient
// of back-propagation (dA = dZ W). Weight gradients (dW = dZ^T A, a
// reduction over the batch) are summed per chunk of rows and the chunks are
// then added in a fixed order, so training is deterministic. The network is
// small (about 50k parameters, ~3e5 flops per row for a training step), so
// a training run costs seconds on the CUDA cores; it runs in FP32 as the
// method specifies.
#include <math.h>
#include <string.h>

#include "../../include/ccz4_mlp.h"
#include "ccz4_internal.cuh"

struct ccz4_mlp {
  int n_in, width, depth, max_batch;
  long long n_params;
  float *theta, *grad, *adam_m, *adam_v;
  float *z;        // [depth][max_batch][width] pre-activations
  float *a;        // [depth][max_batch][width] activations
  float *y;        // [max_batch]
  float *dy;       // [max_batch]
  float *d0, *d1;  // [max_batch][width] gradient ping-pong
  float *wpart;    // weight-gradient partial sums per chunk
  float *lpart;    // loss partial sums
  long long wpart_len;
  int step;
};

namespace {

constexpr int GM_BM = 64, GM_BN = 128, GM_BK = 32, GM_THREADS = 256;
constexpr int WG_CHUNK = 1024;  // rows per weight-gradient partial sum
constexpr int RED_T = 256;

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_prime_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// out[r][j] = bias[j] + sum_k A[r][k] M[k][j] for r < B, j < N, with
// M[k][j] = W[j][k] (transW, W is N x K) or W[k][j] (W is K x N).
// Z (if given) receives out, Act (if given) silu(out).
__global__ void __launch_bounds__(GM_THREADS) gemm_kernel(const float *__restrict__ A, const float *__restrict__ W,
                                                          const float *__restrict__ bias, int B, int K, int N,
                                                          int transW, float *Z, float *Act) {
  __shared__ float As[GM_BK][GM_BM + 4];
  __shared__ float Ws[GM_BK][GM_BN + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int row0 = blockIdx.x * GM_BM;
  const int col0 = blockIdx.y * GM_BN;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += GM_BK) {
    for (int q = tid; q < GM_BM * GM_BK; q += GM_THREADS) {
      const int r = q / GM_BK, kk = q % GM_BK;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < B && gk < K) ? A[(long long)gr * K + gk] : 0.0f;
    }
    for (int q = tid; q < GM_BN * GM_BK; q += GM_THREADS) {
      const int kk = q / GM_BN, j = q % GM_BN;
      const int gj = col0 + j, gk = k0 + kk;
      float w = 0.0f;
      if (gj < N && gk < K) w = transW ? W[(long long)gj * K + gk] : W[(long long)gk * N + gj];
      Ws[kk][j] = w;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GM_BK; ++kk) {
      float a[4], w[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = Ws[kk][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty * 4 + i;
    if (r >= B) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = col0 + tx * 8 + j;
      if (c >= N) continue;
      const float v = acc[i][j] + (bias ? bias[c] : 0.0f);
      if (Z) Z[(long long)r * N + c] = v;
      if (Act) Act[(long long)r * N + c] = silu_f(v);
    }
  }
}

// Partial weight gradient of one chunk of rows: part[chunk][n][k] =
// sum_{r in chunk} dZ[r][n] A[r][k], and (for the tiles with k0 = 0)
// part_b[chunk][n] = sum_r dZ[r][n]. Tiles of 32 x 32 (n, k) per block.
__global__ void __launch_bounds__(256) wgrad_kernel(const float *__restrict__ dZ, const float *__restrict__ A,
                                                    int B, int N, int K, float *part, float *part_b) {
  __shared__ float Ds[32][33];
  __shared__ float Xs[32][33];
  const int chunk = blockIdx.z;
  const int n0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tid = threadIdx.x;
  const int tn = tid / 8, tk4 = (tid % 8) * 4;  // each thread: 1 n x 4 k
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float accb = 0.0f;
  const int r_begin = chunk * WG_CHUNK, r_end = min(B, r_begin + WG_CHUNK);
  for (int r0 = r_begin; r0 < r_end; r0 += 32) {
    for (int q = tid; q < 32 * 32; q += 256) {
      const int rr = q / 32, c = q % 32;
      const int r = r0 + rr;
      Ds[rr][c] = (r < r_end && n0 + c < N) ? dZ[(long long)r * N + n0 + c] : 0.0f;
      Xs[rr][c] = (r < r_end && k0 + c < K) ? A[(long long)r * K + k0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const float d = Ds[rr][tn];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(d, Xs[rr][tk4 + j], acc[j]);
      accb += d;
    }
    __syncthreads();
  }
  const int n = n0 + tn;
  if (n < N) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tk4 + j;
      if (k < K) part[((long long)chunk * N + n) * K + k] = acc[j];
    }
    if (blockIdx.x == 0 && tk4 == 0) part_b[(long long)chunk * N + n] = accb;
  }
}

// g[q] = sum over chunks of part[chunk][q], in chunk order.
__global__ void chunk_sum_kernel(const float *part, int n_chunks, long long len, float *g) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  float s = 0.0f;
  for (int c = 0; c < n_chunks; ++c) s += part[(long long)c * len + q];
  g[q] = s;
}

// dZ = dA * silu'(Z), in place on dA.
__global__ void silu_back_kernel(float *dA, const float *Z, long long len) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < len) dA[q] *= silu_prime_f(Z[q]);
}

// dy = 2 (y - t) / B and per-block partial sums of (y - t)^2.
__global__ void __launch_bounds__(RED_T) loss_kernel(const float *y, const float *t, int B, float *dy,
                                                     float *part) {
  __shared__ float sh[RED_T];
  const int r = blockIdx.x * RED_T + threadIdx.x;
  float e = 0.0f;
  if (r < B) {
    const float d = y[r] - t[r];
    dy[r] = 2.0f * d / (float)B;
    e = d * d;
  }
  sh[threadIdx.x] = e;
  __syncthreads();
  for (int w = RED_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(RED_T) loss_final_kernel(const float *part, int blocks, int B, float *loss) {
  __shared__ float sh[RED_T];
  float s = 0.0f;
  for (int b = threadIdx.x; b < blocks; b += RED_T) s += part[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = RED_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)B;
}

__global__ void adam_kernel(float *theta, float *m, float *v, const float *g, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  theta[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
}

__device__ __forceinline__ void features(int n, double L, long long c, const float *p5, float *x) {
  const int ci = (int)c;  // n <= 1024: 32-bit index arithmetic
  const int i = ci % n, j = (ci / n) % n, k = ci / (n * n);
  const double h = 2.0 * L / n;
  x[0] = (float)((-L + (i + 0.5) * h) / L);
  x[1] = (float)((-L + (j + 0.5) * h) / L);
  x[2] = (float)((-L + (k + 0.5) * h) / L);
  x[3] = (p5[0] - 0.5f) / 0.2f;
  x[4] = (p5[1] - 0.5f) / 0.2f;
  x[5] = (p5[2] - 7.0f) / 5.0f;
  x[6] = (p5[3] - 0.1f) / 0.1f;
  x[7] = (p5[4] - 0.15f) / 0.15f;
}

__global__ void features_grid_kernel(int n, double L, float m1, float m2, float d, float P, float S, float *x) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long long)n * n * n) return;
  const float p5[5] = {m1, m2, d, P, S};
  features(n, L, c, p5, x + c * CCZ4_MLP_N_FEATURES);
}

__global__ void features_sample_kernel(int n, double L, const float *p5, const float *u_store,
                                       const long long *idx, int B, float *x, float *t) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const long long n3 = (long long)n * n * n;
  const long long q = idx[r];
  const long long s = q / n3, c = q - s * n3;
  features(n, L, c, p5 + 5 * s, x + (long long)r * CCZ4_MLP_N_FEATURES);
  t[r] = CCZ4_MLP_U_SCALE * u_store[q];
}

__global__ void output_to_u_kernel(const float *y, long long count, double *u) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < count) u[c] = (double)y[c] / (double)CCZ4_MLP_U_SCALE;
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t gemm(const float *A, const float *W, const float *bias, int B, int K, int N, int transW, float *Z,
                 float *Act, cudaStream_t s) {
  dim3 grid(blocks_for(B, GM_BM), blocks_for(N, GM_BN));
  gemm_kernel<<<grid, GM_THREADS, 0, s>>>(A, W, bias, B, K, N, transW, Z, Act);
  return cudaGetLastError();
}

// Offsets of layer l's weights and bias in the flat vector.
void layer_offsets(const ccz4_mlp *m, int l, long long *w, long long *b, int *out, int *in) {
  long long k = 0;
  for (int q = 0; q <= l; ++q) {
    const int o = q < m->depth ? m->width : 1;
    const int i = q == 0 ? m->n_in : m->width;
    if (q == l) {
      *w = k;
      *b = k + (long long)o * i;
      *out = o;
      *in = i;
      return;
    }
    k += (long long)o * i + o;
  }
}

// Forward through all layers; hidden activations in m->a, output in y.
cudaError_t forward_all(ccz4_mlp *m, const float *x, int B, float *y, cudaStream_t s) {
  const float *in = x;
  const long long lay = (long long)m->max_batch * m->width;
  for (int l = 0; l <= m->depth; ++l) {
    long long wo, bo;
    int o, i;
    layer_offsets(m, l, &wo, &bo, &o, &i);
    if (l < m->depth) {
      cudaError_t e = gemm(in, m->theta + wo, m->theta + bo, B, i, o, 1, m->z + l * lay, m->a + l * lay, s);
      if (e != cudaSuccess) return e;
      in = m->a + l * lay;
    } else {
      cudaError_t e = gemm(in, m->theta + wo, m->theta + bo, B, i, o, 1, y, nullptr, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

using namespace ccz4;

#define ML_TRY(call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                           \
      return CCZ4_ERR_CUDA;                                                                \
    }                                                                                      \
  } while (0)

static void mlp_release(ccz4_mlp *m) {
  float *bufs[] = {m->theta, m->grad, m->adam_m, m->adam_v, m->z, m->a, m->y, m->dy, m->d0, m->d1, m->wpart,
                   m->lpart};
  for (float *b : bufs) cudaFree(b);
  free(m);
}

extern "C" ccz4_status ccz4_mlp_create(int n_in, int width, int depth, int max_batch, ccz4_mlp **out) {
  if (!out || n_in < 1 || n_in > 64 || width < 1 || width > GM_BN || depth < 1 || depth > 8 || max_batch < 1 ||
      max_batch > (1 << 24)) {
    set_error("mlp_create: need n_in 1..64, width 1..%d, depth 1..8, max_batch 1..2^24", GM_BN);
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  ccz4_mlp *m = (ccz4_mlp *)calloc(1, sizeof(ccz4_mlp));
  if (!m) {
    set_error("host allocation failed");
    return CCZ4_ERR_NOMEM;
  }
  m->n_in = n_in;
  m->width = width;
  m->depth = depth;
  m->max_batch = max_batch;
  m->n_params = (long long)width * n_in + width + (long long)(depth - 1) * ((long long)width * width + width) +
                width + 1;
  const long long B = max_batch, W = width;
  const int chunks = (int)((B + WG_CHUNK - 1) / WG_CHUNK);
  m->wpart_len = (long long)chunks * (W * (W > n_in ? W : n_in) + W);
  bool ok = true;
  auto alloc = [&](float **p, long long n) {
    if (ok) ok = cudaMalloc(p, sizeof(float) * (size_t)(n > 0 ? n : 1)) == cudaSuccess;
    if (ok) cudaMemset(*p, 0, sizeof(float) * (size_t)(n > 0 ? n : 1));
  };
  alloc(&m->theta, m->n_params);
  alloc(&m->grad, m->n_params);
  alloc(&m->adam_m, m->n_params);
  alloc(&m->adam_v, m->n_params);
  alloc(&m->z, depth * B * W);
  alloc(&m->a, depth * B * W);
  alloc(&m->y, B);
  alloc(&m->dy, B);
  alloc(&m->d0, B * W);
  alloc(&m->d1, B * W);
  alloc(&m->wpart, m->wpart_len);
  alloc(&m->lpart, (B + RED_T - 1) / RED_T);
  if (!ok) {
    set_error("mlp_create: device allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
    cudaGetLastError();
    mlp_release(m);
    return CCZ4_ERR_NOMEM;
  }
  *out = m;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_free(ccz4_mlp *m) {
  if (!m) return CCZ4_OK;
  cudaDeviceSynchronize();
  mlp_release(m);
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_params(ccz4_mlp *m, float **dev, long long *n) {
  if (!m || !dev) {
    set_error("mlp_params: NULL argument");
    return CCZ4_ERR_INVALID;
  }
  *dev = m->theta;
  if (n) *n = m->n_params;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_grads(ccz4_mlp *m, float **dev, long long *n) {
  if (!m || !dev) {
    set_error("mlp_grads: NULL argument");
    return CCZ4_ERR_INVALID;
  }
  *dev = m->grad;
  if (n) *n = m->n_params;
  return CCZ4_OK;
}

static ccz4_status check_batch(const ccz4_mlp *m, int batch, const void *x) {
  if (!m || !x || batch < 1 || batch > m->max_batch) {
    set_error("mlp: need a network, inputs and 1 <= batch <= max_batch (%d)", m ? m->max_batch : 0);
    return CCZ4_ERR_INVALID;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_forward(ccz4_mlp *m, const float *x, int batch, float *y, void *stream) {
  ccz4_status st = check_batch(m, batch, x);
  if (st != CCZ4_OK) return st;
  if (!y) {
    set_error("mlp_forward: y is NULL");
    return CCZ4_ERR_INVALID;
  }
  ML_TRY(forward_all(m, x, batch, y, (cudaStream_t)stream));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_loss_grad(ccz4_mlp *m, const float *x, const float *t, int batch, float *loss,
                                          void *stream) {
  ccz4_status st = check_batch(m, batch, x);
  if (st != CCZ4_OK) return st;
  if (!t || !loss) {
    set_error("mlp_loss_grad: t and loss must be given");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int B = batch;
  ML_TRY(forward_all(m, x, B, m->y, s));
  const int lblocks = (int)blocks_for(B, RED_T);
  loss_kernel<<<lblocks, RED_T, 0, s>>>(m->y, t, B, m->dy, m->lpart);
  ML_TRY(cudaGetLastError());
  loss_final_kernel<<<1, RED_T, 0, s>>>(m->lpart, lblocks, B, loss);
  ML_TRY(cudaGetLastError());
  const long long lay = (long long)m->max_batch * m->width;
  const int chunks = (int)((B + WG_CHUNK - 1) / WG_CHUNK);
  // dZ of the current layer: the output layer's is dy (B x 1)
  const float *dZ = m->dy;
  float *bufs[2] = {m->d0, m->d1};
  for (int l = m->depth; l >= 0; --l) {
    long long wo, bo;
    int o, i;
    layer_offsets(m, l, &wo, &bo, &o, &i);
    const float *Ain = l == 0 ? x : m->a + (l - 1) * lay;
    // weight and bias gradients of layer l
    const long long wl = (long long)o * i;
    float *pw = m->wpart, *pb = m->wpart + (long long)chunks * wl;
    dim3 g(blocks_for(i, 32), blocks_for(o, 32), chunks);
    wgrad_kernel<<<g, 256, 0, s>>>(dZ, Ain, B, o, i, pw, pb);
    ML_TRY(cudaGetLastError());
    chunk_sum_kernel<<<blocks_for(wl, 256), 256, 0, s>>>(pw, chunks, wl, m->grad + wo);
    ML_TRY(cudaGetLastError());
    chunk_sum_kernel<<<blocks_for(o, 256), 256, 0, s>>>(pb, chunks, o, m->grad + bo);
    ML_TRY(cudaGetLastError());
    if (l == 0) break;
    // dA of the layer below = dZ W (B x i), then dZ below = dA * silu'(Z below)
    float *dA = bufs[l & 1];
    ML_TRY(gemm(dZ, m->theta + wo, nullptr, B, o, i, 0, dA, nullptr, s));
    silu_back_kernel<<<blocks_for((long long)B * i, 256), 256, 0, s>>>(dA, m->z + (l - 1) * lay, (long long)B * i);
    ML_TRY(cudaGetLastError());
    dZ = dA;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_adam(ccz4_mlp *m, float lr, float b1, float b2, float eps, void *stream) {
  if (!m || !(lr >= 0.0f) || !(b1 >= 0.0f && b1 < 1.0f) || !(b2 >= 0.0f && b2 < 1.0f) || !(eps > 0.0f)) {
    set_error("mlp_adam: need lr >= 0, 0 <= b1, b2 < 1, eps > 0");
    return CCZ4_ERR_INVALID;
  }
  m->step += 1;
  const float c1 = (float)(1.0 / (1.0 - pow((double)b1, (double)m->step)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)b2, (double)m->step)));
  adam_kernel<<<blocks_for(m->n_params, 256), 256, 0, (cudaStream_t)stream>>>(m->theta, m->adam_m, m->adam_v,
                                                                              m->grad, m->n_params, lr, b1, b2,
                                                                              eps, c1, c2);
  ML_TRY(cudaGetLastError());
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_features_grid(int n, double L, const double p5[5], float *x, void *stream) {
  if (n < 1 || n > 1024 || !(L > 0.0) || !p5 || !x) {
    set_error("mlp_features_grid: invalid arguments");
    return CCZ4_ERR_INVALID;
  }
  const long long cells = (long long)n * n * n;
  features_grid_kernel<<<blocks_for(cells, 256), 256, 0, (cudaStream_t)stream>>>(
      n, L, (float)p5[0], (float)p5[1], (float)p5[2], (float)p5[3], (float)p5[4], x);
  ML_TRY(cudaGetLastError());
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_features_sample(int n, double L, const float *p5, const float *u_store,
                                                const long long *idx, int batch, float *x, float *t,
                                                void *stream) {
  if (n < 1 || n > 1024 || !(L > 0.0) || !p5 || !u_store || !idx || batch < 1 || !x || !t) {
    set_error("mlp_features_sample: invalid arguments");
    return CCZ4_ERR_INVALID;
  }
  features_sample_kernel<<<blocks_for(batch, 256), 256, 0, (cudaStream_t)stream>>>(n, L, p5, u_store, idx, batch,
                                                                                   x, t);
  ML_TRY(cudaGetLastError());
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mlp_output_to_u(const float *y, long long count, double *u, void *stream) {
  if (!y || !u || count < 0) {
    set_error("mlp_output_to_u: invalid arguments");
    return CCZ4_ERR_INVALID;
  }
  if (count == 0) return CCZ4_OK;
  output_to_u_kernel<<<blocks_for(count, 256), 256, 0, (cudaStream_t)stream>>>(y, count, u);
  ML_TRY(cudaGetLastError());
  return CCZ4_OK;
}
