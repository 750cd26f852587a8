// Learned warm start of the initial-data solve (include/ccz4_mlp.h): the
// perceptron's forward pass, back-propagation and Adam update, in FP32, and
// the kernels that turn solver cells into network inputs and network
// outputs into a solver guess.
//
// The products with the 128-wide hidden layers -- the forward pass (out = A
// W^T + b, SiLU fused, pre-activations kept), the input gradient of
// back-propagation (dA = dZ W) and the weight gradient (dW = dZ^T A, a
// reduction over the batch) -- run in one register-blocked SIMT tile GEMM
// (tile_gemm): a 128 x 128 output tile per 256-thread block, 8 x 8 outputs
// per thread, operands staged through shared memory 16 values of the
// reduction at a time and read back as float4, the next stage's global
// loads in flight while the current one is multiplied. The operand layouts
// (row- or column-major) are template flags, so every product reads its
// operands in place; its epilogues fuse the bias and SiLU of the forward
// pass, the SiLU derivative of back-propagation (dZ = dA * silu'(Z)) and,
// for weight gradients, the bias gradient's column sums. The single-output
// layer has its own kernels (a dot product per row forward, an outer
// product backward), and the weight gradients of the 8-input and the
// single-output layer a kernel that streams rows, 128 columns a warp.
// Weight gradients are summed per chunk of rows and the chunks
// then added in a fixed order, so training is deterministic. The network
// runs in FP32 as the method specifies.
#include <math.h>
#include <stdint.h>
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
constexpr int WG_CHUNK = 1024;  // rows per weight-gradient partial sum (narrow layers)
constexpr int TG_CHUNK = 256;   // rows per weight-gradient partial sum of tile_gemm
constexpr int TG_BM = 128, TG_BN = 128, TG_BK = 16, TG_THREADS = 256;
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

enum { TG_EPI_STORE = 0, TG_EPI_ACT = 1, TG_EPI_DSILU = 2 };

// C = sum over k of Aop(m, k) Bop(k, n) for the 128 x 128 tile at
// (blockIdx.x * 128, blockIdx.y * 128), k over [kc0, kc1) with kc0 =
// blockIdx.z * kchunk (kchunk <= 0: the whole of [0, K)):
//   Aop(m, k) = A_ROW ? A[m * lda + k] : A[k * lda + m]   (m < M)
//   Bop(k, n) = B_ROW ? B[k * ldb + n] : B[n * ldb + k]   (n < N)
// M, N, K, lda, ldb and the pointers multiples of 4 (float4 access); values
// outside the ranges read as zero. EPI_ACT: out = C + bias, Act =
// silu(out); EPI_DSILU: out = C * silu'(aux) (aux indexed like out); both
// with ldc = N. EPI_STORE: out[blockIdx.z][m][n] = C (ldc, stride M * ldc
// between chunks), and with A column-major and bpart given, the blocks of
// the first column of tiles also write bpart[blockIdx.z][m] = sum over the
// chunk's k of Aop(m, k) (warp w adds the k of each stage with k % 8 = w,
// then the eight warps' sums are added in warp order). Thread (ty, tx) = (tid / 16, tid % 16) owns rows ty*4 +
// {0..3} and 64 + ty*4 + {0..3}, columns tx*4 + {0..3} and 64 + tx*4 + {0..3}.
template <bool A_ROW, bool B_ROW, int EPI>
__global__ void __launch_bounds__(TG_THREADS, 2) tile_gemm(const float *__restrict__ A, const float *__restrict__ B,
                                                           int M, int N, int K, int lda, int ldb, int kchunk,
                                                           const float *__restrict__ bias,
                                                           const float *__restrict__ aux, float *__restrict__ out,
                                                           int ldc, float *__restrict__ Act, float *__restrict__ bpart) {
  __shared__ __align__(16) float As[TG_BK][TG_BM + 4];
  __shared__ __align__(16) float Bs[TG_BK][TG_BN + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int m0 = blockIdx.x * TG_BM, n0 = blockIdx.y * TG_BN;
  const int kc0 = kchunk > 0 ? blockIdx.z * kchunk : 0;
  const int kc1 = kchunk > 0 ? min(K, kc0 + kchunk) : K;
  // the two float4 loads of each operand per stage: (row, col) of the staged tile
  // A_ROW: 128 m x 16 k as m = q / 4 (+64), k4 = (q % 4) * 4; column-major: 16 k x 128 m as k = q / 32, m4 = (q % 32) * 4
  float4 ra[2], rb[2];
  float4 bsum = make_float4(0.f, 0.f, 0.f, 0.f);  // column sums of the staged A values (column-major A)
  auto load = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + h * TG_THREADS;
      if (A_ROW) {
        const int m = m0 + q / 4, k = k0 + (q % 4) * 4;
        ra[h] = (m < M && k < kc1) ? *reinterpret_cast<const float4 *>(A + (long long)m * lda + k)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const int k = k0 + q / 32, m = m0 + (q % 32) * 4;
        ra[h] = (m < M && k < kc1) ? *reinterpret_cast<const float4 *>(A + (long long)k * lda + m)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (B_ROW) {
        const int k = k0 + q / 32, n = n0 + (q % 32) * 4;
        rb[h] = (n < N && k < kc1) ? *reinterpret_cast<const float4 *>(B + (long long)k * ldb + n)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const int n = n0 + q / 4, k = k0 + (q % 4) * 4;
        rb[h] = (n < N && k < kc1) ? *reinterpret_cast<const float4 *>(B + (long long)n * ldb + k)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + h * TG_THREADS;
      if (A_ROW) {
        const int m = q / 4, k = (q % 4) * 4;
        As[k][m] = ra[h].x;
        As[k + 1][m] = ra[h].y;
        As[k + 2][m] = ra[h].z;
        As[k + 3][m] = ra[h].w;
      } else {
        *reinterpret_cast<float4 *>(&As[q / 32][(q % 32) * 4]) = ra[h];
        bsum.x += ra[h].x;
        bsum.y += ra[h].y;
        bsum.z += ra[h].z;
        bsum.w += ra[h].w;
      }
      if (B_ROW) {
        *reinterpret_cast<float4 *>(&Bs[q / 32][(q % 32) * 4]) = rb[h];
      } else {
        const int n = q / 4, k = (q % 4) * 4;
        Bs[k][n] = rb[h].x;
        Bs[k + 1][n] = rb[h].y;
        Bs[k + 2][n] = rb[h].z;
        Bs[k + 3][n] = rb[h].w;
      }
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  load(kc0);
  for (int k0 = kc0; k0 < kc1; k0 += TG_BK) {
    __syncthreads();  // the previous stage's readers are done
    stage();
    __syncthreads();
    if (k0 + TG_BK < kc1) load(k0 + TG_BK);  // in flight during the products below
#pragma unroll
    for (int kk = 0; kk < TG_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  if (!A_ROW && EPI == TG_EPI_STORE && bpart != nullptr && blockIdx.y == 0) {  // uniform over the block
    __syncthreads();  // the last stage's readers are done with As
    float *red = &As[0][0];  // [8 warps][128 m]
    *reinterpret_cast<float4 *>(red + (tid / 32) * TG_BM + (tid % 32) * 4) = bsum;
    __syncthreads();
    if (tid < TG_BM && m0 + tid < M) {
      float t = 0.0f;
#pragma unroll
      for (int w = 0; w < TG_THREADS / 32; ++w) t += red[w * TG_BM + tid];
      bpart[(long long)blockIdx.z * M + m0 + tid] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int n = n0 + half * 64 + tx * 4;
      if (n >= N) continue;
      float4 v = make_float4(acc[i][half * 4], acc[i][half * 4 + 1], acc[i][half * 4 + 2], acc[i][half * 4 + 3]);
      if (EPI == TG_EPI_ACT) {
        const float4 bv = *reinterpret_cast<const float4 *>(bias + n);
        v.x += bv.x;
        v.y += bv.y;
        v.z += bv.z;
        v.w += bv.w;
        *reinterpret_cast<float4 *>(out + (long long)m * ldc + n) = v;
        *reinterpret_cast<float4 *>(Act + (long long)m * ldc + n) =
            make_float4(silu_f(v.x), silu_f(v.y), silu_f(v.z), silu_f(v.w));
      } else if (EPI == TG_EPI_DSILU) {
        const float4 zv = *reinterpret_cast<const float4 *>(aux + (long long)m * ldc + n);
        v.x *= silu_prime_f(zv.x);
        v.y *= silu_prime_f(zv.y);
        v.z *= silu_prime_f(zv.z);
        v.w *= silu_prime_f(zv.w);
        *reinterpret_cast<float4 *>(out + (long long)m * ldc + n) = v;
      } else {
        *reinterpret_cast<float4 *>(out + ((long long)blockIdx.z * M + m) * ldc + n) = v;
      }
    }
  }
}

// Partial weight gradient of one chunk of TG_CHUNK rows for a layer whose
// one side is at most 128 wide (a multiple of 4) and the other at most 8:
// part[chunk][n][k] = sum over the chunk's rows of dZ[r][n] A[r][k], and
// part_b[chunk][n] = the sum of dZ[r][n]. WIDE_IS_DZ: dZ is the wide side
// (N <= 128, K <= 8: the first layer); otherwise A is (K <= 128, N <= 8: the
// single-output layer). Lane l of a warp owns wide columns 4l..4l+3 (one
// float4 load per row), warp w takes rows w, w + 8, ... of the chunk; the
// eight warps' sums are then added in warp order.
constexpr int THIN_W = 128, THIN_V = 8;
template <bool WIDE_IS_DZ>
__global__ void __launch_bounds__(256) wgrad_thin_kernel(const float *__restrict__ dZ, const float *__restrict__ A,
                                                         int B, int N, int K, float *__restrict__ part,
                                                         float *__restrict__ part_b) {
  __shared__ float red[8][THIN_W * THIN_V + THIN_W];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int W = WIDE_IS_DZ ? N : K, V = WIDE_IS_DZ ? K : N;
  const float *wide_p = WIDE_IS_DZ ? dZ : A;
  const float *thin_p = WIDE_IS_DZ ? A : dZ;
  const int c4 = lane * 4;
  const bool active = c4 < W;
  const int r_begin = blockIdx.x * TG_CHUNK, r_end = min(B, r_begin + TG_CHUNK);
  float acc[4][THIN_V], bs[WIDE_IS_DZ ? 4 : THIN_V];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int v = 0; v < THIN_V; ++v) acc[c][v] = 0.0f;
#pragma unroll
  for (int c = 0; c < (WIDE_IS_DZ ? 4 : THIN_V); ++c) bs[c] = 0.0f;
#pragma unroll 4
  for (int r = r_begin + w; r < r_end; r += 8) {
    const float4 x4 = active ? *reinterpret_cast<const float4 *>(wide_p + (long long)r * W + c4)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    const float x[4] = {x4.x, x4.y, x4.z, x4.w};
    float t[THIN_V];
#pragma unroll
    for (int v = 0; v < THIN_V; ++v) t[v] = v < V ? thin_p[(long long)r * V + v] : 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int v = 0; v < THIN_V; ++v) acc[c][v] = fmaf(x[c], t[v], acc[c][v]);
    if (WIDE_IS_DZ) {
#pragma unroll
      for (int c = 0; c < 4; ++c) bs[c] += x[c];
    } else {
#pragma unroll
      for (int v = 0; v < THIN_V; ++v) bs[v] += t[v];
    }
  }
  // red[w][c * 8 + v]: wide column c, thin column v; then the bias sums at THIN_W * THIN_V
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int v = 0; v < THIN_V; ++v) red[w][(c4 + c) * THIN_V + v] = acc[c][v];
  if (WIDE_IS_DZ) {
#pragma unroll
    for (int c = 0; c < 4; ++c) red[w][THIN_W * THIN_V + c4 + c] = bs[c];
  } else if (lane == 0) {
#pragma unroll
    for (int v = 0; v < THIN_V; ++v) red[w][THIN_W * THIN_V + v] = bs[v];
  }
  __syncthreads();
  const int NK = N * K;
  for (int q = threadIdx.x; q < NK + N; q += 256) {
    int slot;
    if (q < NK) {
      const int n = q / K, k = q % K;
      slot = WIDE_IS_DZ ? n * THIN_V + k : k * THIN_V + n;
    } else {
      slot = THIN_W * THIN_V + (q - NK);
    }
    float s = 0.0f;
#pragma unroll
    for (int v = 0; v < 8; ++v) s += red[v][slot];
    if (q < NK)
      part[(long long)blockIdx.x * NK + q] = s;
    else
      part_b[(long long)blockIdx.x * N + (q - NK)] = s;
  }
}

// Forward of a single-output layer: y[r] = bias[0] + sum_k A[r][k] W[k],
// one warp per row (lane l takes k = l, l + 32, ...; the lanes' sums are
// combined by a butterfly and lane 0's result is kept).
__global__ void rowdot_kernel(const float *__restrict__ A, const float *__restrict__ W,
                              const float *__restrict__ bias, int B, int K, float *__restrict__ y) {
  const int lane = threadIdx.x % 32;
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (r >= B) return;  // the same for the whole warp
  float s = 0.0f;
  for (int k = lane; k < K; k += 32) s = fmaf(A[r * K + k], W[k], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) y[r] = s + bias[0];
}

// Back-propagation through a single-output layer into the SiLU below:
// dZ[r][n] = (dy[r] W[n]) * silu'(Z[r][n]); N4 = N / 4 float4 groups a row.
__global__ void outer_dsilu_kernel(const float *__restrict__ dy, const float *__restrict__ W,
                                   const float *__restrict__ Z, int B, int N4, float *__restrict__ dZ) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;  // B * N4 < 2^31
  if (q >= (unsigned)B * (unsigned)N4) return;
  const unsigned r = q / (unsigned)N4;
  const int n = (int)(q - r * (unsigned)N4) * 4;
  const float d = dy[r];
  const float4 z = reinterpret_cast<const float4 *>(Z)[q];
  const float4 w = *reinterpret_cast<const float4 *>(W + n);
  reinterpret_cast<float4 *>(dZ)[q] = make_float4((d * w.x) * silu_prime_f(z.x), (d * w.y) * silu_prime_f(z.y),
                                                  (d * w.z) * silu_prime_f(z.z), (d * w.w) * silu_prime_f(z.w));
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

// g[q] = sum over chunks of part[chunk][q]: a block takes 32 consecutive q,
// its warp w adds, in order, the chunks of the w-th of eight equal runs,
// then the eight runs' sums are added in run order.
__global__ void __launch_bounds__(256) chunk_sum_kernel(const float *__restrict__ part, int n_chunks, long long len,
                                                        float *__restrict__ g) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const long long q = (long long)blockIdx.x * 32 + lane;
  const int per = (n_chunks + 7) / 8;
  const int c0 = w * per, c1 = min(n_chunks, c0 + per);
  float s = 0.0f;
  if (q < len) {
#pragma unroll 4
    for (int c = c0; c < c1; ++c) s += part[(long long)c * len + q];
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && q < len) {
    float t = 0.0f;
#pragma unroll
    for (int v = 0; v < 8; ++v) t += red[v][lane];
    g[q] = t;
  }
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

// Whether a product of these sizes and operands takes the 128 x 128 tile
// kernel (its float4 accesses need widths that are multiples of 4 and
// 16-byte aligned operands; the caller's input batch need not be).
bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15) == 0; }
bool wide(int N, int K, const void *p = nullptr, const void *q = nullptr) {
  return N >= 64 && N % 4 == 0 && K >= 4 && K % 4 == 0 && aligned16(p) && aligned16(q);
}

// One layer's forward pass: Z = A W^T + b (W is N x K), Act = silu(Z) if
// given; the single-output layer writes only Z.
cudaError_t layer_forward(const float *A, const float *W, const float *bias, int B, int K, int N, float *Z,
                          float *Act, cudaStream_t s) {
  if (Act && wide(N, K, A, W) && aligned16(bias) && aligned16(Z) && aligned16(Act)) {
    const dim3 grid(blocks_for(B, TG_BM), blocks_for(N, TG_BN), 1);
    tile_gemm<true, false, TG_EPI_ACT><<<grid, TG_THREADS, 0, s>>>(A, W, B, N, K, K, K, 0, bias, nullptr, Z, N,
                                                                    Act, nullptr);
  } else if (N == 1 && !Act) {
    rowdot_kernel<<<blocks_for((long long)B * 32, 256), 256, 0, s>>>(A, W, bias, B, K, Z);
  } else {
    gemm_kernel<<<dim3(blocks_for(B, GM_BM), blocks_for(N, GM_BN)), GM_THREADS, 0, s>>>(A, W, bias, B, K, N, 1, Z,
                                                                                         Act);
  }
  return cudaGetLastError();
}

// Back-propagation from a layer (dZ: B x o, W: o x i) into the SiLU of the
// layer below (pre-activations Zb: B x i): dZb = (dZ W) * silu'(Zb).
cudaError_t layer_backward(const float *dZ, const float *W, const float *Zb, int B, int o, int i, float *dZb,
                           cudaStream_t s) {
  if (o == 1 && i % 4 == 0 && aligned16(W) && aligned16(Zb) && aligned16(dZb)) {
    outer_dsilu_kernel<<<blocks_for((long long)B * (i / 4), 256), 256, 0, s>>>(dZ, W, Zb, B, i / 4, dZb);
    return cudaGetLastError();
  }
  if (wide(i, o, dZ, W) && aligned16(Zb) && aligned16(dZb)) {
    const dim3 grid(blocks_for(B, TG_BM), blocks_for(i, TG_BN), 1);
    tile_gemm<true, true, TG_EPI_DSILU><<<grid, TG_THREADS, 0, s>>>(dZ, W, B, i, o, o, i, 0, nullptr, Zb, dZb, i,
                                                                     nullptr, nullptr);
    return cudaGetLastError();
  }
  gemm_kernel<<<dim3(blocks_for(B, GM_BM), blocks_for(i, GM_BN)), GM_THREADS, 0, s>>>(dZ, W, nullptr, B, o, i, 0,
                                                                                       dZb, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  silu_back_kernel<<<blocks_for((long long)B * i, 256), 256, 0, s>>>(dZb, Zb, (long long)B * i);
  return cudaGetLastError();
}

// The weight and bias gradients from their per-chunk partial sums.
cudaError_t sum_chunks(const float *pw, const float *pb, int n_chunks, long long wl, int o, float *gw, float *gb,
                       cudaStream_t s) {
  chunk_sum_kernel<<<blocks_for(wl, 32), 256, 0, s>>>(pw, n_chunks, wl, gw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  chunk_sum_kernel<<<blocks_for(o, 32), 256, 0, s>>>(pb, n_chunks, o, gb);
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
      cudaError_t e = layer_forward(in, m->theta + wo, m->theta + bo, B, i, o, m->z + l * lay, m->a + l * lay, s);
      if (e != cudaSuccess) return e;
      in = m->a + l * lay;
    } else {
      cudaError_t e = layer_forward(in, m->theta + wo, m->theta + bo, B, i, o, y, nullptr, s);
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
  const int tchunks = (int)((B + TG_CHUNK - 1) / TG_CHUNK);
  m->wpart_len = (long long)(tchunks > chunks ? tchunks : chunks) * (W * (W > n_in ? W : n_in) + W);
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
    const int tch = (int)((B + TG_CHUNK - 1) / TG_CHUNK);
    // a thin layer: dZ at most 128 wide and the inputs at most 8, or the reverse
    const bool thin_dz = o <= THIN_W && o % 4 == 0 && i <= THIN_V && aligned16(dZ);
    const bool thin_a = i <= THIN_W && i % 4 == 0 && o <= THIN_V && aligned16(Ain);
    if (wide(o, 16, dZ, Ain) && wide(i, 16)) {
      // dW[n][k] = sum_r dZ[r][n] Ain[r][k], per chunk of TG_CHUNK rows: Aop(n, r) = dZ[r][n], Bop(r, k) =
      // Ain[r][k]; the bias gradient's chunk sums come with it
      float *pw = m->wpart, *pb = m->wpart + (long long)tch * wl;
      const dim3 g(blocks_for(o, TG_BM), blocks_for(i, TG_BN), tch);
      tile_gemm<false, true, TG_EPI_STORE><<<g, TG_THREADS, 0, s>>>(dZ, Ain, o, i, B, o, i, TG_CHUNK, nullptr,
                                                                     nullptr, pw, i, nullptr, pb);
      ML_TRY(cudaGetLastError());
      ML_TRY(sum_chunks(pw, pb, tch, wl, o, m->grad + wo, m->grad + bo, s));
    } else if (thin_dz || thin_a) {
      float *pw = m->wpart, *pb = m->wpart + (long long)tch * wl;
      if (thin_dz)
        wgrad_thin_kernel<true><<<tch, 256, 0, s>>>(dZ, Ain, B, o, i, pw, pb);
      else
        wgrad_thin_kernel<false><<<tch, 256, 0, s>>>(dZ, Ain, B, o, i, pw, pb);
      ML_TRY(cudaGetLastError());
      ML_TRY(sum_chunks(pw, pb, tch, wl, o, m->grad + wo, m->grad + bo, s));
    } else {
      float *pw = m->wpart, *pb = m->wpart + (long long)chunks * wl;
      dim3 g(blocks_for(i, 32), blocks_for(o, 32), chunks);
      wgrad_kernel<<<g, 256, 0, s>>>(dZ, Ain, B, o, i, pw, pb);
      ML_TRY(cudaGetLastError());
      ML_TRY(sum_chunks(pw, pb, chunks, wl, o, m->grad + wo, m->grad + bo, s));
    }
    if (l == 0) break;
    // dZ of the layer below = (dZ W) * silu'(Z below), W = o x i
    float *dA = bufs[l & 1];
    ML_TRY(layer_backward(dZ, m->theta + wo, m->z + (l - 1) * lay, B, o, i, dA, s));
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
