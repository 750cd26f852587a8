// The first-order CCZ4 formulation (58 variables) and the second-order
// formulation with reconstructed auxiliary variables (Alg. fd4-fo and Alg.
// fd4-so of Sec. "Explicit gradient reconstruction"), on a single uniform
// level, FP64, behind ccz4_fo_*.
//
// A ccz4_fo holds 58-field state buffers on the geometry of a grid (its
// patches, neighbour lookup and Sommerfeld ghost shell). Per RK4 stage:
//  - first order: one halo fill of all 58 fields, the stage kernel (every
//    variable evolved, red terms kept), the ghost-cell kernel;
//  - second order with reconstruction: a halo fill of the 25 primaries, the
//    reconstruction kernel (the auxiliary variables of every interior point
//    from FD4 derivatives of the primaries, written into the stage's input),
//    a halo fill of the 33 auxiliary variables, the stage kernel (the
//    primaries evolved without red terms), the ghost-cell kernel; after the
//    last stage the auxiliary variables are reconstructed from the new
//    primaries. This is the extra mesh sweep the paper's second-order
//    formulation needs.
// The ghost cells of every variable follow the radiative condition of the
// Sommerfeld boundary (speed somm_speed[v] for the primaries, 1 for the
// auxiliary variables).
#include <vector>

#include "fo_stage.cuh"

namespace ccz4 {
namespace {

constexpr int FO_FILL_THREADS = 256;

// Tile of fields [v0, v0 + nv) of a [58][S] state: [58][n_patches][T^3].
__global__ void __launch_bounds__(FO_FILL_THREADS) fo_fill_kernel(GridView g, const double *__restrict__ src,
                                                                  double *__restrict__ tile, int v0, int nv) {
  extern __shared__ long long fo_idx[];
  const int n = blockIdx.x;
  const int p = g.p, T = g.T, T3 = (int)g.T3;
  const int bx = __ldg(g.ijk + 3 * n) * p - HALO, by = __ldg(g.ijk + 3 * n + 1) * p - HALO,
            bz = __ldg(g.ijk + 3 * n + 2) * p - HALO;
  for (int t = threadIdx.x; t < T3; t += blockDim.x) {
    const int lz = t / (T * T), ly = (t / T) % T, lx = t % T;
    fo_idx[t] = locate(g, bx + lx, by + ly, bz + lz);
  }
  __syncthreads();
  for (int v = v0; v < v0 + nv; ++v) {
    const double *sv = src + v * g.S;
    double *tv = tile + ((long long)v * g.n_patches + n) * g.T3;
    for (int t = threadIdx.x; t < T3; t += blockDim.x) {
      const long long s = fo_idx[t];
      tv[t] = s >= 0 ? __ldg(sv + s) : 0.0;
    }
  }
}



// One thread per interior point: its auxiliary variables from the primaries'
// tile, written into the state `out`.
__global__ void __launch_bounds__(128) fo_reconstruct_kernel(GridView g, const double *__restrict__ tile,
                                                             double *__restrict__ out, double c1) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_points) return;
  const Nbhd N = fo_nbhd(g, tile, i);
  const long long S = g.S;
  auto put = [&](int v, double val) { out[v * S + i] = val; };
  fo_reconstruct_point(N, c1, put);
}

// One thread per (Sommerfeld ghost cell, variable): the radiative condition
// (Eq. exa_sommerfeld_inter) with the cell's static geometry, and the stage
// update.
template <int MODE>
__global__ void __launch_bounds__(256) fo_ghost_kernel(GridView g, ccz4_params P, const double *__restrict__ in,
                                                       const double *__restrict__ ini, FoStageArgs a) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (id >= g.n_ghost) return;
  const GhostGeo *gg = g.ghost_geo + id;
  const long long sn = __ldg(&gg->sn);
  if (sn < 0) return;
  const double geo = __ldg(&gg->geo), ir = __ldg(&gg->ir);
  double cv = 1.0;  // selected with static indices (no local copy of the parameters)
#pragma unroll
  for (int q = 0; q < NV; ++q)
    if (q == v) cv = P.somm_speed[q];
  const long long o = v * g.S + g.n_points + id;
  const double qg = __ldg(in + o);
  const double qn = __ldg(in + v * g.S + sn);
  const double k = -cv * geo * (qg - qn) - cv * ir * (qg - __ldg(ini + o));
  if (MODE < 0) {
    a.out[o] = k;
    return;
  }
  double acc = MODE == 0 ? 0.0 : a.acc[o];
  const double un = rk_combine<(MODE < 0 ? 0 : MODE), double>(a.U[o], acc, k, a.dt);
  if (MODE < 3) a.acc[o] = acc;
  a.out[o] = un;
}


template <int MODE, bool RED, bool AUX>
cudaError_t launch_interior(const GridView &g, const ccz4_params &P, const double *tile, const FoStageArgs &a,
                            cudaStream_t s) {
  if (g.p == 9)  // the paper's patch edge, with its strides compiled in
    return launch_fo_interior_p9(MODE, RED, AUX, g, P, tile, a, s);
  return launch_fo_interior_pf<MODE, RED, AUX, 0>(g, P, tile, a, s);
}

template <int MODE>
cudaError_t launch_ghost(const GridView &g, const ccz4_params &P, const double *in, const double *ini,
                         const FoStageArgs &a, cudaStream_t s) {
  if (g.n_ghost == 0) return cudaSuccess;
  const dim3 grid((unsigned)((g.n_ghost + 255) / 256), NVF);
  fo_ghost_kernel<MODE><<<grid, 256, 0, s>>>(g, P, in, ini, a);
  return cudaGetLastError();
}

// stage -1: plain right-hand side (all 58, red terms per `red`); 0..3: RK4 stage
template <int MODE>
cudaError_t launch_fo_mode(const GridView &g, const ccz4_params &P, bool first_order, const double *tile,
                           const double *in, const double *ini, const FoStageArgs &a, cudaStream_t s) {
  cudaError_t e;
  if (MODE < 0)
    e = first_order ? launch_interior<MODE, true, true>(g, P, tile, a, s)
                    : launch_interior<MODE, false, true>(g, P, tile, a, s);
  else
    e = first_order ? launch_interior<MODE, true, true>(g, P, tile, a, s)
                    : launch_interior<MODE, false, false>(g, P, tile, a, s);
  if (e != cudaSuccess) return e;
  return launch_ghost<MODE>(g, P, in, ini, a, s);
}

cudaError_t launch_fo(int stage, const GridView &g, const ccz4_params &P, bool first_order, const double *tile,
                      const double *in, const double *ini, const FoStageArgs &a, cudaStream_t s) {
  switch (stage) {
    case -1: return launch_fo_mode<-1>(g, P, first_order, tile, in, ini, a, s);
    case 0: return launch_fo_mode<0>(g, P, first_order, tile, in, ini, a, s);
    case 1: return launch_fo_mode<1>(g, P, first_order, tile, in, ini, a, s);
    case 2: return launch_fo_mode<2>(g, P, first_order, tile, in, ini, a, s);
    case 3: return launch_fo_mode<3>(g, P, first_order, tile, in, ini, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace ccz4

using namespace ccz4;

struct ccz4_fo {
  ccz4_grid *g;
  int variant;
  double *buf[6];  // U, Y0, Y1, ACC, RHS, INI: [58][S]
  double *tile;    // [58][n_patches][T^3]
};

static const int kFoIn[4] = {CCZ4_BUF_U, CCZ4_BUF_Y0, CCZ4_BUF_Y1, CCZ4_BUF_Y0};
static const int kFoOut[4] = {CCZ4_BUF_Y0, CCZ4_BUF_Y1, CCZ4_BUF_Y0, CCZ4_BUF_U};

#define FO_TRY(call)                                                               \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return CCZ4_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

static void fo_release(ccz4_fo *f) {
  if (!f) return;
  for (double *b : f->buf) cudaFree(b);
  cudaFree(f->tile);
  free(f);
}

static size_t fo_fill_smem(const GridView &v) { return sizeof(long long) * (size_t)v.T3; }

static cudaError_t fo_fill(const ccz4_fo *f, const double *src, int v0, int nv, cudaStream_t s) {
  const GridView &v = f->g->v;
  if (v.n_patches == 0) return cudaSuccess;
  fo_fill_kernel<<<v.n_patches, FO_FILL_THREADS, fo_fill_smem(v), s>>>(v, src, f->tile, v0, nv);
  return cudaGetLastError();
}

static cudaError_t fo_reconstruct_into(const ccz4_fo *f, double *state, cudaStream_t s) {
  const GridView &v = f->g->v;
  cudaError_t e = fo_fill(f, state, 0, NV, s);
  if (e != cudaSuccess || v.n_points == 0) return e;
  fo_reconstruct_kernel<<<(unsigned)((v.n_points + 127) / 128), 128, 0, s>>>(v, f->tile, state, 1.0 / (12.0 * v.dx));
  return cudaGetLastError();
}

static const double *fo_ini(const ccz4_fo *f) {
  return f->buf[CCZ4_BUF_INI] ? f->buf[CCZ4_BUF_INI] : f->buf[CCZ4_BUF_U];
}

static bool fo_check(const ccz4_fo *f, const ccz4_params *P) {
  if (!f || !P) {
    set_error("fo: handle and parameters must be given");
    return false;
  }
  return true;
}

extern "C" ccz4_status ccz4_fo_alloc(ccz4_grid *g, int variant, ccz4_fo **out) {
  if (!out || !g) {
    set_error("fo_alloc: grid and out must be given");
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  if (variant != CCZ4_FO_FIRST_ORDER && variant != CCZ4_FO_SO_RECONSTRUCT) {
    set_error("fo_alloc: unknown variant %d", variant);
    return CCZ4_ERR_INVALID;
  }
  if (g->v.n_levels > 1 || g->v.src) {
    set_error("fo_alloc: the 58-variable formulations run on a single uniform level, not on a refined mesh");
    return CCZ4_ERR_INVALID;
  }
  ccz4_fo *f = (ccz4_fo *)calloc(1, sizeof(ccz4_fo));
  if (!f) {
    set_error("host allocation failed");
    return CCZ4_ERR_NOMEM;
  }
  f->g = g;
  f->variant = variant;
  const GridView &v = g->v;
  const size_t state = sizeof(double) * (size_t)NVF * (size_t)v.S;
  for (int b = 0; b < 6; ++b) {
    if (b == CCZ4_BUF_INI && v.n_ghost == 0) continue;
    if (cudaMalloc(&f->buf[b], state) != cudaSuccess || cudaMemset(f->buf[b], 0, state) != cudaSuccess) {
      set_error("fo_alloc: cudaMalloc of %zu bytes failed: %s", state, cudaGetErrorString(cudaGetLastError()));
      fo_release(f);
      return CCZ4_ERR_NOMEM;
    }
  }
  const size_t tile = sizeof(double) * (size_t)NVF * (size_t)v.n_patches * (size_t)v.T3;
  if (cudaMalloc(&f->tile, tile) != cudaSuccess) {
    set_error("fo_alloc: cudaMalloc of the %zu-byte tile failed: %s", tile, cudaGetErrorString(cudaGetLastError()));
    fo_release(f);
    return CCZ4_ERR_NOMEM;
  }
  cudaError_t e = cudaFuncSetAttribute((const void *)fo_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fo_fill_smem(v));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("fo_alloc: set-up failed: %s", cudaGetErrorString(e));
    fo_release(f);
    return CCZ4_ERR_CUDA;
  }
  *out = f;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_fo_free(ccz4_fo *f) {
  fo_release(f);
  return CCZ4_OK;
}

static ccz4_status fo_copy(ccz4_fo *f, int buf, double *U, double *G, bool to_device, cudaStream_t s) {
  if (!f || buf < CCZ4_BUF_U || buf > CCZ4_BUF_INI || !f->buf[buf] || !U) {
    set_error("fo upload/download: handle, a state buffer of this formulation (U..INI) and U must be given");
    return CCZ4_ERR_INVALID;
  }
  const GridView &v = f->g->v;
  if (v.n_ghost > 0 && !G) {
    set_error("fo upload/download: this grid has %lld Sommerfeld ghost cells; G must be given", v.n_ghost);
    return CCZ4_ERR_INVALID;
  }
  const size_t dp = sizeof(double) * (size_t)v.S;
  double *d = f->buf[buf];
  if (to_device) {
    FO_TRY(cudaMemcpy2DAsync(d, dp, U, sizeof(double) * v.n_points, sizeof(double) * v.n_points, NVF,
                             cudaMemcpyHostToDevice, s));
    if (v.n_ghost)
      FO_TRY(cudaMemcpy2DAsync(d + v.n_points, dp, G, sizeof(double) * v.n_ghost, sizeof(double) * v.n_ghost, NVF,
                               cudaMemcpyHostToDevice, s));
  } else {
    FO_TRY(cudaMemcpy2DAsync(U, sizeof(double) * v.n_points, d, dp, sizeof(double) * v.n_points, NVF,
                             cudaMemcpyDeviceToHost, s));
    if (v.n_ghost)
      FO_TRY(cudaMemcpy2DAsync(G, sizeof(double) * v.n_ghost, d + v.n_points, dp, sizeof(double) * v.n_ghost, NVF,
                               cudaMemcpyDeviceToHost, s));
  }
  FO_TRY(cudaStreamSynchronize(s));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_fo_upload(ccz4_fo *f, int buf, const double *U, const double *G, void *stream) {
  return fo_copy(f, buf, const_cast<double *>(U), const_cast<double *>(G), true, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_fo_download(ccz4_fo *f, int buf, double *U, double *G, void *stream) {
  return fo_copy(f, buf, U, G, false, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_fo_reconstruct(ccz4_fo *f, int buf, void *stream) {
  if (!f || buf < CCZ4_BUF_U || buf > CCZ4_BUF_INI || !f->buf[buf]) {
    set_error("fo_reconstruct: handle and a state buffer (U..INI) must be given");
    return CCZ4_ERR_INVALID;
  }
  FO_TRY(fo_reconstruct_into(f, f->buf[buf], (cudaStream_t)stream));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_fo_rhs(ccz4_fo *f, const ccz4_params *P, int in_buf, int out_buf, void *stream) {
  if (!fo_check(f, P)) return CCZ4_ERR_INVALID;
  if (in_buf < CCZ4_BUF_U || in_buf > CCZ4_BUF_INI || out_buf < CCZ4_BUF_U || out_buf > CCZ4_BUF_INI ||
      in_buf == out_buf || !f->buf[in_buf] || !f->buf[out_buf]) {
    set_error("fo_rhs: in and out must be distinct state buffers of this formulation");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const double *in = f->buf[in_buf];
  FO_TRY(fo_fill(f, in, 0, NVF, s));
  FoStageArgs a{nullptr, nullptr, f->buf[out_buf], 0.0};
  FO_TRY(launch_fo(-1, f->g->v, *P, f->variant == CCZ4_FO_FIRST_ORDER, f->tile, in, fo_ini(f), a, s));
  return CCZ4_OK;
}

// One RK4 stage: the fills (and, second order, the reconstruction), the
// stage kernel and the ghost cells; stage 3 ends the step (enforcement in
// the stage kernel; second order: the auxiliary variables of U_{n+1}
// reconstructed).
static ccz4_status fo_stage(ccz4_fo *f, const ccz4_params *P, int stage, double dt, cudaStream_t s) {
  double *in = f->buf[kFoIn[stage]];
  const bool first = f->variant == CCZ4_FO_FIRST_ORDER;
  if (first) {
    FO_TRY(fo_fill(f, in, 0, NVF, s));
  } else {
    FO_TRY(fo_reconstruct_into(f, in, s));
    FO_TRY(fo_fill(f, in, NV, NVF - NV, s));
  }
  FoStageArgs a{f->buf[CCZ4_BUF_U], f->buf[CCZ4_BUF_ACC], f->buf[kFoOut[stage]], dt};
  FO_TRY(launch_fo(stage, f->g->v, *P, first, f->tile, in, fo_ini(f), a, s));
  if (stage == 3 && !first) FO_TRY(fo_reconstruct_into(f, f->buf[CCZ4_BUF_U], s));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_fo_rk_stage(ccz4_fo *f, const ccz4_params *P, int stage, double dt, void *stream) {
  if (!fo_check(f, P)) return CCZ4_ERR_INVALID;
  if (stage < 0 || stage > 3 || !(dt == dt)) {
    set_error("fo_rk_stage: stage must be 0..3 (got %d) and dt finite", stage);
    return CCZ4_ERR_INVALID;
  }
  return fo_stage(f, P, stage, dt, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_fo_step(ccz4_fo *f, const ccz4_params *P, double dt, int n_steps, void *stream) {
  if (!fo_check(f, P)) return CCZ4_ERR_INVALID;
  if (n_steps < 0 || !(dt == dt)) {
    set_error("fo_step: n_steps must be >= 0 and dt finite");
    return CCZ4_ERR_INVALID;
  }
  for (int n = 0; n < n_steps; ++n)
    for (int st = 0; st < 4; ++st) {
      ccz4_status r = fo_stage(f, P, st, dt, (cudaStream_t)stream);
      if (r != CCZ4_OK) return r;
    }
  return CCZ4_OK;
}
