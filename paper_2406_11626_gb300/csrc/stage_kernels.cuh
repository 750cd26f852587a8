// Right-hand side and fused RK4 stage kernels (templates; rhs.cu
// instantiates them for a single level, rhs_mesh.cu for refined meshes, so
// the two sets compile in parallel).
//
// interior_kernel: one thread per interior point reads its halo'd
// neighbourhood from the tile buffer, evaluates the CCZ4 right-hand side
// plus Kreiss-Oliger dissipation, and either stores it (plain RHS) or
// applies the RK4 stage update in the same pass, so the right-hand side
// never travels through HBM. The last stage also enforces the algebraic
// constraints on the new state. R is the type of the pointwise algebra
// (double: FP64 path; float: mixed path).
// On a refined mesh each thread takes the stencil coefficients of its
// patch's level.
// ghost_kernel: one thread per evolved Sommerfeld ghost cell (Eq.
// exa_sommerfeld_inter; the ghost shell of level 0), same stage update, no
// enforcement, FP64.
#pragma once

#include "ccz4_algebra.cuh"
#include "deriv_tap.cuh"

// Minimum resident blocks of 128 threads per SM requested for the stage
// kernel. 4 caps ptxas at 128 registers per thread (16 warps per SM): the
// kernel spills more than at 255 registers (8 warps per SM), but the extra
// warps hide the latency of the narrow FP64 pipe and of instruction fetch
// (measured on GB300: 51.2 -> 42.5 ms per RK4 step for the mixed path at
// 144^3, 62.7 -> 62.2 ms for the FP64 path).
#ifndef CCZ4_INTERIOR_MIN_BLOCKS
#define CCZ4_INTERIOR_MIN_BLOCKS 4
#endif
// The same for the mixed-precision instances (R = float): 3 blocks (168
// registers). The mixed kernel is held by its register spills rather than
// by the FP64 pipe; with 3 blocks their footprint (resident threads times
// stack) fits in L2, and with the streaming hints below the tiles and the
// state do not push it out (measured on GB300, ms per RK4 step at 144^3:
// 26.16 against 28.30 with 5 blocks and plain loads, 28.21 with 5 blocks
// and streaming, 29.88 with 3 blocks and plain loads).
#ifndef CCZ4_INTERIOR_MIN_BLOCKS_MIXED
#define CCZ4_INTERIOR_MIN_BLOCKS_MIXED 3
#endif
// Register spills of the stage kernel go to shared memory first (the
// kernel uses none otherwise; ptxas places 104 bytes per thread there) and
// only then to local memory. Measured on GB300: mixed path 1 % faster per
// step, FP64 path unchanged. Set to 0 to spill to local memory only.
#ifndef CCZ4_SMEM_SPILL
#define CCZ4_SMEM_SPILL 1
#endif

// The last stage's enforcement reads the new g~ and A~ back from the output
// (written there as soon as they are known, by the same thread) instead of
// holding them in registers through the rest of the right-hand side, which
// frees 12 registers for the algebra. 0: hold them.
#ifndef CCZ4_ENFORCE_RELOAD
#define CCZ4_ENFORCE_RELOAD 1
#endif

// State, accumulator and output of the stage update: streaming
// (evict-first) loads and stores, each value is touched once, which leaves
// L2 to the kernel's register spills; 0 for plain ones.
#ifndef CCZ4_STAGE_STREAM
#define CCZ4_STAGE_STREAM 1
#endif

namespace ccz4 {

__device__ __forceinline__ double st_ld(const double *p) {
#if CCZ4_STAGE_STREAM
  return __ldcs(p);
#else
  return *p;
#endif
}
__device__ __forceinline__ void st_st(double *p, double v) {
#if CCZ4_STAGE_STREAM
  __stcs(p, v);
#else
  *p = v;
#endif
}

struct StageArgs {
  const double *U;  // U_n
  double *acc;      // RK accumulator
  double *out;      // plain RHS (MODE < 0), next stage state, or U_{n+1}
  double dt;
};


// Stencil coefficients of every level, in the differencing type (double)
// and in the algebra type R.
template <class R>
struct LevelCoef {
  StencilCoef<double> C[MAX_LEVELS];
  StencilCoef<R> CR[MAX_LEVELS];
};

// Flat stage-kernel launches of the shapes other than the default (one
// resident block more or fewer, CCZ4_STAGE_SHAPE_*), RK4 stages 0..3 only;
// instantiated in rhs_shapes.cu (single level) and rhs_mesh_shapes.cu.
cudaError_t launch_shaped_uniform(const GridView &g, int stage, const Phys<double> &ph, const LevelCoef<double> &LC,
                                  const double *tile, const double *mix, const StageArgs &a, cudaStream_t s);
cudaError_t launch_shaped_uniform(const GridView &g, int stage, const Phys<float> &ph, const LevelCoef<float> &LC,
                                  const double *tile, const double *mix, const StageArgs &a, cudaStream_t s);
cudaError_t launch_shaped_mesh(const GridView &g, int stage, const Phys<double> &ph, const LevelCoef<double> &LC,
                               const double *tile, const double *mix, const StageArgs &a, cudaStream_t s);
cudaError_t launch_shaped_mesh(const GridView &g, int stage, const Phys<float> &ph, const LevelCoef<float> &LC,
                               const double *tile, const double *mix, const StageArgs &a, cudaStream_t s);

// Raise the shared-memory limits of the two-phase kernels (rhs_shapes.cu,
// rhs_mesh_shapes.cu); once per grid, outside any stream capture.
cudaError_t prepare_shaped_uniform();
cudaError_t prepare_shaped_mesh();

// Launches stage `stage` (-1: plain RHS) with the kernels of a single level
// (rhs.cu) or of a refined mesh (rhs_mesh.cu).
cudaError_t launch_stage_uniform(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                                 const double *mix, const double *in, const double *ini, const StageArgs &a,
                                 cudaStream_t s);
cudaError_t launch_stage_mesh(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                              const double *mix, const double *in, const double *ini, const StageArgs &a,
                              cudaStream_t s);

namespace {


// MODE < 0: store k. MODE = s in 0..3: RK4 stage s.
template <int MODE>
__device__ __forceinline__ void finish_point(const GridView &g, long long i, double k[NV],
                                             const StageArgs &a, bool interior) {
  const long long S = g.S;
  if (MODE < 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a.out[v * S + i] = k[v];
    return;
  }
  double un[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double acc = MODE == 0 ? 0.0 : a.acc[v * S + i];
    un[v] = rk_combine<(MODE < 0 ? 0 : MODE), double>(a.U[v * S + i], acc, k[v], a.dt);
    if (MODE < 3) a.acc[v * S + i] = acc;
  }
  if (MODE == 3 && interior) enforce_point<double>(un + GXX, un + AXX);
#pragma unroll
  for (int v = 0; v < NV; ++v) a.out[v * S + i] = un[v];
}

// Receives d_t Q_v of one interior point field by field and applies the
// stage update at once, so finished values leave the registers early. The
// last stage holds g~ and A~ back for the algebraic enforcement.
template <int MODE>
struct StageSink {
  const GridView &g;
  long long i;
  const StageArgs &a;
  double ug[6], uA[6];
  __device__ __forceinline__ void operator()(int v, double k) {
    const long long o = v * g.S + i;
    if (MODE < 0) {
      st_st(a.out + o, k);
      return;
    }
    double acc = MODE == 0 ? 0.0 : st_ld(a.acc + o);
    const double un = rk_combine<(MODE < 0 ? 0 : MODE), double>(st_ld(a.U + o), acc, k, a.dt);
    if (MODE < 3) st_st(a.acc + o, acc);
    if (!CCZ4_ENFORCE_RELOAD && MODE == 3 && v >= GXX && v <= GZZ) {
      ug[v - GXX] = un;
      return;
    }
    if (!CCZ4_ENFORCE_RELOAD && MODE == 3 && v >= AXX && v <= AZZ) {
      uA[v - AXX] = un;
      return;
    }
    st_st(a.out + o, un);
  }
  __device__ __forceinline__ void finish() {
    if (MODE != 3) return;
    if (CCZ4_ENFORCE_RELOAD) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        ug[c] = st_ld(a.out + (GXX + c) * g.S + i);
        uA[c] = st_ld(a.out + (AXX + c) * g.S + i);
      }
    }
    enforce_point<double>(ug, uA);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      st_st(a.out + (GXX + c) * g.S + i, ug[c]);
      st_st(a.out + (AXX + c) * g.S + i, uA[c]);
    }
  }
};

// Resident blocks of 128 threads per SM that a launch shape asks of the
// stage kernel: the default of the precision, one more (shape 1) or one
// fewer (shape 2).
template <class R, int SHAPE>
struct StageBlocks {
  static constexpr int base = std::is_same<R, float>::value ? CCZ4_INTERIOR_MIN_BLOCKS_MIXED : CCZ4_INTERIOR_MIN_BLOCKS;
  static constexpr int value = SHAPE == 1 ? base + 1 : SHAPE == 2 ? (base > 1 ? base - 1 : 1) : base;
};

// Neighbourhood of interior point i of patch n in the tile and mixed-derivative buffers.
__device__ __forceinline__ Nbhd point_nbhd(const GridView &g, const double *tile, const double *mix, long long i, int n) {
  const int p = g.p, T = g.T;
  const int p3 = p * p * p;
  const int r = (int)(i - n * p3);
  const int z = r / (p * p), y = (r / p) % p, x = r % p;
  Nbhd N;
  N.c = tile + n * g.T3 + ((long long)(z + HALO) * T + (y + HALO)) * T + (x + HALO);
  N.fs = (long long)g.n_patches * g.T3;
  N.st[0] = 1;
  N.st[1] = T;
  N.st[2] = T * T;
  N.mix = mix + i;
  N.ms = g.n_points;
  N.mixf = reinterpret_cast<const float *>(mix) + i;
  N.msf = g.n_points;
  return N;
}

// One interior point of the stage. PF > 0: the patch edge is PF (the
// grid's p must equal it), so the tile strides and the index divisions are
// compile-time constants (immediate offsets in the loads, multiply-shift
// divisions, no registers holding strides).
template <int MODE, class R, bool MESH, int PF = 0>
__device__ __forceinline__ void stage_point(const GridView &g, const Phys<R> &P, const LevelCoef<R> &LC,
                                            const double *__restrict__ tile, const double *__restrict__ mix,
                                            const StageArgs &a, long long i) {
  const int p = PF > 0 ? PF : g.p, T = PF > 0 ? PF + 2 * HALO : g.T;
  // 32-bit division (every state index is below 2^31): a 64-bit integer
  // division is a long software sequence
  const int p3 = p * p * p;
  const int n = (int)i / p3;
  // a run-time index into the parameter array is only taken on a mesh (it
  // makes ptxas keep a local copy of the array)
  const int lev = MESH ? patch_level(g, n) : 0;
  const StencilCoef<double> C = MESH ? LC.C[lev] : LC.C[0];
  const StencilCoef<R> CR = MESH ? LC.CR[lev] : LC.CR[0];
  const int r = (int)(i - n * p3);
  const int z = r / (p * p), y = (r / p) % p, x = r % p;
  Nbhd N;
  const int T3 = PF > 0 ? T * T * T : g.T3;
  N.c = tile + (long long)n * T3 + ((long long)(z + HALO) * T + (y + HALO)) * T + (x + HALO);
  N.fs = (long long)g.n_patches * T3;
  N.st[0] = 1;
  N.st[1] = T;
  N.st[2] = T * T;
  N.mix = mix + i;
  N.ms = g.n_points;
  N.mixf = reinterpret_cast<const float *>(mix) + i;  // read only by the mixed path (R = float)
  N.msf = g.n_points;
  StageSink<MODE> sink{g, i, a};
  ccz4_rhs_point<double, R>(P, N, C, CR, sink);
  sink.finish();
}

// The two-phase launch shape of the mixed-precision stage kernel
// (CCZ4_STAGE_SHAPE_SPLIT): each thread first takes all the stencil values
// of its point and parks them in its shared-memory slots (DerivTap,
// recording with a sink that discards the right-hand side, so the algebra
// is dead code), then, after a barrier, evaluates the right-hand side and
// the stage update reading them back. The first phase holds few values
// live and keeps many tile loads in flight; the second has none in flight.
// 2 resident blocks of 128 threads: 255 registers and 76 KB of slots each.
template <int MODE, bool MESH>
__global__ void __launch_bounds__(128, 2) split_kernel(GridView g, Phys<float> P, LevelCoef<float> LC,
                                                       const double *__restrict__ tile, const double *__restrict__ mix,
                                                       StageArgs a) {
  extern __shared__ double tap_slots[];
  double *sd = tap_slots + threadIdx.x;
  float *sf = reinterpret_cast<float *>(tap_slots + TAP_DOUBLES * blockDim.x) + threadIdx.x;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < g.n_points;
  const int n = active ? (int)i / (g.p * g.p * g.p) : 0;
  const int lev = MESH ? patch_level(g, n) : 0;
  const StencilCoef<double> C = MESH ? LC.C[lev] : LC.C[0];
  const StencilCoef<float> CR = MESH ? LC.CR[lev] : LC.CR[0];
  if (active) {
    const Nbhd N = point_nbhd(g, tile, mix, i, n);
    DerivTap<TAP_RECORD> T(N, sf, sd, blockDim.x);
    NullSink none;
    ccz4_rhs_point<double, float>(P, T, C, CR, none);
  }
  __syncthreads();
  if (active) {
    const Nbhd N = point_nbhd(g, tile, mix, i, n);
    DerivTap<TAP_REPLAY> T(N, sf, sd, blockDim.x);
    StageSink<MODE> sink{g, i, a};
    ccz4_rhs_point<double, float>(P, T, C, CR, sink);
    sink.finish();
  }
}

constexpr size_t SPLIT_SMEM = (sizeof(double) * TAP_DOUBLES + sizeof(float) * TAP_FLOATS) * 128;

// Next 32-point work item of a warp from the device queue (g.queue).
__device__ __forceinline__ long long next_item(const GridView &g, int lane) {
  unsigned long long q = 0;
  if (lane == 0) q = atomicAdd(g.queue, 1ULL);
  return (long long)__shfl_sync(0xffffffffu, q, 0);
}

// Every interior point of every level.
// Flat launch (QUEUE false): one thread per point.
// Queue launch (QUEUE, the grid sized to the resident blocks): each warp
// takes 32-point items from the device counter g.queue until none is left,
// so no block waits for a wave to drain; nothing waits on another thread.
// The two are separate instances: the loop costs the flat kernel registers.
template <int MODE, class R, bool MESH, bool QUEUE, int SHAPE = 0, int PF = 0>
__global__ void __launch_bounds__(128, (StageBlocks<R, SHAPE>::value)) interior_kernel(GridView g, Phys<R> P, LevelCoef<R> LC,
                                                          const double *__restrict__ tile,
                                                          const double *__restrict__ mix, StageArgs a) {
#if CCZ4_SMEM_SPILL
  asm volatile(".pragma \"enable_smem_spilling\";");
#endif
  if (!QUEUE) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.n_points) stage_point<MODE, R, MESH, PF>(g, P, LC, tile, mix, a, i);
    return;
  }
  const int lane = threadIdx.x & 31;
  for (long long item = next_item(g, lane); item * 32 < g.n_points; item = next_item(g, lane)) {
    const long long i = item * 32 + lane;
    if (i < g.n_points) stage_point<MODE, R, MESH, PF>(g, P, LC, tile, mix, a, i);
  }
}

// One thread per (evolved Sommerfeld ghost cell, field): the ghost-cell
// ODE (Eq. exa_sommerfeld_inter) with the cell's static geometry from
// g.ghost_geo, and the same stage update, no enforcement, FP64.
template <int MODE>
__device__ __forceinline__ void ghost_point(const GridView &g, const ccz4_params &P, const double *__restrict__ in,
                                            const double *__restrict__ ini, const StageArgs &a, long long id,
                                            int v) {
  const GhostGeo *gg = g.ghost_geo + id;
  const long long sn = __ldg(&gg->sn);
  if (sn < 0) return;
  const double geo = __ldg(&gg->geo), ir = __ldg(&gg->ir);
  // the field's speed, selected with static indices (a run-time index into
  // the parameter array would copy it to local memory)
  double cv = P.somm_speed[0];
#pragma unroll
  for (int q = 1; q < NV; ++q)
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

// One thread per ghost cell, all fields: the cell's geometry is read once
// and the 25 fields' loads are independent (consecutive cells, coalesced).
template <int MODE>
__global__ void __launch_bounds__(256) ghost_kernel(GridView g, ccz4_params P, const double *__restrict__ in,
                                                    const double *__restrict__ ini, StageArgs a) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= g.n_ghost) return;
#pragma unroll
  for (int v = 0; v < NV; ++v) ghost_point<MODE>(g, P, in, ini, a, id, v);
}

StencilCoef<double> coefs(double dx, const ccz4_params &P) {
  StencilCoef<double> C;
  C.c1 = 1.0 / (12.0 * dx);
  C.c2 = 1.0 / (12.0 * dx * dx);
  C.c3 = 1.0 / (144.0 * dx * dx);
  C.cko = P.ko_eps / (64.0 * dx);
  return C;
}

// Blocks of a queue launch: every SM filled with as many blocks as fit.
template <int MODE, class R, bool MESH>
long long queue_blocks() {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, interior_kernel<MODE, R, MESH, true>, 128, 0);
  return (long long)sms * occ;
}

template <int MODE, class R, bool MESH>
cudaError_t launch_mode(const GridView &g, const ccz4_params &P, const double *tile, const double *mix,
                        const double *in, const double *ini, const StageArgs &a, cudaStream_t s) {
  if (g.n_points > 0) {
    long long blocks = (g.n_points + 127) / 128;
    if (g.queue) {
      const long long qb = queue_blocks<MODE, R, MESH>();
      if (qb <= 0) return cudaErrorInvalidConfiguration;
      blocks = qb < blocks ? qb : blocks;
      cudaError_t e = cudaMemsetAsync(g.queue, 0, sizeof(unsigned long long), s);
      if (e != cudaSuccess) return e;
    }
    LevelCoef<R> LC;
    for (int l = 0; l < MAX_LEVELS; ++l) {
      const StencilCoef<double> C = coefs(g.ldx[l], P);
      LC.C[l] = C;
      LC.CR[l] = StencilCoef<R>{R(C.c1), R(C.c2), R(C.c3), R(C.cko)};
    }
    cudaError_t e;
    if (g.queue) {
      interior_kernel<MODE, R, MESH, true><<<(unsigned)blocks, 128, 0, s>>>(g, make_phys<R>(P), LC, tile, mix, a);
      e = cudaGetLastError();
    } else if (MODE >= 0 && g.stage_shape != 0) {
      e = MESH ? launch_shaped_mesh(g, MODE, make_phys<R>(P), LC, tile, mix, a, s)
               : launch_shaped_uniform(g, MODE, make_phys<R>(P), LC, tile, mix, a, s);
    } else if (g.p == 9) {  // the paper's patch edge, with its strides compiled in
      interior_kernel<MODE, R, MESH, false, 0, 9><<<(unsigned)blocks, 128, 0, s>>>(g, make_phys<R>(P), LC, tile,
                                                                                   mix, a);
      e = cudaGetLastError();
    } else {
      interior_kernel<MODE, R, MESH, false><<<(unsigned)blocks, 128, 0, s>>>(g, make_phys<R>(P), LC, tile, mix, a);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  if (g.n_ghost > 0) {
    ghost_kernel<MODE><<<(unsigned)((g.n_ghost + 255) / 256), 256, 0, s>>>(g, P, in, ini, a);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

template <int MODE, bool MESH>
cudaError_t launch_prec(const GridView &g, const ccz4_params &P, const double *tile, const double *mix,
                        const double *in, const double *ini, const StageArgs &a, cudaStream_t s) {
  if (P.precision == CCZ4_PREC_MIXED) return launch_mode<MODE, float, MESH>(g, P, tile, mix, in, ini, a, s);
  return launch_mode<MODE, double, MESH>(g, P, tile, mix, in, ini, a, s);
}

// stage -1: plain right-hand side; 0..3: RK4 stage
template <bool MESH>
cudaError_t launch_stage(const GridView &g, const ccz4_params &P, int stage, const double *tile,
                         const double *mix, const double *in, const double *ini, const StageArgs &a,
                         cudaStream_t s) {
  switch (stage) {
    case -1: return launch_prec<-1, MESH>(g, P, tile, mix, in, ini, a, s);
    case 0: return launch_prec<0, MESH>(g, P, tile, mix, in, ini, a, s);
    case 1: return launch_prec<1, MESH>(g, P, tile, mix, in, ini, a, s);
    case 2: return launch_prec<2, MESH>(g, P, tile, mix, in, ini, a, s);
    case 3: return launch_prec<3, MESH>(g, P, tile, mix, in, ini, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// Flat launch of stage MODE (0..3) in launch shape SHAPE.
template <class R, bool MESH, int SHAPE>
cudaError_t launch_flat_shape(const GridView &g, int stage, const Phys<R> &ph, const LevelCoef<R> &LC,
                              const double *tile, const double *mix, const StageArgs &a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((g.n_points + 127) / 128);
  switch (stage) {
    case 0: interior_kernel<0, R, MESH, false, SHAPE><<<blocks, 128, 0, s>>>(g, ph, LC, tile, mix, a); break;
    case 1: interior_kernel<1, R, MESH, false, SHAPE><<<blocks, 128, 0, s>>>(g, ph, LC, tile, mix, a); break;
    case 2: interior_kernel<2, R, MESH, false, SHAPE><<<blocks, 128, 0, s>>>(g, ph, LC, tile, mix, a); break;
    case 3: interior_kernel<3, R, MESH, false, SHAPE><<<blocks, 128, 0, s>>>(g, ph, LC, tile, mix, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool MESH>
cudaError_t launch_split(const GridView &g, int stage, const Phys<float> &ph, const LevelCoef<float> &LC,
                         const double *tile, const double *mix, const StageArgs &a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((g.n_points + 127) / 128);
  switch (stage) {
    case 0: split_kernel<0, MESH><<<blocks, 128, SPLIT_SMEM, s>>>(g, ph, LC, tile, mix, a); break;
    case 1: split_kernel<1, MESH><<<blocks, 128, SPLIT_SMEM, s>>>(g, ph, LC, tile, mix, a); break;
    case 2: split_kernel<2, MESH><<<blocks, 128, SPLIT_SMEM, s>>>(g, ph, LC, tile, mix, a); break;
    case 3: split_kernel<3, MESH><<<blocks, 128, SPLIT_SMEM, s>>>(g, ph, LC, tile, mix, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Raises the shared-memory limit of the two-phase kernels (once per grid,
// outside any stream capture).
template <bool MESH>
cudaError_t prepare_split() {
  const void *k[4] = {(const void *)split_kernel<0, MESH>, (const void *)split_kernel<1, MESH>,
                      (const void *)split_kernel<2, MESH>, (const void *)split_kernel<3, MESH>};
  for (const void *f : k) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPLIT_SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class R, bool MESH>
cudaError_t launch_shaped(const GridView &g, int stage, const Phys<R> &ph, const LevelCoef<R> &LC, const double *tile,
                          const double *mix, const StageArgs &a, cudaStream_t s) {
  if (g.stage_shape == 1) return launch_flat_shape<R, MESH, 1>(g, stage, ph, LC, tile, mix, a, s);
  if (g.stage_shape == 2) return launch_flat_shape<R, MESH, 2>(g, stage, ph, LC, tile, mix, a, s);
  if (g.stage_shape == 3) {
    // the two-phase shape exists for the mixed path; the FP64 path keeps its default
    if constexpr (std::is_same<R, float>::value) return launch_split<MESH>(g, stage, ph, LC, tile, mix, a, s);
    else return launch_flat_shape<R, MESH, 0>(g, stage, ph, LC, tile, mix, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace ccz4
