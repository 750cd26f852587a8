// The halo fill of one patch (Sec. "Spatial Discretisation", Fig.
// patch-face-reconstruction) as a block-level device function, with its
// helpers: used by the fill kernel (halo.cu) and by the stage kernel that
// fills and evolves in one cooperative launch (rhs_fused.cu).
#ifndef CCZ4_HALO_FILL_CUH
#define CCZ4_HALO_FILL_CUH

#include "ccz4_algebra.cuh"
#include "ccz4_internal.cuh"

namespace ccz4 {
namespace {

// Launch shapes of the fill (threads per block, independent loads per
// thread in the gather), chosen per grid (CCZ4_FILL_SHAPE_*): 0 the
// default 256 threads and 8 loads, 1 512 threads, 2 16 loads, 3 128
// threads. Each asks for 1024 threads' worth of resident blocks.
constexpr int FILL_SHAPE_THREADS[4] = {256, 512, 256, 128};
constexpr int FILL_SHAPE_BATCH[4] = {8, 8, 16, 8};
constexpr size_t FILL_SMEM_LIMIT = 227 * 1024;  // dynamic shared memory one block may use

// Whether the d_z pass of the mixed derivatives fits on the region widened
// along both x and y (one pass for d_x d_z and d_y d_z).
__host__ __device__ constexpr bool fill_wide(int p) {
  return sizeof(double) * ((size_t)(p + 6) * (p + 6) * (p + 6) + (size_t)(p + 4) * (p + 4) * p) +
             sizeof(int) * (size_t)(p + 6) * (p + 6) * (p + 6) <=
         FILL_SMEM_LIMIT;
}

// Scale of the mixed derivatives, 1 / (144 dx^2), per level (and rounded
// to FP32 for the FP32 weights of the mixed path).
struct LevelScale {
  double cmix[MAX_LEVELS];
  float cmixf[MAX_LEVELS];
};

// First stage of a mixed derivative at point e of the widened region: the
// (unscaled) first derivative of the tile along stride si. FP64 differences
// of the FP64 tile and FP64 weights; or, for the fields whose mixed
// derivatives the mixed path's stage kernel uses in FP32 (g~ and beta, f32
// set; their shared-memory tile holds the split pairs), the differences of
// the pairs, (hi+ - hi-) + (lo+ - lo-), and the weights in FP32, with the
// result kept as FP32 (as the stage kernel takes its own first derivatives).
__device__ __forceinline__ void mixed_in(double *ext, int e, const double *ts, int c0, int si, bool f32) {
  if (f32) {
    const float2 *tf = reinterpret_cast<const float2 *>(ts);
    const float2 p1 = tf[c0 + si], m1 = tf[c0 - si], p2 = tf[c0 + 2 * si], m2 = tf[c0 - 2 * si];
    const float a = (p1.x - m1.x) + (p1.y - m1.y), b = (p2.x - m2.x) + (p2.y - m2.y);
    reinterpret_cast<float *>(ext)[e] = fmaf(8.0f, a, -b);
  } else {
    const double a = ts[c0 + si] - ts[c0 - si], b = ts[c0 + 2 * si] - ts[c0 - 2 * si];
    ext[e] = fma(8.0, a, -b);
  }
}

// Second stage: d_a of the first derivatives at ext[e] along stride s, stored
// to mixed-derivative slot `slot` of this patch's point q. FP64 differences
// and weights and an FP64 slot; or (f32) the differences of the FP32 first
// derivatives in FP32 (a subtraction of two FP32 numbers is exact when it
// cancels and otherwise within half an ulp of its result), the weights in
// FP32 and an FP32 slot (half the traffic).
__device__ __forceinline__ void mixed_out(const double *ext, int e, int s, double cmix, float cmixf, bool f32,
                                          double *mix, long long n_points, long long pbase, int slot, int q) {
  if (f32) {
    const float *ef = reinterpret_cast<const float *>(ext) + e;
    const float d1 = ef[s] - ef[-s], d2 = ef[2 * s] - ef[-2 * s];
    float *mf = reinterpret_cast<float *>(mix) + (long long)mix_fslot(slot) * n_points + pbase;
    __stcs(mf + q, fmaf(8.0f, d1, -d2) * cmixf);
  } else {
    const double *ed = ext + e;
    const double d1 = ed[s] - ed[-s], d2 = ed[2 * s] - ed[-2 * s];
    __stcs(mix + (long long)slot * n_points + pbase + q, fma(8.0, d1, -d2) * cmix);
  }
}

// Linear-interpolation weights between coarse cell centres for remainder
// r = (i - 1) mod 3 of fine index i: the rows (1), (2/3, 1/3), (1/3, 2/3)
// of the printed matrices P^par and P^perp.
__device__ __forceinline__ double pw(int r, int k) {
  return r == 0 ? (k == 0 ? 1.0 : 0.0) : r == 1 ? (k == 0 ? 2.0 / 3.0 : 1.0 / 3.0) : (k == 0 ? 1.0 / 3.0 : 2.0 / 3.0);
}

// Value of an interpolated halo point of a refined mesh from the corner
// indices c[8] and remainders (rx, ry, rz) of its entry: the tensor product
// of three linear maps, along x, then y, then z; every product and sum is
// rounded on its own (no fused multiply-add), in that order. A corner along
// an axis with remainder 0 has weight zero and is not read.
__device__ __forceinline__ double interp_value(const int (&c)[8], int rx, int ry, int rz,
                                               const double *__restrict__ sv) {
  double t[2][2], u[2];
#pragma unroll
  for (int cz = 0; cz < 2; ++cz) {
    if (cz == 1 && rz == 0) break;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (b == 1 && ry == 0) break;
      const double q0 = __ldg(sv + c[(cz * 2 + b) * 2]);
      t[cz][b] = rx ? __dadd_rn(__dmul_rn(pw(rx, 0), q0), __dmul_rn(pw(rx, 1), __ldg(sv + c[(cz * 2 + b) * 2 + 1])))
                    : q0;
    }
    u[cz] = ry ? __dadd_rn(__dmul_rn(pw(ry, 0), t[cz][0]), __dmul_rn(pw(ry, 1), t[cz][1])) : t[cz][0];
  }
  return rz ? __dadd_rn(__dmul_rn(pw(rz, 0), u[0]), __dmul_rn(pw(rz, 1), u[1])) : u[0];
}

// Whether field v's tile holds split pairs: in the mixed path (F32W) every
// field but alpha and phi, whose differences the mixed stage kernel takes
// in FP64 (see split_pair).
__device__ __forceinline__ bool split_field(bool f32w, int v) { return f32w && v != ALPHA && v != PHI; }

// A tile value as the stage kernel reads it: the FP64 value or its split
// pair. The fill's shared-memory tile of a field holds the same encoding.
__device__ __forceinline__ double tile_enc(double u, bool split) { return split ? split_pair(u) : u; }

// One linear map of the interpolation between a and b for remainder r, the
// product and the sum each rounded on its own; r = 0: a.
__device__ __forceinline__ double lerp3(int r, double a, double b) {
  return r ? __dadd_rn(__dmul_rn(pw(r, 0), a), __dmul_rn(pw(r, 1), b)) : a;
}

// MESH: the tile sources come from the host-built table of a refined mesh
// (and may be interpolations); otherwise they are resolved here. F32W: FP32
// weights for the mixed derivatives (see mixed_out). PF > 0: the patch edge
// is PF (the grid's p must equal it), so the index divisions of the tile
// and of the widened regions are by compile-time constants.
// The fill of patch n by one block of FILL_THREADS threads (blockDim.x ==
// FILL_THREADS), smem the block's dynamic shared memory (fill_smem_bytes).
template <bool MESH, bool F32W, int FILL_THREADS, int GATHER_BATCH, int PF = 0>
__device__ __forceinline__ void fill_patch(const GridView &g, const double *__restrict__ src,
                                           double *__restrict__ tile, double *__restrict__ mix,
                                           const LevelScale &ls, int n, double *smem) {
  const int p = PF > 0 ? PF : g.p, T = PF > 0 ? PF + 2 * HALO : g.T;
  const int T3 = PF > 0 ? T * T * T : (int)g.T3;
  const int pe = p + 4;             // patch edge widened by two points on each side
  const int next = pe * p * p;      // widened region of one first-derivative pass
  const bool wide = fill_wide(p);   // room for the region widened along two axes
  double *ts = smem;                // [T3] tile of the current field
  double *ext = smem + T3;          // [next or pe^2 p] first derivatives on the widened region
  int *idx = (int *)(ext + (wide ? pe * pe * p : next));  // [T3] source index of each tile point
  const int bx = __ldg(g.ijk + 3 * n) * p - HALO;
  const int by = __ldg(g.ijk + 3 * n + 1) * p - HALO;
  const int bz = __ldg(g.ijk + 3 * n + 2) * p - HALO;
  if (MESH) {
    // refined mesh: sources resolved once on the host
    const int *sp = g.src + (long long)n * T3;
    for (int t = threadIdx.x; t < T3; t += blockDim.x) idx[t] = __ldg(sp + t);
    // A patch without separable tables: its interpolated halo points, one
    // entry per thread, all fields at once (the entry is read once and the
    // fields' corner loads are independent). The fields that need mixed
    // derivatives read these values back from the tile after the barrier
    // below.
    const int e1 = __ldg(g.ibeg + n + 1);
    const bool by_entry = __ldg(g.xbeg + n + 1) == __ldg(g.xbeg + n);
    for (int e = by_entry ? __ldg(g.ibeg + n) + (int)threadIdx.x : e1; e < e1; e += FILL_THREADS) {
      const InterpEntry *ep = g.interp + e;
      int c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] = __ldg(&ep->src[k]);
      const int r = __ldg(&ep->r), t = __ldg(&ep->t);
      const int rx = r & 3, ry = (r >> 2) & 3, rz = (r >> 4) & 3;
      double *tp = tile + (long long)n * T3 + t;
#pragma unroll 5
      for (int v = 0; v < NV; ++v)
        __stcs(tp + (long long)v * g.n_patches * T3, tile_enc(interp_value(c, rx, ry, rz, src + v * g.S), split_field(F32W, v)));
    }
  } else {
    for (int t = threadIdx.x; t < T3; t += blockDim.x) {
      const int lz = t / (T * T), ly = (t / T) % T, lx = t % T;
      const long long s = locate(g, bx + lx, by + ly, bz + lz);
      idx[t] = (int)s;
    }
  }
  const double cmix = MESH ? ls.cmix[patch_level(g, n)] : ls.cmix[0];
  const float cmixf = MESH ? ls.cmixf[patch_level(g, n)] : ls.cmixf[0];
  __syncthreads();
  const long long p3 = (long long)p * p * p;
  const long long pbase = (long long)n * p3;
  // separable interpolation of this patch's halo points (see XJob)
  int e0 = 0, e1 = 0, xb0 = 0, nx = 0, yb0 = 0, ny = 0;
  if (MESH) {
    e0 = __ldg(g.ibeg + n);
    e1 = __ldg(g.ibeg + n + 1);
    xb0 = __ldg(g.xbeg + n);
    nx = __ldg(g.xbeg + n + 1) - xb0;
    yb0 = __ldg(g.ybeg + n);
    ny = __ldg(g.ybeg + n + 1) - yb0;
  }
  constexpr int JM = (1 << JOB_BITS) - 1;
  for (int v = 0; v < NV; ++v) {
    const double *sv = src + v * g.S;
    double *tv = tile + ((long long)v * g.n_patches + n) * T3;
    const int slot = mix_slot(v);
    const bool sp = split_field(F32W, v);
    if (MESH && nx > 0) {
      // x, then y, then z: the x and y results of the patch in the tile's
      // shared memory (host-checked to fit), the z results to the tile
      double *xv = ts, *yv = ts + nx;
      for (int j = threadIdx.x; j < nx; j += FILL_THREADS) {
        const XJob *J = g.xjob + xb0 + j;
        const int rx = __ldg(&J->rx);
        const double q0 = __ldg(sv + __ldg(&J->s0));
        xv[j] = rx ? lerp3(rx, q0, __ldg(sv + __ldg(&J->s1))) : q0;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < ny; j += FILL_THREADS) {
        const int k = __ldg(g.yjob + yb0 + j);
        yv[j] = lerp3((k >> (2 * JOB_BITS)) & 3, xv[k & JM], xv[(k >> JOB_BITS) & JM]);
      }
      __syncthreads();
      for (int e = e0 + threadIdx.x; e < e1; e += FILL_THREADS) {
        const int k = __ldg(&g.zjob[e].yab);
        __stcs(tv + __ldg(&g.zjob[e].t), tile_enc(lerp3((k >> (2 * JOB_BITS)) & 3, yv[k & JM], yv[(k >> JOB_BITS) & JM]), sp));
      }
      __syncthreads();  // the gather below overwrites the tile's shared memory
    }
    // Gather in batches of GATHER_BATCH independent loads per thread, so a
    // field costs a couple of memory latencies rather than one per point.
    for (int t0 = threadIdx.x; t0 < T3; t0 += GATHER_BATCH * FILL_THREADS) {
      double val[GATHER_BATCH];
      int sx[GATHER_BATCH];
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int t = t0 + u * FILL_THREADS;
        sx[u] = t < T3 ? idx[t] : -1;
        // on a mesh, interpolated points (s <= -2) were written by the pass
        // above: read back (through L2, already encoded) only where the mixed
        // derivatives need them
        val[u] = sx[u] >= 0 ? __ldg(sv + sx[u]) : (MESH && slot >= 0 && sx[u] <= -2) ? __ldcg(tv + t) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < GATHER_BATCH; ++u) {
        const int t = t0 + u * FILL_THREADS;
        if (t < T3) {
          // encoded after all the batch's loads are in flight
          const double w = (sp && sx[u] >= 0) ? split_pair(val[u]) : val[u];
          if (slot >= 0) ts[t] = w;
          if (!MESH || sx[u] > -2) __stcs(tv + t, w);  // read once, by the stage kernel
        }
      }
    }
    if (slot < 0) continue;  // uniform across the block
    const bool f32 = F32W && mix_fslot(slot) >= 0;
    __syncthreads();
    // pass 0: d_y on the region widened along x, then d_x of it -> d_x d_y.
    // wide: d_z once on the region widened along x and y (corners skipped),
    // then d_x and d_y of it -> d_x d_z, d_y d_z; otherwise (the block does
    // not fit in shared memory) pass 1: d_z widened along x -> d_x d_z and
    // pass 2: d_z widened along y -> d_y d_z. Both give the same values.
#pragma unroll 1
    for (int pass = 0; pass < (wide ? 1 : 3); ++pass) {
      const int si = pass == 0 ? T : T * T;  // stride of the inner derivative in the tile
      for (int e = threadIdx.x; e < next; e += blockDim.x) {
        const int a = e % pe - 2, b = (e / pe) % p, c = e / (pe * p);
        // a runs along the widened axis (x for passes 0, 1; y for pass 2)
        const int x = pass == 2 ? b : a, y = pass == 2 ? a : b, z = c;
        const int c0 = ((z + HALO) * T + (y + HALO)) * T + (x + HALO);
        mixed_in(ext, e, ts, c0, si, f32);
      }
      __syncthreads();
      for (int q = threadIdx.x; q < p3; q += blockDim.x) {
        const int x = q % p, y = (q / p) % p, z = q / (p * p);
        const int a = pass == 2 ? y : x, b = pass == 2 ? x : y;
        const int e = (z * p + b) * pe + (a + 2);
        mixed_out(ext, e, 1, cmix, cmixf, f32, mix, g.n_points, pbase, slot + pass, q);
      }
      __syncthreads();
    }
    if (!wide) continue;
    const int T2 = T * T;
    for (int e = threadIdx.x; e < pe * pe * p; e += blockDim.x) {
      const int a = e % pe - 2, b = (e / pe) % pe - 2, c = e / (pe * pe);
      if ((a < 0 || a >= p) && (b < 0 || b >= p)) continue;  // corner: not needed
      const int c0 = ((c + HALO) * T + (b + HALO)) * T + (a + HALO);
      mixed_in(ext, e, ts, c0, T2, f32);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < p3; q += blockDim.x) {
      const int x = q % p, y = (q / p) % p, z = q / (p * p);
      const int e = (z * pe + (y + 2)) * pe + (x + 2);
      mixed_out(ext, e, 1, cmix, cmixf, f32, mix, g.n_points, pbase, slot + 1, q);
      mixed_out(ext, e, pe, cmix, cmixf, f32, mix, g.n_points, pbase, slot + 2, q);
    }
    __syncthreads();
  }
}

// Dynamic shared memory of fill_patch for patch edge p: the tile of one
// field, the widened first-derivative region and the source index table.
inline size_t fill_smem_bytes(int p) {
  const size_t T = (size_t)p + 2 * HALO, pe = (size_t)p + 4;
  return sizeof(double) * (T * T * T + (fill_wide(p) ? pe * pe * p : pe * p * p)) + sizeof(int) * T * T * T;
}

// The mixed derivatives' scale per level for the fill.
inline LevelScale level_scale(const GridView &g) {
  LevelScale ls;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    ls.cmix[l] = 1.0 / (144.0 * g.ldx[l] * g.ldx[l]);
    ls.cmixf[l] = (float)ls.cmix[l];
  }
  return ls;
}

}  // namespace
}  // namespace ccz4

#endif
