// Particle tracers and puncture trackers (Sec. "Particle Tracers as Data
// Probes"; Sec. "Particle tracers" on puncture trackers).
//
// A tracer records the 25 fields at its position by trilinear
// interpolation from the 2^3 closest sample points (cell centres) and may
// move with three of them as its velocity by the explicit Euler step
// x <- x + dt v. The sample points are those of the finest level that holds
// all eight as interior points of its patches; where no refined level does,
// those of level 0 with its boundary rule (periodic wrap, clamped copy, or
// the cells of the Sommerfeld ghost shell). A puncture tracker is a tracer
// dropped at a black hole whose velocity is the opposite shift, -beta.
//
// One thread per tracer; the products and sums are rounded one by one in
// a fixed order (no fused multiply-add), so the projection and the move are
// the same double operations as those of a plain sequential evaluation.
#include <vector>

#include "ccz4_internal.cuh"

namespace ccz4 {
namespace {

// Patch-slot tables of the refined levels: level l >= 1 covers the
// bounding box lo + [0, ext) of its slots; owner[off[l] + (z * ext_y + y) *
// ext_x + x] is the patch in that slot, or -1.
struct TrackLevels {
  int n_levels;
  long long off[MAX_LEVELS];
  int lo[MAX_LEVELS][3], ext[MAX_LEVELS][3];
  const int *owner;
};

// Patch of level l >= 1 holding level-l point (x, y, z), or -1.
__device__ __forceinline__ int level_owner(const TrackLevels &L, int l, int p, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0) return -1;
  const int s0 = x / p - L.lo[l][0], s1 = y / p - L.lo[l][1], s2 = z / p - L.lo[l][2];
  if (s0 < 0 || s1 < 0 || s2 < 0 || s0 >= L.ext[l][0] || s1 >= L.ext[l][1] || s2 >= L.ext[l][2]) return -1;
  return __ldg(L.owner + L.off[l] + ((long long)s2 * L.ext[l][1] + s1) * L.ext[l][0] + s0);
}

__global__ void __launch_bounds__(128) tracers_kernel(GridView g, TrackLevels L, const double *__restrict__ U,
                                                      double *__restrict__ pos, double *__restrict__ val,
                                                      int *__restrict__ bad, int n, double dt, int vel_field,
                                                      double vel_scale) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double x[3] = {pos[3 * s], pos[3 * s + 1], pos[3 * s + 2]};
  const int p = g.p;
  const long long p3 = (long long)p * p * p;
  long long idx[8];
  double t[3];
  bool found = false;
  for (int l = L.n_levels - 1; l >= 0 && !found; --l) {
    int i0[3];
    bool finite = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double sd = __dsub_rn(__ddiv_rn(__dsub_rn(x[d], g.origin[d]), g.ldx[l]), 0.5);
      if (!(fabs(sd) < 1.0e9)) finite = false;
      const double f = finite ? floor(sd) : 0.0;
      i0[d] = (int)f;
      t[d] = __dsub_rn(sd, f);
    }
    if (!finite) break;
    bool ok = true;
    for (int k = 0; k < 8 && ok; ++k) {
      const int px = i0[0] + (k & 1), py = i0[1] + ((k >> 1) & 1), pz = i0[2] + (k >> 2);
      if (l > 0) {
        const int m = level_owner(L, l, p, px, py, pz);
        if (m < 0) {
          ok = false;
        } else {
          const int *ij = g.ijk + 3 * m;
          idx[k] = m * p3 + ((long long)(pz - __ldg(ij + 2) * p) * p + (py - __ldg(ij + 1) * p)) * p +
                   (px - __ldg(ij) * p);
        }
      } else {
        // level 0: its boundary rule; beyond the Sommerfeld ghost shell nothing resolves the point
        if (g.bc == CCZ4_BC_SOMMERFELD && (px < -HALO || px >= g.N[0] + HALO || py < -HALO ||
                                           py >= g.N[1] + HALO || pz < -HALO || pz >= g.N[2] + HALO)) {
          ok = false;
        } else {
          idx[k] = locate(g, px, py, pz);
          ok = idx[k] >= 0;
        }
      }
    }
    found = ok;
  }
  if (!found) {
    bad[s] = 1;
    for (int v = 0; v < NV; ++v) val[(long long)s * NV + v] = __longlong_as_double(0x7FF8000000000000LL);
    return;
  }
  bad[s] = 0;
  const double wx[2] = {__dsub_rn(1.0, t[0]), t[0]}, wy[2] = {__dsub_rn(1.0, t[1]), t[1]},
               wz[2] = {__dsub_rn(1.0, t[2]), t[2]};
  double w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = __dmul_rn(__dmul_rn(wx[k & 1], wy[(k >> 1) & 1]), wz[k >> 2]);
  double vel[3] = {0.0, 0.0, 0.0};
  for (int v = 0; v < NV; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = __dadd_rn(acc, __dmul_rn(w[k], __ldg(U + v * g.S + idx[k])));
    val[(long long)s * NV + v] = acc;
    if (v >= vel_field && v < vel_field + 3) vel[v - vel_field] = acc;
  }
  if (vel_field >= 0) {
    const double c = __dmul_rn(dt, vel_scale);
#pragma unroll
    for (int d = 0; d < 3; ++d) pos[3 * s + d] = __dadd_rn(x[d], __dmul_rn(c, vel[d]));
  }
}

}  // namespace
}  // namespace ccz4

using namespace ccz4;

struct ccz4_tracers {
  ccz4_grid *g;
  int n, vel_field;
  double vel_scale;
  double *d_pos, *d_val;  // [n][3], [n][25]
  int *d_bad;             // [n] 1 where the last step could not project the tracer
  int *d_owner;           // slot tables of the refined levels
  TrackLevels L;
};

static void tracers_release(ccz4_tracers *t) {
  if (!t) return;
  cudaFree(t->d_pos);
  cudaFree(t->d_val);
  cudaFree(t->d_bad);
  cudaFree(t->d_owner);
  free(t);
}

extern "C" ccz4_status ccz4_tracers_new(ccz4_grid *g, int n, const double *pos, int vel_field, double vel_scale,
                                        ccz4_tracers **out) {
  if (!out || !g || !pos || n < 1 || vel_field < -1 || vel_field > NV - 3 || !(vel_scale == vel_scale)) {
    set_error("tracers_new: grid, positions and out must be given, n >= 1, vel_field in [-1, %d]", NV - 3);
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  ccz4_tracers *t = (ccz4_tracers *)calloc(1, sizeof(ccz4_tracers));
  if (!t) {
    set_error("host allocation failed");
    return CCZ4_ERR_NOMEM;
  }
  t->g = g;
  t->n = n;
  t->vel_field = vel_field;
  t->vel_scale = vel_scale;
  const GridView &v = g->v;
  // slot tables of the refined levels from the grid's patch coordinates and levels
  std::vector<int> ijk(3 * (size_t)v.n_patches), lev((size_t)v.n_patches, 0);
  bool ok = cudaMemcpy(ijk.data(), v.ijk, sizeof(int) * ijk.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
  if (ok && v.plev)
    ok = cudaMemcpy(lev.data(), v.plev, sizeof(int) * lev.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
  std::vector<int> table;
  t->L.n_levels = v.n_levels;
  for (int l = 1; l < v.n_levels && ok; ++l) {
    int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
    bool any = false;
    for (int m = 0; m < v.n_patches; ++m) {
      if (lev[m] != l) continue;
      for (int d = 0; d < 3; ++d) {
        const int c = ijk[3 * m + d];
        if (!any || c < lo[d]) lo[d] = c;
        if (!any || c > hi[d]) hi[d] = c;
      }
      any = true;
    }
    t->L.off[l] = (long long)table.size();
    long long size = 1;
    for (int d = 0; d < 3; ++d) {
      t->L.lo[l][d] = lo[d];
      t->L.ext[l][d] = any ? hi[d] - lo[d] + 1 : 0;
      size *= t->L.ext[l][d];
    }
    table.resize(table.size() + (size_t)size, -1);
    for (int m = 0; m < v.n_patches; ++m) {
      if (lev[m] != l) continue;
      const long long k = ((long long)(ijk[3 * m + 2] - lo[2]) * t->L.ext[l][1] + (ijk[3 * m + 1] - lo[1])) *
                              t->L.ext[l][0] + (ijk[3 * m] - lo[0]);
      table[(size_t)(t->L.off[l] + k)] = m;
    }
  }
  ok = ok && cudaMalloc(&t->d_pos, sizeof(double) * 3 * (size_t)n) == cudaSuccess &&
       cudaMalloc(&t->d_val, sizeof(double) * NV * (size_t)n) == cudaSuccess &&
       cudaMalloc(&t->d_bad, sizeof(int) * (size_t)n) == cudaSuccess &&
       cudaMalloc(&t->d_owner, sizeof(int) * (table.empty() ? 1 : table.size())) == cudaSuccess;
  ok = ok && cudaMemcpy(t->d_pos, pos, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(t->d_bad, 0, sizeof(int) * (size_t)n) == cudaSuccess &&
       cudaMemset(t->d_val, 0, sizeof(double) * NV * (size_t)n) == cudaSuccess;
  if (ok && !table.empty())
    ok = cudaMemcpy(t->d_owner, table.data(), sizeof(int) * table.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    set_error("tracers_new: device allocation or copy failed: %s", cudaGetErrorString(cudaGetLastError()));
    tracers_release(t);
    return CCZ4_ERR_NOMEM;
  }
  t->L.owner = t->d_owner;
  *out = t;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_tracers_step(ccz4_tracers *t, int buf, double dt, void *stream) {
  if (!t || buf < CCZ4_BUF_U || buf > CCZ4_BUF_INI || !(dt == dt)) {
    set_error("tracers_step: tracers must be given, buf a state buffer (U..INI), dt finite");
    return CCZ4_ERR_INVALID;
  }
  const double *U = t->g->buf[buf];
  if (!U) {
    set_error("tracers_step: buffer %d is not allocated for this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  const int blocks = (t->n + 127) / 128;
  tracers_kernel<<<blocks, 128, 0, (cudaStream_t)stream>>>(t->g->v, t->L, U, t->d_pos, t->d_val, t->d_bad, t->n,
                                                           dt, t->vel_field, t->vel_scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tracers_step launch failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_tracers_read(ccz4_tracers *t, double *pos, double *values, void *stream) {
  if (!t) {
    set_error("tracers_read: tracers must be given");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> bad((size_t)t->n);
  cudaError_t e = cudaSuccess;
  if (pos) e = cudaMemcpyAsync(pos, t->d_pos, sizeof(double) * 3 * (size_t)t->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && values)
    e = cudaMemcpyAsync(values, t->d_val, sizeof(double) * NV * (size_t)t->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad.data(), t->d_bad, sizeof(int) * bad.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("tracers_read failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  int n_bad = 0, first = -1;
  for (int k = 0; k < t->n; ++k)
    if (bad[(size_t)k]) {
      if (first < 0) first = k;
      ++n_bad;
    }
  if (n_bad) {
    set_error("%d tracer(s) outside the grid in the last step (first: %d); they were left in place", n_bad, first);
    return CCZ4_ERR_BOUNDS;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_tracers_free(ccz4_tracers *t) {
  tracers_release(t);
  return CCZ4_OK;
}
