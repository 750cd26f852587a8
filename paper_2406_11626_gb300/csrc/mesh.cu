// Statically refined meshes (appendix "refinement transition"): the host
// planner that validates a ratio-3 mesh and resolves the source of every
// halo'd tile point once, and the restriction kernel.
//
// The mesh is static, so the fill kernel does not search for neighbours at
// run time on a mesh: the planner writes, per patch and tile point, either
// the index of the value in the state vector (a same-level patch, or on
// level 0 the boundary rule) or an interpolation entry holding the eight
// coarse source indices and the remainders that pick the weights. The
// coarse level overlaps the fine one, so every fine halo point interpolates
// between interior coarse points; no extrapolation is needed.
#include <stdint.h>
#include <string.h>

#include <unordered_map>
#include <vector>

#include "ccz4_internal.cuh"
#include "mesh_plan.h"

namespace ccz4 {

namespace {

inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((b - 1 - a) / b); }

inline uint64_t slot_key(int l, int a, int b, int c) {
  return ((uint64_t)l << 60) | ((uint64_t)a << 40) | ((uint64_t)b << 20) | (uint64_t)c;
}

// Level-0 source of global point (x, y, z), by the boundary kind (the same
// rules as the fill kernel's run-time lookup), or -1.
long long locate0(const GridView &v, const std::vector<int> &owner0, int x, int y, int z) {
  const bool inside = x >= 0 && x < v.N[0] && y >= 0 && y < v.N[1] && z >= 0 && z < v.N[2];
  if (!inside) {
    if (v.bc == CCZ4_BC_PERIODIC) {
      x = wrap(x, v.N[0]);
      y = wrap(y, v.N[1]);
      z = wrap(z, v.N[2]);
    } else if (v.bc == CCZ4_BC_COPY) {
      x = clampi(x, 0, v.N[0] - 1);
      y = clampi(y, 0, v.N[1] - 1);
      z = clampi(z, 0, v.N[2] - 1);
    } else {
      if (x < -HALO || x >= v.N[0] + HALO || y < -HALO || y >= v.N[1] + HALO || z < -HALO ||
          z >= v.N[2] + HALO)
        return -1;
      return v.n_points + ghost_rank(v, x, y, z);
    }
  }
  const int p = v.p;
  const int px = x / p, py = y / p, pz = z / p;
  const int n = owner0[((size_t)pz * v.np[1] + py) * v.np[0] + px];
  return (long long)n * p * p * p + ((long long)(z - pz * p) * p + (y - py * p)) * p + (x - px * p);
}

struct Planner {
  const ccz4_mesh_desc *d;
  GridView v;                // sizes of level 0
  std::vector<int> owner0;
  std::unordered_map<uint64_t, int> slots;  // levels >= 1
  std::vector<int> level;

  // Interior index of level-l point (x, y, z), or -1 if level l holds no
  // patch there (level 0: outside the domain).
  long long interior(int l, int x, int y, int z) const {
    const int p = d->p;
    if (l == 0) {
      if (x < 0 || x >= v.N[0] || y < 0 || y >= v.N[1] || z < 0 || z >= v.N[2]) return -1;
      return locate0(v, owner0, x, y, z);
    }
    const int a = floordiv(x, p), b = floordiv(y, p), c = floordiv(z, p);
    if (a < 0 || b < 0 || c < 0) return -1;
    auto it = slots.find(slot_key(l, a, b, c));
    if (it == slots.end()) return -1;
    const int n = it->second;
    return (long long)n * p * p * p + ((long long)(z - c * p) * p + (y - b * p)) * p + (x - a * p);
  }
};

}  // namespace

ccz4_status plan_mesh(const ccz4_mesh_desc *d, bool want_tables, MeshPlan &out) {
  if (!d || !d->level || !d->ijk) {
    set_error("mesh descriptor, level and ijk must be given");
    return CCZ4_ERR_INVALID;
  }
  if (d->p < 1 || d->p > MAX_P || d->np[0] < 1 || d->np[1] < 1 || d->np[2] < 1 || !(d->dx > 0.0) ||
      d->n_patches < 1) {
    set_error("invalid mesh sizes: p=%d (1..%d) np=(%d,%d,%d) n_patches=%d dx=%g", d->p, MAX_P, d->np[0],
              d->np[1], d->np[2], d->n_patches, d->dx);
    return CCZ4_ERR_INVALID;
  }
  if (d->bc != CCZ4_BC_PERIODIC && d->bc != CCZ4_BC_COPY && d->bc != CCZ4_BC_SOMMERFELD) {
    set_error("unknown boundary kind %d", d->bc);
    return CCZ4_ERR_INVALID;
  }
  Planner P;
  P.d = d;
  const int p = d->p, n = d->n_patches;
  int n_levels = 1;
  P.level.assign(d->level, d->level + n);
  for (int m = 0; m < n; ++m) {
    if (P.level[m] < 0 || P.level[m] >= MAX_LEVELS) {
      set_error("patch %d has level %d outside 0..%d", m, P.level[m], MAX_LEVELS - 1);
      return CCZ4_ERR_INVALID;
    }
    if (P.level[m] + 1 > n_levels) n_levels = P.level[m] + 1;
  }
  long long scale = 1;
  for (int l = 1; l < n_levels; ++l) scale *= 3;
  for (int q = 0; q < 3; ++q)
    if ((long long)d->np[q] * p * scale + 2 * HALO >= (1LL << 30) || (long long)d->np[q] * scale >= (1LL << 20)) {
      set_error("mesh too large for 32-bit point coordinates");
      return CCZ4_ERR_INVALID;
    }
  GridView &v = P.v;
  v = GridView{};
  v.p = p;
  v.T = p + 2 * HALO;
  for (int q = 0; q < 3; ++q) {
    v.np[q] = d->np[q];
    v.N[q] = d->np[q] * p;
  }
  v.bc = d->bc;
  v.n_patches = n;
  v.n_points = (long long)n * p * p * p;
  v.T3 = (long long)v.T * v.T * v.T;
  // level 0 covers its slots exactly once
  const long long slots0 = (long long)d->np[0] * d->np[1] * d->np[2];
  P.owner0.assign((size_t)slots0, -1);
  long long count0 = 0;
  for (int m = 0; m < n; ++m) {
    const int a = d->ijk[3 * m], b = d->ijk[3 * m + 1], c = d->ijk[3 * m + 2];
    if (P.level[m] == 0) {
      if (a < 0 || a >= d->np[0] || b < 0 || b >= d->np[1] || c < 0 || c >= d->np[2]) {
        set_error("level-0 patch %d has slot (%d,%d,%d) outside the %dx%dx%d block", m, a, b, c, d->np[0],
                  d->np[1], d->np[2]);
        return CCZ4_ERR_INVALID;
      }
      const long long cell = ((long long)c * d->np[1] + b) * d->np[0] + a;
      if (P.owner0[cell] >= 0) {
        set_error("level-0 slot (%d,%d,%d) is listed twice", a, b, c);
        return CCZ4_ERR_INVALID;
      }
      P.owner0[cell] = m;
      ++count0;
    } else {
      if (a < 0 || b < 0 || c < 0 || a >= (1 << 20) || b >= (1 << 20) || c >= (1 << 20)) {
        set_error("level-%d patch %d has slot (%d,%d,%d) out of range", P.level[m], m, a, b, c);
        return CCZ4_ERR_INVALID;
      }
      if (!P.slots.emplace(slot_key(P.level[m], a, b, c), m).second) {
        set_error("level-%d slot (%d,%d,%d) is listed twice", P.level[m], a, b, c);
        return CCZ4_ERR_INVALID;
      }
    }
  }
  if (count0 != slots0) {
    set_error("level 0 must cover all %lld slots of the base grid (has %lld patches)", slots0, count0);
    return CCZ4_ERR_INVALID;
  }
  // parents and complete child sets
  std::vector<int> nchild((size_t)n, 0);
  std::vector<int> parent((size_t)n, -1);
  for (int m = 0; m < n; ++m) {
    const int l = P.level[m];
    if (l == 0) continue;
    const int a = d->ijk[3 * m] / 3, b = d->ijk[3 * m + 1] / 3, c = d->ijk[3 * m + 2] / 3;
    int par = -1;
    if (l - 1 == 0) {
      if (a < d->np[0] && b < d->np[1] && c < d->np[2]) par = P.owner0[((size_t)c * d->np[1] + b) * d->np[0] + a];
    } else {
      auto it = P.slots.find(slot_key(l - 1, a, b, c));
      if (it != P.slots.end()) par = it->second;
    }
    if (par < 0) {
      set_error("level-%d patch %d at (%d,%d,%d) has no parent on level %d", l, m, d->ijk[3 * m],
                d->ijk[3 * m + 1], d->ijk[3 * m + 2], l - 1);
      return CCZ4_ERR_INVALID;
    }
    parent[m] = par;
    ++nchild[par];
  }
  for (int m = 0; m < n; ++m)
    if (nchild[m] != 0 && nchild[m] != 27) {
      set_error("patch %d has %d children; a refined patch has all 27", m, nchild[m]);
      return CCZ4_ERR_INVALID;
    }
  // ghost shell of level 0 (Sommerfeld): sizes for the ghost ranks
  if (d->bc == CCZ4_BC_SOMMERFELD)
    v.n_ghost = ((long long)v.N[0] + 6) * (v.N[1] + 6) * (v.N[2] + 6) - (long long)v.N[0] * v.N[1] * v.N[2];
  // tile sources
  out = MeshPlan();
  out.n_levels = n_levels;
  out.level = P.level;
  out.leaf.assign((size_t)n, 0);
  out.n_leaf_points = 0;
  for (int m = 0; m < n; ++m) {
    out.leaf[m] = nchild[m] == 0;
    if (out.leaf[m]) out.n_leaf_points += (long long)p * p * p;
  }
  out.owner0 = P.owner0;
  const int T = v.T;
  if (want_tables) {
    out.src.assign((size_t)n * v.T3, -1);
    out.ibeg.assign((size_t)n + 1, 0);
  }
  out.n_interp = 0;
  for (int m = 0; m < n; ++m) {
    const int l = P.level[m];
    if (want_tables) out.ibeg[m] = (int)out.n_interp;
    const int bx = d->ijk[3 * m] * p - HALO, by = d->ijk[3 * m + 1] * p - HALO, bz = d->ijk[3 * m + 2] * p - HALO;
    for (int t = 0; t < (int)v.T3; ++t) {
      const int x = bx + t % T, y = by + (t / T) % T, z = bz + t / (T * T);
      long long s;
      if (l == 0) {
        s = locate0(v, P.owner0, x, y, z);
      } else {
        s = P.interior(l, x, y, z);
        if (s < 0) {
          // interpolate from level l-1: coarse cell c = floor((i-1)/3), remainder r
          int c0[3], r[3];
          const int fi[3] = {x, y, z};
          for (int q = 0; q < 3; ++q) {
            c0[q] = floordiv(fi[q] - 1, 3);
            r[q] = fi[q] - 1 - 3 * c0[q];
          }
          InterpEntry e;
          e.r = r[0] | (r[1] << 2) | (r[2] << 4);
          e.t = t;
          for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
              for (int cx = 0; cx < 2; ++cx) {
                // a corner along an axis with remainder 0 has weight zero: reuse the used one
                const int ux = r[0] ? cx : 0, uy = r[1] ? cy : 0, uz = r[2] ? cz : 0;
                const long long cs = P.interior(l - 1, c0[0] + ux, c0[1] + uy, c0[2] + uz);
                if (cs < 0) {
                  set_error("level-%d patch %d: halo point (%d,%d,%d) needs level-%d point (%d,%d,%d), which "
                            "is not an interior point of that level (refined levels must be nested with two "
                            "coarse cells to spare and keep off the domain boundary)",
                            l, m, x, y, z, l - 1, c0[0] + ux, c0[1] + uy, c0[2] + uz);
                  return CCZ4_ERR_INVALID;
                }
                e.src[(cz * 2 + cy) * 2 + cx] = (int)cs;
              }
          if (want_tables) out.interp.push_back(e);
          s = -2 - out.n_interp;
          ++out.n_interp;
        }
      }
      if (s == -1 || s >= (1LL << 31) || s < -(1LL << 31)) {
        set_error("patch %d: tile point (%d,%d,%d) cannot be resolved", m, x, y, z);
        return CCZ4_ERR_INVALID;
      }
      if (want_tables) out.src[(size_t)m * v.T3 + t] = (int)s;
    }
  }
  if (want_tables) {
    if (out.n_interp >= (1LL << 31)) {
      set_error("mesh has too many interpolated halo points (%lld)", out.n_interp);
      return CCZ4_ERR_INVALID;
    }
    out.ibeg[n] = (int)out.n_interp;
  }
  // restriction lists: per level l >= 1, the parents on level l-1 and their children
  for (int l = 1; l < n_levels; ++l) {
    std::vector<int> &par = out.rpar[l];
    std::vector<int> &kid = out.rkid[l];
    for (int m = 0; m < n; ++m) {
      if (P.level[m] != l - 1 || nchild[m] == 0) continue;
      par.push_back(m);
      const int a = d->ijk[3 * m], b = d->ijk[3 * m + 1], c = d->ijk[3 * m + 2];
      for (int kz = 0; kz < 3; ++kz)
        for (int ky = 0; ky < 3; ++ky)
          for (int kx = 0; kx < 3; ++kx)
            kid.push_back(P.slots.at(slot_key(l, 3 * a + kx, 3 * b + ky, 3 * c + kz)));
    }
  }
  return CCZ4_OK;
}

namespace {

// Coarse point q of parent k <- mean of its 27 fine cells (x, then y, then
// z; products and sums rounded separately, in this order).
__global__ void __launch_bounds__(128) restrict_kernel(GridView g, const int *__restrict__ par,
                                                       const int *__restrict__ kid, int n_par, double *U) {
  const int p = g.p;
  const int p3 = p * p * p;
  // n_par * p^3 points of coarse patches: below 2^31 (32-bit division)
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_par * p3) return;
  const int k = i / p3;
  const int q = i - k * p3;
  const int cz = q / (p * p), cy = (q / p) % p, cx = q % p;
  const int *kk = kid + 27 * k;
  int idx[27];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int X = 3 * cx + a, Y = 3 * cy + b, Z = 3 * cz + c;
        const int child = __ldg(kk + ((Z / p) * 3 + Y / p) * 3 + X / p);
        idx[(c * 3 + b) * 3 + a] = child * p3 + ((Z % p) * p + Y % p) * p + X % p;
      }
  const long long dst = (long long)__ldg(par + k) * p3 + q;  // below 2^31 too
  const double third = 1.0 / 3.0;
  for (int v = 0; v < NV; ++v) {
    const double *f = U + v * g.S;
    double sy[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double sx[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int *id = idx + (c * 3 + b) * 3;
        sx[b] = __dadd_rn(__dadd_rn(__dmul_rn(third, f[id[0]]), __dmul_rn(third, f[id[1]])),
                          __dmul_rn(third, f[id[2]]));
      }
      sy[c] = __dadd_rn(__dadd_rn(__dmul_rn(third, sx[0]), __dmul_rn(third, sx[1])), __dmul_rn(third, sx[2]));
    }
    U[v * g.S + dst] = __dadd_rn(__dadd_rn(__dmul_rn(third, sy[0]), __dmul_rn(third, sy[1])),
                                 __dmul_rn(third, sy[2]));
  }
}

}  // namespace

cudaError_t launch_restrict(const GridView &g, const int *par, const int *kid, int n_par, double *U,
                            cudaStream_t s) {
  if (n_par <= 0) return cudaSuccess;
  const long long work = (long long)n_par * g.p * g.p * g.p;
  restrict_kernel<<<(unsigned)((work + 127) / 128), 128, 0, s>>>(g, par, kid, n_par, U);
  return cudaGetLastError();
}

// The x jobs of an entry are its (up to four) x-pairs, the y jobs its (up
// to two) pairs of x results, in the order of the per-entry evaluation, so
// every job computes the same products and sums as the entry itself.
void plan_separable(MeshPlan &out, long long T3) {
  const int n = (int)out.ibeg.size() - 1;
  out.xjob.clear();
  out.yjob.clear();
  out.zjob.assign(out.interp.size(), ZJob{0, 0});
  out.xbeg.assign((size_t)n + 1, 0);
  out.ybeg.assign((size_t)n + 1, 0);
  std::unordered_map<unsigned long long, int> xs;
  std::unordered_map<int, int> ys;
  std::vector<XJob> px;
  std::vector<int> py;
  for (int m = 0; m < n; ++m) {
    out.xbeg[m] = (int)out.xjob.size();
    out.ybeg[m] = (int)out.yjob.size();
    const int e0 = out.ibeg[m], e1 = out.ibeg[m + 1];
    if (e1 == e0) continue;
    xs.clear();
    ys.clear();
    px.clear();
    py.clear();
    bool fits = true;
    for (int e = e0; e < e1 && fits; ++e) {
      const InterpEntry &E = out.interp[e];
      const int rx = E.r & 3, ry = (E.r >> 2) & 3, rz = (E.r >> 4) & 3;
      int yi[2] = {0, 0};
      for (int c = 0; c < (rz ? 2 : 1); ++c) {
        int xi[2] = {0, 0};
        for (int b = 0; b < (ry ? 2 : 1); ++b) {
          const int s0 = E.src[(c * 2 + b) * 2], s1 = rx ? E.src[(c * 2 + b) * 2 + 1] : s0;
          const unsigned long long key =
              ((unsigned long long)(unsigned)s0 << 33) | ((unsigned long long)(unsigned)s1 << 2) | (unsigned)rx;
          auto it = xs.find(key);
          if (it == xs.end()) {
            it = xs.emplace(key, (int)px.size()).first;
            px.push_back(XJob{s0, s1, rx});
          }
          xi[b] = it->second;
        }
        if (!ry) xi[1] = xi[0];
        const int key = xi[0] | (xi[1] << JOB_BITS) | (ry << (2 * JOB_BITS));
        auto it = ys.find(key);
        if (it == ys.end()) {
          it = ys.emplace(key, (int)py.size()).first;
          py.push_back(key);
        }
        yi[c] = it->second;
      }
      if (!rz) yi[1] = yi[0];
      out.zjob[e] = ZJob{yi[0] | (yi[1] << JOB_BITS) | (rz << (2 * JOB_BITS)), E.t};
      fits = (long long)(px.size() + py.size()) <= T3 && px.size() < (1u << JOB_BITS) &&
             py.size() < (1u << JOB_BITS);
    }
    if (!fits) continue;  // interpolated entry by entry
    out.xjob.insert(out.xjob.end(), px.begin(), px.end());
    out.yjob.insert(out.yjob.end(), py.begin(), py.end());
  }
  out.xbeg[n] = (int)out.xjob.size();
  out.ybeg[n] = (int)out.yjob.size();
}

}  // namespace ccz4

using namespace ccz4;

extern "C" ccz4_status ccz4_mesh_plan(const ccz4_mesh_desc *desc, long long *n_interp, int *src, int *interp) {
  MeshPlan plan;
  ccz4_status st = plan_mesh(desc, src != nullptr || interp != nullptr, plan);
  if (st != CCZ4_OK) return st;
  if (n_interp) *n_interp = plan.n_interp;
  if (src) memcpy(src, plan.src.data(), sizeof(int) * plan.src.size());
  if (interp)
    for (size_t e = 0; e < plan.interp.size(); ++e) {
      for (int c = 0; c < 8; ++c) interp[9 * e + c] = plan.interp[e].src[c];
      interp[9 * e + 8] = plan.interp[e].r;
    }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_mesh_info(const ccz4_grid *g, int *n_levels, long long *n_leaf_points) {
  if (!g) {
    set_error("grid is NULL");
    return CCZ4_ERR_INVALID;
  }
  if (n_levels) *n_levels = g->v.n_levels;
  if (n_leaf_points) *n_leaf_points = g->v.n_leaf_points;
  return CCZ4_OK;
}
