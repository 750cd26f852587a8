// Test support: the oracle's arithmetic counted. The oracle's C source is
// compiled unchanged as C++ with every `double` replaced by a scalar that
// counts its operations (add and subtract, multiply, divide, square and
// cube roots; a negation, a comparison or a conversion is not an
// operation), and one RK4 step of a single-puncture grid is run. Built by
// tests/test_oracle_opcount.py with g++ into a temporary directory; the
// count is the algorithmic work of a point-stage as the oracle's plain,
// unfactored restatement of the paper performs it (full index loops, no
// symmetry used, no fused multiply-adds).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace opcount {
long long n_add = 0, n_mul = 0, n_div = 0, n_root = 0;
}

struct CountedDouble {
  double v;
  CountedDouble() = default;
  CountedDouble(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator bool() const { return v != 0.0; }
  CountedDouble operator-() const { return CountedDouble(-v); }
  CountedDouble &operator+=(const CountedDouble &o) { ++opcount::n_add; v += o.v; return *this; }
  CountedDouble &operator-=(const CountedDouble &o) { ++opcount::n_add; v -= o.v; return *this; }
  CountedDouble &operator*=(const CountedDouble &o) { ++opcount::n_mul; v *= o.v; return *this; }
  CountedDouble &operator/=(const CountedDouble &o) { ++opcount::n_div; v /= o.v; return *this; }
};
typedef CountedDouble CD;
inline CD operator+(CD a, CD b) { ++opcount::n_add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++opcount::n_add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++opcount::n_mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++opcount::n_div; return CD(a.v / b.v); }
inline bool operator<(CD a, CD b) { return a.v < b.v; }
inline bool operator>(CD a, CD b) { return a.v > b.v; }
inline bool operator<=(CD a, CD b) { return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { return a.v >= b.v; }
inline bool operator==(CD a, CD b) { return a.v == b.v; }
inline bool operator!=(CD a, CD b) { return a.v != b.v; }
inline CD sqrt(CD a) { ++opcount::n_root; return CD(std::sqrt(a.v)); }
inline CD cbrt(CD a) { ++opcount::n_root; return CD(std::cbrt(a.v)); }
inline CD fabs(CD a) { return CD(std::fabs(a.v)); }
inline CD floor(CD a) { return CD(std::floor(a.v)); }
inline bool isfinite(CD a) { return std::isfinite(a.v); }

#define double CountedDouble
#include "../oracle/ccz4_oracle.c"
#undef double

// One RK4 step of a single puncture (Brill-Lindquist data, every field
// perturbed) on n^3 patches of p^3 with a Sommerfeld shell; out = operations
// per interior point-stage: [add, mul, div, root], and the total.
extern "C" void oracle_ops_per_point_stage(int p, int n, const og_params *Pin, double out[5]) {
  std::vector<int> ijk;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        ijk.push_back(a);
        ijk.push_back(b);
        ijk.push_back(c);
      }
  const CD dx(2.0 / (n * p));
  og_grid *g = og_grid_new(p, n, n, n, n * n * n, ijk.data(), -1.0, -1.0, -1.0, dx, OG_BC_SOMMERFELD);
  const long pts = (long)n * n * n * p * p * p, ng = og_n_ghost(g);
  std::vector<CD> U((size_t)OG_NV * pts), G((size_t)OG_NV * (ng > 0 ? ng : 1));
  std::vector<int> gc((size_t)3 * (ng > 0 ? ng : 1));
  og_ghost_coords(g, gc.data());
  auto state = [&](double x, double y, double z, int v) {
    const double r = std::sqrt(x * x + y * y + z * z);
    const double psi = 1.0 + 0.5 / r;
    double q = 0.0;
    if (v == GXX || v == GYY || v == GZZ) q = 1.0;
    if (v == PHI) q = 1.0 / (psi * psi);
    if (v == ALPHA) q = 1.0 / psi;
    return q + 1e-3 * std::sin(1.3 * x + 0.7 * y - 0.4 * z + v);
  };
  const double h = (double)dx;
  for (int m = 0; m < n * n * n; ++m)
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) {
          const long li = (long)m * p * p * p + ((long)k * p + j) * p + i;
          const double x = -1.0 + (ijk[3 * m] * p + i + 0.5) * h, y = -1.0 + (ijk[3 * m + 1] * p + j + 0.5) * h,
                       z = -1.0 + (ijk[3 * m + 2] * p + k + 0.5) * h;
          for (int v = 0; v < OG_NV; ++v) U[(size_t)v * pts + li] = CD(state(x, y, z, v));
        }
  for (long c = 0; c < ng; ++c)
    for (int v = 0; v < OG_NV; ++v)
      G[(size_t)v * ng + c] = CD(state(-1.0 + (gc[3 * c] + 0.5) * h, -1.0 + (gc[3 * c + 1] + 0.5) * h,
                                       -1.0 + (gc[3 * c + 2] + 0.5) * h, v));
  std::vector<CD> Gini = G;
  og_params P = *Pin;
  opcount::n_add = opcount::n_mul = opcount::n_div = opcount::n_root = 0;
  og_rk4_step(g, &P, CD(0.1) * dx, U.data(), G.data(), Gini.data());
  const double units = 4.0 * (double)pts;
  out[0] = opcount::n_add / units;
  out[1] = opcount::n_mul / units;
  out[2] = opcount::n_div / units;
  out[3] = opcount::n_root / units;
  out[4] = (opcount::n_add + opcount::n_mul + opcount::n_div + opcount::n_root) / units;
  og_grid_free(g);
}
