// Pointwise FD4 stencils and the second-order CCZ4 right-hand side.
//
// Stencils (appendix "Formulation for the kernel FD4 Solver"):
//   first derivative  [8 (Q+ - Q-) - (Q++ - Q--)] / (12 dx)      (Eq. exa_fd4_central_difference)
//   pure second       [-(Q++ + Q--) + 16 (Q+ + Q-) - 30 Q] / (12 dx^2)
//   mixed second      the first-derivative stencil along one axis applied
//                     to the first-derivative stencil along the other
//                     (the tensor-product approach of Sec. "Finite Differences")
//   Kreiss-Oliger     eps/(64 dx) (Q--- - 6 Q-- + 15 Q- - 20 Q + 15 Q+ - 6 Q++ + Q+++),
//                     summed over x, y, z                             (Eq. exa_fd4_ko)
// Right-hand side: the nine primary evolution equations of the appendix
// "Spacetime foliation" with the red (first-order-only) terms removed, the
// auxiliary quantities A_i, B_k^i, D_kij, P_i replaced by FD4 derivatives of
// the primaries, closed by the listed relations and the modified Ricci
// tensor of Eq. NR_foccz4_modified_ricci.
//
// Two scalar types: D carries the state, the differences of alpha and phi,
// the terms with inverse powers of the conformal factor phi (which grow
// without bound at a puncture) and the time update; R carries the rest of
// the pointwise algebra. D = R = double is the FP64 path, where D also
// takes every difference; D = double, R = float the mixed path, where the
// differences of the other fields are taken with FP64 accuracy on split
// FP32 pairs (sp_second and its neighbours below). Constants are written in
// the type they are used in, so no expression silently widens.
//
// Arithmetic is arranged for the FP64 pipe: reciprocals are taken once,
// symmetric tensors are stored as six components, contractions use the
// symmetry, and stencil sums are paired so that most operations fuse into
// FMAs.
#pragma once

#include <type_traits>

#include "ccz4_internal.cuh"

namespace ccz4 {

// Host-side section marker of the operation count (no code on the device).
void count_mark(const char *section);
#ifdef __CUDA_ARCH__
#define CCZ4_MARK(name)
#else
#define CCZ4_MARK(name) ::ccz4::count_mark(name)
#endif

__host__ __device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double rcbrtT(double a) {
#ifdef __CUDA_ARCH__
  return rcbrt(a);
#else
  return 1.0 / cbrt(a);
#endif
}

// Precision conversions. GB300 executes the F2F double <-> float conversion
// instructions on its narrow FP64 pipe, the bottleneck of this kernel, so on
// the device they are done with integer operations on the bit patterns:
// double -> float rounds to nearest (ties away from zero), flushes values
// below the single-precision normal range to signed zero and maps values
// beyond it to infinity (NaN if mantissa bits survive); float -> double is
// exact for normal numbers and flushes subnormals to zero.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u, e = (hi >> 20) & 0x7FFu;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned f = (sgn | ((e - 896u) << 23) | m) + ((lo >> 28) & 1u);
  f = e < 897u ? sgn : f;
  f = e > 1150u ? (sgn | 0x7F800000u | (m ? 0x400000u : 0u)) : f;
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d_bits(float v) {
  const unsigned u = __float_as_uint(v), sgn = u & 0x80000000u, e = (u >> 23) & 0xFFu;
  unsigned hi = sgn | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  unsigned lo = u << 29;
  hi = e == 0u ? sgn : hi;
  lo = e == 0u ? 0u : lo;
  hi = e == 255u ? (sgn | 0x7FF00000u | ((u & 0x7FFFFFu) >> 3)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}
// The split pair of the mixed path's tiles: hi = d2f_bits(x) and lo = the
// FP32 rounding (to nearest even) of x - hi, returned as the 8 bytes of a
// float2 {hi, lo} (the bit pattern of a double, for a store in place of x).
// x - hi is read off the 29 mantissa bits that hi drops: with r the rounding
// bit (the highest of them), x - hi = sign(x) (low29 - r 2^29) 2^(e - 52);
// its magnitude (below 2^28 units) is made an FP32 number from two exact
// 14-bit halves and one fused multiply-add (a single rounding), then scaled
// by the power of two. Integer and FP32 operations only. Where hi is zero
// (x below the FP32 normal range) or infinite, or the power of two leaves
// the FP32 normal range, lo is zero.
__device__ __forceinline__ double split_pair(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const float h = d2f_bits(x);
  const unsigned E = (hw >> 20) & 0x7FFu;
  const unsigned r = (lw >> 28) & 1u;
  const unsigned low = lw & 0x1FFFFFFFu;
  const unsigned mag = r ? (0x20000000u - low) : low;  // |x - hi| in units of 2^(e - 52), at most 2^28
  const float a = __uint_as_float(0x4B000000u | (mag >> 14)) - 8388608.0f;     // exact: below 2^15
  const float b = __uint_as_float(0x4B000000u | (mag & 0x3FFFu)) - 8388608.0f;  // exact: below 2^14
  const float m = fmaf(a, 16384.0f, b);
  const int se = (int)E - 948;  // FP32 exponent field of 2^(e - 52)
  const float scale = (se >= 1 && se <= 254 && E >= 897u && E <= 1150u) ? __uint_as_float((unsigned)se << 23) : 0.0f;
  float l = m * scale;
  // sign: x - hi has the sign of x when hi was rounded down in magnitude
  l = ((hw >> 31) ^ r) ? -l : l;
  return __hiloint2double((int)__float_as_uint(l), (int)__float_as_uint(h));
}
template <class To, class From>
__host__ __device__ __forceinline__ To cvt(const From &x) { return To(x); }
template <>
__host__ __device__ __forceinline__ float cvt<float, double>(const double &x) {
#ifdef __CUDA_ARCH__
  return d2f_bits(x);
#else
  return (float)x;
#endif
}
template <>
__host__ __device__ __forceinline__ double cvt<double, float>(const float &x) {
#ifdef __CUDA_ARCH__
  return f2d_bits(x);
#else
  return (double)x;
#endif
}

// index of the symmetric pair (i, j) among xx, xy, xz, yy, yz, zz. Written
// without recursion: the index must fold to a constant as soon as the
// loops around it are unrolled, or the arrays it indexes stay in local
// memory (a recursive form left the mixed stage kernel a 624-byte stack
// frame of such arrays).
__host__ __device__ constexpr int S6(int i, int j) {
  return i > j ? (j == 0 ? i : (j == 1 ? 2 + i : 5)) : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

// Tile loads through Nbhd (the stage kernel and the constraint monitors):
// the streaming (evict-first) hint, which leaves L2 to the stage kernel's
// register spills (a tile is reused within a block, through L1); 0 for the
// read-only path.
#ifndef CCZ4_TILE_LOAD_CS
#define CCZ4_TILE_LOAD_CS 1
#endif
#if CCZ4_TILE_LOAD_CS
#define CCZ4_TLD __ldcs
#else
#define CCZ4_TLD __ldg
#endif
// Loads of the mixed derivatives: through the read-only path, except in a
// translation unit whose kernel writes them itself before reading them (the
// fused stage launch defines this as a coherent load before including).
#ifndef CCZ4_MIX_LOAD
#define CCZ4_MIX_LOAD __ldg
#endif

// Read-only view of the halo'd neighbourhood of one point.
struct Nbhd {
  const double *__restrict__ c;    // field 0 at the centre point
  long long fs;                    // distance between fields
  int st[3];                       // distance between neighbours along x, y, z
  const double *__restrict__ mix;  // mixed second derivatives of this point, slot 0
  long long ms;                    // distance between slots
  const float *__restrict__ mixf;  // mixed path: those of g~ and beta in FP32 (mix_fslot order)
  long long msf;                   // distance between FP32 slots
  __host__ __device__ __forceinline__ double at(int v, int off) const {
#ifdef __CUDA_ARCH__
    return CCZ4_TLD(c + v * fs + off);
#else
    return c[v * fs + off];
#endif
  }
  __host__ __device__ __forceinline__ double mixed(int slot) const {
#ifdef __CUDA_ARCH__
    return CCZ4_MIX_LOAD(mix + slot * ms);
#else
    return mix[slot * ms];
#endif
  }
  __host__ __device__ __forceinline__ float mixedf(int fslot) const {
#ifdef __CUDA_ARCH__
    return CCZ4_MIX_LOAD(mixf + fslot * msf);
#else
    return mixf[fslot * msf];
#endif
  }
  // mixed path: the split pair (hi, lo) stored in place of the FP64 value
  __host__ __device__ __forceinline__ float2 at2(int v, int off) const {
    const float2 *q = reinterpret_cast<const float2 *>(c) + (v * fs + off);
#ifdef __CUDA_ARCH__
    return CCZ4_TLD(q);
#else
    return *q;
#endif
  }
};

template <class D>
struct StencilCoef {
  D c1;   // 1 / (12 dx)
  D c2;   // 1 / (12 dx^2)
  D c3;   // 1 / (144 dx^2)
  D cko;  // eps / (64 dx)
};

template <class D>
__host__ __device__ __forceinline__ D ld(const Nbhd &N, int v, int off) {
  return D(N.at(v, off));
}

template <class D>
__host__ __device__ __forceinline__ D fd1(const Nbhd &N, int v, int s, const D &c1) {
  const D a = ld<D>(N, v, s) - ld<D>(N, v, -s);
  const D b = ld<D>(N, v, 2 * s) - ld<D>(N, v, -2 * s);
  return fmaT(D(8.0), a, -b) * c1;
}

// First derivative whose neighbour differences are taken in D and whose
// stencil weights are applied in O (O = D: identical to fd1).
template <class D, class O>
__host__ __device__ __forceinline__ O fd1o(const Nbhd &N, int v, int s, const O &c1) {
  const D a = ld<D>(N, v, s) - ld<D>(N, v, -s);
  const D b = ld<D>(N, v, 2 * s) - ld<D>(N, v, -2 * s);
  return fmaT(O(8.0), cvt<O>(a), -cvt<O>(b)) * c1;
}

// The same without the factor 1 / (12 dx), for callers that fold it into
// a coefficient they apply anyway.
template <class D, class O>
__host__ __device__ __forceinline__ O fd1u(const Nbhd &N, int v, int s) {
  const D a = ld<D>(N, v, s) - ld<D>(N, v, -s);
  const D b = ld<D>(N, v, 2 * s) - ld<D>(N, v, -2 * s);
  return fmaT(O(8.0), cvt<O>(a), -cvt<O>(b));
}

template <class D>
__host__ __device__ __forceinline__ D fd2(const Nbhd &N, int v, int s, const D &c2) {
  const D s1 = ld<D>(N, v, s) + ld<D>(N, v, -s);
  const D s2 = ld<D>(N, v, 2 * s) + ld<D>(N, v, -2 * s);
  return fmaT(D(-30.0), ld<D>(N, v, 0), fmaT(D(16.0), s1, -s2)) * c2;
}

// sum over the four quadrants of one (a, b) offset pair of the mixed stencil
template <class D>
__host__ __device__ __forceinline__ D quad(const Nbhd &N, int v, int oa, int ob) {
  return (ld<D>(N, v, oa + ob) - ld<D>(N, v, -oa + ob)) - (ld<D>(N, v, oa - ob) - ld<D>(N, v, -oa - ob));
}

template <class D, class O>
__host__ __device__ __forceinline__ O fd11(const Nbhd &N, int v, int sa, int sb, const O &c3) {
  const D s11 = quad<D>(N, v, sa, sb);
  const D s12 = quad<D>(N, v, sa, 2 * sb);
  const D s21 = quad<D>(N, v, 2 * sa, sb);
  const D s22 = quad<D>(N, v, 2 * sa, 2 * sb);
  return fmaT(O(64.0), cvt<O>(s11), fmaT(O(-8.0), cvt<O>(s12) + cvt<O>(s21), cvt<O>(s22))) * c3;
}

// second derivative d_k d_l of field v (k, l known at compile time after unrolling)
template <class D>
__host__ __device__ __forceinline__ D fdkl(const Nbhd &N, int v, int k, int l, const StencilCoef<D> &C) {
  return k == l ? fd2<D>(N, v, N.st[k], C.c2) : fd11<D, D>(N, v, N.st[k], N.st[l], C.c3);
}

// Kreiss-Oliger sum of field v over the three axes, without its factor
// eps / (64 dx): the caller applies that factor in the fused multiply-add
// that adds the dissipation to the right-hand side.
template <class D>
__host__ __device__ __forceinline__ D ko_sum(const Nbhd &N, int v) {
  const int s0 = N.st[0], s1 = N.st[1], s2 = N.st[2];
  const D p1 = (ld<D>(N, v, s0) + ld<D>(N, v, -s0)) + (ld<D>(N, v, s1) + ld<D>(N, v, -s1)) +
               (ld<D>(N, v, s2) + ld<D>(N, v, -s2));
  const D p2 = (ld<D>(N, v, 2 * s0) + ld<D>(N, v, -2 * s0)) + (ld<D>(N, v, 2 * s1) + ld<D>(N, v, -2 * s1)) +
               (ld<D>(N, v, 2 * s2) + ld<D>(N, v, -2 * s2));
  const D p3 = (ld<D>(N, v, 3 * s0) + ld<D>(N, v, -3 * s0)) + (ld<D>(N, v, 3 * s1) + ld<D>(N, v, -3 * s1)) +
               (ld<D>(N, v, 3 * s2) + ld<D>(N, v, -3 * s2));
  return fmaT(D(-60.0), ld<D>(N, v, 0), fmaT(D(15.0), p1, fmaT(D(-6.0), p2, p3)));
}

// Pure second derivatives d_x d_x, d_y d_y, d_z d_z of field v and its
// Kreiss-Oliger sum, computed together: both use the same neighbour pair
// sums Q+ + Q- and Q++ + Q--. The second derivatives come out in O: for
// O != D the second differences Q+ + Q- - 2Q and Q++ + Q-- - 2Q are taken
// in D and only their weighted combination is done in O.
template <class D, class O, bool SCALED = true>
__host__ __device__ __forceinline__ void pure2_ko(const Nbhd &N, int v, const StencilCoef<D> &C, const O &c2o,
                                                  O d2[3], D &ko) {
  const D q0 = ld<D>(N, v, 0);
  D s1[3], s2[3], s3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
    s1[k] = ld<D>(N, v, s) + ld<D>(N, v, -s);
    s2[k] = ld<D>(N, v, 2 * s) + ld<D>(N, v, -2 * s);
    s3[k] = ld<D>(N, v, 3 * s) + ld<D>(N, v, -3 * s);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if constexpr (std::is_same<D, O>::value) {
      d2[k] = fmaT(D(-30.0), q0, fmaT(D(16.0), s1[k], -s2[k]));
      if constexpr (SCALED) d2[k] = d2[k] * C.c2;
    } else {
      const D t1 = fmaT(D(-2.0), q0, s1[k]), t2 = fmaT(D(-2.0), q0, s2[k]);
      d2[k] = fmaT(O(16.0), cvt<O>(t1), -cvt<O>(t2));
      if constexpr (SCALED) d2[k] = d2[k] * c2o;
    }
  }
  const D p1 = s1[0] + s1[1] + s1[2], p2 = s2[0] + s2[1] + s2[2], p3 = s3[0] + s3[1] + s3[2];
  ko = fmaT(D(-60.0), q0, fmaT(D(15.0), p1, fmaT(D(-6.0), p2, p3)));  // unscaled, as ko_sum
}

// All six second derivatives of field v, in the order xx, xy, xz, yy, yz, zz,
// in O, and its Kreiss-Oliger sum in D. The pure ones are taken here; the
// mixed ones were formed by the halo fill while the tile was in shared
// memory, sharing first derivatives between neighbouring points.
// SCALED false: the pure ones without their factor 1 / (12 dx^2), for a
// caller that folds it into its own coefficients.
template <class D, class O, bool SCALED = true>
__host__ __device__ __forceinline__ void second_ko(const Nbhd &N, int v, const StencilCoef<D> &C,
                                                   const StencilCoef<O> &CO, O dd[6], D &ko) {
  O d2[3];
  pure2_ko<D, O, SCALED>(N, v, C, CO.c2, d2, ko);
  dd[0] = d2[0];
  dd[3] = d2[1];
  dd[5] = d2[2];
  // the mixed derivatives come from the halo fill (CCZ4_BUF_MIX); the
  // mixed path's fill stores those it uses in FP32 as FP32
  const int m = mix_slot(v);
  if constexpr (std::is_same<O, float>::value) {
    const int fm = mix_fslot(m);
    dd[1] = N.mixedf(fm);
    dd[2] = N.mixedf(fm + 1);
    dd[4] = N.mixedf(fm + 2);
  } else {
    dd[1] = cvt<O>(D(N.mixed(m)));
    dd[2] = cvt<O>(D(N.mixed(m + 1)));
    dd[4] = cvt<O>(D(N.mixed(m + 2)));
  }
}

// A right-hand side (algebra type R) plus the dissipation eps/(64 dx) times
// the Kreiss-Oliger sum ko (taken in D): the sum is the differencing and
// stays in D; its factor and the addition are algebra, done in R.
template <class D, class R>
__host__ __device__ __forceinline__ D with_ko(const R &rhs, const D &ko, const StencilCoef<D> &C,
                                              const StencilCoef<R> &CR) {
  if constexpr (std::is_same<D, R>::value) {
    return fmaT(C.cko, ko, rhs);
  } else {
    return cvt<D>(fmaT(CR.cko, cvt<R>(ko), rhs));
  }
}

// ---- mixed path: differences on split pairs ----------------------------------------
// In the mixed path the halo fill stores every field but alpha and phi as
// a pair of FP32 numbers per tile point: hi = u rounded to FP32 and lo =
// u - hi (exact in FP64) rounded to FP32, so hi + lo = u to within
// 2^-48 |u| (split_pair below). The stencil differences are taken on the
// pairs with FP32 operations, whose pipe is 64 times wider than the FP64
// one on this GPU, and carry the accuracy of FP64 differences rounded once
// to FP32:
//  - a difference of two neighbours, u(+o) - u(-o) = (hi+ - hi-) + (lo+ -
//    lo-): the FP32 subtraction of the high parts is exact when they are
//    within a factor of two (Sterbenz) and otherwise within half an ulp of
//    a result that does not cancel further in the first-derivative
//    stencil;
//  - a second difference u(+o) + u(-o) - 2 u(0), which cancels to O(dx^2 u''),
//    from error-free differences of the high parts (Knuth's two-sum, sp_two_diff):
//    (d+ + d-) + ((e+ + e-) + (lo+ + lo- - 2 lo0)), where d+ + d- is exact
//    whenever it cancels (Sterbenz) and every other term is of order
//    2^-24 |u|, so the result is the exact second difference up to its own
//    rounding and 2^-48 |u|.
// The FD4 stencil weights and the Kreiss-Oliger combination are then applied
// in FP32 to these differences, as the mixed path applied them to the FP64
// differences before.
template <class R>
__host__ __device__ __forceinline__ void ld2(const Nbhd &N, int v, int off, R &h, R &l) {
  const float2 q = N.at2(v, off);
  h = R(q.x);
  l = R(q.y);
}

// a - b = s + e exactly (Knuth's two-sum applied to a and -b); returns s
template <class R>
__host__ __device__ __forceinline__ R sp_two_diff(const R &a, const R &b, R &e) {
  const R s = a - b;
  const R bv = s - a;
  e = (a - (s - bv)) - (b + bv);
  return s;
}

// u(+o) - u(-o)
template <class R>
__host__ __device__ __forceinline__ R sp_diff(const Nbhd &N, int v, int o) {
  R hp, lp, hm, lm;
  ld2<R>(N, v, o, hp, lp);
  ld2<R>(N, v, -o, hm, lm);
  return (hp - hm) + (lp - lm);
}

// u(+o) + u(-o) - 2 u(0), the centre pair (h0, l0) given
template <class R>
__host__ __device__ __forceinline__ R sp_second(const Nbhd &N, int v, int o, const R &h0, const R &l0) {
  R hp, lp, hm, lm, ep, em;
  ld2<R>(N, v, o, hp, lp);
  ld2<R>(N, v, -o, hm, lm);
  const R dp = sp_two_diff<R>(hp, h0, ep), dm = sp_two_diff<R>(hm, h0, em);
  return (dp + dm) + ((ep + em) + fmaT(R(-2.0), l0, lp + lm));
}

// first derivative along stride s without the factor 1 / (12 dx)
template <class R>
__host__ __device__ __forceinline__ R sp_fd1u(const Nbhd &N, int v, int s) {
  return fmaT(R(8.0), sp_diff<R>(N, v, s), -sp_diff<R>(N, v, 2 * s));
}

// Pure second derivatives along x, y, z (unscaled unless SCALED, which
// applies c2 = 1 / (12 dx^2)) and the Kreiss-Oliger sum over the three
// axes without its factor: sum over axes of b3 - 6 b2 + 15 b1, b_j the
// second difference at distance j (the -20 u(0) of each axis is inside the
// b_j). KO only: d2 == nullptr.
template <class R, bool SCALED>
__host__ __device__ __forceinline__ void sp_pure2_ko(const Nbhd &N, int v, const R &c2, R *d2, R &ko) {
  R h0, l0;
  ld2<R>(N, v, 0, h0, l0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
    const R b1 = sp_second<R>(N, v, s, h0, l0), b2 = sp_second<R>(N, v, 2 * s, h0, l0);
    const R b3 = sp_second<R>(N, v, 3 * s, h0, l0);
    if (d2) {
      d2[k] = fmaT(R(16.0), b1, -b2);
      if constexpr (SCALED) d2[k] = d2[k] * c2;
    }
    const R t = fmaT(R(15.0), b1, fmaT(R(-6.0), b2, b3));
    ko = k == 0 ? t : ko + t;
  }
}

// The mixed path's counterparts of fd1u, fd1o, ko_sum, second_ko and of
// the centre value, dispatched on the precision split: D == R reads FP64
// tiles, D != R split pairs (every field but alpha and phi).
template <class D, class R>
__host__ __device__ __forceinline__ R centre(const Nbhd &N, int v) {
  if constexpr (std::is_same<D, R>::value) {
    return ld<D>(N, v, 0);
  } else {
    R h, l;
    ld2<R>(N, v, 0, h, l);
    return h;
  }
}
template <class D, class R>
__host__ __device__ __forceinline__ R d1u(const Nbhd &N, int v, int s) {
  if constexpr (std::is_same<D, R>::value) return fd1u<D, R>(N, v, s);
  else return sp_fd1u<R>(N, v, s);
}
template <class D, class R>
__host__ __device__ __forceinline__ R d1o(const Nbhd &N, int v, int s, const R &c1) {
  if constexpr (std::is_same<D, R>::value) return fd1o<D, R>(N, v, s, c1);
  else return sp_fd1u<R>(N, v, s) * c1;
}
template <class D, class R>
__host__ __device__ __forceinline__ R kosum(const Nbhd &N, int v) {
  if constexpr (std::is_same<D, R>::value) {
    return ko_sum<D>(N, v);
  } else {
    R ko;
    sp_pure2_ko<R, false>(N, v, R(0.0), nullptr, ko);
    return ko;
  }
}
template <class D, class R, bool SCALED>
__host__ __device__ __forceinline__ void second_sp(const Nbhd &N, int v, const StencilCoef<D> &C,
                                                   const StencilCoef<R> &CR, R dd[6], R &ko) {
  if constexpr (std::is_same<D, R>::value) {
    second_ko<D, R, SCALED>(N, v, C, CR, dd, ko);
  } else {
    R d2[3];
    sp_pure2_ko<R, SCALED>(N, v, CR.c2, d2, ko);
    dd[0] = d2[0];
    dd[3] = d2[1];
    dd[5] = d2[2];
    const int m = mix_slot(v);
    if constexpr (std::is_same<R, float>::value) {
      const int fm = mix_fslot(m);
      dd[1] = N.mixedf(fm);
      dd[2] = N.mixedf(fm + 1);
      dd[4] = N.mixedf(fm + 2);
    } else {  // the counting types read the FP64 slots
      dd[1] = R(N.mixed(m));
      dd[2] = R(N.mixed(m + 1));
      dd[4] = R(N.mixed(m + 2));
    }
  }
}

// A right-hand side plus the dissipation of a Kreiss-Oliger sum ko taken
// in D (alpha, phi, and every field of the FP64 path) or in R (the other
// fields of the mixed path).
template <class D, class R, class K>
__host__ __device__ __forceinline__ D add_ko(const R &rhs, const K &ko, const StencilCoef<D> &C,
                                             const StencilCoef<R> &CR) {
  if constexpr (std::is_same<D, R>::value) return fmaT(C.cko, ko, rhs);
  else if constexpr (std::is_same<K, R>::value) return cvt<D>(fmaT(CR.cko, ko, rhs));
  else return cvt<D>(fmaT(CR.cko, cvt<R>(ko), rhs));
}

// Parameters of the equations, combined on the host and stored in the
// algebra type R (no per-point division or widening).
template <class R>
struct Phys {
  R itau;   // 1 / tau
  R c;      // c
  R c2;     // 2 c
  R K0;     // K0
  R k1a;    // 3 kappa1 (1 + kappa2)
  R k1b;    // kappa1 (2 + kappa2)
  R e2h;    // e^2 / 2
  R s3;     // s / 3
  R k3x2;   // 2 kappa3
  R kappa1, f, eta;
  int slicing, shift;
};

template <class R>
inline Phys<R> make_phys(const ccz4_params &P) {
  Phys<R> q;
  q.itau = R(1.0 / P.tau);
  q.c = R(P.c);
  q.c2 = R(2.0 * P.c);
  q.K0 = R(P.K0);
  q.k1a = R(3.0 * P.kappa1 * (1.0 + P.kappa2));
  q.k1b = R(P.kappa1 * (2.0 + P.kappa2));
  q.e2h = R(0.5 * P.e * P.e);
  q.s3 = R(P.s / 3.0);
  q.k3x2 = R(2.0 * P.kappa3);
  q.kappa1 = R(P.kappa1);
  q.f = R(P.f);
  q.eta = R(P.eta);
  q.slicing = P.slicing;
  q.shift = P.shift;
  return q;
}

// inverse of a symmetric 3x3 matrix stored as six components; returns det
template <class T>
__host__ __device__ __forceinline__ T sym_inverse(const T g[6], T ig[6]) {
  ig[0] = g[3] * g[5] - g[4] * g[4];
  ig[1] = g[2] * g[4] - g[1] * g[5];
  ig[2] = g[1] * g[4] - g[2] * g[3];
  ig[3] = g[0] * g[5] - g[2] * g[2];
  ig[4] = g[1] * g[2] - g[0] * g[4];
  ig[5] = g[0] * g[3] - g[1] * g[1];
  const T det = g[0] * ig[0] + g[1] * ig[1] + g[2] * ig[2];
  const T idet = T(1.0) / det;
#pragma unroll
  for (int c = 0; c < 6; ++c) ig[c] *= idet;
  return det;
}

// Right-hand side, Kreiss-Oliger dissipation included, at one interior point.
// Each field's value d_t Q_v is handed to sink(v, value) as soon as it is
// known, in the order g~, A~, alpha, phi, K, Theta, Gamma-hat, beta, b; the
// work is ordered so that every derivative is taken right before its first
// use, which keeps the number of live values (and so register spills) low.
// NB: the neighbourhood (Nbhd), or a type that supplies the same stencil
// values another way (the two-phase stage kernel's DerivTap).
template <class D, class R, class Sink, class NB>
__host__ __device__ __forceinline__ void ccz4_rhs_point(const Phys<R> &P, NB &N, const StencilCoef<D> &C,
                                                        const StencilCoef<R> &CR, Sink &sink) {
  constexpr bool SAME = std::is_same<D, R>::value;
  // ---- conformal metric, its inverse and its first derivatives ----------------
  D gD[6];
  R g[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    if constexpr (SAME) {
      gD[c] = ld<D>(N, GXX + c, 0);
      g[c] = cvt<R>(gD[c]);
    } else {
      // the FP64 metric (for the conformal-factor terms) from the split pair
      R l;
      ld2<R>(N, GXX + c, 0, g[c], l);
      gD[c] = cvt<D>(g[c]) + cvt<D>(l);
    }
  }
  // igw: the inverse with the off-diagonal entries doubled, for contractions
  // with a symmetric pair stored as six components
  R ig[6];
  const R det = sym_inverse<R>(g, ig);
  const R igw[6] = {ig[0], ig[1] + ig[1], ig[2] + ig[2], ig[3], ig[4] + ig[4], ig[5]};
  D igD[6], igwD[6];
  if constexpr (SAME) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      igD[c] = ig[c];
      igwD[c] = igw[c];
    }
  } else {
    sym_inverse<D>(gD, igD);
    igwD[0] = igD[0];
    igwD[1] = igD[1] + igD[1];
    igwD[2] = igD[2] + igD[2];
    igwD[3] = igD[3];
    igwD[4] = igD[4] + igD[4];
    igwD[5] = igD[5];
  }
  R be[3], Gh[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    be[i] = centre<D, R>(N, BETAX + i);
    Gh[i] = centre<D, R>(N, GHX + i);
  }
  CCZ4_MARK("inverse metric");

  // ---- Christoffel symbols of g~ --------------------------------------------
  // Gd[k][ij] = G~_kij = (d_i g~_jk + d_j g~_ik - d_k g~_ij) / 2 ; Gu[k][ij] = G~^k_ij
  R Gd[3][6], Gu[3][6], Gc[3];
  R advg[6], Ghdg[6];  // beta^k d_k g~_ij and Gamma-hat^k d_k g~_ij
  {
    // half the derivatives, so that the 1/2 of G~_kij costs nothing; the
    // contractions with beta and Gamma-hat take them doubled (all exact
    // powers of two: the same values as with full derivatives)
    const R c1h = R(0.5) * CR.c1;
    const R be2[3] = {be[0] + be[0], be[1] + be[1], be[2] + be[2]};
    const R Gh2[3] = {Gh[0] + Gh[0], Gh[1] + Gh[1], Gh[2] + Gh[2]};
    R dg[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) dg[k][c] = d1o<D, R>(N, GXX + c, N.st[k], c1h);  // (1/2) d_k g~_ij
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
          Gd[k][S6(i, j)] = dg[i][S6(j, k)] + dg[j][S6(i, k)] - dg[k][S6(i, j)];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      advg[c] = fmaT(be2[0], dg[0][c], fmaT(be2[1], dg[1][c], be2[2] * dg[2][c]));
      Ghdg[c] = fmaT(Gh2[0], dg[0][c], fmaT(Gh2[1], dg[1][c], Gh2[2] * dg[2][c]));
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      Gu[k][c] = fmaT(ig[S6(k, 0)], Gd[0][c], fmaT(ig[S6(k, 1)], Gd[1][c], ig[S6(k, 2)] * Gd[2][c]));
    R s = igw[0] * Gu[k][0];
#pragma unroll
    for (int c = 1; c < 6; ++c) s = fmaT(igw[c], Gu[k][c], s);
    Gc[k] = s;  // G~^k = g~^ij G~^k_ij
  }
  // Gamma-hat - G~ and 2 Z_i = g~_ij (Gamma-hat^j - G~^j) (Z only enters doubled)
  R dGam[3], Z2[3];  // Gamma-hat - G~ and 2 Z_i
#pragma unroll
  for (int i = 0; i < 3; ++i) dGam[i] = Gh[i] - Gc[i];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    Z2[i] = fmaT(g[S6(i, 0)], dGam[0], fmaT(g[S6(i, 1)], dGam[1], g[S6(i, 2)] * dGam[2]));
  CCZ4_MARK("christoffel");

  // ---- quadratic Christoffel part of the Ricci tensor -------------------------
  // Cm[k][i][m] = g~^lm G~^k_li. With it, g~^lm G~^k_li G~_jkm = sum_km Cm[k][i][m] G~_jkm
  // and g~^lm G~^k_im G~_klj = sum_kl Cm[k][i][l] G~_klj; Q6_ij collects the three terms.
  R Q6[6];
  {
    R Cm[3][3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int m = 0; m < 3; ++m)
          Cm[k][i][m] = fmaT(ig[S6(0, m)], Gu[k][S6(0, i)],
                             fmaT(ig[S6(1, m)], Gu[k][S6(1, i)], ig[S6(2, m)] * Gu[k][S6(2, i)]));
    R X[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R s = Cm[0][i][0] * Gd[j][S6(0, 0)];
#pragma unroll
        for (int q = 1; q < 9; ++q) s = fmaT(Cm[q / 3][i][q % 3], Gd[j][S6(q / 3, q % 3)], s);
        X[i][j] = s;
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        R q3 = X[i][j] + X[j][i];
#pragma unroll
        for (int q = 0; q < 9; ++q) q3 = fmaT(Cm[q / 3][i][q % 3], Gd[q / 3][S6(q % 3, j)], q3);
        Q6[S6(i, j)] = q3;
      }
  }
  CCZ4_MARK("ricci quadratic");

  // ---- conformal-factor terms and nabla nabla alpha, in D ---------------------
  // the parts of R_ij + 2 nabla_(i Z_j) and of nabla_i nabla_j alpha with
  // inverse powers of phi:
  //   (1/phi)(nabla~_i nabla~_j phi + g~_ij g~^kl nabla~_k nabla~_l phi)
  //   - (2/phi^2) g~_ij g~^kl P_k P_l + (2/phi^3) Z^k (g~_ik P_j + g~_jk P_i - g~_ij P_k)
  //   and (1/phi)(P_i A_j + P_j A_i - g~_ij g~^kl P_k A_l)
  const D phD = ld<D>(N, PHI, 0);
  const R ph = cvt<R>(phD), al = cvt<R>(ld<D>(N, ALPHA, 0));
  D daD[3], dPD[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    daD[k] = fd1<D>(N, ALPHA, N.st[k], C.c1);
    dPD[k] = fd1<D>(N, PHI, N.st[k], C.c1);
  }
  const D iph = D(1.0) / phD;
  const R da[3] = {cvt<R>(daD[0]), cvt<R>(daD[1]), cvt<R>(daD[2])};
  R phiRZ[6], DDa[6];
  D koP, koA;
  {
    D PuD[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      PuD[k] = fmaT(igD[S6(k, 0)], dPD[0], fmaT(igD[S6(k, 1)], dPD[1], igD[S6(k, 2)] * dPD[2]));
    const D PP = fmaT(PuD[0], dPD[0], fmaT(PuD[1], dPD[1], PuD[2] * dPD[2]));
    const D PA = fmaT(PuD[0], daD[0], fmaT(PuD[1], daD[1], PuD[2] * daD[2]));
    D dGamD[3], Z2D[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dGamD[i] = cvt<D>(dGam[i]);
      Z2D[i] = cvt<D>(Z2[i]);  // 2 Z_i
    }
    const D dGP = fmaT(dGamD[0], dPD[0], fmaT(dGamD[1], dPD[1], dGamD[2] * dPD[2]));
    D cdph[6];  // nabla~_i nabla~_j phi
    {
      D ddP[6];
      second_ko<D, D>(N, PHI, C, C, ddP, koP);
#pragma unroll
      for (int c = 0; c < 6; ++c)
        cdph[c] = fmaT(-cvt<D>(Gu[0][c]), dPD[0], fmaT(-cvt<D>(Gu[1][c]), dPD[1], fmaT(-cvt<D>(Gu[2][c]), dPD[2], ddP[c])));
    }
    D trcdph = igwD[0] * cdph[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) trcdph = fmaT(igwD[c], cdph[c], trcdph);
    // (1/phi)(cdph_ij + g~_ij (trcdph - dGP - 2 PP / phi) + 2 Z_i P_j + 2 Z_j P_i): the
    // g~_ij terms of the Ricci part share one coefficient
    const D iphPP = iph * PP;
    const D gco = (trcdph - dGP) - (iphPP + iphPP);
    D ddA[6];
    second_ko<D, D>(N, ALPHA, C, C, ddA, koA);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int c = S6(i, j);
        const D zt = fmaT(Z2D[i], dPD[j], Z2D[j] * dPD[i]);
        phiRZ[c] = cvt<R>(iph * (cdph[c] + fmaT(gD[c], gco, zt)));
        // nabla_i nabla_j alpha with the physical Christoffel symbols
        const D DDaD = fmaT(iph, fmaT(dPD[i], daD[j], fmaT(dPD[j], daD[i], -gD[c] * PA)), ddA[c]);
        DDa[c] = fmaT(-Gu[0][c], da[0], fmaT(-Gu[1][c], da[1], fmaT(-Gu[2][c], da[2], cvt<R>(DDaD))));
      }
  }
  R trDDa = igw[0] * DDa[0];
#pragma unroll
  for (int c = 1; c < 6; ++c) trDDa = fmaT(igw[c], DDa[c], trDDa);
  CCZ4_MARK("phi terms");

  // ---- R_ij + 2 nabla_(i Z_j) -----------------------------------------------------
  // -1/2 g~^kl d_k d_l g~_ij + g~_k(i d_j) Gamma-hat^k + 1/2 Gamma-hat^k d_k g~_ij + Q6_ij + phi terms
  // FP64 path: g~^kl with the factor 1 / (12 dx^2) of the pure second
  // differences on its diagonal, for the Laplacians of g~ and beta (taken
  // from unscaled pure ones: fewer FP64 multiplies). Mixed path: g~^kl and
  // scaled pure ones (the saving would be FP32 work, and the six weights
  // would stay live across the kernel).
  R igwc[6];
  if constexpr (SAME) {
    igwc[0] = igw[0] * CR.c2;
    igwc[1] = igw[1];
    igwc[2] = igw[2];
    igwc[3] = igw[3] * CR.c2;
    igwc[4] = igw[4];
    igwc[5] = igw[5] * CR.c2;
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) igwc[c] = igw[c];
  }
  R RZ[6], advGh[3];
  R kog[6];
  {
    R dG[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) dG[k][i] = d1o<D, R>(N, GHX + i, N.st[k], CR.c1);  // d_k Gamma-hat^i
#pragma unroll
    for (int i = 0; i < 3; ++i) advGh[i] = fmaT(be[0], dG[0][i], fmaT(be[1], dG[1][i], be[2] * dG[2][i]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int c = S6(i, j);
        R dd[6];
        second_sp<D, R, !SAME>(N, GXX + c, C, CR, dd, kog[c]);  // FP64 path: pure ones unscaled
        R lap = igwc[0] * dd[0];
#pragma unroll
        for (int q = 1; q < 6; ++q) lap = fmaT(igwc[q], dd[q], lap);
        R u = Ghdg[c];
#pragma unroll
        for (int k = 0; k < 3; ++k) u = fmaT(g[S6(k, i)], dG[j][k], fmaT(g[S6(k, j)], dG[i][k], u));
        RZ[c] = fmaT(R(-0.5), lap, fmaT(R(0.5), u, Q6[c] + phiRZ[c]));
      }
  }
  R trRZ = igw[0] * RZ[0];
#pragma unroll
  for (int c = 1; c < 6; ++c) trRZ = fmaT(igw[c], RZ[c], trRZ);
  const R ph2 = ph * ph;
  const R RpZ = ph2 * trRZ;     // R + 2 nabla_k Z^k
  const R lapal = ph2 * trDDa;  // nabla^i nabla_i alpha
  CCZ4_MARK("ricci assembly");

  // ---- A~ contractions ---------------------------------------------------------------
  R A[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) A[c] = centre<D, R>(N, AXX + c);
  R Au[6], AgA[6];
  {
    R Am[3][3];  // A~_i^m = A~_il g~^lm
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        Am[i][m] = fmaT(A[S6(i, 0)], ig[S6(0, m)], fmaT(A[S6(i, 1)], ig[S6(1, m)], A[S6(i, 2)] * ig[S6(2, m)]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        Au[S6(i, j)] = fmaT(ig[S6(i, 0)], Am[0][j], fmaT(ig[S6(i, 1)], Am[1][j], ig[S6(i, 2)] * Am[2][j]));
        AgA[S6(i, j)] = fmaT(Am[i][0], A[S6(0, j)], fmaT(Am[i][1], A[S6(1, j)], Am[i][2] * A[S6(2, j)]));
      }
  }
  const R trA = fmaT(igw[0], A[0], fmaT(igw[1], A[1], fmaT(igw[2], A[2], fmaT(igw[3], A[3],
                fmaT(igw[4], A[4], igw[5] * A[5])))));
  const R Auw[6] = {Au[0], Au[1] + Au[1], Au[2] + Au[2], Au[3], Au[4] + Au[4], Au[5]};
  R AA = A[0] * Auw[0];
#pragma unroll
  for (int c = 1; c < 6; ++c) AA = fmaT(A[c], Auw[c], AA);
  R GA[3];  // G~^i_jk A~^jk
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R s = Gu[i][0] * Auw[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) s = fmaT(Gu[i][c], Auw[c], s);
    GA[i] = s;
  }
  CCZ4_MARK("A contractions");

  // ---- d_t g~_ij, d_t A~_ij ---------------------------------------------------------------
  // beta / (12 dx): the advection of A~ and b takes unscaled first differences
  const R bec1[3] = {be[0] * CR.c1, be[1] * CR.c1, be[2] * CR.c1};
  R dB[3][3];  // B_k^i = d_k beta^i
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) dB[k][i] = d1o<D, R>(N, BETAX + i, N.st[k], CR.c1);
  const R third = R(1.0 / 3.0), twothird = R(2.0 / 3.0);
  const R trB = dB[0][0] + dB[1][1] + dB[2][2];
  const R trB23 = twothird * trB;
  const R Th = centre<D, R>(N, THETA), Kt = centre<D, R>(N, KTR);
  const R Kc = fmaT(-P.c2, Th, Kt);  // K - 2 c Theta
  const R al2 = al + al;
  {
    // Lie-derivative parts: Xg_ij = g~_ki B_j^k, XA_ij = A~_ki B_j^k, used as X_ij + X_ji
    R Xg[3][3], XA[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Xg[i][j] = fmaT(g[S6(0, i)], dB[j][0], fmaT(g[S6(1, i)], dB[j][1], g[S6(2, i)] * dB[j][2]));
        XA[i][j] = fmaT(A[S6(0, i)], dB[j][0], fmaT(A[S6(1, i)], dB[j][1], A[S6(2, i)] * dB[j][2]));
      }
    const R trMx = fmaT(al, trRZ, -trDDa);  // g~^ij (-nabla_i nabla_j alpha + alpha RZ_ij)
    const R sg = fmaT(twothird * al, trA, -trB23) - P.itau * (det - R(1.0));
    const R ph2al = ph2 * al;
    const R sA1 = -third * ph2 * trMx;
    const R sA2 = fmaT(al, Kc, -trB23);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int c = S6(i, j);
        sink(GXX + c, add_ko<D, R>(fmaT(g[c], sg, fmaT(-al2, A[c], advg[c] + (Xg[i][j] + Xg[j][i]))), kog[c], C, CR));
        R advA = XA[i][j] + XA[j][i];  // the advection and Lie-derivative terms
#pragma unroll
        for (int k = 0; k < 3; ++k) advA = fmaT(bec1[k], d1u<D, R>(N, AXX + c, N.st[k]), advA);
        const R rA = fmaT(ph2al, RZ[c], fmaT(-ph2, DDa[c], fmaT(g[c], sA1, fmaT(A[c], sA2, fmaT(-al2, AgA[c], advA)))));
        sink(AXX + c, add_ko<D, R>(rA, kosum<D, R>(N, AXX + c), C, CR));
      }
  }
  CCZ4_MARK("rhs g A");

  // ---- scalars ---------------------------------------------------------------------------------
  const R gK = (P.slicing == CCZ4_SLICING_ONE_PLUS_LOG) ? al2 : al * al;  // alpha^2 g(alpha)
  const R dP[3] = {cvt<R>(dPD[0]), cvt<R>(dPD[1]), cvt<R>(dPD[2])};
  sink(ALPHA, add_ko<D, R>(fmaT(be[0], da[0], fmaT(be[1], da[1], fmaT(be[2], da[2], -gK * (Kc - P.K0)))), koA, C, CR));
  sink(PHI, add_ko<D, R>(fmaT(be[0], dP[0], fmaT(be[1], dP[1], fmaT(be[2], dP[2], third * ph * fmaT(al, Kt, -trB)))), koP,
                          C, CR));
  // first differences of K and Theta without 1 / (12 dx): their advection
  // takes beta / (12 dx), the Gamma-hat equation coefficients with the factor
  R dK[3], dT[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dK[k] = d1u<D, R>(N, KTR, N.st[k]);
    dT[k] = d1u<D, R>(N, THETA, N.st[k]);
  }
  // the advection terms seeded with the other terms outside the factor alpha
  const R advK = fmaT(bec1[0], dK[0], fmaT(bec1[1], dK[1], fmaT(bec1[2], dK[2], -lapal)));
  sink(KTR, add_ko<D, R>(fmaT(al, RpZ + fmaT(Kt, Kc, -P.k1a * Th), advK), kosum<D, R>(N, KTR), C, CR));
  const R ZA = R(0.5) * ph2 * fmaT(dGam[0], da[0], fmaT(dGam[1], da[1], dGam[2] * da[2]));  // Z^i A_i
  const R advT = fmaT(bec1[0], dT[0], fmaT(bec1[1], dT[1], fmaT(bec1[2], dT[2], -ZA)));
  sink(THETA, add_ko<D, R>(fmaT(al, fmaT(P.e2h, RpZ + fmaT(twothird * Kt, Kt, -AA), -Th * fmaT(Kt, P.c, P.k1b)), advT),
                            kosum<D, R>(N, THETA), C, CR));
  CCZ4_MARK("rhs scalars");

  // ---- d_t Gamma-hat^i, gauge --------------------------------------------------------------------
  R lapB[3], gdivB[3];  // g~^kl d_k d_l beta^i and d_k (d_l beta^l)
  R koB[3];
  {
    R ddB[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      second_sp<D, R, !SAME>(N, BETAX + i, C, CR, ddB[i], koB[i]);  // FP64 path: pure ones unscaled
      R s = igwc[0] * ddB[i][0];
#pragma unroll
      for (int q = 1; q < 6; ++q) s = fmaT(igwc[q], ddB[i][q], s);
      lapB[i] = s;
    }
    // d_k d_l beta^l (FP64 path: the l = k term is the unscaled pure one)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if constexpr (SAME)
        gdivB[k] = fmaT(CR.c2, ddB[k][S6(k, k)],
                        ddB[(k + 1) % 3][S6(k, (k + 1) % 3)] + ddB[(k + 2) % 3][S6(k, (k + 2) % 3)]);
      else
        gdivB[k] = ddB[0][S6(k, 0)] + ddB[1][S6(k, 1)] + ddB[2][S6(k, 2)];
    }
  }
  const R al43 = R(4.0 / 3.0) * al;
  const R al6 = R(6.0) * al;
  const R Th2 = Th + Th;
  // coefficient of Gamma-hat^i - G~^i: (1/2)(-(4/3) alpha K - 2 alpha kappa1 + 2 kappa3 (2/3) tr B)
  const R zc = R(0.5) * fmaT(-al43, Kt, fmaT(-al2, P.kappa1, P.k3x2 * trB23));
  const R k3h = R(-0.5) * P.k3x2;
  // the terms g~^ik (2 alpha d_k Theta - (4/3) alpha d_k K + (s/3) d_k d_l beta^l
  // - 2 Theta d_k alpha) contract one vector with g~^ik
  const R al2c = al2 * CR.c1, al43c = al43 * CR.c1;
  R wv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) wv[k] = fmaT(al2c, dT[k], fmaT(-al43c, dK[k], fmaT(P.s3, gdivB[k], -Th2 * da[k])));
  R dbK[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R AuA = fmaT(Au[S6(i, 0)], da[0], fmaT(Au[S6(i, 1)], da[1], Au[S6(i, 2)] * da[2]));
    const R ZB = fmaT(dGam[0], dB[0][i], fmaT(dGam[1], dB[1][i], dGam[2] * dB[2][i]));
    // the 3 A~^ij P_j / phi term, in D
    const D AuP = fmaT(cvt<D>(Au[S6(i, 0)]), dPD[0], fmaT(cvt<D>(Au[S6(i, 1)]), dPD[1], cvt<D>(Au[S6(i, 2)]) * dPD[2]));
    const R AuPphi = cvt<R>(AuP * iph);
    R t = fmaT(ig[S6(i, 0)], wv[0], fmaT(ig[S6(i, 1)], wv[1], fmaT(ig[S6(i, 2)], wv[2], lapB[i])));
    t = fmaT(al2, GA[i], t);
    t = fmaT(trB23, Gc[i], t);
    t = fmaT(-al6, AuPphi, t);
    t = fmaT(R(-2.0), AuA, t);
    t = fmaT(zc, dGam[i], t);
    t = fmaT(k3h, ZB, t);
    // - G~^k B_k^i; d_t Gamma-hat^i - beta^k d_k Gamma-hat^i
    dbK[i] = fmaT(-Gc[0], dB[0][i], fmaT(-Gc[1], dB[1][i], fmaT(-Gc[2], dB[2][i], t)));
    sink(GHX + i, add_ko<D, R>(advGh[i] + dbK[i], kosum<D, R>(N, GHX + i), C, CR));
  }
  if (P.shift == CCZ4_SHIFT_GAMMA_DRIVER) {
    const R bb[3] = {centre<D, R>(N, BBX), centre<D, R>(N, BBY), centre<D, R>(N, BBZ)};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sink(BETAX + i, add_ko<D, R>(fmaT(be[0], dB[0][i], fmaT(be[1], dB[1][i], fmaT(be[2], dB[2][i], P.f * bb[i]))), koB[i],
                                C, CR));
      R advb = fmaT(-P.eta, bb[i], dbK[i]);
#pragma unroll
      for (int k = 0; k < 3; ++k) advb = fmaT(bec1[k], d1u<D, R>(N, BBX + i, N.st[k]), advb);
      sink(BBX + i, add_ko<D, R>(advb, kosum<D, R>(N, BBX + i), C, CR));
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sink(BETAX + i, add_ko<D, R>(R(0.0), koB[i], C, CR));
      sink(BBX + i, add_ko<D, R>(R(0.0), kosum<D, R>(N, BBX + i), C, CR));
    }
  }
  CCZ4_MARK("rhs gamma-hat gauge");
}

// Algebraic constraints after a time step (Sec. "Evolution equations"):
// rescale g~ by det(g~)^(-1/3) so that its determinant is one, then remove
// from A~ the trace taken with the rescaled metric.
template <class T>
__host__ __device__ __forceinline__ void enforce_point(T g[6], T A[6]) {
  const T det0 = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
                 g[2] * (g[1] * g[4] - g[3] * g[2]);
  const T sc = rcbrtT(det0);
#pragma unroll
  for (int c = 0; c < 6; ++c) g[c] *= sc;
  T ig[6];
  ig[0] = g[3] * g[5] - g[4] * g[4];
  ig[1] = g[2] * g[4] - g[1] * g[5];
  ig[2] = g[1] * g[4] - g[2] * g[3];
  ig[3] = g[0] * g[5] - g[2] * g[2];
  ig[4] = g[1] * g[2] - g[0] * g[4];
  ig[5] = g[0] * g[3] - g[1] * g[1];
  const T det = g[0] * ig[0] + g[1] * ig[1] + g[2] * ig[2];
  const T tr = (ig[0] * A[0] + ig[3] * A[3] + ig[5] * A[5] +
                T(2.0) * (ig[1] * A[1] + ig[2] * A[2] + ig[4] * A[4])) / det;
#pragma unroll
  for (int c = 0; c < 6; ++c) A[c] -= T(1.0 / 3.0) * g[c] * tr;
}

// RK4 stage update of one value: returns the new state value and updates acc.
// MODE 0..2: stage states; MODE 3: the final combination.
template <int MODE, class D>
__host__ __device__ __forceinline__ D rk_combine(const D &u, D &acc, const D &k, const D &dt) {
  if (MODE == 0) {
    acc = k;
    return fmaT(D(0.5) * dt, k, u);
  }
  if (MODE == 1 || MODE == 2) {
    acc = fmaT(D(2.0), k, acc);
    return fmaT(MODE == 2 ? dt : D(0.5) * dt, k, u);
  }
  return fmaT(dt * D(1.0 / 6.0), acc + k, u);
}

}  // namespace ccz4
