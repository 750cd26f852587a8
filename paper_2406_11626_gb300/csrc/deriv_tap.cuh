// Two-phase evaluation of the mixed-precision stage kernel.
//
// DerivTap stands in for the neighbourhood (Nbhd) of ccz4_rhs_point. In
// the recording phase (TAP_RECORD) every stencil value the right-hand side
// asks for -- first derivatives, pure second derivatives with their
// Kreiss-Oliger sum, Kreiss-Oliger sums -- is computed from the tile as
// before and also stored in this thread's slots in shared memory; run with
// a sink that discards the right-hand side, the algebra is dead code and
// only the differencing remains. In the replay phase (TAP_REPLAY) the same
// requests, made in the same order, read the slots back: the algebra runs
// with no tile loads in flight. Centre values and the mixed derivatives of
// the halo fill are read from memory in both phases (one load each).
//
// Slot k of a thread is at slots[k * stride] (stride = threads per block,
// so a warp's accesses fall in distinct banks); the request order is fixed
// by the code of ccz4_rhs_point, so after inlining k is a constant at each
// request. Floats and doubles have slots of their own.
#pragma once

#include "ccz4_algebra.cuh"

namespace ccz4 {

enum { TAP_RECORD = 0, TAP_REPLAY = 1 };

// Slots a point of the mixed path needs (checked by the host count of the
// kernel templates, ccz4_flops_per_point_stage's counting run).
constexpr int TAP_FLOATS = 120;
constexpr int TAP_DOUBLES = 16;

template <int MODE>
struct DerivTap {
  const Nbhd &nb;
  float *sf;    // this thread's float slots
  double *sd;   // and double slots
  int stride;
  int kf, kd;   // next slot of each kind
  int st[3];    // strides of the neighbourhood (the arguments ccz4_rhs_point passes along)
  __host__ __device__ __forceinline__ DerivTap(const Nbhd &n, float *f, double *d, int s)
      : nb(n), sf(f), sd(d), stride(s), kf(0), kd(0) {
    st[0] = n.st[0];
    st[1] = n.st[1];
    st[2] = n.st[2];
  }
  // a request beyond the slots (k is a constant at each request after
  // inlining, so the test costs nothing) is not stored: the host check of
  // the slot count keeps the code within them
  __host__ __device__ __forceinline__ float tap(float v) {
    if (kf < TAP_FLOATS) {
      if (MODE == TAP_RECORD) sf[kf * stride] = v;
      else v = sf[kf * stride];
    }
    ++kf;
    return v;
  }
  __host__ __device__ __forceinline__ double tap(double v) {
    if (kd < TAP_DOUBLES) {
      if (MODE == TAP_RECORD) sd[kd * stride] = v;
      else v = sd[kd * stride];
    }
    ++kd;
    return v;
  }
};

// centre values: read in both phases
template <class D, int M>
__host__ __device__ __forceinline__ D ld(DerivTap<M> &T, int v, int off) { return ld<D>(T.nb, v, off); }
template <class R, int M>
__host__ __device__ __forceinline__ void ld2(DerivTap<M> &T, int v, int off, R &h, R &l) { ld2<R>(T.nb, v, off, h, l); }
template <class D, class R, int M>
__host__ __device__ __forceinline__ R centre(DerivTap<M> &T, int v) { return centre<D, R>(T.nb, v); }

// stencil values: computed and stored, or read back
template <class D, class R, int M>
__host__ __device__ __forceinline__ R d1o(DerivTap<M> &T, int v, int s, const R &c1) {
  return T.tap(M == TAP_RECORD ? d1o<D, R>(T.nb, v, s, c1) : R(0));
}
template <class D, class R, int M>
__host__ __device__ __forceinline__ R d1u(DerivTap<M> &T, int v, int s) {
  return T.tap(M == TAP_RECORD ? d1u<D, R>(T.nb, v, s) : R(0));
}
template <class D, int M>
__host__ __device__ __forceinline__ D fd1(DerivTap<M> &T, int v, int s, const D &c1) {
  return T.tap(M == TAP_RECORD ? fd1<D>(T.nb, v, s, c1) : D(0));
}
template <class D, class R, int M>
__host__ __device__ __forceinline__ R kosum(DerivTap<M> &T, int v) {
  return T.tap(M == TAP_RECORD ? kosum<D, R>(T.nb, v) : R(0));
}
// six second derivatives: the three pure ones and the dissipation sum
// through the slots, the three mixed ones (xy, xz, yz) from the fill's
// buffer in both phases
template <class D, class O, bool SCALED = true, int M>
__host__ __device__ __forceinline__ void second_ko(DerivTap<M> &T, int v, const StencilCoef<D> &C, const StencilCoef<O> &CO,
                                          O dd[6], D &ko) {
  if (M == TAP_RECORD) second_ko<D, O, SCALED>(T.nb, v, C, CO, dd, ko);
  else {
    const int m = mix_slot(v);
    dd[1] = cvt<O>(D(T.nb.mixed(m)));
    dd[2] = cvt<O>(D(T.nb.mixed(m + 1)));
    dd[4] = cvt<O>(D(T.nb.mixed(m + 2)));
  }
  dd[0] = T.tap(dd[0]);
  dd[3] = T.tap(dd[3]);
  dd[5] = T.tap(dd[5]);
  ko = T.tap(ko);
}
template <class D, class R, bool SCALED, int M>
__host__ __device__ __forceinline__ void second_sp(DerivTap<M> &T, int v, const StencilCoef<D> &C, const StencilCoef<R> &CR,
                                          R dd[6], R &ko) {
  if (M == TAP_RECORD) second_sp<D, R, SCALED>(T.nb, v, C, CR, dd, ko);
  else {
    const int fm = mix_fslot(mix_slot(v));
    dd[1] = T.nb.mixedf(fm);
    dd[2] = T.nb.mixedf(fm + 1);
    dd[4] = T.nb.mixedf(fm + 2);
  }
  dd[0] = T.tap(dd[0]);
  dd[3] = T.tap(dd[3]);
  dd[5] = T.tap(dd[5]);
  ko = T.tap(ko);
}

// A sink that discards the right-hand side (the recording phase).
struct NullSink {
  __host__ __device__ __forceinline__ void operator()(int, double) {}
  __host__ __device__ __forceinline__ void finish() {}
};

}  // namespace ccz4
