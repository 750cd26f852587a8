// Operation-counting scalar types for the host-side flop count of the
// pointwise kernels (the algorithmic flops of the roofline).
//
// Cnt<T> wraps a double or a float and, on the host, tallies every
// arithmetic operation into the counter of its precision: add, sub and mul
// count one flop, an FMA two, a division one (tallied separately as well),
// conversions between precisions are tallied but carry no flops. Only
// same-type operations are defined, so instantiating the kernel templates
// with Cnt<double> and Cnt<float> also proves that the mixed-precision
// algebra contains no silent float -> double promotion.
#pragma once

#include <math.h>

namespace ccz4 {

struct OpTally {
  long long add = 0, mul = 0, fma = 0, div = 0, sqrt = 0, cvt = 0;
  double flops() const { return (double)(add + mul + div + sqrt) + 2.0 * (double)fma; }
};

// host-side tallies; index 0 = FP64, 1 = FP32
OpTally &tally(int precision_index);

template <class T>
struct Cnt {
  T v;
  static constexpr int PI = sizeof(T) == 8 ? 0 : 1;
  __host__ __device__ Cnt() : v(0) {}
  __host__ __device__ explicit Cnt(double x) : v((T)x) {}
  template <class U>
  __host__ __device__ explicit Cnt(const Cnt<U> &o) : v((T)o.v) {
#ifndef __CUDA_ARCH__
    tally(PI).cvt++;
#endif
  }
  __host__ __device__ static void tick(long long OpTally::*f) {
#ifndef __CUDA_ARCH__
    tally(PI).*f += 1;
#endif
  }
  __host__ __device__ Cnt operator-() const { return Cnt((double)-v); }
  __host__ __device__ Cnt &operator+=(const Cnt &o) { v += o.v; tick(&OpTally::add); return *this; }
  __host__ __device__ Cnt &operator-=(const Cnt &o) { v -= o.v; tick(&OpTally::add); return *this; }
  __host__ __device__ Cnt &operator*=(const Cnt &o) { v *= o.v; tick(&OpTally::mul); return *this; }
};

template <class T>
__host__ __device__ inline Cnt<T> operator+(Cnt<T> a, const Cnt<T> &b) { a += b; return a; }
template <class T>
__host__ __device__ inline Cnt<T> operator-(Cnt<T> a, const Cnt<T> &b) { a -= b; return a; }
template <class T>
__host__ __device__ inline Cnt<T> operator*(Cnt<T> a, const Cnt<T> &b) { a *= b; return a; }
template <class T>
__host__ __device__ inline Cnt<T> operator/(const Cnt<T> &a, const Cnt<T> &b) {
  Cnt<T>::tick(&OpTally::div);
  return Cnt<T>((double)(a.v / b.v));
}
template <class T>
__host__ __device__ inline Cnt<T> fmaT(const Cnt<T> &a, const Cnt<T> &b, const Cnt<T> &c) {
  Cnt<T>::tick(&OpTally::fma);
  return Cnt<T>((double)(a.v * b.v + c.v));
}
template <class T>
__host__ __device__ inline Cnt<T> sqrtT(const Cnt<T> &a) {
  Cnt<T>::tick(&OpTally::sqrt);
  return Cnt<T>(sqrt((double)a.v));
}
template <class T>
__host__ __device__ inline Cnt<T> rcbrtT(const Cnt<T> &a) {
  Cnt<T>::tick(&OpTally::sqrt);
  return Cnt<T>(1.0 / cbrt((double)a.v));
}

}  // namespace ccz4
