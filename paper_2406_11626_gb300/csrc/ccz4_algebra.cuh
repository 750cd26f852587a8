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
// Two scalar types: D carries the state, every finite difference, the
// contractions of second derivatives, the terms with inverse powers of the
// conformal factor phi (which grow without bound at a puncture) and the
// time update; R carries the rest of the pointwise algebra. D = R = double
// is the FP64 path; D = double, R = float the mixed path. Constants are
// written in the type they are used in, so no expression silently widens.
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

// index of the symmetric pair (i, j) among xx, xy, xz, yy, yz, zz
__host__ __device__ constexpr int S6(int i, int j) {
  return i > j ? S6(j, i) : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

// Read-only view of the halo'd neighbourhood of one point.
struct Nbhd {
  const double *__restrict__ c;  // field 0 at the centre point
  long long fs;                  // distance between fields
  int st[3];                     // distance between neighbours along x, y, z
  __host__ __device__ __forceinline__ double at(int v, int off) const {
#ifdef __CUDA_ARCH__
    return __ldg(c + v * fs + off);
#else
    return c[v * fs + off];
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

template <class D>
__host__ __device__ __forceinline__ D fd11(const Nbhd &N, int v, int sa, int sb, const D &c3) {
  const D s11 = quad<D>(N, v, sa, sb);
  const D s12 = quad<D>(N, v, sa, 2 * sb);
  const D s21 = quad<D>(N, v, 2 * sa, sb);
  const D s22 = quad<D>(N, v, 2 * sa, 2 * sb);
  return fmaT(D(64.0), s11, fmaT(D(-8.0), s12 + s21, s22)) * c3;
}

// second derivative d_k d_l of field v (k, l known at compile time after unrolling)
template <class D>
__host__ __device__ __forceinline__ D fdkl(const Nbhd &N, int v, int k, int l, const StencilCoef<D> &C) {
  return k == l ? fd2<D>(N, v, N.st[k], C.c2) : fd11<D>(N, v, N.st[k], N.st[l], C.c3);
}

template <class D>
__host__ __device__ __forceinline__ D ko_sum(const Nbhd &N, int v, const D &cko) {
  D p1 = D(0.0), p2 = D(0.0), p3 = D(0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
    p1 += ld<D>(N, v, s) + ld<D>(N, v, -s);
    p2 += ld<D>(N, v, 2 * s) + ld<D>(N, v, -2 * s);
    p3 += ld<D>(N, v, 3 * s) + ld<D>(N, v, -3 * s);
  }
  return fmaT(D(-60.0), ld<D>(N, v, 0), fmaT(D(15.0), p1, fmaT(D(-6.0), p2, p3))) * cko;
}

// Parameters of the equations, combined on the host and stored in the
// algebra type R (no per-point division or widening).
template <class R>
struct Phys {
  R itau;   // 1 / tau
  R c;      // c
  R K0;     // K0
  R k1a;    // 3 kappa1 (1 + kappa2)
  R k1b;    // kappa1 (2 + kappa2)
  R e2;     // e^2
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
  q.K0 = R(P.K0);
  q.k1a = R(3.0 * P.kappa1 * (1.0 + P.kappa2));
  q.k1b = R(P.kappa1 * (2.0 + P.kappa2));
  q.e2 = R(P.e * P.e);
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

// Right-hand side (without the dissipation term) at one interior point.
template <class D, class R>
__host__ __device__ __forceinline__ void ccz4_rhs_point(const Phys<R> &P, const Nbhd &N,
                                                        const StencilCoef<D> &C, D r[NV]) {
  constexpr bool SAME = std::is_same<D, R>::value;
  // ---- state and first derivatives, in D ------------------------------------
  D gD[6];
  R g[6], A[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    gD[c] = ld<D>(N, GXX + c, 0);
    g[c] = R(gD[c]);
    A[c] = R(ld<D>(N, AXX + c, 0));
  }
  const D phD = ld<D>(N, PHI, 0);
  const R al = R(ld<D>(N, ALPHA, 0)), ph = R(phD), Kt = R(ld<D>(N, KTR, 0)), Th = R(ld<D>(N, THETA, 0));
  R be[3], Gh[3], bb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    be[i] = R(ld<D>(N, BETAX + i, 0));
    Gh[i] = R(ld<D>(N, GHX + i, 0));
    bb[i] = R(ld<D>(N, BBX + i, 0));
  }
  D daD[3], dPD[3];
  R dg[3][6], dA[3][6], da[3], dB[3][3], dP[3], dK[3], dT[3], dG[3][3], db[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dg[k][c] = R(fd1<D>(N, GXX + c, s, C.c1));
      dA[k][c] = R(fd1<D>(N, AXX + c, s, C.c1));
    }
    daD[k] = fd1<D>(N, ALPHA, s, C.c1);
    dPD[k] = fd1<D>(N, PHI, s, C.c1);
    da[k] = R(daD[k]);
    dP[k] = R(dPD[k]);
    dK[k] = R(fd1<D>(N, KTR, s, C.c1));
    dT[k] = R(fd1<D>(N, THETA, s, C.c1));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dB[k][i] = R(fd1<D>(N, BETAX + i, s, C.c1));  // B_k^i = d_k beta^i
      dG[k][i] = R(fd1<D>(N, GHX + i, s, C.c1));    // d_k Gamma-hat^i
      db[k][i] = R(fd1<D>(N, BBX + i, s, C.c1));    // d_k b^i
    }
  }

  CCZ4_MARK("first derivatives");
  // ---- inverse conformal metric ---------------------------------------------
  R ig[6];
  const R det = sym_inverse<R>(g, ig);
  D igD[6];
  if constexpr (SAME) {
#pragma unroll
    for (int c = 0; c < 6; ++c) igD[c] = ig[c];
  } else {
    sym_inverse<D>(gD, igD);
  }
  const R w6[6] = {R(1.0), R(2.0), R(2.0), R(1.0), R(2.0), R(1.0)};
  const D w6D[6] = {D(1.0), D(2.0), D(2.0), D(1.0), D(2.0), D(1.0)};

  CCZ4_MARK("inverse metric");
  // ---- Christoffel symbols of g~ --------------------------------------------
  // Gd[k][ij] = G~_kij = (d_i g~_jk + d_j g~_ik - d_k g~_ij) / 2 ; Gu[k][ij] = G~^k_ij
  R Gd[3][6], Gu[3][6], Gc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        Gd[k][S6(i, j)] = R(0.5) * (dg[i][S6(j, k)] + dg[j][S6(i, k)] - dg[k][S6(i, j)]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      Gu[k][c] = fmaT(ig[S6(k, 0)], Gd[0][c], fmaT(ig[S6(k, 1)], Gd[1][c], ig[S6(k, 2)] * Gd[2][c]));
    R s = R(0.0);
#pragma unroll
    for (int c = 0; c < 6; ++c) s = fmaT(w6[c] * ig[c], Gu[k][c], s);
    Gc[k] = s;  // G~^k = g~^ij G~^k_ij
  }
  // Gamma-hat - G~ and Z_i = g~_ij (Gamma-hat^j - G~^j) / 2
  R dGam[3], Zd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) dGam[i] = Gh[i] - Gc[i];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    Zd[i] = R(0.5) * fmaT(g[S6(i, 0)], dGam[0], fmaT(g[S6(i, 1)], dGam[1], g[S6(i, 2)] * dGam[2]));

  CCZ4_MARK("christoffel");
  // ---- conformal-factor terms, in D -----------------------------------------
  // the parts of R_ij + 2 nabla_(i Z_j) and of nabla_i nabla_j alpha with
  // inverse powers of phi:
  //   (1/phi)(nabla~_i nabla~_j phi + g~_ij g~^kl nabla~_k nabla~_l phi)
  //   - (2/phi^2) g~_ij g~^kl P_k P_l + (2/phi^3) Z^k (g~_ik P_j + g~_jk P_i - g~_ij P_k)
  //   and (1/phi)(P_i A_j + P_j A_i - g~_ij g~^kl P_k A_l)
  const D iph = D(1.0) / phD;
  D PuD[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    PuD[k] = fmaT(igD[S6(k, 0)], dPD[0], fmaT(igD[S6(k, 1)], dPD[1], igD[S6(k, 2)] * dPD[2]));
  const D PP = fmaT(PuD[0], dPD[0], fmaT(PuD[1], dPD[1], PuD[2] * dPD[2]));
  const D PA = fmaT(PuD[0], daD[0], fmaT(PuD[1], daD[1], PuD[2] * daD[2]));
  D dGamD[3], ZdD[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dGamD[i] = D(dGam[i]);
    ZdD[i] = D(Zd[i]);
  }
  const D dGP = fmaT(dGamD[0], dPD[0], fmaT(dGamD[1], dPD[1], dGamD[2] * dPD[2]));
  D cdph[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      const D Gp = fmaT(D(Gu[0][c]), dPD[0], fmaT(D(Gu[1][c]), dPD[1], D(Gu[2][c]) * dPD[2]));
      cdph[c] = fdkl<D>(N, PHI, i, j, C) - Gp;  // nabla~_i nabla~_j phi
    }
  D trcdph = D(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) trcdph = fmaT(w6D[c] * igD[c], cdph[c], trcdph);
  const D two_iph2PP = D(2.0) * iph * iph * PP;
  R phiRZ[6], phiDDa[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      const D zt = D(2.0) * (ZdD[i] * dPD[j] + ZdD[j] * dPD[i]) - gD[c] * dGP;
      phiRZ[c] = R(iph * (cdph[c] + fmaT(gD[c], trcdph, zt)) - two_iph2PP * gD[c]);
      phiDDa[c] = R(iph * (dPD[i] * daD[j] + dPD[j] * daD[i] - gD[c] * PA));
    }

  CCZ4_MARK("phi terms");
  // ---- second derivatives of alpha, g~ and beta, contracted in D ----------------
  R DDa[6];  // nabla_i nabla_j alpha (physical Christoffel symbols)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      const R Ga = fmaT(Gu[0][c], da[0], fmaT(Gu[1][c], da[1], Gu[2][c] * da[2]));
      DDa[c] = R(fdkl<D>(N, ALPHA, i, j, C)) - Ga + phiDDa[c];
    }
  R lapg[6];  // g~^kl d_k d_l g~_ij
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    D s = D(0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) s = fmaT(w6D[S6(k, l)] * igD[S6(k, l)], fdkl<D>(N, GXX + c, k, l, C), s);
    lapg[c] = R(s);
  }
  R lapB[3], gdivB[3];  // g~^kl d_k d_l beta^i and d_k (d_l beta^l)
  {
    D lb[3] = {D(0.0), D(0.0), D(0.0)}, gd[3] = {D(0.0), D(0.0), D(0.0)};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) {
        const D w = w6D[S6(k, l)] * igD[S6(k, l)];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const D u = fdkl<D>(N, BETAX + i, k, l, C);
          lb[i] = fmaT(w, u, lb[i]);
          if (i == l) gd[k] += u;
          if (i == k && k != l) gd[l] += u;
        }
      }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lapB[i] = R(lb[i]);
      gdivB[i] = R(gd[i]);
    }
  }
  R trDDa = R(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) trDDa = fmaT(w6[c] * ig[c], DDa[c], trDDa);

  CCZ4_MARK("second derivatives");
  // ---- quadratic Christoffel part of the Ricci tensor ---------------------------
  // Cm[k][i][m] = g~^lm G~^k_li ; Em[k][j][m] = g~^lm G~_klj ; X_ij = g~^lm G~^k_li G~_jkm
  R Cm[3][3][3], Em[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Cm[k][i][m] = fmaT(ig[S6(0, m)], Gu[k][S6(0, i)],
                           fmaT(ig[S6(1, m)], Gu[k][S6(1, i)], ig[S6(2, m)] * Gu[k][S6(2, i)]));
        Em[k][i][m] = fmaT(ig[S6(0, m)], Gd[k][S6(0, i)],
                           fmaT(ig[S6(1, m)], Gd[k][S6(1, i)], ig[S6(2, m)] * Gd[k][S6(2, i)]));
      }
  R X[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R s = R(0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) s = fmaT(Cm[k][i][m], Gd[j][S6(k, m)], s);
      X[i][j] = s;
    }

  CCZ4_MARK("ricci quadratic");
  // ---- R_ij + 2 nabla_(i Z_j) -------------------------------------------------------
  R RZ[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      R t = R(-0.5) * lapg[c];
      // g~_k(i d_j) Gamma-hat^k + 1/2 Gamma-hat^k d_k g~_ij
      R u = R(0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        u += fmaT(g[S6(k, i)], dG[j][k], fmaT(g[S6(k, j)], dG[i][k], Gh[k] * dg[k][c]));
      t = fmaT(R(0.5), u, t);
      // g~^lm (G~^k_li G~_jkm + G~^k_lj G~_ikm + G~^k_im G~_klj)
      R q3 = R(0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) q3 = fmaT(Gu[k][S6(i, m)], Em[k][j][m], q3);
      RZ[c] = t + X[i][j] + X[j][i] + q3 + phiRZ[c];
    }
  R trRZ = R(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) trRZ = fmaT(w6[c] * ig[c], RZ[c], trRZ);
  const R ph2 = ph * ph;
  const R RpZ = ph2 * trRZ;    // R + 2 nabla_k Z^k
  const R lapal = ph2 * trDDa;  // nabla^i nabla_i alpha

  CCZ4_MARK("ricci assembly");
  // ---- A~ contractions ---------------------------------------------------------------
  R Am[3][3];  // A~_i^m = A~_il g~^lm
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m)
      Am[i][m] = fmaT(A[S6(i, 0)], ig[S6(0, m)], fmaT(A[S6(i, 1)], ig[S6(1, m)], A[S6(i, 2)] * ig[S6(2, m)]));
  const R trA = Am[0][0] + Am[1][1] + Am[2][2];
  R Au[6], AgA[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      Au[S6(i, j)] = fmaT(ig[S6(i, 0)], Am[0][j], fmaT(ig[S6(i, 1)], Am[1][j], ig[S6(i, 2)] * Am[2][j]));
      AgA[S6(i, j)] = fmaT(Am[i][0], A[S6(0, j)], fmaT(Am[i][1], A[S6(1, j)], Am[i][2] * A[S6(2, j)]));
    }
  R AA = R(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) AA = fmaT(w6[c] * A[c], Au[c], AA);

  const R trB = dB[0][0] + dB[1][1] + dB[2][2];
  const R Kc = Kt - R(2.0) * P.c * Th;  // K - 2 Theta c
  const R third = R(1.0 / 3.0), twothird = R(2.0 / 3.0);

  CCZ4_MARK("A contractions");
  // ---- d_t g~_ij, d_t A~_ij ---------------------------------------------------------------
  const R trMx = al * trRZ - trDDa;  // g~^ij (-nabla_i nabla_j alpha + alpha RZ_ij)
  R rr[NV];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      R advg = R(0.0), lieg = R(0.0), advA = R(0.0), lieA = R(0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        advg = fmaT(be[k], dg[k][c], advg);
        lieg += fmaT(g[S6(k, i)], dB[j][k], g[S6(k, j)] * dB[i][k]);
        advA = fmaT(be[k], dA[k][c], advA);
        lieA += fmaT(A[S6(k, i)], dB[j][k], A[S6(k, j)] * dB[i][k]);
      }
      rr[GXX + c] = advg + lieg - twothird * g[c] * trB - R(2.0) * al * (A[c] - third * g[c] * trA) -
                    P.itau * (det - R(1.0)) * g[c];
      const R Mij = al * RZ[c] - DDa[c];
      rr[AXX + c] = advA + ph2 * (Mij - third * g[c] * trMx) + lieA - twothird * A[c] * trB +
                    al * A[c] * Kc - R(2.0) * al * AgA[c];
    }

  CCZ4_MARK("rhs g A");
  // ---- scalars ---------------------------------------------------------------------------------
  const R advK = fmaT(be[0], dK[0], fmaT(be[1], dK[1], be[2] * dK[2]));
  const R advT = fmaT(be[0], dT[0], fmaT(be[1], dT[1], be[2] * dT[2]));
  const R gK = (P.slicing == CCZ4_SLICING_ONE_PLUS_LOG) ? R(2.0) * al : al * al;  // alpha^2 g(alpha)
  rr[ALPHA] = fmaT(be[0], da[0], fmaT(be[1], da[1], be[2] * da[2])) - gK * (Kt - P.K0 - R(2.0) * P.c * Th);
  rr[PHI] = fmaT(be[0], dP[0], fmaT(be[1], dP[1], be[2] * dP[2])) + third * ph * (al * Kt - trB);
  rr[KTR] = advK - lapal + al * RpZ + al * Kt * Kc - al * P.k1a * Th;
  const R ZA = R(0.5) * ph2 * fmaT(dGam[0], da[0], fmaT(dGam[1], da[1], dGam[2] * da[2]));  // Z^i A_i
  const R e2 = P.e2;
  rr[THETA] = advT + R(0.5) * al * e2 * (RpZ + twothird * Kt * Kt - AA) - al * Th * Kt * P.c - ZA -
              al * P.k1b * Th;

  CCZ4_MARK("rhs scalars");
  // ---- d_t Gamma-hat^i, gauge --------------------------------------------------------------------
  // the 3 A~^ij P_j / phi term of the Gamma-hat equation, in D
  R AuPphi[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const D s = fmaT(D(Au[S6(i, 0)]), dPD[0], fmaT(D(Au[S6(i, 1)]), dPD[1], D(Au[S6(i, 2)]) * dPD[2]));
    AuPphi[i] = R(s * iph);
  }
  const R s3 = P.s3;
  R dbK[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R adv = R(0.0), gT = R(0.0), gKk = R(0.0), gdv = R(0.0), gA = R(0.0), GB = R(0.0), AuA = R(0.0), ZB = R(0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      adv = fmaT(be[k], dG[k][i], adv);
      gT = fmaT(ig[S6(i, k)], dT[k], gT);
      gKk = fmaT(ig[S6(i, k)], dK[k], gKk);
      gdv = fmaT(ig[S6(i, k)], gdivB[k], gdv);
      gA = fmaT(ig[S6(i, k)], da[k], gA);
      GB = fmaT(Gc[k], dB[k][i], GB);
      AuA = fmaT(Au[S6(i, k)], da[k], AuA);
      ZB = fmaT(dGam[k], dB[k][i], ZB);
    }
    R GA = R(0.0);  // G~^i_jk A~^jk
#pragma unroll
    for (int c = 0; c < 6; ++c) GA = fmaT(w6[c] * Gu[i][c], Au[c], GA);
    const R Zc = R(0.5) * dGam[i];  // g~^ij Z_j
    const R rG = adv + R(2.0) * al * gT + lapB[i] + s3 * gdv - R(4.0 / 3.0) * al * gKk +
                 twothird * Gc[i] * trB - GB + R(2.0) * al * (GA - R(3.0) * AuPphi[i]) - R(2.0) * Th * gA -
                 R(4.0 / 3.0) * al * Kt * Zc - R(2.0) * AuA - R(2.0) * al * P.kappa1 * Zc +
                 P.k3x2 * (twothird * Zc * trB - R(0.5) * ZB);
    rr[GHX + i] = rG;
    dbK[i] = rG - adv;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (P.shift == CCZ4_SHIFT_GAMMA_DRIVER) {
      rr[BETAX + i] = fmaT(be[0], dB[0][i], fmaT(be[1], dB[1][i], be[2] * dB[2][i])) + P.f * bb[i];
      rr[BBX + i] = fmaT(be[0], db[0][i], fmaT(be[1], db[1][i], be[2] * db[2][i])) + dbK[i] - P.eta * bb[i];
    } else {
      rr[BETAX + i] = R(0.0);
      rr[BBX + i] = R(0.0);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) r[v] = D(rr[v]);
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
