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
// Arithmetic is arranged for the FP64 pipe: reciprocals of det g~, phi and
// the grid spacing are taken once, symmetric tensors are stored as six
// components, contractions use the symmetry, and stencil sums are paired so
// that most operations fuse into FMAs.
#pragma once

#include "ccz4_internal.cuh"

namespace ccz4 {

// index of the symmetric pair (i, j) among xx, xy, xz, yy, yz, zz
__host__ __device__ constexpr int S6(int i, int j) {
  return i > j ? S6(j, i) : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

// Read-only view of the halo'd neighbourhood of one point.
struct Nbhd {
  const double *__restrict__ c;  // field 0 at the centre point
  long long fs;                  // distance between fields
  int st[3];                     // distance between neighbours along x, y, z
  __device__ __forceinline__ double at(int v, int off) const { return __ldg(c + v * fs + off); }
};

struct StencilCoef {
  double c1;   // 1 / (12 dx)
  double c2;   // 1 / (12 dx^2)
  double c3;   // 1 / (144 dx^2)
  double cko;  // eps / (64 dx)
};

__device__ __forceinline__ double fd1(const Nbhd &N, int v, int s, double c1) {
  const double a = N.at(v, s) - N.at(v, -s);
  const double b = N.at(v, 2 * s) - N.at(v, -2 * s);
  return fma(8.0, a, -b) * c1;
}

__device__ __forceinline__ double fd2(const Nbhd &N, int v, int s, double c2) {
  const double s1 = N.at(v, s) + N.at(v, -s);
  const double s2 = N.at(v, 2 * s) + N.at(v, -2 * s);
  return fma(-30.0, N.at(v, 0), fma(16.0, s1, -s2)) * c2;
}

// sum over the four quadrants of one (a, b) offset pair of the mixed stencil
__device__ __forceinline__ double quad(const Nbhd &N, int v, int oa, int ob) {
  return (N.at(v, oa + ob) - N.at(v, -oa + ob)) - (N.at(v, oa - ob) - N.at(v, -oa - ob));
}

__device__ __forceinline__ double fd11(const Nbhd &N, int v, int sa, int sb, double c3) {
  const double s11 = quad(N, v, sa, sb);
  const double s12 = quad(N, v, sa, 2 * sb);
  const double s21 = quad(N, v, 2 * sa, sb);
  const double s22 = quad(N, v, 2 * sa, 2 * sb);
  return fma(64.0, s11, fma(-8.0, s12 + s21, s22)) * c3;
}

// second derivative d_k d_l of field v, k and l known at compile time after unrolling
__device__ __forceinline__ double fdkl(const Nbhd &N, int v, int k, int l, const StencilCoef &C) {
  return k == l ? fd2(N, v, N.st[k], C.c2) : fd11(N, v, N.st[k], N.st[l], C.c3);
}

__device__ __forceinline__ double ko_sum(const Nbhd &N, int v, double cko) {
  double p1 = 0.0, p2 = 0.0, p3 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
    p1 += N.at(v, s) + N.at(v, -s);
    p2 += N.at(v, 2 * s) + N.at(v, -2 * s);
    p3 += N.at(v, 3 * s) + N.at(v, -3 * s);
  }
  return fma(-60.0, N.at(v, 0), fma(15.0, p1, fma(-6.0, p2, p3))) * cko;
}

// Right-hand side (without the dissipation term) at one interior point.
__device__ __forceinline__ void ccz4_rhs_point(const ccz4_params &P, const Nbhd &N,
                                               const StencilCoef &C, double r[NV]) {
  // ---- state and first derivatives --------------------------------------
  double g[6], A[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    g[c] = N.at(GXX + c, 0);
    A[c] = N.at(AXX + c, 0);
  }
  const double al = N.at(ALPHA, 0), ph = N.at(PHI, 0), Kt = N.at(KTR, 0), Th = N.at(THETA, 0);
  double be[3], Gh[3], bb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    be[i] = N.at(BETAX + i, 0);
    Gh[i] = N.at(GHX + i, 0);
    bb[i] = N.at(BBX + i, 0);
  }
  double dg[3][6], dA[3][6], da[3], dB[3][3], dP[3], dK[3], dT[3], dG[3][3], db[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dg[k][c] = fd1(N, GXX + c, s, C.c1);
      dA[k][c] = fd1(N, AXX + c, s, C.c1);
    }
    da[k] = fd1(N, ALPHA, s, C.c1);
    dP[k] = fd1(N, PHI, s, C.c1);
    dK[k] = fd1(N, KTR, s, C.c1);
    dT[k] = fd1(N, THETA, s, C.c1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dB[k][i] = fd1(N, BETAX + i, s, C.c1);  // B_k^i = d_k beta^i
      dG[k][i] = fd1(N, GHX + i, s, C.c1);    // d_k Gamma-hat^i
      db[k][i] = fd1(N, BBX + i, s, C.c1);    // d_k b^i
    }
  }

  // ---- inverse conformal metric -----------------------------------------
  double ig[6];
  ig[0] = g[3] * g[5] - g[4] * g[4];
  ig[1] = g[2] * g[4] - g[1] * g[5];
  ig[2] = g[1] * g[4] - g[2] * g[3];
  ig[3] = g[0] * g[5] - g[2] * g[2];
  ig[4] = g[1] * g[2] - g[0] * g[4];
  ig[5] = g[0] * g[3] - g[1] * g[1];
  const double det = g[0] * ig[0] + g[1] * ig[1] + g[2] * ig[2];
  const double idet = 1.0 / det;
#pragma unroll
  for (int c = 0; c < 6; ++c) ig[c] *= idet;
  // contraction weights for sums over a symmetric pair
  const double w6[6] = {1.0, 2.0, 2.0, 1.0, 2.0, 1.0};

  // ---- Christoffel symbols of g~ ------------------------------------------
  // Gd[k][ij] = G~_kij = (d_i g~_jk + d_j g~_ik - d_k g~_ij) / 2
  double Gd[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        Gd[k][S6(i, j)] = 0.5 * (dg[i][S6(j, k)] + dg[j][S6(i, k)] - dg[k][S6(i, j)]);
  // Gu[k][ij] = G~^k_ij
  double Gu[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 6; ++c)
      Gu[k][c] = ig[S6(k, 0)] * Gd[0][c] + ig[S6(k, 1)] * Gd[1][c] + ig[S6(k, 2)] * Gd[2][c];
  // contracted G~^k = g~^ij G~^k_ij
  double Gc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) s = fma(w6[c] * ig[c], Gu[k][c], s);
    Gc[k] = s;
  }

  // ---- conformal factor, Z ---------------------------------------------------
  const double iph = 1.0 / ph;
  const double ph2 = ph * ph;
  double dGam[3], Zd[3];  // Gamma-hat - G~, and Z_i = g~_ij dGam^j / 2
#pragma unroll
  for (int i = 0; i < 3; ++i) dGam[i] = Gh[i] - Gc[i];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    Zd[i] = 0.5 * (g[S6(i, 0)] * dGam[0] + g[S6(i, 1)] * dGam[1] + g[S6(i, 2)] * dGam[2]);
  double Pu[3];  // g~^kl P_l
#pragma unroll
  for (int k = 0; k < 3; ++k) Pu[k] = ig[S6(k, 0)] * dP[0] + ig[S6(k, 1)] * dP[1] + ig[S6(k, 2)] * dP[2];
  const double PP = Pu[0] * dP[0] + Pu[1] * dP[1] + Pu[2] * dP[2];
  const double PA = Pu[0] * da[0] + Pu[1] * da[1] + Pu[2] * da[2];
  const double dGP = dGam[0] * dP[0] + dGam[1] * dP[1] + dGam[2] * dP[2];

  // ---- second derivatives of alpha and phi ----------------------------------
  double DDa[6], cdph[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      const double ua = fdkl(N, ALPHA, i, j, C);
      const double up = fdkl(N, PHI, i, j, C);
      const double Ga = Gu[0][c] * da[0] + Gu[1][c] * da[1] + Gu[2][c] * da[2];
      const double Gp = Gu[0][c] * dP[0] + Gu[1][c] * dP[1] + Gu[2][c] * dP[2];
      // nabla_i nabla_j alpha with the physical Christoffel symbols
      DDa[c] = ua - Ga + iph * (dP[i] * da[j] + dP[j] * da[i] - g[c] * PA);
      cdph[c] = up - Gp;  // nabla~_i nabla~_j phi
    }
  double trDDa = 0.0, trcdph = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    trDDa = fma(w6[c] * ig[c], DDa[c], trDDa);
    trcdph = fma(w6[c] * ig[c], cdph[c], trcdph);
  }

  // ---- quadratic Christoffel part of the Ricci tensor -------------------------
  // Cm[k][i][m] = g~^lm G~^k_li ; Em[k][j][m] = g~^lm G~_klj
  double Cm[3][3][3], Em[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Cm[k][i][m] = ig[S6(0, m)] * Gu[k][S6(0, i)] + ig[S6(1, m)] * Gu[k][S6(1, i)] +
                      ig[S6(2, m)] * Gu[k][S6(2, i)];
        Em[k][i][m] = ig[S6(0, m)] * Gd[k][S6(0, i)] + ig[S6(1, m)] * Gd[k][S6(1, i)] +
                      ig[S6(2, m)] * Gd[k][S6(2, i)];
      }
  double X[3][3];  // X_ij = g~^lm G~^k_li G~_jkm
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) s = fma(Cm[k][i][m], Gd[j][S6(k, m)], s);
      X[i][j] = s;
    }

  // ---- R_ij + 2 nabla_(i Z_j) --------------------------------------------------
  double RZ[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      // -1/2 g~^kl d_k d_l g~_ij
      double lap = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = k; l < 3; ++l) lap = fma(w6[S6(k, l)] * ig[S6(k, l)], fdkl(N, GXX + c, k, l, C), lap);
      double t = -0.5 * lap;
      // g~_k(i d_j) Gamma-hat^k + 1/2 Gamma-hat^k d_k g~_ij
#pragma unroll
      for (int k = 0; k < 3; ++k)
        t += 0.5 * (g[S6(k, i)] * dG[j][k] + g[S6(k, j)] * dG[i][k] + Gh[k] * dg[k][c]);
      // g~^lm (G~^k_li G~_jkm + G~^k_lj G~_ikm + G~^k_im G~_klj)
      double q3 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) q3 = fma(Gu[k][S6(i, m)], Em[k][j][m], q3);
      t += X[i][j] + X[j][i] + q3;
      // conformal-factor terms
      t += iph * (cdph[c] + g[c] * trcdph) - 2.0 * iph * iph * g[c] * PP +
           iph * (2.0 * Zd[i] * dP[j] + 2.0 * Zd[j] * dP[i] - g[c] * dGP);
      RZ[c] = t;
    }
  double trRZ = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) trRZ = fma(w6[c] * ig[c], RZ[c], trRZ);
  const double RpZ = ph2 * trRZ;   // R + 2 nabla_k Z^k
  const double lapal = ph2 * trDDa; // nabla^i nabla_i alpha

  // ---- A~ contractions ------------------------------------------------------------
  double Am[3][3];  // A~_i^m = A~_il g~^lm
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m)
      Am[i][m] = A[S6(i, 0)] * ig[S6(0, m)] + A[S6(i, 1)] * ig[S6(1, m)] + A[S6(i, 2)] * ig[S6(2, m)];
  const double trA = Am[0][0] + Am[1][1] + Am[2][2];
  double Au[6], AgA[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      Au[S6(i, j)] = ig[S6(i, 0)] * Am[0][j] + ig[S6(i, 1)] * Am[1][j] + ig[S6(i, 2)] * Am[2][j];
      AgA[S6(i, j)] = Am[i][0] * A[S6(0, j)] + Am[i][1] * A[S6(1, j)] + Am[i][2] * A[S6(2, j)];
    }
  double AA = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) AA = fma(w6[c] * A[c], Au[c], AA);

  const double trB = dB[0][0] + dB[1][1] + dB[2][2];
  const double Kc = Kt - 2.0 * P.c * Th;  // K - 2 Theta c

  // ---- d_t g~_ij, d_t A~_ij -------------------------------------------------------------
  const double itau = 1.0 / P.tau;
  const double trMx = -trDDa + al * trRZ;  // g~^ij (-nabla_i nabla_j alpha + alpha RZ_ij)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      double advg = 0.0, lieg = 0.0, advA = 0.0, lieA = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        advg = fma(be[k], dg[k][c], advg);
        lieg += g[S6(k, i)] * dB[j][k] + g[S6(k, j)] * dB[i][k];
        advA = fma(be[k], dA[k][c], advA);
        lieA += A[S6(k, i)] * dB[j][k] + A[S6(k, j)] * dB[i][k];
      }
      r[GXX + c] = advg + lieg - (2.0 / 3.0) * g[c] * trB -
                   2.0 * al * (A[c] - (1.0 / 3.0) * g[c] * trA) - itau * (det - 1.0) * g[c];
      const double Mij = -DDa[c] + al * RZ[c];
      r[AXX + c] = advA + ph2 * (Mij - (1.0 / 3.0) * g[c] * trMx) + lieA -
                   (2.0 / 3.0) * A[c] * trB + al * A[c] * Kc - 2.0 * al * AgA[c];
    }

  // ---- scalars ---------------------------------------------------------------------------
  const double advK = be[0] * dK[0] + be[1] * dK[1] + be[2] * dK[2];
  const double advT = be[0] * dT[0] + be[1] * dT[1] + be[2] * dT[2];
  const double gK = (P.slicing == CCZ4_SLICING_ONE_PLUS_LOG) ? 2.0 * al : al * al;  // alpha^2 g(alpha)
  r[ALPHA] = be[0] * da[0] + be[1] * da[1] + be[2] * da[2] - gK * (Kt - P.K0 - 2.0 * P.c * Th);
  r[PHI] = be[0] * dP[0] + be[1] * dP[1] + be[2] * dP[2] + (1.0 / 3.0) * ph * (al * Kt - trB);
  r[KTR] = advK - lapal + al * RpZ + al * Kt * Kc - 3.0 * al * P.kappa1 * (1.0 + P.kappa2) * Th;
  const double ZA = 0.5 * ph2 * (dGam[0] * da[0] + dGam[1] * da[1] + dGam[2] * da[2]);  // Z^i A_i
  const double e2 = P.e * P.e;
  r[THETA] = advT + 0.5 * al * e2 * (RpZ + (2.0 / 3.0) * Kt * Kt - AA) - al * Th * Kt * P.c - ZA -
             al * P.kappa1 * (2.0 + P.kappa2) * Th;

  // ---- d_t Gamma-hat^i, gauge ----------------------------------------------------------------
  // d_k d_l beta^i contracted with g~^kl, and d_k (d_l beta^l)
  double lapB[3] = {0.0, 0.0, 0.0}, gdivB[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = k; l < 3; ++l) {
      const double w = w6[S6(k, l)] * ig[S6(k, l)];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double u = fdkl(N, BETAX + i, k, l, C);
        lapB[i] = fma(w, u, lapB[i]);
        if (i == l) gdivB[k] += u;        // d_k d_i beta^i
        if (i == k && k != l) gdivB[l] += u;
      }
    }
  double dbK[3];  // g~^ij d_j K etc. folded below
  const double s3 = P.s / 3.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double adv = 0.0, gT = 0.0, gKk = 0.0, gdv = 0.0, gA = 0.0, GB = 0.0, AuP = 0.0, AuA = 0.0, ZB = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      adv = fma(be[k], dG[k][i], adv);
      gT = fma(ig[S6(i, k)], dT[k], gT);
      gKk = fma(ig[S6(i, k)], dK[k], gKk);
      gdv = fma(ig[S6(i, k)], gdivB[k], gdv);
      gA = fma(ig[S6(i, k)], da[k], gA);
      GB = fma(Gc[k], dB[k][i], GB);
      AuP = fma(Au[S6(i, k)], dP[k], AuP);
      AuA = fma(Au[S6(i, k)], da[k], AuA);
      ZB = fma(dGam[k], dB[k][i], ZB);
    }
    double GA = 0.0;  // G~^i_jk A~^jk
#pragma unroll
    for (int c = 0; c < 6; ++c) GA = fma(w6[c] * Gu[i][c], Au[c], GA);
    const double Zc = 0.5 * dGam[i];  // g~^ij Z_j
    const double rG = adv + 2.0 * al * gT + lapB[i] + s3 * gdv - (4.0 / 3.0) * al * gKk +
                      (2.0 / 3.0) * Gc[i] * trB - GB + 2.0 * al * (GA - 3.0 * iph * AuP) -
                      2.0 * Th * gA - (4.0 / 3.0) * al * Kt * Zc - 2.0 * AuA -
                      2.0 * al * P.kappa1 * Zc +
                      2.0 * P.kappa3 * ((2.0 / 3.0) * Zc * trB - 0.5 * ZB);
    r[GHX + i] = rG;
    dbK[i] = rG - adv;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (P.shift == CCZ4_SHIFT_GAMMA_DRIVER) {
      r[BETAX + i] = be[0] * dB[0][i] + be[1] * dB[1][i] + be[2] * dB[2][i] + P.f * bb[i];
      r[BBX + i] = be[0] * db[0][i] + be[1] * db[1][i] + be[2] * db[2][i] + dbK[i] - P.eta * bb[i];
    } else {
      r[BETAX + i] = 0.0;
      r[BBX + i] = 0.0;
    }
  }
}

// Algebraic constraints after a time step (Sec. "Evolution equations"):
// rescale g~ by det(g~)^(-1/3) so that its determinant is one, then remove
// from A~ the trace taken with the rescaled metric.
__device__ __forceinline__ void enforce_point(double g[6], double A[6]) {
  const double det0 = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
                      g[2] * (g[1] * g[4] - g[3] * g[2]);
  const double sc = rcbrt(det0);
#pragma unroll
  for (int c = 0; c < 6; ++c) g[c] *= sc;
  double ig[6];
  ig[0] = g[3] * g[5] - g[4] * g[4];
  ig[1] = g[2] * g[4] - g[1] * g[5];
  ig[2] = g[1] * g[4] - g[2] * g[3];
  ig[3] = g[0] * g[5] - g[2] * g[2];
  ig[4] = g[1] * g[2] - g[0] * g[4];
  ig[5] = g[0] * g[3] - g[1] * g[1];
  const double det = g[0] * ig[0] + g[1] * ig[1] + g[2] * ig[2];
  const double tr = (ig[0] * A[0] + ig[3] * A[3] + ig[5] * A[5] +
                     2.0 * (ig[1] * A[1] + ig[2] * A[2] + ig[4] * A[4])) / det;
#pragma unroll
  for (int c = 0; c < 6; ++c) A[c] -= (1.0 / 3.0) * g[c] * tr;
}

}  // namespace ccz4
