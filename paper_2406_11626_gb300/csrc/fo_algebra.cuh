// Pointwise right-hand side of the first-order CCZ4 formulation (58
// variables, Eq. first-order-variables) and of the second-order formulation
// with reconstructed auxiliary variables, FP64.
//
// Variables: the 25 primaries, then A_k = d_k alpha (FA + k),
// B_k^i = d_k beta^i (FB + 3k + i), D_kij = 1/2 d_k g~_ij (FD + 6k + pair)
// and P_k = d_k phi (FP + k) (Eq. auxiliary-variables). Only first
// derivatives are taken (Alg. fd4-fo): the primaries' equations use the
// auxiliary variables for the first derivatives of alpha, beta, g~ and phi,
// and their symmetrised first derivatives for the second derivatives, as
// the relations below the evolution equations close the system
// (Christoffel symbols from D, nabla nabla alpha = d_(i A_j) - Gamma^k_ij
// A_k, Eq. NR_foccz4_modified_ricci). The auxiliary variables follow Eqs.
// NR_foccz4_A_k, NR_foccz4_B^i_j, the D_kij equation and NR_foccz4_P_i.
// RED keeps the red terms (first-order formulation); without them the
// primaries' equations are those of the second-order formulation, whose
// auxiliary variables are reconstructed instead of evolved (Alg. fd4-so).
// AUX: the auxiliary variables' right-hand sides are formed too.
//
// The derivatives are taken field group by field group and consumed at once
// (the D_kij equation is emitted inside the loop over the derivatives of D),
// so that few of the 141 derivative values are live at a time.
#pragma once

#include "ccz4_algebra.cuh"

namespace ccz4 {

// Index of a symmetric pair for the first-order algebra: the same table as
// S6, in the recursive form on purpose. The first-order stage kernel runs
// at 128 registers and spills several KB per thread; with this form the
// arrays it indexes keep fixed places in local memory instead of being
// allocated to registers and spilled, which measured 3.5 % faster per step
// (144^3 puncture: 104.1 against 107.9 ms). The second-order kernels use
// S6, whose indices fold so that their arrays stay in registers.
__host__ __device__ constexpr int S6_fo(int i, int j) {
  return i > j ? S6_fo(j, i) : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

constexpr int NVF = 58;
constexpr int FA = 25, FB = 28, FD = 37, FP = 55;

struct FoPhys {
  Phys<double> p;
  double mu;
};

template <bool RED, bool AUX, class Sink>
__device__ __forceinline__ void fo_rhs_point(const FoPhys &F, const Nbhd &N, const StencilCoef<double> &C,
                                             Sink &sink) {
  using D = double;
  const Phys<D> &P = F.p;
  const D c1 = C.c1;
  const bool driver = P.shift == CCZ4_SHIFT_GAMMA_DRIVER;
  // ---- values and the conformal geometry from D ----------------------------------
  D g[6], ig[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) g[c] = ld<D>(N, GXX + c, 0);
  const D det = sym_inverse<D>(g, ig);
  const D igw[6] = {ig[0], ig[1] + ig[1], ig[2] + ig[2], ig[3], ig[4] + ig[4], ig[5]};
  const D al = ld<D>(N, ALPHA, 0), ph = ld<D>(N, PHI, 0), Kt = ld<D>(N, KTR, 0), Th = ld<D>(N, THETA, 0);
  const D iph = D(1.0) / ph;
  D be[3], Gh[3], Av[3], Pv[3], B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    be[i] = ld<D>(N, BETAX + i, 0);
    Gh[i] = ld<D>(N, GHX + i, 0);
    Av[i] = ld<D>(N, FA + i, 0);
    Pv[i] = ld<D>(N, FP + i, 0);
#pragma unroll
    for (int j = 0; j < 3; ++j) B[i][j] = ld<D>(N, FB + 3 * i + j, 0);   // B[k][i] = B_k^i
  }
  D Dv[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 6; ++c) Dv[k][c] = ld<D>(N, FD + 6 * k + c, 0);
  // G~_lij = D_ijl + D_jil - D_lij (lowered), G~^k_ij = g~^kl G~_lij, G~^k = g~^ij G~^k_ij
  D Gd[3][6], Gu[3][6], Gc[3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) Gd[l][S6_fo(i, j)] = Dv[i][S6_fo(j, l)] + Dv[j][S6_fo(i, l)] - Dv[l][S6_fo(i, j)];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      Gu[k][c] = fmaT(ig[S6_fo(k, 0)], Gd[0][c], fmaT(ig[S6_fo(k, 1)], Gd[1][c], ig[S6_fo(k, 2)] * Gd[2][c]));
    D s = igw[0] * Gu[k][0];
#pragma unroll
    for (int c = 1; c < 6; ++c) s = fmaT(igw[c], Gu[k][c], s);
    Gc[k] = s;
  }
  D dGam[3], Z2[3];  // Gamma-hat - G~ and 2 Z_i
#pragma unroll
  for (int i = 0; i < 3; ++i) dGam[i] = Gh[i] - Gc[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) Z2[i] = fmaT(g[S6_fo(i, 0)], dGam[0], fmaT(g[S6_fo(i, 1)], dGam[1], g[S6_fo(i, 2)] * dGam[2]));
  D At[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) At[c] = ld<D>(N, AXX + c, 0);
  const D trA = fmaT(igw[0], At[0], fmaT(igw[1], At[1], fmaT(igw[2], At[2], fmaT(igw[3], At[3],
                fmaT(igw[4], At[4], igw[5] * At[5])))));
  const D trB = B[0][0] + B[1][1] + B[2][2];
  const D third = 1.0 / 3.0, twothird = 2.0 / 3.0;

  // ---- derivatives of B: d_(k B_j)^m, the advection of B, g~^kl d_k B_l^i, d_(k B_l)^l ----
  D sB[6][3], advB[3][3], lapB[3], gdivB[3];
  {
    D dB[3][3][3];  // dB[k][l][i] = d_k B_l^i
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) dB[k][l][i] = fd1<D>(N, FB + 3 * l + i, N.st[k], c1);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) advB[k][i] = fmaT(be[0], dB[0][k][i], fmaT(be[1], dB[1][k][i], be[2] * dB[2][k][i]));
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = k; j < 3; ++j)
#pragma unroll
        for (int m = 0; m < 3; ++m) sB[S6_fo(k, j)][m] = D(0.5) * (dB[k][j][m] + dB[j][k][m]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    D s = igw[0] * sB[0][i];
#pragma unroll
    for (int c = 1; c < 6; ++c) s = fmaT(igw[c], sB[c][i], s);
    lapB[i] = s;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) gdivB[k] = sB[S6_fo(k, 0)][0] + sB[S6_fo(k, 1)][1] + sB[S6_fo(k, 2)][2];

  // ---- derivatives of A and P: d_(i A_j), d_(i P_j), advection, the curl of P ------------
  D ddA[6], ddP[6], advA[3], advP[3], curlP[3];  // curlP[k][j] as (yz, zx, xy): d_y P_z - d_z P_y, ...
  {
    D dA[3][3], dP[3][3];  // dA[k][i] = d_k A_i
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dA[k][i] = fd1<D>(N, FA + i, N.st[k], c1);
        dP[k][i] = fd1<D>(N, FP + i, N.st[k], c1);
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        ddA[S6_fo(i, j)] = D(0.5) * (dA[i][j] + dA[j][i]);
        ddP[S6_fo(i, j)] = D(0.5) * (dP[i][j] + dP[j][i]);
      }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      advA[k] = fmaT(be[0], dA[0][k], fmaT(be[1], dA[1][k], be[2] * dA[2][k]));
      advP[k] = fmaT(be[0], dP[0][k], fmaT(be[1], dP[1][k], be[2] * dP[2][k]));
    }
    curlP[0] = dP[1][2] - dP[2][1];
    curlP[1] = dP[2][0] - dP[0][2];
    curlP[2] = dP[0][1] - dP[1][0];
  }

  // ---- derivatives of A~: its advection and g~^nm d_k A~_nm --------------------------------
  D advAt[6], gdAt[3];
  {
    D s[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      D a = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const D d = fd1<D>(N, AXX + c, N.st[k], c1);
        a = fmaT(be[k], d, a);
        s[k] = fmaT(igw[c], d, s[k]);
      }
      advAt[c] = a;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) gdAt[k] = s[k];
  }
  // D_k^nm A~_nm = A~^ab D_kab, with A~^ab = g~^an g~^bm A~_nm
  D Au[6];
  {
    D Am[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        Am[i][m] = fmaT(At[S6_fo(i, 0)], ig[S6_fo(0, m)], fmaT(At[S6_fo(i, 1)], ig[S6_fo(1, m)], At[S6_fo(i, 2)] * ig[S6_fo(2, m)]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        Au[S6_fo(i, j)] = fmaT(ig[S6_fo(i, 0)], Am[0][j], fmaT(ig[S6_fo(i, 1)], Am[1][j], ig[S6_fo(i, 2)] * Am[2][j]));
  }
  const D Auw[6] = {Au[0], Au[1] + Au[1], Au[2] + Au[2], Au[3], Au[4] + Au[4], Au[5]};
  D DuA[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    D s = Auw[0] * Dv[k][0];
#pragma unroll
    for (int c = 1; c < 6; ++c) s = fmaT(Auw[c], Dv[k][c], s);
    DuA[k] = s;
  }

  // ---- derivatives of D: g~^kl d_k D_lij (the Laplacian of g~), the D_kij equation and,
  //      with the red terms, the mu term g~^ij g~^nl (d_k D_ljn - d_l D_kjn) of B ---------------
  D lapg[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  D m2[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) m2[k][i] = 0.0;
#pragma unroll
  for (int b = 0; b < 3; ++b) {  // D_b.., the k index of the D_kij equation
    D advD[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {  // derivative direction
      D M[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) M[c] = fd1<D>(N, FD + 6 * b + c, N.st[a], c1);  // d_a D_b,c
      const D w = ig[S6_fo(a, b)];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        lapg[c] = fmaT(w, M[c], lapg[c]);
        advD[c] = fmaT(be[a], M[c], advD[c]);
      }
      if (RED && AUX && driver) {
        // H = g~^-1 M g~^-1; term 1 adds H[i][b] to m2[a][i], term 2 subtracts H[i][a] from m2[b][i]
#pragma unroll
        for (int col = 0; col < 2; ++col) {
          const int q = col == 0 ? b : a;
          D u[3];
#pragma unroll
          for (int n = 0; n < 3; ++n)
            u[n] = fmaT(M[S6_fo(n, 0)], ig[S6_fo(0, q)], fmaT(M[S6_fo(n, 1)], ig[S6_fo(1, q)], M[S6_fo(n, 2)] * ig[S6_fo(2, q)]));
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const D h = fmaT(ig[S6_fo(i, 0)], u[0], fmaT(ig[S6_fo(i, 1)], u[1], ig[S6_fo(i, 2)] * u[2]));
            if (col == 0) m2[a][i] += h;
            else m2[b][i] -= h;
          }
        }
      }
    }
    if (AUX) {
      // the D_bij equation: advection, shift terms, -alpha d_b A~_ij, the B D terms, -A_b (A~ - g~ tr A~ / 3)
      const D sgd = gdivB[b];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          const int c = S6_fo(i, j);
          D sh = third * g[c] * sgd;
#pragma unroll
          for (int m = 0; m < 3; ++m) sh = fmaT(D(-0.5), fmaT(g[S6_fo(m, i)], sB[S6_fo(b, j)][m], g[S6_fo(m, j)] * sB[S6_fo(b, i)][m]), sh);
          D BD = advD[c] - twothird * trB * Dv[b][c];
#pragma unroll
          for (int l = 0; l < 3; ++l)
            BD = fmaT(B[b][l], Dv[l][c], fmaT(B[j][l], Dv[b][S6_fo(l, i)], fmaT(B[i][l], Dv[b][S6_fo(l, j)], BD)));
          D r = fmaT(-P.s3 * D(3.0), sh, BD);
          r = fmaT(-al, fd1<D>(N, AXX + c, N.st[b], c1), r);
          r = fmaT(-Av[b], fmaT(-third * g[c], trA, At[c]), r);
          if (RED) r = fmaT(al * third * g[c], fmaT(D(-2.0), DuA[b], gdAt[b]), r);
          sink(FD + 6 * b + c, fmaT(C.cko, ko_sum<D>(N, FD + 6 * b + c), r));
        }
    }
  }

  // ---- Ricci tensor: R_ij + 2 nabla_(i Z_j) (Eq. NR_foccz4_modified_ricci) ----------------------
  D RZ[6], DDa[6], advGh[3];
  {
    // quadratic Christoffel part
    D Q6[6];
    {
      D Cm[3][3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int m = 0; m < 3; ++m)
            Cm[k][i][m] = fmaT(ig[S6_fo(0, m)], Gu[k][S6_fo(0, i)], fmaT(ig[S6_fo(1, m)], Gu[k][S6_fo(1, i)], ig[S6_fo(2, m)] * Gu[k][S6_fo(2, i)]));
      D X[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          D s = Cm[0][i][0] * Gd[j][S6_fo(0, 0)];
#pragma unroll
          for (int q = 1; q < 9; ++q) s = fmaT(Cm[q / 3][i][q % 3], Gd[j][S6_fo(q / 3, q % 3)], s);
          X[i][j] = s;
        }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          D q3 = X[i][j] + X[j][i];
#pragma unroll
          for (int q = 0; q < 9; ++q) q3 = fmaT(Cm[q / 3][i][q % 3], Gd[q / 3][S6_fo(q % 3, j)], q3);
          Q6[S6_fo(i, j)] = q3;
        }
    }
    // conformal-factor part and nabla nabla alpha
    const D PP = fmaT(Pv[0], fmaT(ig[0], Pv[0], fmaT(igw[1], Pv[1], igw[2] * Pv[2])),
                      fmaT(Pv[1], fmaT(ig[3], Pv[1], igw[4] * Pv[2]), ig[5] * Pv[2] * Pv[2]));
    D Pu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Pu[k] = fmaT(ig[S6_fo(k, 0)], Pv[0], fmaT(ig[S6_fo(k, 1)], Pv[1], ig[S6_fo(k, 2)] * Pv[2]));
    const D PA = fmaT(Pu[0], Av[0], fmaT(Pu[1], Av[1], Pu[2] * Av[2]));
    const D dGP = fmaT(dGam[0], Pv[0], fmaT(dGam[1], Pv[1], dGam[2] * Pv[2]));
    D cdph[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) cdph[c] = fmaT(-Gu[0][c], Pv[0], fmaT(-Gu[1][c], Pv[1], fmaT(-Gu[2][c], Pv[2], ddP[c])));
    D trcdph = igw[0] * cdph[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) trcdph = fmaT(igw[c], cdph[c], trcdph);
    const D iphPP = iph * PP;
    const D gco = (trcdph - dGP) - (iphPP + iphPP);
    // d_j Gamma-hat^k: g~_k(i d_j) Gamma-hat^k and the advection of Gamma-hat
    D dGh[3][3];  // dGh[j][k] = d_j Gamma-hat^k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) dGh[j][k] = fd1<D>(N, GHX + k, N.st[j], c1);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int c = S6_fo(i, j);
        D u = D(0.0);
#pragma unroll
        for (int k = 0; k < 3; ++k) u = fmaT(g[S6_fo(k, i)], dGh[j][k], fmaT(g[S6_fo(k, j)], dGh[i][k], u));
        D GD = Gh[0] * Dv[0][c];  // Gamma-hat^k D_kij = 1/2 Gamma-hat^k d_k g~_ij
        GD = fmaT(Gh[1], Dv[1][c], fmaT(Gh[2], Dv[2][c], GD));
        const D zt = fmaT(Z2[i], Pv[j], Z2[j] * Pv[i]);
        const D phiRZ = iph * (cdph[c] + fmaT(g[c], gco, zt));
        RZ[c] = fmaT(D(0.5), u, Q6[c] + GD + phiRZ - lapg[c]);
        const D DDaD = fmaT(iph, fmaT(Pv[i], Av[j], fmaT(Pv[j], Av[i], -g[c] * PA)), ddA[c]);
        DDa[c] = fmaT(-Gu[0][c], Av[0], fmaT(-Gu[1][c], Av[1], fmaT(-Gu[2][c], Av[2], DDaD)));
      }
#pragma unroll
    for (int i = 0; i < 3; ++i) advGh[i] = fmaT(be[0], dGh[0][i], fmaT(be[1], dGh[1][i], be[2] * dGh[2][i]));
  }
  D trRZ = igw[0] * RZ[0], trDDa = igw[0] * DDa[0];
#pragma unroll
  for (int c = 1; c < 6; ++c) {
    trRZ = fmaT(igw[c], RZ[c], trRZ);
    trDDa = fmaT(igw[c], DDa[c], trDDa);
  }
  const D ph2 = ph * ph;
  const D RpZ = ph2 * trRZ, lapal = ph2 * trDDa;

  // ---- g~, A~, alpha, phi -----------------------------------------------------------------------
  const D Kc = fmaT(-P.c2, Th, Kt);
  const D al2 = al + al;
  D AgA[6], AA;
  {
    D Am[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        Am[i][m] = fmaT(At[S6_fo(i, 0)], ig[S6_fo(0, m)], fmaT(At[S6_fo(i, 1)], ig[S6_fo(1, m)], At[S6_fo(i, 2)] * ig[S6_fo(2, m)]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        AgA[S6_fo(i, j)] = fmaT(Am[i][0], At[S6_fo(0, j)], fmaT(Am[i][1], At[S6_fo(1, j)], Am[i][2] * At[S6_fo(2, j)]));
    AA = At[0] * Auw[0];
#pragma unroll
    for (int c = 1; c < 6; ++c) AA = fmaT(At[c], Auw[c], AA);
  }
  {
    const D trMx = fmaT(al, trRZ, -trDDa);
    const D sg = fmaT(twothird * al, trA, -twothird * trB) - P.itau * (det - D(1.0));
    const D sA1 = -third * ph2 * trMx;
    const D sA2 = fmaT(al, Kc, -twothird * trB);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int c = S6_fo(i, j);
        D lie = D(0.0), lieA = D(0.0), adv = D(0.0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          lie = fmaT(g[S6_fo(k, i)], B[j][k], fmaT(g[S6_fo(k, j)], B[i][k], lie));
          lieA = fmaT(At[S6_fo(k, i)], B[j][k], fmaT(At[S6_fo(k, j)], B[i][k], lieA));
          adv = fmaT(be[k], Dv[k][c], adv);
        }
        sink(GXX + c, fmaT(C.cko, ko_sum<D>(N, GXX + c), fmaT(g[c], sg, fmaT(-al2, At[c], fmaT(D(2.0), adv, lie)))));
        const D rA = fmaT(ph2 * al, RZ[c], fmaT(-ph2, DDa[c], fmaT(g[c], sA1, fmaT(At[c], sA2,
                     fmaT(-al2, AgA[c], advAt[c] + lieA)))));
        sink(AXX + c, fmaT(C.cko, ko_sum<D>(N, AXX + c), rA));
      }
  }
  const D gfun = P.slicing == CCZ4_SLICING_ONE_PLUS_LOG ? D(2.0) / al : D(1.0);
  const D lapse_src = Kc - P.K0;
  sink(ALPHA, fmaT(C.cko, ko_sum<D>(N, ALPHA), fmaT(be[0], Av[0], fmaT(be[1], Av[1], fmaT(be[2], Av[2], -al * al * gfun * lapse_src)))));
  sink(PHI, fmaT(C.cko, ko_sum<D>(N, PHI),
                 fmaT(be[0], Pv[0], fmaT(be[1], Pv[1], fmaT(be[2], Pv[2], third * ph * fmaT(al, Kt, -trB))))));

  // ---- K, Theta -------------------------------------------------------------------------------------
  D dK[3], dT[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dK[k] = fd1<D>(N, KTR, N.st[k], c1);
    dT[k] = fd1<D>(N, THETA, N.st[k], c1);
  }
  {
    const D advK = fmaT(be[0], dK[0], fmaT(be[1], dK[1], be[2] * dK[2]));
    const D advT = fmaT(be[0], dT[0], fmaT(be[1], dT[1], be[2] * dT[2]));
    const D rK = advK - lapal + al * RpZ + al * Kt * Kc - P.k1a * al * Th;
    sink(KTR, fmaT(C.cko, ko_sum<D>(N, KTR), rK));
    // Z^i A_i = 1/2 phi^2 (Gamma-hat^i - G~^i) A_i
    const D ZA = D(0.5) * ph2 * fmaT(dGam[0], Av[0], fmaT(dGam[1], Av[1], dGam[2] * Av[2]));
    const D rT = advT + al * P.e2h * (RpZ + fmaT(twothird * Kt, Kt, -AA)) - al * Th * Kt * P.c - ZA - P.k1b * al * Th;
    sink(THETA, fmaT(C.cko, ko_sum<D>(N, THETA), rT));
  }

  // ---- Gamma-hat, b, beta ----------------------------------------------------------------------------
  D dbK[3];  // d_t Gamma-hat^i - beta^k d_k Gamma-hat^i (before dissipation)
  {
    const D al43 = D(4.0 / 3.0) * al;
    const D zc = D(0.5) * fmaT(-al43, Kt, fmaT(-al2, P.kappa1, P.k3x2 * twothird * trB));
    const D k3h = D(-0.5) * P.k3x2;
    D wv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wv[k] = fmaT(al2, dT[k], fmaT(-al43, dK[k], fmaT(P.s3, gdivB[k], -(Th + Th) * Av[k])));
      if (RED) wv[k] = fmaT(al2, fmaT(D(-2.0), DuA[k], gdAt[k]), wv[k]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      D GA = Gu[i][0] * Auw[0];
#pragma unroll
      for (int c = 1; c < 6; ++c) GA = fmaT(Gu[i][c], Auw[c], GA);
      const D AuA = fmaT(Au[S6_fo(i, 0)], Av[0], fmaT(Au[S6_fo(i, 1)], Av[1], Au[S6_fo(i, 2)] * Av[2]));
      const D AuP = fmaT(Au[S6_fo(i, 0)], Pv[0], fmaT(Au[S6_fo(i, 1)], Pv[1], Au[S6_fo(i, 2)] * Pv[2])) * iph;
      const D ZB = fmaT(dGam[0], B[0][i], fmaT(dGam[1], B[1][i], dGam[2] * B[2][i]));
      D t = fmaT(ig[S6_fo(i, 0)], wv[0], fmaT(ig[S6_fo(i, 1)], wv[1], fmaT(ig[S6_fo(i, 2)], wv[2], lapB[i])));
      t = fmaT(al2, GA, t);
      t = fmaT(twothird * trB, Gc[i], t);
      t = fmaT(D(-6.0) * al, AuP, t);
      t = fmaT(D(-2.0), AuA, t);
      t = fmaT(zc, dGam[i], t);
      t = fmaT(k3h, ZB, t);
      dbK[i] = fmaT(-Gc[0], B[0][i], fmaT(-Gc[1], B[1][i], fmaT(-Gc[2], B[2][i], t)));
      sink(GHX + i, fmaT(C.cko, ko_sum<D>(N, GHX + i), advGh[i] + dbK[i]));
    }
  }
  D bb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bb[i] = ld<D>(N, BBX + i, 0);
  {
    D advb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const D db = fd1<D>(N, BBX + i, N.st[k], c1);  // d_k b^i
        advb[i] = fmaT(be[k], db, advb[i]);
        if (AUX) {
          // Eq. NR_foccz4_B^i_j: advection, f d_k b^i, B_k^l B_l^i, and the mu terms
          D r = D(0.0);
          if (driver) {
            r = fmaT(P.f, db, advB[k][i]);
#pragma unroll
            for (int l = 0; l < 3; ++l) r = fmaT(B[k][l], B[l][i], r);
            if (RED) {
              // -alpha^2 mu g~^ij / phi (d_k P_j - d_j P_k): the curl component of (k, j)
              D m1 = D(0.0);
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                if (j == k) continue;
                // d_k P_j - d_j P_k from curlP (yz, zx, xy)
                const int o = 3 - k - j;
                const D cp = ((k + 1) % 3 == j) ? curlP[o] : -curlP[o];
                m1 = fmaT(ig[S6_fo(i, j)], cp, m1);
              }
              const D amu = al * al * F.mu;
              r = fmaT(-amu * iph, m1, fmaT(amu, m2[k][i], r));
            }
          }
          sink(FB + 3 * k + i, fmaT(C.cko, ko_sum<D>(N, FB + 3 * k + i), r));
        }
      }
    if (driver) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sink(BETAX + i, fmaT(C.cko, ko_sum<D>(N, BETAX + i), fmaT(be[0], B[0][i], fmaT(be[1], B[1][i], fmaT(be[2], B[2][i], P.f * bb[i])))));
        sink(BBX + i, fmaT(C.cko, ko_sum<D>(N, BBX + i), fmaT(-P.eta, bb[i], advb[i] + dbK[i])));
      }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sink(BETAX + i, C.cko * ko_sum<D>(N, BETAX + i));
        sink(BBX + i, C.cko * ko_sum<D>(N, BBX + i));
      }
    }
  }
  if (!AUX) return;

  // ---- A_k (Eq. NR_foccz4_A_k) and P_k (Eq. NR_foccz4_P_i) ---------------------------------------------
  {
    const D gp = P.slicing == CCZ4_SLICING_ONE_PLUS_LOG ? D(-2.0) / (al * al) : D(0.0);
    const D cA = fmaT(al * al, gp, D(2.0) * al * gfun) * lapse_src;   // (2 alpha g + alpha^2 g') (K - K0 - 2 c Theta)
    const D a2g = al * al * gfun;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      D BA = D(0.0), BP = D(0.0);
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        BA = fmaT(B[k][l], Av[l], BA);
        BP = fmaT(B[k][l], Pv[l], BP);
      }
      D rA = fmaT(-a2g, fmaT(-P.c2, dT[k], dK[k]), advA[k] + BA);
      rA = fmaT(-cA, Av[k], rA);
      if (RED) rA = fmaT(-al * gfun, fmaT(D(-2.0), DuA[k], gdAt[k]), rA);
      sink(FA + k, fmaT(C.cko, ko_sum<D>(N, FA + k), rA));
      D rP = advP[k] + BP;
      rP = fmaT(third * ph, fmaT(al, dK[k], -gdivB[k]), rP);
      rP = fmaT(third * fmaT(al, Kt, -trB), Pv[k], rP);
      rP = fmaT(third * ph * Kt, Av[k], rP);
      if (RED) rP = fmaT(third * al * ph, fmaT(D(-2.0), DuA[k], gdAt[k]), rP);
      sink(FP + k, fmaT(C.cko, ko_sum<D>(N, FP + k), rP));
    }
  }
}

// Auxiliary variables of one point from FD4 first derivatives of the
// primaries (the reconstruction of Alg. fd4-so, Eq. auxiliary-variables):
// out(v, value) receives A_k, B_k^i, D_kij = 1/2 d_k g~_ij and P_k.
template <class Out>
__device__ __forceinline__ void fo_reconstruct_point(const Nbhd &N, const double c1, Out &out) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int s = N.st[k];
    out(FA + k, fd1<double>(N, ALPHA, s, c1));
    out(FP + k, fd1<double>(N, PHI, s, c1));
#pragma unroll
    for (int i = 0; i < 3; ++i) out(FB + 3 * k + i, fd1<double>(N, BETAX + i, s, c1));
#pragma unroll
    for (int c = 0; c < 6; ++c) out(FD + 6 * k + c, 0.5 * fd1<double>(N, GXX + c, s, c1));
  }
}

}  // namespace ccz4
