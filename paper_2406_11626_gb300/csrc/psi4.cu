// psi_4 at every interior point (appendix "psi_4 in ExaGRyPE"): the
// electric and magnetic parts of the Weyl tensor in their Z4 form
// (Eqs. eq_NR_psi4_E_ij, eq_NR_psi4_B_ij, vacuum), contracted with mbar of
// the Gram-Schmidt tetrad (Eqs. eq_NR_psi4_m_conj,
// eq_NR_psi_code_implementation). A monitor, evaluated from the halo'd
// tiles of the halo fill in FP64 with the stage kernel's stencils; Re and Im
// go to fields 0 and 1 of a state-shaped buffer, where the particle tracers
// can sample them (the paper attaches psi_4 to the solution vector and
// interpolates it onto tracers arranged on a sphere).
//
// The physical Ricci tensor is taken through the conformal decomposition,
// R_ij = R~_ij + R^phi_ij, with R~_ij of the conformal metric alone (its
// contracted Christoffel symbol G~^k from the metric's derivatives) and
// R^phi_ij = (nabla~_i nabla~_j phi + g~_ij nabla~^l nabla~_l phi) / phi
//            - 2 g~_ij g~^kl d_k phi d_l phi / phi^2;
// Z_i = 1/2 g~_ij (Gamma-hat^j - G~^j) enters through D_(i Z_j).
#include "ccz4_algebra.cuh"
#include "ccz4_internal.cuh"

namespace ccz4 {
namespace {

struct Psi4Coef {
  StencilCoef<double> C[MAX_LEVELS];
};

__device__ __forceinline__ double eps3(int i, int j, int k) { return (double)((i - j) * (j - k) * (k - i)) * 0.5; }

__device__ void psi4_point(const Nbhd &N, const StencilCoef<double> &C, const double X[3], double out[2]) {
  // state and derivatives
  double g[3][3], A[3][3], dg[3][3][3], dA[3][3][3], ddg[3][3][3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int c = S6(i, j);
      g[i][j] = g[j][i] = N.at(GXX + c, 0);
      A[i][j] = A[j][i] = N.at(AXX + c, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dg[k][i][j] = dg[k][j][i] = fd1<double>(N, GXX + c, N.st[k], C.c1);
        dA[k][i][j] = dA[k][j][i] = fd1<double>(N, AXX + c, N.st[k], C.c1);
#pragma unroll
        for (int l = k; l < 3; ++l) {
          const double v = fdkl<double>(N, GXX + c, k, l, C);
          ddg[k][l][i][j] = ddg[k][l][j][i] = ddg[l][k][i][j] = ddg[l][k][j][i] = v;
        }
      }
    }
  const double ph = N.at(PHI, 0), Kt = N.at(KTR, 0), Th = N.at(THETA, 0);
  double dph[3], ddph[3][3], dKt[3], Gh[3], dGh[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dph[k] = fd1<double>(N, PHI, N.st[k], C.c1);
    dKt[k] = fd1<double>(N, KTR, N.st[k], C.c1);
    Gh[k] = N.at(GHX + k, 0);
#pragma unroll
    for (int l = 0; l < 3; ++l) dGh[l][k] = fd1<double>(N, GHX + k, N.st[l], C.c1);  // d_l Gamma-hat^k
#pragma unroll
    for (int l = k; l < 3; ++l) ddph[k][l] = ddph[l][k] = fdkl<double>(N, PHI, k, l, C);
  }
  // inverse conformal metric
  double ig[3][3];
  ig[0][0] = g[1][1] * g[2][2] - g[1][2] * g[1][2];
  ig[0][1] = g[0][2] * g[1][2] - g[0][1] * g[2][2];
  ig[0][2] = g[0][1] * g[1][2] - g[0][2] * g[1][1];
  ig[1][1] = g[0][0] * g[2][2] - g[0][2] * g[0][2];
  ig[1][2] = g[0][1] * g[0][2] - g[0][0] * g[1][2];
  ig[2][2] = g[0][0] * g[1][1] - g[0][1] * g[0][1];
  const double det = g[0][0] * ig[0][0] + g[0][1] * ig[0][1] + g[0][2] * ig[0][2];
  const double idet = 1.0 / det;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) ig[j][i] = (ig[i][j] *= idet);
  // conformal Christoffels: first kind Gd[k][i][j] = G~_kij, second kind Gu[k][i][j] = G~^k_ij
  double Gd[3][3][3], Gu[3][3][3], Gt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Gd[k][i][j] = 0.5 * (dg[i][j][k] + dg[j][i][k] - dg[k][i][j]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Gu[k][i][j] = ig[k][0] * Gd[0][i][j] + ig[k][1] * Gd[1][i][j] + ig[k][2] * Gd[2][i][j];
        t += ig[i][j] * Gu[k][i][j];
      }
    Gt[k] = t;
  }
  // d_l G~^k = d_l (g~^ij G~^k_ij), with d_l g~^ab = -g~^ac d_l g~_cd g~^db
  double dig[3][3][3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) s -= ig[a][c] * dg[l][c][d] * ig[d][b];
        dig[l][a][b] = s;
      }
  double dGt[3][3];  // dGt[l][k] = d_l G~^k
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          // d_l G~^k_ij = d_l g~^km G~_mij + g~^km d_l G~_mij
          double dG = 0.0;
#pragma unroll
          for (int m = 0; m < 3; ++m)
            dG += dig[l][k][m] * Gd[m][i][j] +
                  ig[k][m] * 0.5 * (ddg[l][i][j][m] + ddg[l][j][i][m] - ddg[l][m][i][j]);
          s += dig[l][i][j] * Gu[k][i][j] + ig[i][j] * dG;
        }
      dGt[l][k] = s;
    }
  // R~_ij = -1/2 g~^lm d_l d_m g~_ij + g~_k(i d_j) G~^k + G~^k G~_(ij)k
  //         + g~^lm (G~^k_li G~_jkm + G~^k_lj G~_ikm + G~^k_im G~_klj)
  // and the phi part; Ric[i][j] = R_ij (physical)
  double cdph[3][3], trcd = 0.0, PP = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      cdph[i][j] = ddph[i][j] - (Gu[0][i][j] * dph[0] + Gu[1][i][j] * dph[1] + Gu[2][i][j] * dph[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      trcd += ig[k][l] * cdph[k][l];
      PP += ig[k][l] * dph[k] * dph[l];
    }
  const double iph = 1.0 / ph;
  double Ric[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double r = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          r -= 0.5 * ig[l][m] * ddg[l][m][i][j];
#pragma unroll
          for (int k = 0; k < 3; ++k)
            r += ig[l][m] * (Gu[k][l][i] * Gd[j][k][m] + Gu[k][l][j] * Gd[i][k][m] + Gu[k][i][m] * Gd[k][l][j]);
        }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        r += 0.5 * (g[k][i] * dGt[j][k] + g[k][j] * dGt[i][k]);
        r += 0.5 * Gt[k] * (Gd[i][j][k] + Gd[j][i][k]);
      }
      r += (cdph[i][j] + g[i][j] * trcd) * iph - 2.0 * g[i][j] * PP * iph * iph;
      Ric[i][j] = Ric[j][i] = r;
    }
  // physical Christoffels Gamma^k_ij = G~^k_ij - (d^k_i d_j phi + d^k_j d_i phi - g~_ij g~^kl d_l phi) / phi
  double Pu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) Pu[k] = ig[k][0] * dph[0] + ig[k][1] * dph[1] + ig[k][2] * dph[2];
  double Gp[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Gp[k][i][j] = Gu[k][i][j] - ((k == i ? dph[j] : 0.0) + (k == j ? dph[i] : 0.0) - g[i][j] * Pu[k]) * iph;
  // Z_i = 1/2 g~_ij (Gamma-hat^j - G~^j) and D_(i Z_j)
  double Z[3], dZ[3][3];  // dZ[k][i] = d_k Z_i
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) s += 0.5 * g[i][j] * (Gh[j] - Gt[j]);
    Z[i] = s;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) s += 0.5 * (dg[k][i][j] * (Gh[j] - Gt[j]) + g[i][j] * (dGh[k][j] - dGt[k][j]));
      dZ[k][i] = s;
    }
  // extrinsic curvature: covariant K_ij = (A~_ij + g~_ij K / 3) / phi^2, mixed K^n_j = g~^nk A~_kj + d^n_j K / 3
  double Kd[3][3], Km[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Kd[i][j] = (A[i][j] + g[i][j] * Kt * (1.0 / 3.0)) * iph * iph;
      Km[i][j] = ig[i][0] * A[0][j] + ig[i][1] * A[1][j] + ig[i][2] * A[2][j] + (i == j ? Kt * (1.0 / 3.0) : 0.0);
    }
  // E_ij = R_ij - K_im K^m_j + K_ij (K - Theta) + D_(i Z_j)
  double E[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = Ric[i][j] + Kd[i][j] * (Kt - Th) + 0.5 * (dZ[i][j] + dZ[j][i]);
#pragma unroll
      for (int m = 0; m < 3; ++m) s -= Kd[i][m] * Km[m][j] + Gp[m][i][j] * Z[m];
      E[i][j] = s;
    }
  // D_l K^n_j = d_l K^n_j + Gamma^n_lp K^p_j - Gamma^p_lj K^n_p, raised with gamma^ml = phi^2 g~^ml
  double DK[3][3][3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double s = n == j ? dKt[l] * (1.0 / 3.0) : 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) s += dig[l][n][k] * A[k][j] + ig[n][k] * dA[l][k][j];
#pragma unroll
        for (int q = 0; q < 3; ++q) s += Gp[n][l][q] * Km[q][j] - Gp[q][l][j] * Km[n][q];
        DK[l][n][j] = s;
      }
  const double sdet = sqrt(det) * iph * iph * iph;  // sqrt(det gamma), gamma = g~ / phi^2
  double B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          if (m == n) continue;
          double um_j = 0.0, um_i = 0.0;  // D^m K^n_j, D^m K^n_i
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            um_j += ig[m][l] * DK[l][n][j];
            um_i += ig[m][l] * DK[l][n][i];
          }
          s += eps3(m, n, i) * um_j + eps3(m, n, j) * um_i;
        }
      B[i][j] = 0.5 * sdet * ph * ph * s;
    }
  // trace-free parts with the physical metric (gamma_ij gamma^kl = g~_ij g~^kl)
  double trE = 0.0, trB = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      trE += ig[i][j] * E[i][j];
      trB += ig[i][j] * B[i][j];
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      E[i][j] -= g[i][j] * trE * (1.0 / 3.0);
      B[i][j] -= g[i][j] * trB * (1.0 / 3.0);
    }
  // the tetrad: Gram-Schmidt of v = (-y, x, 0), u = (x, y, z), w = gamma^-1 eps(v, u) with gamma = g~ / phi^2
  const double i2 = iph * iph;
  auto dot = [&](const double a[3], const double b[3]) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) s += g[i][j] * a[i] * b[j];
    return s * i2;
  };
  double v[3] = {-X[1], X[0], 0.0}, u[3] = {X[0], X[1], X[2]}, w[3];
  double nrm = rsqrt(dot(v, v));
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] *= nrm;
  const double vu = dot(v, u);
#pragma unroll
  for (int i = 0; i < 3; ++i) u[i] -= vu * v[i];
  nrm = rsqrt(dot(u, u));
#pragma unroll
  for (int i = 0; i < 3; ++i) u[i] *= nrm;
  const double c[3] = {sdet * (v[1] * u[2] - v[2] * u[1]), sdet * (v[2] * u[0] - v[0] * u[2]),
                       sdet * (v[0] * u[1] - v[1] * u[0])};  // eps_jkl v^k u^l
#pragma unroll
  for (int i = 0; i < 3; ++i) w[i] = ph * ph * (ig[i][0] * c[0] + ig[i][1] * c[1] + ig[i][2] * c[2]);
  const double vw = dot(v, w), uw = dot(u, w);
#pragma unroll
  for (int i = 0; i < 3; ++i) w[i] -= vw * v[i] + uw * u[i];
  nrm = rsqrt(dot(w, w));
#pragma unroll
  for (int i = 0; i < 3; ++i) w[i] *= nrm;
  double Eww = 0.0, Evv = 0.0, Ewv = 0.0, Bww = 0.0, Bvv = 0.0, Bwv = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Eww += E[i][j] * w[i] * w[j];
      Evv += E[i][j] * v[i] * v[j];
      Ewv += E[i][j] * w[i] * v[j];
      Bww += B[i][j] * w[i] * w[j];
      Bvv += B[i][j] * v[i] * v[j];
      Bwv += B[i][j] * w[i] * v[j];
    }
  // (E - i B)_ij mbar^i mbar^j, mbar = (w - i v) / sqrt 2
  out[0] = 0.5 * (Eww - Evv) - Bwv;
  out[1] = -Ewv - 0.5 * (Bww - Bvv);
}

__global__ void __launch_bounds__(128) psi4_kernel(GridView g, Psi4Coef PC, const double *__restrict__ tile,
                                                   double cx, double cy, double cz, double *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n_points) return;
  const int p = g.p, T = g.T;
  const int p3 = p * p * p;
  const int n = (int)i / p3;
  const int r = (int)i - n * p3;
  const int z = r / (p * p), y = (r / p) % p, x = r % p;
  Nbhd N;
  N.c = tile + n * g.T3 + ((long long)(z + HALO) * T + (y + HALO)) * T + (x + HALO);
  N.fs = (long long)g.n_patches * g.T3;
  N.st[0] = 1;
  N.st[1] = T;
  N.st[2] = T * T;
  N.mix = nullptr;
  N.ms = 0;
  N.mixf = nullptr;
  N.msf = 0;
  const int lev = patch_level(g, n);
  const double h = g.ldx[lev];
  const double X[3] = {g.origin[0] + (__ldg(g.ijk + 3 * n) * p + x + 0.5) * h - cx,
                       g.origin[1] + (__ldg(g.ijk + 3 * n + 1) * p + y + 0.5) * h - cy,
                       g.origin[2] + (__ldg(g.ijk + 3 * n + 2) * p + z + 0.5) * h - cz};
  double v[2];
  psi4_point(N, PC.C[lev], X, v);
  out[i] = v[0];
  out[g.S + i] = v[1];
}

}  // namespace

cudaError_t launch_psi4(const GridView &g, const double *tile, const double centre[3], double *out, cudaStream_t s) {
  if (g.n_points == 0) return cudaSuccess;
  Psi4Coef PC;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    const double dx = g.ldx[l];
    PC.C[l].c1 = 1.0 / (12.0 * dx);
    PC.C[l].c2 = 1.0 / (12.0 * dx * dx);
    PC.C[l].c3 = 1.0 / (144.0 * dx * dx);
    PC.C[l].cko = 0.0;
  }
  psi4_kernel<<<(unsigned)((g.n_points + 127) / 128), 128, 0, s>>>(g, PC, tile, centre[0], centre[1], centre[2],
                                                                    out);
  return cudaGetLastError();
}

}  // namespace ccz4
