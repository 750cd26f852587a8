// Test support: the stage kernel's pointwise templates (ccz4_algebra.cuh)
// evaluated on the host, so that their FP64 and mixed-precision right-hand
// sides can be compared with the oracle on a machine without a GPU. Built by
// tests/test_host_rhs.py with nvcc into a temporary directory.
//
// Inputs: halo'd FP64 tiles [25][n_patches][(p+6)^3] (the oracle's fill),
// patch edge p, patch count, spacing dx and the parameters. The mixed
// second derivatives are formed here with the same FD4 tensor-product
// stencil as the halo fill (fd11). For the mixed path the tiles of every
// field but alpha and phi are turned into split FP32 pairs (hi = u rounded
// to FP32, lo = u - hi rounded to FP32), and the mixed derivatives of g~ and
// beta into FP32 slots, as the mixed halo fill lays them out.
// mixed = 2: the mixed path in two phases (DerivTap: the stencil values
// recorded into slots with the algebra discarded, then replayed), as the
// two-phase launch shape of the stage kernel evaluates it.
// Output: d_t Q, [25][n_patches * p^3].
#include <string.h>

#include <vector>

#include "../paper_2406_11626_gb300/csrc/ccz4_algebra.cuh"
#include "../paper_2406_11626_gb300/csrc/deriv_tap.cuh"

namespace ccz4 {
void count_mark(const char *) {}
}  // namespace ccz4

using namespace ccz4;

extern "C" void host_rhs(const double *tiles, int p, int n_patches, double dx, const ccz4_params *P, int mixed,
                         double *out) {
  const int T = p + 6;
  const long long T3 = (long long)T * T * T, np = (long long)n_patches * p * p * p;
  const long long fs = (long long)n_patches * T3;
  StencilCoef<double> C;
  C.c1 = 1.0 / (12 * dx);
  C.c2 = 1.0 / (12 * dx * dx);
  C.c3 = 1.0 / (144 * dx * dx);
  C.cko = P->ko_eps / (64 * dx);
  const StencilCoef<float> CF{(float)C.c1, (float)C.c2, (float)C.c3, (float)C.cko};

  auto view = [&](const double *base, int n, int x, int y, int z) {
    Nbhd N;
    N.c = base + n * T3 + ((long long)(z + 3) * T + (y + 3)) * T + (x + 3);
    N.fs = fs;
    N.st[0] = 1;
    N.st[1] = T;
    N.st[2] = T * T;
    return N;
  };

  // mixed second derivatives of g~, alpha, beta, phi
  std::vector<double> mixb((size_t)NMIX * np);
  for (int n = 0; n < n_patches; ++n)
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          const Nbhd N = view(tiles, n, x, y, z);
          const long long i = (long long)n * p * p * p + ((long long)z * p + y) * p + x;
          for (int v = 0; v < NV; ++v) {
            const int m = mix_slot(v);
            if (m < 0) continue;
            mixb[(m + 0) * np + i] = fd11<double, double>(N, v, N.st[0], N.st[1], C.c3);
            mixb[(m + 1) * np + i] = fd11<double, double>(N, v, N.st[0], N.st[2], C.c3);
            mixb[(m + 2) * np + i] = fd11<double, double>(N, v, N.st[1], N.st[2], C.c3);
          }
        }

  // the mixed path's layout: split pairs and FP32 slots
  std::vector<double> split;
  std::vector<float> mixf((size_t)NMIXF * np);
  const double *src = tiles;
  if (mixed) {
    split.resize((size_t)NV * fs);
    for (int v = 0; v < NV; ++v)
      for (long long t = 0; t < fs; ++t) {
        const double u = tiles[v * fs + t];
        if (v == ALPHA || v == PHI) {
          split[v * fs + t] = u;
          continue;
        }
        float pr[2];
        pr[0] = (float)u;
        pr[1] = (float)(u - (double)pr[0]);
        memcpy(&split[v * fs + t], pr, 8);
      }
    src = split.data();
    for (int v = 0; v < NV; ++v) {
      const int m = mix_slot(v);
      if (m < 0 || mix_fslot(m) < 0) continue;
      for (int k = 0; k < 3; ++k)
        for (long long i = 0; i < np; ++i) mixf[(mix_fslot(m) + k) * np + i] = (float)mixb[(m + k) * np + i];
    }
  }

  for (int n = 0; n < n_patches; ++n)
    for (int z = 0; z < p; ++z)
      for (int y = 0; y < p; ++y)
        for (int x = 0; x < p; ++x) {
          Nbhd N = view(src, n, x, y, z);
          const long long i = (long long)n * p * p * p + ((long long)z * p + y) * p + x;
          N.mix = mixb.data() + i;
          N.ms = np;
          N.mixf = mixf.data() + i;
          N.msf = np;
          auto sink = [&](int v, double k) { out[v * np + i] = k; };
          if (mixed == 2) {
            float sf[TAP_FLOATS];
            double sd[TAP_DOUBLES];
            DerivTap<TAP_RECORD> rec(N, sf, sd, 1);
            NullSink none;
            ccz4_rhs_point<double, float>(make_phys<float>(*P), rec, C, CF, none);
            DerivTap<TAP_REPLAY> rep(N, sf, sd, 1);
            ccz4_rhs_point<double, float>(make_phys<float>(*P), rep, C, CF, sink);
          } else if (mixed) {
            ccz4_rhs_point<double, float>(make_phys<float>(*P), N, C, CF, sink);
          } else {
            ccz4_rhs_point<double, double>(make_phys<double>(*P), N, C, C, sink);
          }
        }
}

// Slots the two-phase evaluation asks for at one point with parameters P:
// *nf floats and *nd doubles (must not exceed TAP_FLOATS, TAP_DOUBLES).
extern "C" void host_tap_slots(const ccz4_params *P, int *nf, int *nd, int *max_f, int *max_d) {
  const int T = 7;
  std::vector<double> tile(NV * T * T * T, 1.0);
  std::vector<double> mix(NMIX, 0.0);
  std::vector<float> mixf(NMIXF, 0.0f);
  Nbhd N;
  N.c = tile.data() + (3 * T + 3) * T + 3;
  N.fs = T * T * T;
  N.st[0] = 1;
  N.st[1] = T;
  N.st[2] = T * T;
  N.mix = mix.data();
  N.ms = 1;
  N.mixf = mixf.data();
  N.msf = 1;
  StencilCoef<double> C{1.0, 1.0, 1.0, 0.1};
  const StencilCoef<float> CF{1.0f, 1.0f, 1.0f, 0.1f};
  float sf[TAP_FLOATS];
  double sd[TAP_DOUBLES];
  DerivTap<TAP_RECORD> rec(N, sf, sd, 1);
  NullSink none;
  ccz4_rhs_point<double, float>(make_phys<float>(*P), rec, C, CF, none);
  *nf = rec.kf;
  *nd = rec.kd;
  *max_f = TAP_FLOATS;
  *max_d = TAP_DOUBLES;
}
