// Host-side count of the arithmetic of one interior point-stage, obtained by
// running the kernel templates (right-hand side, dissipation, RK4 update,
// enforcement) with the counting scalar types of ccz4_count.cuh. These are
// the algorithmic flops the roofline divides by the kernel time.
#include <stdio.h>

#include <string>
#include <utility>
#include <vector>

#include "ccz4_algebra.cuh"
#include "ccz4_count.cuh"

namespace ccz4 {

static OpTally g_tally[2];
OpTally &tally(int precision_index) { return g_tally[precision_index]; }

// section breakdown of the last count: label -> FP64 and FP32 flops since the previous mark
static std::vector<std::pair<std::string, std::pair<double, double>>> g_sections;
static double g_last[2] = {0.0, 0.0};
static bool g_sections_on = false;

void count_mark(const char *section) {
  if (!g_sections_on) return;
  const double f64 = g_tally[0].flops(), f32 = g_tally[1].flops();
  g_sections.push_back({section, {f64 - g_last[0], f32 - g_last[1]}});
  g_last[0] = f64;
  g_last[1] = f32;
}

namespace {

template <int MODE>
struct CountSink {
  Cnt<double> dt{0.01};
  void operator()(int, const Cnt<double> &k) {
    Cnt<double> u(1.0), acc(0.5);
    rk_combine<MODE, Cnt<double>>(u, acc, k, dt);
  }
};

template <class R>
void count_point_stage(const ccz4_params &P, const Nbhd &N) {
  using D = Cnt<double>;
  StencilCoef<D> C{D(1.0), D(1.0), D(1.0), D(P.ko_eps)};
  StencilCoef<R> CR{R(1.0), R(1.0), R(1.0), R(P.ko_eps)};
  const Phys<R> ph = make_phys<R>(P);
  // four stages: right-hand side + dissipation + update each
  g_sections_on = true;
  CountSink<0> s0;
  ccz4_rhs_point<D, R>(ph, N, C, CR, s0);
  count_mark("rk update");
  g_sections_on = false;
  CountSink<1> s1;
  ccz4_rhs_point<D, R>(ph, N, C, CR, s1);
  CountSink<2> s2;
  ccz4_rhs_point<D, R>(ph, N, C, CR, s2);
  CountSink<3> s3;
  ccz4_rhs_point<D, R>(ph, N, C, CR, s3);
  // enforcement after the last stage
  D g[6] = {D(1.0), D(0.01), D(0.0), D(1.0), D(0.0), D(1.0)};
  D A[6] = {D(0.1), D(0.0), D(0.0), D(-0.05), D(0.0), D(-0.05)};
  enforce_point<D>(g, A);
}

}  // namespace
}  // namespace ccz4

using namespace ccz4;

extern "C" ccz4_status ccz4_flops_per_point_stage(const ccz4_params *P, double out[6]) {
  if (!P || !out || (P->precision != CCZ4_PREC_FP64 && P->precision != CCZ4_PREC_MIXED)) {
    set_error("flops_per_point_stage: invalid arguments");
    return CCZ4_ERR_INVALID;
  }
  // 7^3 neighbourhood of flat space (the values do not change the count)
  const int W = 7;
  std::vector<double> buf((size_t)NV * W * W * W, 0.0);
  for (int v : {GXX, GYY, GZZ, ALPHA, PHI})
    for (int t = 0; t < W * W * W; ++t) buf[(size_t)v * W * W * W + t] = 1.0;
  std::vector<double> mixbuf(NMIX, 0.0);
  Nbhd N;
  N.mix = mixbuf.data();
  N.ms = 1;
  N.mixf = nullptr;  // the counting types read the FP64 slots
  N.msf = 0;
  N.c = buf.data() + (3 * W * W + 3 * W + 3);
  N.fs = W * W * W;
  N.st[0] = 1;
  N.st[1] = W;
  N.st[2] = W * W;
  g_tally[0] = OpTally();
  g_tally[1] = OpTally();
  g_sections.clear();
  g_last[0] = g_last[1] = 0.0;
  if (P->precision == CCZ4_PREC_MIXED) count_point_stage<Cnt<float>>(*P, N);
  else count_point_stage<Cnt<double>>(*P, N);
  const double per = 1.0 / 4.0;  // the counts above cover the four stages of one step
  out[0] = g_tally[0].flops() * per;
  out[1] = g_tally[1].flops() * per;
  out[2] = (double)(g_tally[0].div + g_tally[0].sqrt) * per;
  out[3] = (double)(g_tally[0].cvt + g_tally[1].cvt) * per;
  out[4] = (double)g_tally[0].fma * per;
  out[5] = (double)(g_tally[0].add + g_tally[0].mul) * per;
  return CCZ4_OK;
}

// Breakdown of the last ccz4_flops_per_point_stage call by kernel section
// (stage 0 only): writes up to `cap` labels into `labels` (each at most 31
// chars + NUL, 32 bytes apart) and FP64/FP32 flops into fp64[] and fp32[].
// Returns the number of sections.
extern "C" int ccz4_flops_sections(int cap, char *labels, double *fp64, double *fp32) {
  int n = 0;
  for (const auto &e : g_sections) {
    if (n >= cap) break;
    snprintf(labels + 32 * n, 32, "%s", e.first.c_str());
    fp64[n] = e.second.first;
    fp32[n] = e.second.second;
    ++n;
  }
  return n;
}
