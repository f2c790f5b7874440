// Launch shape of the sweep kernel.
#include <cstdio>
#include <cstdlib>

#include "lmdg_internal.h"

namespace lmdg {

SweepGeom env_override(SweepGeom best, int nq, int n) {
  if (const char *e = std::getenv("LMDG_SWEEP_GEOM")) {
    int a = 0, b = 0, c = 0;
    if (std::sscanf(e, "%d,%d,%d", &a, &b, &c) == 3 && a >= 1 && a <= nq && b >= 1 && b <= 8 && c >= 1 &&
        c <= kMaxA && b * c >= (nq + a - 1) / a && (a - 1) * ((nq + a - 1) / a) < nq)
      best = SweepGeom{a, b, c, (n + 31) / 32};
  }
  return best;
}

// One CTA per (quadrant, group, strip), W warps of APW directions, with the fewest groups for that shape (one
// partial reduction array per quadrant-group).  Measured on the GB300 at 1024^2 cells, S16: the latency-bound
// FP32 sweeps run fastest with one direction per warp and 8 warps per CTA (the most independent
// cell-direction chains), even though not every CTA is then resident (the ticket order keeps the wavefront
// deadlock-free); the FP64 sweeps, bound by the FP64 pipe, with two directions per warp and up to 6 warps.
SweepGeom choose_geom(int variant, int n, int nq, bool fp64) {
  (void)variant;
  const int apw = fp64 ? 2 : 1, wmax = fp64 ? 6 : 8;
  int G = (nq + apw * wmax - 1) / (apw * wmax);
  while (G > 1 && (G - 1) * ((nq + G - 1) / G) >= nq) --G;
  const int gsize = (nq + G - 1) / G;
  const int a = gsize < apw ? gsize : apw;
  const int W = (gsize + a - 1) / a;
  return env_override(SweepGeom{G, W, a, (n + 31) / 32}, nq, n);
}

}  // namespace lmdg
