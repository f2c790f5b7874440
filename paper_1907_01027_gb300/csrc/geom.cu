// Launch shape of the sweep kernel.
#include <cstdio>
#include <cstdlib>

#include "lmdg_internal.h"

namespace lmdg {

SweepGeom env_override(SweepGeom best, int nq, int nj, int amax) {
  if (const char *e = std::getenv("LMDG_SWEEP_GEOM")) {
    int a = 0, b = 0, c = 0;
    if (std::sscanf(e, "%d,%d,%d", &a, &b, &c) == 3 && a >= 1 && a <= nq && b >= 1 && b <= 8 && c >= 1 &&
        c <= amax && b * c >= (nq + a - 1) / a && (a - 1) * ((nq + a - 1) / a) < nq)
      best = SweepGeom{a, b, c, (nj + 31) / 32};
  }
  return best;
}

// One CTA per (quadrant, group, strip), W warps of APW directions, with the fewest groups for that shape (one
// partial reduction array per quadrant-group).  Measured on the GB300 at 1024^2 cells, S16 (sweep times in
// ms of the chosen shape against the runner-up):
//   FP32: one direction per warp, 8 warps for Q1-DG and RLMDG (2.42, 2.69; the latency-bound sweeps want
//         the most independent cell-direction chains, even though not every CTA is then resident -- the
//         ticket order keeps the wavefront deadlock-free); LMDG, whose per-direction work is smallest, two
//         directions per warp and 6 warps (2.08 against 2.15);
//   FP64 (FP64-pipe bound): Q1-DG one direction per warp, 4 warps (15.2 against 16.8 with two directions and
//         6 warps); LMDG and RLMDG two directions per warp, 3 warps (9.2, 17.5).
//   float-float (FP32-pipe bound, FP64-like registers; at most two directions per warp, the instances
//         compiled): Q1-DG one direction per warp, 4 warps (4.45 against 4.68 with 8 warps); LMDG and P0-DG two
//         directions per warp, 4 warps (3.18 against 3.29 with 2 warps); RLMDG one direction per warp, 8 warps
//         (5.32 against 5.96 with two directions and 6 warps).
SweepGeom choose_geom(int variant, int nj, int nq, int prec) {
  int apw, wmax;
  if (prec == 0) { apw = variant == LMDG_STD ? 1 : 2; wmax = variant == LMDG_STD ? 4 : 3; }
  else if (prec == 2) {
    const bool row0 = variant == LMDG_LM || variant == kP0;
    apw = row0 ? 2 : 1;
    wmax = (row0 || variant == LMDG_STD) ? 4 : 8;
  } else { apw = variant == LMDG_LM ? 2 : 1; wmax = variant == LMDG_LM ? 6 : 8; }
  // the Q1-type reconstruction's eight reduced values per cell: at most 6 warps keep a CTA's shared memory within
  // two CTAs per SM (FP32) and within the per-CTA limit (float-float)
  if (variant == kRlmQ1 && prec != 0 && wmax > 6) wmax = 6;
  int G = (nq + apw * wmax - 1) / (apw * wmax);
  while (G > 1 && (G - 1) * ((nq + G - 1) / G) >= nq) --G;
  const int gsize = (nq + G - 1) / G;
  const int a = gsize < apw ? gsize : apw;
  const int W = (gsize + a - 1) / a;
  return env_override(SweepGeom{G, W, a, (nj + 31) / 32}, nq, nj, prec == 2 ? 2 : kMaxA);
}

}  // namespace lmdg
