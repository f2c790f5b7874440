// Transport sweep kernels: the upwind inversion of the streaming-plus-collision operator for every
// discrete ordinate (L^-1 of Section 2.1.1, L00^-1 of Section 3.2, Ltilde00^-1 of Section 3.3.2), with the
// angular reduction fused into the sweep.
//
// Work decomposition.  The mesh is cut into strips of 32 rows (in the sweep direction of a quadrant).  One
// CTA owns one (quadrant, angle group, strip); its warps hold disjoint directions of the group.  Lane k of a
// warp owns row k of the strip and at step t solves the cell in column t - k, so the cell below (row k-1,
// same column) was solved by lane k-1 at step t-1 and arrives by a warp shuffle, and the cell to the left is
// the lane's own previous result.  Lane 0 takes its inflow from the strip below through a global trace
// buffer guarded by a per-strip progress counter; lane 31 publishes the traces for the strip above.  CTAs
// take their (strip, quadrant, group) from an atomic ticket in strip-major order, so a CTA only ever waits for
// a strip owned by a CTA that started earlier: the wavefront cannot deadlock whatever the residency.  Every
// wait is bounded (spin_limit polls); on expiry the CTA raises the error word and returns.
//
// Local coordinates.  Each quadrant is swept with the mesh mirrored so that its directions have
// Omega_x, Omega_y > 0; a cell's Legendre coefficients transform as (u0, sx u1, sy u2, sx sy u3).  With
// a = |Omega_x|, b = |Omega_y|, sigma-hat = sigma_t h, the per-cell Q1 block of L (eq-Ljk, times 2/h) is
//   [ 2(a+b+s)   2a              2b              0                  ]
//   [ -2a        2a+2/3(b+s)     0               2/3 b              ]
//   [ -2b        0               2b+2/3(a+s)     2/3 a              ]
//   [ 0          -2/3 b          -2/3 a          2/3(a+b)+2/9 s     ]
// and the upwind neighbours enter through their outflow traces: left face (U0 + U1 eta) with U0 = u0 + u1,
// U1 = u2 + u3; bottom face (V0 + V1 xi) with V0 = u0 + u2, V1 = u1 + u3.
//
// Reductions per cell (summed over the group's directions in a fixed order, one partial per quadrant-group):
//   LMDG_STD : P psi = sum w psi                                  (4 moments)
//   LMDG_LM  : P0 psi0 and sum_l w_l L_l(u_l; b_r), r = 1..3      (u_l the full per-direction trial function)
//   LMDG_RLM : as LM, plus P1 R psi0 (2 slope moments)
// from which the epilogue forms the reduced operator (see epilogue_kernel).
#include "lmdg_internal.h"

namespace lmdg {

namespace {

// Reciprocal by Newton's iteration r <- r (2 - x r) from a single-precision seed: each step squares the
// relative error, so two steps take the seed's ~2^-23 to below double rounding.
__device__ __forceinline__ double rcp(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ void store_psi0(void *psi, size_t idx, T v, int bf16) {
  if (bf16) reinterpret_cast<__nv_bfloat16 *>(psi)[idx] = __float2bfloat16((float)v);
  else reinterpret_cast<T *>(psi)[idx] = v;
}

constexpr unsigned kFull = 0xffffffffu;

}  // namespace

template <typename T, int VAR, bool STORE>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepArgs<T> A) {
  constexpr int NR = (VAR == 2) ? 6 : 4;   // reduced values per cell
  constexpr int NS = (VAR == 2) ? 3 : 2;   // trace values passed downwind per face
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);  // [2][W][NR][32]
  __shared__ int s_unit, s_abort;
  __shared__ unsigned s_avail;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = A.g.warps;
  const int n = A.n, nx = A.nx;
  if (threadIdx.x == 0) {
    s_unit = (int)atomicAdd(&A.ctrl[0], 1u);
    s_abort = 0;
    s_avail = 0;
  }
  __syncthreads();
  const int unit = s_unit;
  const int per_strip = 4 * A.g.groups;
  const int strip = unit / per_strip;
  const int pq = unit - strip * per_strip;          // partial index = quadrant * groups + group
  const int quad = pq / A.g.groups, grp = pq - quad * A.g.groups;
  const int sx = (quad == 0 || quad == 3) ? 1 : -1;
  const int sy = (quad <= 1) ? 1 : -1;
  const T fsx = (T)sx, fsy = (T)sy, fsxy = (T)(sx * sy);
  const int gsize = (A.nq + A.g.groups - 1) / A.g.groups;
  const int g0 = grp * gsize;
  const int gcount = min(gsize, A.nq - g0);

  int ang[kMaxA], uA[kMaxA];
  T wA[kMaxA], aA[kMaxA], bA[kMaxA];
  int nA = 0;
#pragma unroll
  for (int k = 0; k < kMaxA; ++k) {
    const int idx = warp + k * W;
    ang[k] = quad * A.nq + g0 + min(idx, gcount - 1);
    if (k < A.g.apw && idx < gcount) nA = k + 1;
    uA[k] = A.perm[ang[k]];
    wA[k] = A.pd.w[ang[k]];
    aA[k] = fabs(A.pd.ox[ang[k]]);
    bA[k] = fabs(A.pd.oy[ang[k]]);
  }

  const int row = strip * 32 + lane;
  const bool row_ok = row < n;
  const int j = sy > 0 ? row : n - 1 - row;
  const T h = A.h, h2 = A.h * A.h;
  const T c23 = (T)(2.0 / 3.0), c29 = (T)(2.0 / 9.0);

  T xs[kMaxA][NS], ys[kMaxA][NS];
#pragma unroll
  for (int k = 0; k < kMaxA; ++k)
#pragma unroll
    for (int c = 0; c < NS; ++c) xs[k][c] = ys[k][c] = (T)0;

  const unsigned *prog_below = strip > 0 ? &A.ctrl[2 + unit - per_strip] : nullptr;
  unsigned *prog_mine = &A.ctrl[2 + unit];
  const bool has_above = strip + 1 < A.g.strips;
  int avail = 0;
  const int nsteps = n + 31;

  for (int t = 0; t < nsteps; ++t) {
    // ---- inflow from the strip below must be published up to column t (block-uniform condition)
    if (strip > 0 && t < n && t >= avail) {
      if (threadIdx.x == 0) {
        const unsigned need = (unsigned)min(n, t + kPublish);
        long long spins = 0;
        unsigned v = ld_acquire(prog_below);
        while (v < need) {
          if (++spins > A.spin_limit || ld_relaxed(&A.ctrl[1]) != 0u) {
            atomicExch(&A.ctrl[1], 1u);
            s_abort = 1;
            break;
          }
          __nanosleep(128);
          v = ld_acquire(prog_below);
        }
        __threadfence();
        s_avail = v;
      }
      __syncthreads();
      if (s_abort) return;
      avail = (int)s_avail;
    }

    const int x = t - lane;
    const bool act = row_ok && x >= 0 && x < n;
    const int i = sx > 0 ? x : n - 1 - x;
    const int K = act ? j * n + i : 0;
    const bool xbnd = (x == 0);
    const bool ybnd = (strip == 0 && lane == 0);

    // ---- per-cell data shared by the warp's directions
    T st = 0, sse = 0, s[4] = {0, 0, 0, 0}, iso[3] = {0, 0, 0};
    if (act) {
      st = A.pd.sigt[K] * h;
      sse = A.pd.sse[K];
      const double2 Xa = *reinterpret_cast<const double2 *>(A.X + 4 * (size_t)K);
      const double2 Xb = *reinterpret_cast<const double2 *>(A.X + 4 * (size_t)K + 2);
      const struct { double x, y, z, w; } X = {Xa.x, Xa.y, Xb.x, Xb.y};
      T q4[4] = {0, 0, 0, 0};
      if (A.source && !A.q_per_angle) {
        const T *qp = A.pd.q + 4 * (size_t)K;
        q4[0] = qp[0]; q4[1] = qp[1]; q4[2] = qp[2]; q4[3] = qp[3];
      }
      const T eps = A.eps;
      if (VAR == 0) {
        // 2h D_r (sigma_s/eps X_r + eps q_r), D = (1, 1/3, 1/3, 1/9), in local coordinates
        s[0] = 2 * h * (sse * (T)X.x + eps * q4[0]);
        s[1] = fsx * (2 * h / 3) * (sse * (T)X.y + eps * q4[1]);
        s[2] = fsy * (2 * h / 3) * (sse * (T)X.z + eps * q4[2]);
        s[3] = fsxy * (2 * h / 9) * (sse * (T)X.w + eps * q4[3]);
      } else {
        s[0] = 2 * h * (sse * (T)X.x + eps * q4[0]);
        T p1 = 0, p2 = 0;
        if (VAR == 2 && A.source && A.p1ra) {
          p1 = A.p1ra[2 * (size_t)K];
          p2 = A.p1ra[2 * (size_t)K + 1];
        }
        // isotropic slopes of the trial function: -X1 (minus P1 r_alpha in source sweeps)
        iso[0] = -fsx * ((T)X.y + p1);
        iso[1] = -fsy * ((T)X.z + p2);
        iso[2] = -fsxy * (T)X.w;
      }
    }

    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;

#pragma unroll
    for (int k = 0; k < kMaxA; ++k) {
      if (k < nA) {
        T yin[NS];
#pragma unroll
        for (int c = 0; c < NS; ++c) yin[c] = __shfl_up_sync(kFull, ys[k][c], 1);
        if (act) {
          const int ua = uA[k];
          if (lane == 0 && !ybnd) {
            const T *yp = A.ytr + (((size_t)ang[k] * A.g.strips + (strip - 1)) * n + x) * 3;
#pragma unroll
            for (int c = 0; c < NS; ++c) yin[c] = ldcg(yp + c);
          }
          const T a = aA[k], b = bA[k], wl = wA[k];
          // inflow boundary data (local coordinates): left face side 0/1 row j, bottom face side 2/3 col i
          T xa0 = 0, xa1 = 0, ya0 = 0, ya1 = 0;
          if (A.source && A.pd.alpha) {
            if (xbnd) {
              const T *ap = A.pd.alpha + ((((size_t)ang[k] * 4 + (sx > 0 ? 0 : 1)) * n + j) * 2);
              xa0 = ap[0];
              xa1 = fsy * ap[1];
            }
            if (ybnd) {
              const T *ap = A.pd.alpha + ((((size_t)ang[k] * 4 + (sy > 0 ? 2 : 3)) * n + i) * 2);
              ya0 = ap[0];
              ya1 = fsx * ap[1];
            }
          }
          T sa[4] = {s[0], s[1], s[2], s[3]};
          if (A.source && A.q_per_angle) {
            const T *qp = A.pd.q + ((size_t)ang[k] * nx + K) * 4;
            const T eps = A.eps;
            sa[0] += 2 * h * eps * qp[0];
            if (VAR == 0) {
              sa[1] += fsx * (2 * h / 3) * eps * qp[1];
              sa[2] += fsy * (2 * h / 3) * eps * qp[2];
              sa[3] += fsxy * (2 * h / 9) * eps * qp[3];
            }
          }
          if (VAR == 0) {
            // ---------------- standard Q1 block solve
            const T U0 = xbnd ? xa0 : xs[k][0], U1 = xbnd ? xa1 : xs[k][1];
            const T V0 = ybnd ? ya0 : yin[0], V1 = ybnd ? ya1 : yin[1];
            const T r0 = sa[0] + 2 * a * U0 + 2 * b * V0;
            const T r1 = sa[1] - 2 * a * U0 + c23 * b * V1;
            const T r2 = sa[2] + c23 * a * U1 - 2 * b * V0;
            const T r3 = sa[3] - c23 * a * U1 - c23 * b * V1;
            const T d0 = 2 * (a + b + st);
            const T d1 = 2 * a + c23 * (b + st);
            const T d2 = 2 * b + c23 * (a + st);
            const T d3 = c23 * (a + b) + c29 * st;
            const T i1 = rcp(d1), i2 = rcp(d2);
            const T a00 = d0 + 4 * a * a * i1 + 4 * b * b * i2;
            const T a03 = -(T)(4.0 / 3.0) * a * b * (i1 + i2);
            const T a33 = d3 + (T)(4.0 / 9.0) * (b * b * i1 + a * a * i2);
            const T b0 = r0 - 2 * a * r1 * i1 - 2 * b * r2 * i2;
            const T b3 = r3 + c23 * (b * r1 * i1 + a * r2 * i2);
            const T idet = rcp(a00 * a33 - a03 * a03);
            const T u0 = (a33 * b0 - a03 * b3) * idet;
            const T u3 = (a00 * b3 - a03 * b0) * idet;
            const T u1 = (r1 + 2 * a * u0 - c23 * b * u3) * i1;
            const T u2 = (r2 + 2 * b * u0 - c23 * a * u3) * i2;
            acc[0] += wl * u0;
            acc[1] += wl * fsx * u1;
            acc[2] += wl * fsy * u2;
            acc[3] += wl * fsxy * u3;
            xs[k][0] = u0 + u1; xs[k][1] = u2 + u3;
            ys[k][0] = u0 + u2; ys[k][1] = u1 + u3;
            if (STORE) {
              T *pp = reinterpret_cast<T *>(A.psi) + ((size_t)ua * nx + K) * 4;
              pp[0] = u0; pp[1] = fsx * u1; pp[2] = fsy * u2; pp[3] = fsxy * u3;
            }
          } else {
            // ---------------- low-memory row-0 solve (L00, or Ltilde00 with reconstruction)
            const T U0s = xbnd ? xa0 : xs[k][0];
            const T V0s = ybnd ? ya0 : yin[0];
            const T d0 = 2 * (a + b + st);
            T rhs = sa[0] + 2 * a * (U0s - iso[0]) + 2 * b * (V0s - iso[1]);
            T u0, rec1 = 0, rec2 = 0;
            if (VAR == 1) {
              u0 = rhs * rcp(d0);
            } else {
              // reconstructed slopes (h/2) delta: interior (u0 - u0_up)/2, inflow boundary u0 - alpha_mid
              const T cx = xbnd ? 2 * a : a, cy = ybnd ? 2 * b : b;
              rhs += xbnd ? 2 * a * xa0 : a * xs[k][2];
              rhs += ybnd ? 2 * b * ya0 : b * yin[2];
              u0 = rhs * rcp(d0 + cx + cy);
              rec1 = xbnd ? (u0 - xa0) : (T)0.5 * (u0 - xs[k][2]);
              rec2 = ybnd ? (u0 - ya0) : (T)0.5 * (u0 - yin[2]);
            }
            const T u1 = iso[0] + rec1, u2 = iso[1] + rec2, u3 = iso[2];
            // rows 1..3 of L applied to the trial function (inflow traces of L vanish on the boundary)
            const T U0L = xbnd ? (T)0 : xs[k][0], U1L = xbnd ? (T)0 : xs[k][1];
            const T V0L = ybnd ? (T)0 : yin[0], V1L = ybnd ? (T)0 : yin[1];
            const T d1 = 2 * a + c23 * (b + st);
            const T d2 = 2 * b + c23 * (a + st);
            const T d3 = c23 * (a + b) + c29 * st;
            const T T1 = -2 * a * u0 + d1 * u1 + c23 * b * u3 + 2 * a * U0L - c23 * b * V1L;
            const T T2 = -2 * b * u0 + d2 * u2 + c23 * a * u3 - c23 * a * U1L + 2 * b * V0L;
            const T T3 = -c23 * b * u1 - c23 * a * u2 + d3 * u3 + c23 * (a * U1L + b * V1L);
            acc[0] += wl * u0;
            acc[1] += wl * fsx * T1;
            acc[2] += wl * fsy * T2;
            acc[3] += wl * fsxy * T3;
            if (VAR == 2) {
              acc[4] += wl * fsx * rec1;
              acc[5] += wl * fsy * rec2;
            }
            xs[k][0] = u0 + u1; xs[k][1] = u2 + u3;
            ys[k][0] = u0 + u2; ys[k][1] = u1 + u3;
            if (VAR == 2) { xs[k][2] = u0; ys[k][2] = u0; }
            if (STORE) store_psi0<T>(A.psi, (size_t)ua * nx + K, u0, A.psi_bf16);
          }
          if (lane == 31 && has_above) {
            T *yp = A.ytr + (((size_t)ang[k] * A.g.strips + strip) * n + x) * 3;
#pragma unroll
            for (int c = 0; c < NS; ++c) yp[c] = ys[k][c];
          }
        }
      }
    }

    // ---- fixed-order reduction over the CTA's warps (double-buffered shared memory, one barrier a step)
    T *bb = buf + ((size_t)((t & 1) * W + warp) * NR) * 32 + lane;
#pragma unroll
    for (int r = 0; r < NR; ++r) bb[r * 32] = acc[r];
    const bool publish = has_above && t >= 31 && (((t - 30) % kPublish) == 0 || t == nsteps - 1);
    if (publish && lane == 31) __threadfence();
    __syncthreads();
    if (warp == 0 && act) {
      T sum[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) sum[r] = 0;
      for (int ww = 0; ww < W; ++ww) {
        const T *src = buf + ((size_t)((t & 1) * W + ww) * NR) * 32 + lane;
#pragma unroll
        for (int r = 0; r < NR; ++r) sum[r] += src[r * 32];
      }
      T *dst = A.part + ((size_t)pq * nx + K) * NR;
#pragma unroll
      for (int r = 0; r < NR; ++r) dst[r] = sum[r];
    }
    if (publish && threadIdx.x == 0) {
      __threadfence();
      st_release(prog_mine, (unsigned)min(n, t - 30));
    }
  }
}

// y = K X - source * b from the partial reductions, one thread per cell.
//   STD : y = X - sum_p part_p                       (K = I - P L^-1 M; b = P L^-1 Q)
//   LM/RLM: y0 = X0 - P0 psi0
//           y_r = (sigma_s/eps) h^2 D_r (S_r - source P1r_alpha_r - X_r) - (h/2) T_r + source SigmaQ1_r
// where T_r = sum_l w_l L_l(u_l; b_r) over the full trial functions u_l = psi0_l + (R psi0)_l - X1 and S = P1 R
// psi0.  For the homogeneous sweep this equals the second block row B11 X1 - (Sigma Ltilde10 + B11 P1 R) psi0
// of the reduced operator, because Sigma L11 Sigma^T = B11 + Sigma M1 (eq-lmdg-psi1).
template <typename T, int VAR>
__global__ void epilogue_kernel(int nx, int P, double h, const T *__restrict__ part,
                                const double *__restrict__ X, const double *__restrict__ sse,
                                const double *__restrict__ p1ra, const double *__restrict__ sq1, int source,
                                double *__restrict__ y) {
  constexpr int NR = (VAR == 2) ? 6 : 4;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  double s[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) s[r] = 0;
  for (int p = 0; p < P; ++p) {
    const T *pp = part + ((size_t)p * nx + K) * NR;
#pragma unroll
    for (int r = 0; r < NR; ++r) s[r] += (double)pp[r];
  }
  const double2 xa = *reinterpret_cast<const double2 *>(X + 4 * (size_t)K);
  const double2 xb = *reinterpret_cast<const double2 *>(X + 4 * (size_t)K + 2);
  const struct { double x, y, z, w; } x = {xa.x, xa.y, xb.x, xb.y};
  struct { double x, y, z, w; } out;
  if (VAR == 0) {
    out.x = x.x - s[0]; out.y = x.y - s[1]; out.z = x.z - s[2]; out.w = x.w - s[3];
  } else {
    const double m = sse[K] * h * h;
    double S1 = 0, S2 = 0;
    if (VAR == 2) {
      S1 = s[4]; S2 = s[5];
      if (source && p1ra) { S1 -= p1ra[2 * (size_t)K]; S2 -= p1ra[2 * (size_t)K + 1]; }
    }
    out.x = x.x - s[0];
    out.y = m * (1.0 / 3.0) * (S1 - x.y) - 0.5 * h * s[1];
    out.z = m * (1.0 / 3.0) * (S2 - x.z) - 0.5 * h * s[2];
    out.w = m * (1.0 / 9.0) * (0.0 - x.w) - 0.5 * h * s[3];
    if (source) { out.y += sq1[3 * (size_t)K]; out.z += sq1[3 * (size_t)K + 1]; out.w += sq1[3 * (size_t)K + 2]; }
  }
  *reinterpret_cast<double2 *>(y + 4 * (size_t)K) = make_double2(out.x, out.y);
  *reinterpret_cast<double2 *>(y + 4 * (size_t)K + 2) = make_double2(out.z, out.w);
}

template <typename T, int VAR>
static cudaError_t launch_var(const SweepArgs<T> &a, bool store, cudaStream_t s) {
  constexpr int NR = (VAR == 2) ? 6 : 4;
  const size_t smem = 2ull * a.g.warps * NR * 32 * sizeof(T);
  const dim3 grid(a.g.units()), block(a.g.warps * 32);
  cudaError_t e = cudaMemsetAsync(a.ctrl, 0, (2 + (size_t)a.g.units()) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  add_launches(1);
  if (store) sweep_kernel<T, VAR, true><<<grid, block, smem, s>>>(a);
  else sweep_kernel<T, VAR, false><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep(int variant, const SweepArgs<T> &a, cudaStream_t s) {
  const bool store = a.psi != nullptr;
  switch (variant) {
    case LMDG_STD: return launch_var<T, 0>(a, store, s);
    case LMDG_LM: return launch_var<T, 1>(a, store, s);
    default: return launch_var<T, 2>(a, store, s);
  }
}

template <typename T>
cudaError_t launch_epilogue(int variant, int n, int nx, int P, double h, const T *part, const double *X,
                            const double *sse, const double *p1ra, const double *sq1, int source, double *y,
                            cudaStream_t s) {
  (void)n;
  const int bs = 256, gs = (nx + bs - 1) / bs;
  add_launches(1);
  switch (variant) {
    case LMDG_STD: epilogue_kernel<T, 0><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, p1ra, sq1, source, y); break;
    case LMDG_LM: epilogue_kernel<T, 1><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, p1ra, sq1, source, y); break;
    default: epilogue_kernel<T, 2><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, p1ra, sq1, source, y); break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_sweep<double>(int, const SweepArgs<double> &, cudaStream_t);
template cudaError_t launch_sweep<float>(int, const SweepArgs<float> &, cudaStream_t);
template cudaError_t launch_epilogue<double>(int, int, int, int, double, const double *, const double *,
                                             const double *, const double *, const double *, int, double *,
                                             cudaStream_t);
template cudaError_t launch_epilogue<float>(int, int, int, int, double, const float *, const double *,
                                            const double *, const double *, const double *, int, double *,
                                            cudaStream_t);

}  // namespace lmdg
