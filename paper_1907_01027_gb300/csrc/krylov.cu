// Vector kernels for GMRES (classical Gram-Schmidt applied twice) and conjugate gradients, plus the B11
// stencil.  All reductions are two-pass with a fixed block count and a fixed summation order, so results
// are bitwise reproducible run to run.
#include "lmdg_internal.h"
#include "krylov.h"
#include <atomic>
#include <cstdint>

namespace lmdg {

namespace {
constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kDotChunk = 8;         // vectors reduced per pass over w

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

// partial[b * nv + i] = sum over this block's slice of V_i[k] * w[k], i < nv.  PAIRS: entries move as 16-byte
// pairs (N, ldv even and 16-byte aligned vectors, as the [nx][4] Krylov vectors are); the summation order is fixed
// by the launch shape.
template <bool PAIRS>
__global__ void mdot_kernel(const double *__restrict__ V, size_t ldv, int nv, const double *__restrict__ w,
                            size_t N, double *__restrict__ partial) {
  __shared__ double sh[kRedThreads / 32][kDotChunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nv; c0 += kDotChunk) {
    const int nc = min(kDotChunk, nv - c0);
    double acc[kDotChunk];
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) acc[c] = 0;
    if (PAIRS) {
      const double2 *w2 = reinterpret_cast<const double2 *>(w);
      for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N / 2; k += (size_t)gridDim.x * blockDim.x) {
        const double2 wk = w2[k];
#pragma unroll
        for (int c = 0; c < kDotChunk; ++c)
          if (c < nc) {
            const double2 v = reinterpret_cast<const double2 *>(V + (size_t)(c0 + c) * ldv)[k];
            acc[c] = fma(v.y, wk.y, fma(v.x, wk.x, acc[c]));
          }
      }
    } else {
      for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const double wk = w[k];
#pragma unroll
        for (int c = 0; c < kDotChunk; ++c)
          if (c < nc) acc[c] = fma(V[(size_t)(c0 + c) * ldv + k], wk, acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) sh[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      double s = 0;
      for (int ww = 0; ww < kRedThreads / 32; ++ww) s += sh[ww][threadIdx.x];
      partial[(size_t)blockIdx.x * nv + c0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// out[i] = sum_b partial[b * nv + i]   (+ out[i] if accumulate); one warp per output: lane l sums the blocks
// b = l, l + 32, ... in order, then a fixed butterfly combines the lanes (deterministic)
__global__ void mdot_fin_kernel(const double *__restrict__ partial, int nb, int nv, double *__restrict__ out,
                                int accumulate) {
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= nv) return;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += partial[(size_t)b * nv + i];
  s = warp_sum(s);
  if (lane == 0) out[i] = accumulate ? out[i] + s : s;
}

// w -= sum_i V_i coef_i (pairs of entries per thread, coefficients staged in shared memory; nv <= 128)
__global__ void maxpy_kernel(double *__restrict__ w, const double *__restrict__ V, size_t ldv, int nv,
                             const double *__restrict__ coef, size_t N) {
  __shared__ double cs[128];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = coef[i];
  __syncthreads();
  double2 *w2 = reinterpret_cast<double2 *>(w);
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N / 2; k += (size_t)gridDim.x * blockDim.x) {
    double2 s = w2[k];
    for (int i = 0; i < nv; ++i) {
      const double2 v = reinterpret_cast<const double2 *>(V + (size_t)i * ldv)[k];
      s.x = fma(-cs[i], v.x, s.x);
      s.y = fma(-cs[i], v.y, s.y);
    }
    w2[k] = s;
  }
}

// y = x * (1 / sqrt(*nrm2))  (nrm2 on the device; the reciprocal is formed once per block -- FP64 square root
// and division are long instruction sequences on a part where FP64 is scarce)
__global__ void scale_by_inv_kernel(double *__restrict__ y, const double *__restrict__ x,
                                    const double *__restrict__ nrm2, size_t N) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / sqrt(*nrm2);
  __syncthreads();
  const double inv = s_inv;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N / 2; k += (size_t)gridDim.x * blockDim.x) {
    const double2 v = reinterpret_cast<const double2 *>(x)[k];
    reinterpret_cast<double2 *>(y)[k] = make_double2(v.x * inv, v.y * inv);
  }
}

__global__ void axpby_kernel(double *__restrict__ y, double a, const double *__restrict__ x, double b, size_t N) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
    y[k] = fma(a, x[k], b * y[k]);
}

// y = Minv x for the right preconditioner diag(I, diag(B11))^-1 on [nx][4] vectors (mode 1), copy (mode 0);
// dinv holds the reciprocal diagonal
__global__ void precond_kernel(double *__restrict__ y, const double *__restrict__ x,
                               const double *__restrict__ dinv, int nx, int mode) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  double2 va = reinterpret_cast<const double2 *>(x)[2 * K];
  double2 vb = reinterpret_cast<const double2 *>(x)[2 * K + 1];
  if (mode == 1) {
    va.y *= dinv[3 * (size_t)K];
    vb.x *= dinv[3 * (size_t)K + 1];
    vb.y *= dinv[3 * (size_t)K + 2];
  }
  reinterpret_cast<double2 *>(y)[2 * K] = va;
  reinterpret_cast<double2 *>(y)[2 * K + 1] = vb;
}

// B11 = Sigma L11 Sigma^T - Sigma M1 on slope fields u = (c1, c2, c3) per cell (eq-lmdg-psi1):
//   (B11 u)_r(K) = eps sigma_a int_K u b_r + sum over faces F of K of
//        [ (outflow weight of F) int_F u^K b_r  -  (inflow weight of F) int_F u^nbr b_r ],
// where for the east face the outflow weight is Ax+ = sum_{Omega_x>0} w Omega_x and the inflow weight is
// Ax- = sum_{Omega_x<0} w |Omega_x| (mirror for west, likewise y), and u^nbr = 0 outside the domain.  The
// volume streaming term vanishes because sum_l w_l Omega_l = 0 (eq-polyquad (ii)).  Face integrals of the
// slope basis (xi, eta, xi eta), with s = +-1 the side of the face:
//   x-face (xi = s): traces (s, eta, s eta): int b_r b_q ds = h [[1,0,0],[0,1/3,s/3],[0,s/3,1/3]] with the
//   neighbour's trace (-s, eta, -s eta) entering as h [[-1,0,0],[0,1/3,-s/3],[0,s/3,-1/3]]  (rows own, cols nbr)
__global__ void b11_kernel(int ni, int nj, double h, double eps, const double *__restrict__ sigma_a, double Axp,
                           double Axm, double Ayp, double Aym, const double *__restrict__ u,
                           double *__restrict__ y) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= ni * nj) return;
  const int i = K % ni, j = K / ni;
  const double *uk = u + 3 * (size_t)K;
  const double c1 = uk[0], c2 = uk[1], c3 = uk[2];
  const double m = eps * sigma_a[K] * h * h;
  double y1 = m * c1 / 3.0, y2 = m * c2 / 3.0, y3 = m * c3 / 9.0;
  // x faces: s = +1 east (outflow weight Axp, inflow Axm), s = -1 west (outflow Axm, inflow Axp)
  for (int side = 0; side < 2; ++side) {
    const double s = side == 0 ? 1.0 : -1.0;
    const double wo = side == 0 ? Axp : Axm, wi = side == 0 ? Axm : Axp;
    const int in = side == 0 ? i + 1 : i - 1;
    // own trace: (c1 s) + (c2 + s c3) eta ; test traces b1 = s, b2 = eta, b3 = s eta
    const double o0 = c1 * s, o1 = c2 + s * c3;
    y1 += wo * h * (s * o0);
    y2 += wo * h * (o1 / 3.0);
    y3 += wo * h * (s * o1 / 3.0);
    if (in >= 0 && in < ni) {
      const double *un = u + 3 * (size_t)(j * ni + in);
      // neighbour trace on the shared face (its xi = -s): (-s n1) + (n2 - s n3) eta
      const double e0 = -s * un[0], e1 = un[1] - s * un[2];
      y1 -= wi * h * (s * e0);
      y2 -= wi * h * (e1 / 3.0);
      y3 -= wi * h * (s * e1 / 3.0);
    }
  }
  for (int side = 0; side < 2; ++side) {
    const double s = side == 0 ? 1.0 : -1.0;
    const double wo = side == 0 ? Ayp : Aym, wi = side == 0 ? Aym : Ayp;
    const int jn = side == 0 ? j + 1 : j - 1;
    // own trace at eta = s: (c2 s) + (c1 + s c3) xi ; tests b1 = xi, b2 = s, b3 = s xi
    const double o0 = c2 * s, o1 = c1 + s * c3;
    y1 += wo * h * (o1 / 3.0);
    y2 += wo * h * (s * o0);
    y3 += wo * h * (s * o1 / 3.0);
    if (jn >= 0 && jn < nj) {
      const double *un = u + 3 * (size_t)(jn * ni + i);
      const double e0 = -s * un[1], e1 = un[0] - s * un[2];
      y1 -= wi * h * (e1 / 3.0);
      y2 -= wi * h * (s * e0);
      y3 -= wi * h * (s * e1 / 3.0);
    }
  }
  double *yk = y + 3 * (size_t)K;
  yk[0] = y1; yk[1] = y2; yk[2] = y3;
}

// Per-cell sensitivities of the standard scheme from the correlation partials C_r = sum_l w_l lam_l,r psi_l,r,
// the forward scalar flux Phi and the multiplier Lam (mass = h^2 diag(1, 1/3, 1/3, 1/9)):
//   dJ/dsigma_s = (Lam^T mass Phi - sum_r mass_r C_r) / eps,  dJ/dsigma_a = -eps sum_r mass_r C_r,
//   dJ/dq = eps mass_0 Lam_0.
__global__ void adjoint_grad_kernel(int nx, int P, double h, double eps, const double *__restrict__ part,
                                    const double *__restrict__ Phi, const double *__restrict__ Lam,
                                    double *__restrict__ out) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double D[4] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0};
  double corr = 0, lp = 0;
  for (int r = 0; r < 4; ++r) {
    double c = 0;
    for (int p = 0; p < P; ++p) c += part[((size_t)p * nx + K) * 4 + r];
    corr += h * h * D[r] * c;
    lp += h * h * D[r] * Lam[4 * (size_t)K + r] * Phi[4 * (size_t)K + r];
  }
  out[K] = (lp - corr) / eps;
  out[nx + K] = -eps * corr;
  out[2 * (size_t)nx + K] = eps * h * h * Lam[4 * (size_t)K];
}

// Low-memory scheme (V_h^lm trial = test space): with the forward scalar-flux moments Phi = (X0, Phi1), the
// adjoint solution's moments A = (Lam0, mu1) and C0 = sum_l w_l mu0_l psi0_l (correlation partials, r = 0):
//   dJ/dsigma_s = h^2 (Lam0 X0 - C0) / eps,  dJ/dsigma_a = -eps h^2 (C0 + sum_{r>=1} D_r mu1_r Phi1_r),
//   dJ/dq = eps h^2 Lam0   (the isotropic slope terms of dJ/dsigma_s cancel).
__global__ void adjoint_grad_lm_kernel(int nx, int P, double h, double eps, const double *__restrict__ part,
                                       const double *__restrict__ Phi, const double *__restrict__ Adj,
                                       double *__restrict__ out) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  double c0 = 0;
  for (int p = 0; p < P; ++p) c0 += part[((size_t)p * nx + K) * 4];
  const double *f = Phi + 4 * (size_t)K, *a = Adj + 4 * (size_t)K;
  const double h2 = h * h;
  const double slopes = (a[1] * f[1] + a[2] * f[2]) / 3.0 + a[3] * f[3] / 9.0;
  out[K] = h2 * (a[0] * f[0] - c0) / eps;
  out[nx + K] = -eps * h2 * (c0 + slopes);
  out[2 * (size_t)nx + K] = eps * h2 * a[0];
}

__global__ void fill_u32_kernel(unsigned *__restrict__ p, unsigned v, size_t N) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) p[k] = v;
}

// Stored angular unknowns to the user layout: the sweeps keep each direction's plane in its own wavefront order
// (psi_slot in the quadrant's mirrored frame, per values a slot); the user layout is row-major, [u][j][i][per], in
// double.  Item o runs over the sorted directions (quadrant = sorted index / nq), u = perm[sorted index].
__global__ void psi_to_user_kernel(double *__restrict__ y, const void *__restrict__ x, int kind, int per, int ni,
                                   int nj, int nang, int nq, const int *__restrict__ perm) {
  const size_t nx = (size_t)ni * nj, N = (size_t)nang * nx * per, plane = psi_plane(ni, nj);
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < N; o += (size_t)gridDim.x * blockDim.x) {
    const size_t c = o % per, cell = o / per;
    const size_t ks = cell / nx, K = cell - ks * nx;
    const int j = (int)(K / ni), i = (int)(K - (size_t)j * ni);
    const int quad = (int)ks / nq, u = perm[ks];
    const int lx = (quad == 0 || quad == 3) ? i : ni - 1 - i, lr = quad <= 1 ? j : nj - 1 - j;
    const size_t k = ((size_t)u * plane + psi_slot(ni, lx, lr)) * per + c;
    const size_t out = ((size_t)u * nx + K) * per + c;
    if (kind == 1) y[out] = (double)reinterpret_cast<const float *>(x)[k];
    else if (kind == 2) y[out] = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(x)[k]);
    else y[out] = reinterpret_cast<const double *>(x)[k];
  }
}

// ------------------------------------------------------------------------------------------ host wrappers
static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void add_launches(long long k) { g_launches += k; }

static int grid_for(size_t N) {
  size_t g = (N + 255) / 256;
  return (int)(g < 2048 ? (g == 0 ? 1 : g) : 2048);
}

static bool pairs_ok(size_t N, size_t ldv, const void *a, const void *b) {
  return N % 2 == 0 && ldv % 2 == 0 && reinterpret_cast<uintptr_t>(a) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(b) % 16 == 0;
}

cudaError_t mdot(const double *V, size_t ldv, int nv, const double *w, size_t N, double *partial, double *out,
                 int accumulate, cudaStream_t s) {
  add_launches(2);
  if (pairs_ok(N, ldv, V, w)) mdot_kernel<true><<<kRedBlocks, kRedThreads, 0, s>>>(V, ldv, nv, w, N, partial);
  else mdot_kernel<false><<<kRedBlocks, kRedThreads, 0, s>>>(V, ldv, nv, w, N, partial);
  mdot_fin_kernel<<<(nv + 3) / 4, 128, 0, s>>>(partial, kRedBlocks, nv, out, accumulate);
  return cudaGetLastError();
}
size_t mdot_partial_len(int nvmax) { return (size_t)kRedBlocks * nvmax; }

cudaError_t maxpy(double *w, const double *V, size_t ldv, int nv, const double *coef, size_t N, cudaStream_t s) {
  if (nv > 128 || !pairs_ok(N, ldv, V, w)) return cudaErrorInvalidValue;
  add_launches(1);
  maxpy_kernel<<<grid_for(N), 256, 0, s>>>(w, V, ldv, nv, coef, N);
  return cudaGetLastError();
}
cudaError_t scale_by_inv(double *y, const double *x, const double *nrm2, size_t N, cudaStream_t s) {
  if (!pairs_ok(N, 0, x, y)) return cudaErrorInvalidValue;
  add_launches(1);
  scale_by_inv_kernel<<<grid_for(N), 256, 0, s>>>(y, x, nrm2, N);
  return cudaGetLastError();
}
cudaError_t axpby(double *y, double a, const double *x, double b, size_t N, cudaStream_t s) {
  add_launches(1);
  axpby_kernel<<<grid_for(N), 256, 0, s>>>(y, a, x, b, N);
  return cudaGetLastError();
}
__global__ void unit_kernel(double *__restrict__ x, int nx, int r) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  for (int q = 0; q < 4; ++q) x[4 * (size_t)K + q] = q == r ? 1.0 : 0.0;
}

// One 4 x 4 inverse per cell by Gauss-Jordan elimination on [B | I] with partial pivoting.
__global__ void block_inverse_kernel(const double *__restrict__ y0, const double *__restrict__ y1,
                                     const double *__restrict__ y2, const double *__restrict__ y3, int nx,
                                     double *__restrict__ binv, unsigned *__restrict__ bad) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double *col[4] = {y0, y1, y2, y3};
  double a[4][8];
  double scale = 0;
  for (int q = 0; q < 4; ++q)
    for (int r = 0; r < 4; ++r) {
      a[q][r] = col[r][4 * (size_t)K + q];
      a[q][4 + r] = q == r ? 1.0 : 0.0;
      scale = fmax(scale, fabs(a[q][r]));
    }
  bool ok = scale > 0 && isfinite(scale);
  for (int c = 0; c < 4 && ok; ++c) {
    int piv = c;
    for (int q = c + 1; q < 4; ++q)
      if (fabs(a[q][c]) > fabs(a[piv][c])) piv = q;
    if (!(fabs(a[piv][c]) > 1e-14 * scale)) { ok = false; break; }
    if (piv != c)
      for (int r = 0; r < 8; ++r) { const double t = a[c][r]; a[c][r] = a[piv][r]; a[piv][r] = t; }
    const double inv = 1.0 / a[c][c];
    for (int r = 0; r < 8; ++r) a[c][r] *= inv;
    for (int q = 0; q < 4; ++q) {
      if (q == c) continue;
      const double f = a[q][c];
      if (f != 0.0)
        for (int r = 0; r < 8; ++r) a[q][r] -= f * a[c][r];
    }
  }
  double *o = binv + 16 * (size_t)K;
  for (int q = 0; q < 4; ++q)
    for (int r = 0; r < 4; ++r) o[4 * q + r] = ok ? a[q][4 + r] : (q == r ? 1.0 : 0.0);
  if (!ok) atomicAdd(bad, 1u);
}

__global__ void block_step_kernel(double *__restrict__ y, const double *__restrict__ x,
                                  const double *__restrict__ binv, const double *__restrict__ dinv, int nx, int mode) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double *xk = x + 4 * (size_t)K;
  const double *b = binv + 16 * (size_t)K;
  double *yk = y + 4 * (size_t)K;
  for (int q = 0; q < 4; ++q) {
    const double jx = (mode == 1 && q > 0) ? xk[q] * dinv[3 * (size_t)K + q - 1] : xk[q];
    const double bx = b[4 * q] * xk[0] + b[4 * q + 1] * xk[1] + b[4 * q + 2] * xk[2] + b[4 * q + 3] * xk[3];
    yk[q] += bx - jx;
  }
}

cudaError_t unit_vectors(double *x, int nx, int r, cudaStream_t s) {
  add_launches(1);
  unit_kernel<<<(nx + 255) / 256, 256, 0, s>>>(x, nx, r);
  return cudaGetLastError();
}
cudaError_t block_inverses(const double *y0, const double *y1, const double *y2, const double *y3, int nx,
                           double *binv, unsigned *bad, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  add_launches(1);
  block_inverse_kernel<<<(nx + 127) / 128, 128, 0, s>>>(y0, y1, y2, y3, nx, binv, bad);
  return cudaGetLastError();
}
cudaError_t block_step(double *y, const double *x, const double *binv, const double *dinv, int nx, int mode,
                       cudaStream_t s) {
  add_launches(1);
  block_step_kernel<<<(nx + 255) / 256, 256, 0, s>>>(y, x, binv, dinv, nx, mode);
  return cudaGetLastError();
}

cudaError_t precond(double *y, const double *x, const double *dinv, int nx, int mode, cudaStream_t s) {
  add_launches(1);
  precond_kernel<<<(nx + 255) / 256, 256, 0, s>>>(y, x, dinv, nx, mode);
  return cudaGetLastError();
}
cudaError_t b11_apply(int ni, int nj, double h, double eps, const double *sigma_a, const double *A4, const double *u,
                      double *y, cudaStream_t s) {
  add_launches(1);
  b11_kernel<<<(ni * nj + 255) / 256, 256, 0, s>>>(ni, nj, h, eps, sigma_a, A4[0], A4[1], A4[2], A4[3], u, y);
  return cudaGetLastError();
}
cudaError_t adjoint_gradients(int variant, int nx, int P, double h, double eps, const double *part,
                              const double *Phi, const double *Lam, double *out, cudaStream_t s) {
  add_launches(1);
  if (variant == LMDG_STD) adjoint_grad_kernel<<<(nx + 255) / 256, 256, 0, s>>>(nx, P, h, eps, part, Phi, Lam, out);
  else adjoint_grad_lm_kernel<<<(nx + 255) / 256, 256, 0, s>>>(nx, P, h, eps, part, Phi, Lam, out);
  return cudaGetLastError();
}
cudaError_t fill_u32(unsigned *p, unsigned v, size_t N, cudaStream_t s) {
  add_launches(1);
  fill_u32_kernel<<<grid_for(N), 256, 0, s>>>(p, v, N);
  return cudaGetLastError();
}
cudaError_t psi_to_user(double *y, const void *x, int kind, int per, int ni, int nj, int nang, int nq, const int *perm,
                        cudaStream_t s) {
  const size_t N = (size_t)nang * ni * nj * per;
  add_launches(1);
  psi_to_user_kernel<<<grid_for(N), 256, 0, s>>>(y, x, kind, per, ni, nj, nang, nq, perm);
  return cudaGetLastError();
}

}  // namespace lmdg
