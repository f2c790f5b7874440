// Vertex diffusion correction: the right preconditioner of GMRES in the diffusive regime, with a geometric
// multigrid V-cycle on the mesh vertices.
//
// In the diffusive regime the source iteration behind the reduced operator K converges slowly on every mode up
// to the mesh scale; on them K ~ D_t^-1 D_a with D_a = -div D grad + eps sigma_a, D = 1/(3 sigma_t), so
// K^-1 ~ I + D_a^-1 (sigma_s/eps).  D_a is discretised as each scheme behaves in its diffusion limit (Section
// 3.1): continuous Q1 Galerkin for Q1-DG (eq-lmdg-cg), and continuous Q1 with the cell-averaged gradient for the
// low-memory schemes (eq-difflimPF, whose gradient part couples a vertex only to its diagonal neighbours), plus
// the consistent Q1 mass eps sigma_a and the vacuum boundary term A_n int d v (A_n the half-range outflow weight
// sum_{Omega.n > 0} w Omega.n of the side).  The paper leaves preconditioners to future work; this is the
// diffusion-synthetic construction written for its schemes.
//
// Vertex (I, J), I along x, of the (ni + 1) x (nj + 1) vertices of ni x nj cells has index J (ni + 1) + I.
// Operators are nine-point stencils of bs x bs blocks, A[v][k][r][c] with k = (dJ + 1) * 3 + (dI + 1) the
// neighbour (I + dI, J + dJ).  Levels halve the cells along x and y while both numbers are even and above 2.
// Prolongation is bilinear per component; for the cell-average stiffness the first coarsening carries two
// components per coarse vertex, P = [P_bl, C P_bl] with
// C = diag((-1)^(I+J)) (its gradient part leaves the two lattices I + J even / odd decoupled, so functions smooth
// on each lattice are what the coarse space must hold).  Coarse operators are Galerkin products P^T A P computed
// on the device, one coarse vertex per thread in a fixed order.  Smoothing: nu damped block-Jacobi steps before
// and after the coarse correction; the coarsest level is solved with a dense inverse (formed on the host at
// setup) when it has at most kMaxDense unknowns, else with damped-Jacobi steps.
#include <cmath>
#include <cstring>
#include <vector>

#include "lmdg_internal.h"

namespace lmdg {

namespace {

// element matrices on the bilinear corner functions of a square cell, corners (0,0), (1,0), (0,1), (1,1)
__constant__ double c_kfull[16] = {4 / 6.0, -1 / 6.0, -1 / 6.0, -2 / 6.0, -1 / 6.0, 4 / 6.0, -2 / 6.0, -1 / 6.0,
                                   -1 / 6.0, -2 / 6.0, 4 / 6.0, -1 / 6.0, -2 / 6.0, -1 / 6.0, -1 / 6.0, 4 / 6.0};
__constant__ double c_kavg[16] = {0.5, 0, 0, -0.5, 0, 0.5, -0.5, 0, 0, -0.5, 0.5, 0, -0.5, 0, 0, 0.5};
__constant__ double c_mass[16] = {4 / 36.0, 2 / 36.0, 2 / 36.0, 1 / 36.0, 2 / 36.0, 4 / 36.0, 1 / 36.0, 2 / 36.0,
                                  2 / 36.0, 1 / 36.0, 4 / 36.0, 2 / 36.0, 1 / 36.0, 2 / 36.0, 2 / 36.0, 4 / 36.0};

constexpr int kBlock = 256;
inline int grid_of(long long n) { return (int)((n + kBlock - 1) / kBlock); }

// Fine-level row of vertex (I, J): the cells around it (corner a of cell (i, j)), every other corner b of those
// cells, then the boundary edges through the vertex.
__global__ void fine_matrix_kernel(int ni, int nj, double h, double eps, const double *__restrict__ sigt,
                                   const double *__restrict__ sigma_a, double Ax, double Ay, int avg,
                                   double *__restrict__ A) {
  const int nv = ni + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv * (nj + 1)) return;
  const int I = v % nv, J = v / nv;
  double row[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) row[k] = 0.0;
  const double *Ke = avg ? c_kavg : c_kfull;
  for (int cj = 0; cj < 2; ++cj)
    for (int ci = 0; ci < 2; ++ci) {
      const int i = I - 1 + ci, j = J - 1 + cj;           // cell whose corner (1 - ci, 1 - cj) is this vertex
      if (i < 0 || i >= ni || j < 0 || j >= nj) continue;
      const size_t K = (size_t)j * ni + i;
      const double D = 1.0 / (3.0 * sigt[K]);
      const double m = eps * sigma_a[K] * h * h;
      const int a = (1 - ci) + 2 * (1 - cj);
      for (int b = 0; b < 4; ++b) {
        const int dI = (b & 1) - (1 - ci), dJ = (b >> 1) - (1 - cj);
        row[(dJ + 1) * 3 + (dI + 1)] += D * Ke[a * 4 + b] + m * c_mass[a * 4 + b];
      }
    }
  // boundary edges: A_n h (2 1; 1 2) / 6 on the edge's two vertices
  const double e2 = h * 2.0 / 6.0, e1 = h / 6.0;
  if (J == 0 || J == nj) {    // south / north side: edges (I-1, I) and (I, I+1)
    if (I > 0) { row[4] += Ay * e2; row[3] += Ay * e1; }
    if (I < ni) { row[4] += Ay * e2; row[5] += Ay * e1; }
  }
  if (I == 0 || I == ni) {    // west / east side
    if (J > 0) { row[4] += Ax * e2; row[1] += Ax * e1; }
    if (J < nj) { row[4] += Ax * e2; row[7] += Ax * e1; }
  }
  double *o = A + (size_t)v * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[k] = row[k];
}

// interpolation weight of fine coordinate f from coarse coordinate c (1, 1/2 or 0)
__device__ __forceinline__ double w1d(int f, int c) {
  const int d = f - 2 * c;
  return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);
}

// T(f): bsf x bsc block of the prolongation at fine vertex f; identity, or [1, (-1)^(I+J)] when split
__device__ __forceinline__ double tval(int split, int r, int c, int I, int J) {
  if (split) return c == 0 ? 1.0 : (((I + J) & 1) ? -1.0 : 1.0);
  return r == c ? 1.0 : 0.0;
}

// Galerkin product, one coarse vertex C per thread: Ac[C][C'] = sum over fine f1 near 2C and its stencil
// neighbours f2 of w(f1, C) w(f2, C') T(f1)^T A[f1][f2] T(f2).
template <int BSF, int BSC>
__global__ void galerkin_kernel(int nfi, int nfj, const double *__restrict__ Af, int nci, int ncj,
                                double *__restrict__ Ac) {
  constexpr int split = (BSF == 1 && BSC == 2) ? 1 : 0;
  const int nvf = nfi + 1, nvc = nci + 1;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= nvc * (ncj + 1)) return;
  const int CI = C % nvc, CJ = C / nvc;
  double acc[9][BSC][BSC];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int r = 0; r < BSC; ++r)
#pragma unroll
      for (int c = 0; c < BSC; ++c) acc[k][r][c] = 0.0;
  for (int b1 = -1; b1 <= 1; ++b1)
    for (int a1 = -1; a1 <= 1; ++a1) {
      const int I1 = 2 * CI + a1, J1 = 2 * CJ + b1;
      if (I1 < 0 || I1 > nfi || J1 < 0 || J1 > nfj) continue;
      const double wa = (a1 == 0 ? 1.0 : 0.5) * (b1 == 0 ? 1.0 : 0.5);
      const double *Arow = Af + (size_t)(J1 * nvf + I1) * 9 * BSF * BSF;
      for (int k = 0; k < 9; ++k) {
        const int I2 = I1 + (k % 3) - 1, J2 = J1 + (k / 3) - 1;
        if (I2 < 0 || I2 > nfi || J2 < 0 || J2 > nfj) continue;
        const double *Ab = Arow + k * BSF * BSF;
        // M = T(f1)^T A_blk T(f2)  (BSC x BSC)
        double M[BSC][BSC];
#pragma unroll
        for (int r = 0; r < BSC; ++r)
#pragma unroll
          for (int c = 0; c < BSC; ++c) {
            double s = 0.0;
#pragma unroll
            for (int p = 0; p < BSF; ++p)
#pragma unroll
              for (int q = 0; q < BSF; ++q)
                s += tval(split, p, r, I1, J1) * Ab[p * BSF + q] * tval(split, q, c, I2, J2);
            M[r][c] = s;
          }
        // coarse vertices interpolating f2
        const int cx0 = I2 >> 1, cy0 = J2 >> 1;
        for (int cy = cy0; cy <= cy0 + (J2 & 1); ++cy)
          for (int cx = cx0; cx <= cx0 + (I2 & 1); ++cx) {
            const double wb = w1d(I2, cx) * w1d(J2, cy);
            const int kk = (cy - CJ + 1) * 3 + (cx - CI + 1);
#pragma unroll
            for (int r = 0; r < BSC; ++r)
#pragma unroll
              for (int c = 0; c < BSC; ++c) acc[kk][r][c] += wa * wb * M[r][c];
          }
      }
    }
  double *o = Ac + (size_t)C * 9 * BSC * BSC;
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int r = 0; r < BSC; ++r)
#pragma unroll
      for (int c = 0; c < BSC; ++c) o[(k * BSC + r) * BSC + c] = acc[k][r][c];
}

// inverse of the diagonal block of every vertex
template <int BS>
__global__ void dinv_kernel(int nvv, const double *__restrict__ A, double *__restrict__ dinv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvv) return;
  const double *d = A + ((size_t)v * 9 + 4) * BS * BS;
  if (BS == 1) {
    dinv[v] = 1.0 / d[0];
  } else {
    const double det = d[0] * d[3] - d[1] * d[2];
    double *o = dinv + (size_t)v * 4;
    o[0] = d[3] / det; o[1] = -d[1] / det; o[2] = -d[2] / det; o[3] = d[0] / det;
  }
}

// (A x)_v for one vertex
template <int BS>
__device__ __forceinline__ void stencil_apply(int ni, int nj, int I, int J, const double *__restrict__ Arow,
                                              const double *__restrict__ x, double *out) {
  const int nv = ni + 1;
#pragma unroll
  for (int r = 0; r < BS; ++r) out[r] = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int I2 = I + (k % 3) - 1, J2 = J + (k / 3) - 1;
    if (I2 < 0 || I2 > ni || J2 < 0 || J2 > nj) continue;
    const double *xv = x + (size_t)(J2 * nv + I2) * BS;
    const double *Ab = Arow + k * BS * BS;
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) out[r] += Ab[r * BS + c] * xv[c];
  }
}

// x_out = x_in + omega Dinv (b - A x_in); x_in = null means zero
template <int BS>
__global__ void jacobi_kernel(int ni, int nj, const double *__restrict__ A, const double *__restrict__ dinv,
                              const double *__restrict__ b, const double *__restrict__ xin, double *__restrict__ xout,
                              double omega) {
  const int nv = ni + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv * (nj + 1)) return;
  double r[BS];
  if (xin) {
    double ax[BS];
    stencil_apply<BS>(ni, nj, v % nv, v / nv, A + (size_t)v * 9 * BS * BS, xin, ax);
#pragma unroll
    for (int q = 0; q < BS; ++q) r[q] = b[(size_t)v * BS + q] - ax[q];
  } else {
#pragma unroll
    for (int q = 0; q < BS; ++q) r[q] = b[(size_t)v * BS + q];
  }
  const double *di = dinv + (size_t)v * BS * BS;
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < BS; ++c) s += di[q * BS + c] * r[c];
    xout[(size_t)v * BS + q] = (xin ? xin[(size_t)v * BS + q] : 0.0) + omega * s;
  }
}

template <int BS>
__global__ void residual_kernel(int ni, int nj, const double *__restrict__ A, const double *__restrict__ b,
                                const double *__restrict__ x, double *__restrict__ r) {
  const int nv = ni + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv * (nj + 1)) return;
  double ax[BS];
  stencil_apply<BS>(ni, nj, v % nv, v / nv, A + (size_t)v * 9 * BS * BS, x, ax);
#pragma unroll
  for (int q = 0; q < BS; ++q) r[(size_t)v * BS + q] = b[(size_t)v * BS + q] - ax[q];
}

// bc[C] = sum over fine f near 2C of w(f, C) T(f)^T r[f]
template <int BSF, int BSC>
__global__ void restrict_kernel(int nfi, int nfj, const double *__restrict__ r, int nci, int ncj,
                                double *__restrict__ bc) {
  constexpr int split = (BSF == 1 && BSC == 2) ? 1 : 0;
  const int nvf = nfi + 1, nvc = nci + 1;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= nvc * (ncj + 1)) return;
  const int CI = C % nvc, CJ = C / nvc;
  double acc[BSC];
#pragma unroll
  for (int c = 0; c < BSC; ++c) acc[c] = 0.0;
  for (int b1 = -1; b1 <= 1; ++b1)
    for (int a1 = -1; a1 <= 1; ++a1) {
      const int I = 2 * CI + a1, J = 2 * CJ + b1;
      if (I < 0 || I > nfi || J < 0 || J > nfj) continue;
      const double w = (a1 == 0 ? 1.0 : 0.5) * (b1 == 0 ? 1.0 : 0.5);
      const double *rv = r + (size_t)(J * nvf + I) * BSF;
#pragma unroll
      for (int c = 0; c < BSC; ++c) {
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < BSF; ++p) s += tval(split, p, c, I, J) * rv[p];
        acc[c] += w * s;
      }
    }
#pragma unroll
  for (int c = 0; c < BSC; ++c) bc[(size_t)C * BSC + c] = acc[c];
}

// x[f] += sum over coarse C interpolating f of w(f, C) T(f) xc[C]
template <int BSF, int BSC>
__global__ void prolong_kernel(int nfi, int nfj, double *__restrict__ x, int nci, const double *__restrict__ xc) {
  constexpr int split = (BSF == 1 && BSC == 2) ? 1 : 0;
  const int nvf = nfi + 1, nvc = nci + 1;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nvf * (nfj + 1)) return;
  const int I = f % nvf, J = f / nvf;
  double acc[BSF];
#pragma unroll
  for (int p = 0; p < BSF; ++p) acc[p] = 0.0;
  const int cx0 = I >> 1, cy0 = J >> 1;
  for (int cy = cy0; cy <= cy0 + (J & 1); ++cy)
    for (int cx = cx0; cx <= cx0 + (I & 1); ++cx) {
      const double w = w1d(I, cx) * w1d(J, cy);
      const double *xv = xc + (size_t)(cy * nvc + cx) * BSC;
#pragma unroll
      for (int p = 0; p < BSF; ++p) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < BSC; ++c) s += tval(split, p, c, I, J) * xv[c];
        acc[p] += w * s;
      }
    }
#pragma unroll
  for (int p = 0; p < BSF; ++p) x[(size_t)f * BSF + p] += acc[p];
}

// x = inv b, one warp per row (rows of inv contiguous)
__global__ void dense_apply_kernel(int N, const double *__restrict__ inv, const double *__restrict__ b,
                                   double *__restrict__ x) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N) return;
  double s = 0.0;
  for (int c = lane; c < N; c += 32) s += inv[(size_t)row * N + c] * b[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = s;
}

// f_v = sum over the cells K touching v of (sigma_s/eps)_K int_K u_K phi_v, with int_K b_m phi_c =
// h^2/4 (1, cx/3, cy/3, cx cy/9) for the corner c = (cx, cy) of the reference square; lowmem: u holds (X0, X1)
// and the scalar-flux slopes are -X1
__global__ void load_kernel(int ni, int nj, double h, const double *__restrict__ sse, const double *__restrict__ u,
                            int lowmem, double *__restrict__ f) {
  const int nv = ni + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv * (nj + 1)) return;
  const int I = v % nv, J = v / nv;
  const double q = 0.25 * h * h, sg = lowmem ? -1.0 : 1.0;
  double s = 0.0;
  for (int cj = 0; cj < 2; ++cj)
    for (int ci = 0; ci < 2; ++ci) {
      const int i = I - 1 + ci, j = J - 1 + cj;
      if (i < 0 || i >= ni || j < 0 || j >= nj) continue;
      const size_t K = (size_t)j * ni + i;
      const double cx = ci ? -1.0 : 1.0, cy = cj ? -1.0 : 1.0;   // corner of cell K at this vertex
      const double *uk = u + 4 * K;
      s += sse[K] * q * (uk[0] + sg * (uk[1] * cx / 3.0 + uk[2] * cy / 3.0 + uk[3] * cx * cy / 9.0));
    }
  f[v] = s;
}

// u += Legendre moments of the bilinear interpolant of d (slopes subtracted for the low-memory unknowns)
__global__ void interp_add_kernel(int ni, int nj, const double *__restrict__ d, int lowmem, double *__restrict__ u) {
  const int nv = ni + 1;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= ni * nj) return;
  const int i = K % ni, j = K / ni;
  const double d00 = d[(size_t)j * nv + i], d10 = d[(size_t)j * nv + i + 1];
  const double d01 = d[(size_t)(j + 1) * nv + i], d11 = d[(size_t)(j + 1) * nv + i + 1];
  const double sg = lowmem ? -1.0 : 1.0;
  double *o = u + 4 * (size_t)K;
  o[0] += (d00 + d10 + d01 + d11) / 4.0;
  o[1] += sg * ((-d00 + d10 - d01 + d11) / 4.0);
  o[2] += sg * ((-d00 - d10 + d01 + d11) / 4.0);
  o[3] += sg * ((d00 - d10 - d01 + d11) / 4.0);
}

size_t nvert(const MgLevel &L) { return (size_t)(L.ni + 1) * (L.nj + 1); }

// Gauss-Jordan inverse with partial pivoting (host, coarsest level only)
bool dense_inverse(std::vector<double> &a, int N) {
  std::vector<double> inv((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) inv[(size_t)i * N + i] = 1.0;
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (std::fabs(a[(size_t)r * N + c]) > std::fabs(a[(size_t)p * N + c])) p = r;
    if (a[(size_t)p * N + c] == 0.0) return false;
    if (p != c)
      for (int k = 0; k < N; ++k) {
        std::swap(a[(size_t)p * N + k], a[(size_t)c * N + k]);
        std::swap(inv[(size_t)p * N + k], inv[(size_t)c * N + k]);
      }
    const double piv = 1.0 / a[(size_t)c * N + c];
    for (int k = 0; k < N; ++k) { a[(size_t)c * N + k] *= piv; inv[(size_t)c * N + k] *= piv; }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * N + c];
      if (f == 0.0) continue;
      for (int k = 0; k < N; ++k) {
        a[(size_t)r * N + k] -= f * a[(size_t)c * N + k];
        inv[(size_t)r * N + k] -= f * inv[(size_t)c * N + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

template <int BS>
cudaError_t jacobi(const MgLevel &L, const double *b, const double *xin, double *xout, double omega, cudaStream_t s) {
  add_launches(1);
  jacobi_kernel<BS><<<grid_of((long long)nvert(L)), kBlock, 0, s>>>(L.ni, L.nj, L.A, L.dinv, b, xin, xout, omega);
  return cudaGetLastError();
}

// steps damped-Jacobi steps on level L into x, from zero or from x; they ping-pong through L.y and end in x
cudaError_t smooth(const MgLevel &L, const double *b, double *x, bool from_zero, int steps, double omega,
                   cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < steps; ++k) {
    const double *in = (k == 0 && from_zero) ? nullptr : ((k % 2 == 0) ? x : L.y);
    double *out = (k % 2 == 0) ? L.y : x;
    e = L.bs == 1 ? jacobi<1>(L, b, in, out, omega, s) : jacobi<2>(L, b, in, out, omega, s);
    if (e != cudaSuccess) return e;
  }
  if (steps % 2 == 1) e = cudaMemcpyAsync(x, L.y, sizeof(double) * nvert(L) * L.bs, cudaMemcpyDeviceToDevice, s);
  return e;
}

cudaError_t vcycle(const VertexDsa &d, int l, cudaStream_t s) {
  const MgLevel &L = d.lev[l];
  cudaError_t e;
  if (l == d.nlev) {   // coarsest: x = A^-1 b
    if (d.cinv) {
      const int N = (int)(nvert(L) * L.bs);
      add_launches(1);
      dense_apply_kernel<<<(N + 7) / 8, 256, 0, s>>>(N, d.cinv, L.b, L.x);
      return cudaGetLastError();
    }
    return smooth(L, L.b, L.x, true, d.coarse_sweeps, d.omega, s);
  }
  const MgLevel &Cl = d.lev[l + 1];
  if ((e = smooth(L, L.b, L.x, true, d.nu, d.omega, s)) != cudaSuccess) return e;
  add_launches(2);
  const int gf = grid_of((long long)nvert(L)), gc = grid_of((long long)nvert(Cl));
  if (L.bs == 1) residual_kernel<1><<<gf, kBlock, 0, s>>>(L.ni, L.nj, L.A, L.b, L.x, L.r);
  else residual_kernel<2><<<gf, kBlock, 0, s>>>(L.ni, L.nj, L.A, L.b, L.x, L.r);
  if (L.bs == 1 && Cl.bs == 1) restrict_kernel<1, 1><<<gc, kBlock, 0, s>>>(L.ni, L.nj, L.r, Cl.ni, Cl.nj, Cl.b);
  else if (L.bs == 1) restrict_kernel<1, 2><<<gc, kBlock, 0, s>>>(L.ni, L.nj, L.r, Cl.ni, Cl.nj, Cl.b);
  else restrict_kernel<2, 2><<<gc, kBlock, 0, s>>>(L.ni, L.nj, L.r, Cl.ni, Cl.nj, Cl.b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = vcycle(d, l + 1, s)) != cudaSuccess) return e;
  add_launches(1);
  if (L.bs == 1 && Cl.bs == 1) prolong_kernel<1, 1><<<gf, kBlock, 0, s>>>(L.ni, L.nj, L.x, Cl.ni, Cl.x);
  else if (L.bs == 1) prolong_kernel<1, 2><<<gf, kBlock, 0, s>>>(L.ni, L.nj, L.x, Cl.ni, Cl.x);
  else prolong_kernel<2, 2><<<gf, kBlock, 0, s>>>(L.ni, L.nj, L.x, Cl.ni, Cl.x);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return smooth(L, L.b, L.x, false, d.nu, d.omega, s);   // post-smoothing from the corrected x
}

}  // namespace

void dsa_free(VertexDsa &d) {
  for (auto &L : d.lev) {
    lmdg::dfree(L.A); lmdg::dfree(L.dinv); lmdg::dfree(L.x); lmdg::dfree(L.y); lmdg::dfree(L.b); lmdg::dfree(L.r);
    L = MgLevel();
  }
  lmdg::dfree(d.cinv);
  d.cinv = nullptr;
  if (d.vcycle_graph) cudaGraphExecDestroy(d.vcycle_graph);
  d.vcycle_graph = nullptr;
  d.nlev = -1;
}

int dsa_build(VertexDsa &d, int avg, int ni, int nj, double h, double eps, const double *sigt, const double *sigma_a,
              double Ax, double Ay, cudaStream_t s) {
  dsa_free(d);
  d.avg = avg;
  int nl = 0, bs = 1, ci = ni, cj = nj;
  while (true) {
    if (nl >= kMaxMgLevels) return LMDG_ERR_ARG;
    MgLevel &L = d.lev[nl];
    L.ni = ci; L.nj = cj; L.bs = bs;
    const size_t nv = nvert(L);
    if (lmdg::dmalloc(&L.A, sizeof(double) * nv * 9 * bs * bs) != cudaSuccess ||
        lmdg::dmalloc(&L.dinv, sizeof(double) * nv * bs * bs) != cudaSuccess ||
        lmdg::dmalloc(&L.x, sizeof(double) * nv * bs) != cudaSuccess ||
        lmdg::dmalloc(&L.y, sizeof(double) * nv * bs) != cudaSuccess ||
        lmdg::dmalloc(&L.b, sizeof(double) * nv * bs) != cudaSuccess ||
        lmdg::dmalloc(&L.r, sizeof(double) * nv * bs) != cudaSuccess)
      return LMDG_ERR_NOMEM;
    const int gv = grid_of((long long)nv);
    add_launches(2);
    if (nl == 0) {
      fine_matrix_kernel<<<gv, kBlock, 0, s>>>(ci, cj, h, eps, sigt, sigma_a, Ax, Ay, avg, L.A);
    } else {
      const MgLevel &F = d.lev[nl - 1];
      if (F.bs == 1 && bs == 1) galerkin_kernel<1, 1><<<gv, kBlock, 0, s>>>(F.ni, F.nj, F.A, ci, cj, L.A);
      else if (F.bs == 1) galerkin_kernel<1, 2><<<gv, kBlock, 0, s>>>(F.ni, F.nj, F.A, ci, cj, L.A);
      else galerkin_kernel<2, 2><<<gv, kBlock, 0, s>>>(F.ni, F.nj, F.A, ci, cj, L.A);
    }
    if (bs == 1) dinv_kernel<1><<<gv, kBlock, 0, s>>>((int)nv, L.A, L.dinv);
    else dinv_kernel<2><<<gv, kBlock, 0, s>>>((int)nv, L.A, L.dinv);
    if (cudaGetLastError() != cudaSuccess) return LMDG_ERR_CUDA;
    if (ci % 2 != 0 || cj % 2 != 0 || ci <= 2 || cj <= 2) break;
    ci /= 2;
    cj /= 2;
    if (nl == 0 && avg) bs = 2;
    ++nl;
  }
  d.nlev = nl;
  // coarsest level: dense inverse from the host when small enough
  const MgLevel &Lc = d.lev[nl];
  const int N = (int)(nvert(Lc) * Lc.bs);
  if (N <= kMaxDense) {
    const int bsc = Lc.bs, nvi = Lc.ni + 1, nvj = Lc.nj + 1;
    std::vector<double> st(nvert(Lc) * 9 * bsc * bsc), M((size_t)N * N, 0.0);
    if (cudaMemcpyAsync(st.data(), Lc.A, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LMDG_ERR_CUDA;
    for (int v = 0; v < nvi * nvj; ++v) {
      const int I = v % nvi, J = v / nvi;
      for (int k = 0; k < 9; ++k) {
        const int I2 = I + k % 3 - 1, J2 = J + k / 3 - 1;
        if (I2 < 0 || I2 >= nvi || J2 < 0 || J2 >= nvj) continue;
        const int v2 = J2 * nvi + I2;
        for (int r = 0; r < bsc; ++r)
          for (int c = 0; c < bsc; ++c)
            M[(size_t)(v * bsc + r) * N + v2 * bsc + c] = st[((size_t)v * 9 + k) * bsc * bsc + r * bsc + c];
      }
    }
    if (!dense_inverse(M, N)) return LMDG_ERR_BREAKDOWN;
    if (lmdg::dmalloc(&d.cinv, sizeof(double) * M.size()) != cudaSuccess) return LMDG_ERR_NOMEM;
    if (cudaMemcpyAsync(d.cinv, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return LMDG_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return LMDG_ERR_CUDA;
  // The V-cycle is the same sequence of about 7 launches per level on fixed buffers (lev[0].b in, lev[0].x out)
  // every time: capture it once on a private stream and replay it as one graph launch, so the coarse levels' tiny
  // kernels do not each pay a launch.  If capture is not available the cycle is launched kernel by kernel.
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
    cudaGraph_t g = nullptr;
    const long long l0 = launch_count();
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const cudaError_t ev = vcycle(d, 0, cs);
      ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && ev == cudaSuccess && g != nullptr;
    }
    d.vcycle_launches = launch_count() - l0;
    add_launches(-d.vcycle_launches);          // counted when replayed
    if (ok && cudaGraphInstantiate(&d.vcycle_graph, g, 0) != cudaSuccess) d.vcycle_graph = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();                        // a refused capture leaves no error behind: the fallback runs
  }
  return 0;
}

cudaError_t dsa_apply(const VertexDsa &d, int ni, int nj, double h, const double *sse, int lowmem, double *u,
                      cudaStream_t s) {
  const MgLevel &L0 = d.lev[0];
  add_launches(1);
  load_kernel<<<grid_of((long long)nvert(L0)), kBlock, 0, s>>>(ni, nj, h, sse, u, lowmem, L0.b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d.vcycle_graph) {                                 // one V-cycle from zero
    add_launches(d.vcycle_launches);
    if ((e = cudaGraphLaunch(d.vcycle_graph, s)) != cudaSuccess) return e;
  } else if ((e = vcycle(d, 0, s)) != cudaSuccess) {
    return e;
  }
  add_launches(1);
  interp_add_kernel<<<grid_of((long long)ni * nj), kBlock, 0, s>>>(ni, nj, L0.x, lowmem, u);
  return cudaGetLastError();
}

}  // namespace lmdg
