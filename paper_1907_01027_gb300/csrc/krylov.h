// Host wrappers of the Krylov vector kernels (krylov.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace lmdg {
// out[i] (+)= sum_k V_i[k] w[k], i < nv (N and ldv even); partial needs mdot_partial_len(nv) doubles
cudaError_t mdot(const double *V, size_t ldv, int nv, const double *w, size_t N, double *partial, double *out,
                 int accumulate, cudaStream_t s);
size_t mdot_partial_len(int nvmax);
// w -= sum_i V_i coef_i (coef on the device, nv <= 128; N and ldv even)
cudaError_t maxpy(double *w, const double *V, size_t ldv, int nv, const double *coef, size_t N, cudaStream_t s);
// y = x / sqrt(*nrm2) (N even)
cudaError_t scale_by_inv(double *y, const double *x, const double *nrm2, size_t N, cudaStream_t s);
// y = a x + b y
cudaError_t axpby(double *y, double a, const double *x, double b, size_t N, cudaStream_t s);
// y = diag(I, 1/dinv)^-1 x on [nx][4] (mode 1) or y = x (mode 0); dinv = reciprocal diagonal
cudaError_t precond(double *y, const double *x, const double *dinv, int nx, int mode, cudaStream_t s);
// y = B11 u on [nx][3] (ni x nj cells); A4 = {Ax+, Ax-, Ay+, Ay-}
cudaError_t b11_apply(int ni, int nj, double h, double eps, const double *sigma_a, const double *A4, const double *u,
                      double *y, cudaStream_t s);
// out[0..nx) = dJ/dsigma_s, out[nx..2nx) = dJ/dsigma_a, out[2nx..3nx) = dJ/dq; Phi, Lam: forward and adjoint
// reduced solutions (standard) or scalar-flux moments (low-memory)
cudaError_t adjoint_gradients(int variant, int nx, int P, double h, double eps, const double *part,
                              const double *Phi, const double *Lam, double *out, cudaStream_t s);
// x[4K + q] = (q == r) for every cell K < nx: one unit Legendre moment in every cell
cudaError_t unit_vectors(double *x, int nx, int r, cudaStream_t s);
// binv[K] = B_K^-1 with B_K[q][r] = y_r[4K + q] (Gauss-Jordan elimination with partial pivoting, FP64); cells
// whose block has no usable pivot add 1 to *bad (zeroed here first) and get the identity
cudaError_t block_inverses(const double *y0, const double *y1, const double *y2, const double *y3, int nx,
                           double *binv, unsigned *bad, cudaStream_t s);
// y += binv x - J x per cell, J = diag(I, 1/dinv)^-1 (mode 1) or the identity (mode 0): turns J x + C(J x) into the
// cell-block step B^-1 x + C(J x)
cudaError_t block_step(double *y, const double *x, const double *binv, const double *dinv, int nx, int mode,
                       cudaStream_t s);
// p[0..N) = v
cudaError_t fill_u32(unsigned *p, unsigned v, size_t N, cudaStream_t s);
// stored psi (one wavefront-ordered plane per direction, psi_slot; kind 0 double, 1 float, 2 bfloat16; per values
// per slot) to the user layout [u][nj*ni][per] in double; perm maps sorted to user directions, nq per quadrant
cudaError_t psi_to_user(double *y, const void *x, int kind, int per, int ni, int nj, int nang, int nq, const int *perm,
                        cudaStream_t s);
}  // namespace lmdg
