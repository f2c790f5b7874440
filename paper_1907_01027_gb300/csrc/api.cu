// C ABI of liblmdg: problem setup, sweeps, GMRES solve with FP64 or mixed-precision iterative refinement,
// B11 apply/CG, and the angular-flux store.  See include/lmdg.h for the contract of every entry point.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lmdg_internal.h"
#include "krylov.h"

using namespace lmdg;

namespace {

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return LMDG_ERR_CUDA;   \
  } while (0)

int quadrant(double ox, double oy) { return oy > 0 ? (ox > 0 ? 0 : 1) : (ox < 0 ? 2 : 3); }

// n host doubles to a new device array of T (converted on the host when T is not double)
template <typename T>
int upload(T **dst, const double *src, size_t n) {
  if (lmdg::dmalloc(dst, sizeof(T) * std::max<size_t>(1, n)) != cudaSuccess) return LMDG_ERR_NOMEM;
  if (n == 0) return 0;
  if constexpr (std::is_same<T, double>::value) {
    CK(cudaMemcpy(*dst, src, sizeof(double) * n, cudaMemcpyHostToDevice));
  } else {
    std::vector<T> tmp(src, src + n);
    CK(cudaMemcpy(*dst, tmp.data(), sizeof(T) * n, cudaMemcpyHostToDevice));
  }
  return 0;
}
template <typename T>
int upload(T **dst, const std::vector<double> &src) {
  return upload(dst, src.data(), src.size());
}

template <typename T>
void free_pd(ProblemData<T> &p) {
  lmdg::dfree(p.ox); lmdg::dfree(p.oy); lmdg::dfree(p.w); lmdg::dfree(p.sigt); lmdg::dfree(p.sse); lmdg::dfree(p.q);
  lmdg::dfree(p.alpha);
  p = ProblemData<T>();
}


// Add the device time of the last recorded sweep launch to its precision's total (after a synchronisation,
// or waiting for it when wait is set).
void harvest(lmdg_ctx *c, bool wait) {
  if (c->ev_pending < 0) return;
  if (wait) cudaEventSynchronize(c->ev1);
  float ms = 0;
  if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->sweep_ms[c->ev_pending] += ms;
  c->ev_pending = -1;
}

// Float-float copies of the problem data and coefficient tables, made from the FP64 ones on the first
// float-float sweep.
int ensure_f2(lmdg_ctx *c, cudaStream_t s) {
  if (c->f2_ready) return 0;
  const size_t na = c->nang, nx = c->nx;
  const size_t nq = c->q_layout == 2 ? na * nx * 4 : nx * 4;
  const size_t nal = c->has_alpha ? na * 2 * (size_t)(c->ni + c->nj) * 2 : 0;
  const size_t ntab = c->coef ? (size_t)c->nmat * c->ncls * c->ncoef : 0;
  struct Item { const double *src; f2 **dst; size_t n; } items[] = {
      {c->d64.ox, &c->d2.ox, na}, {c->d64.oy, &c->d2.oy, na}, {c->d64.w, &c->d2.w, na},
      {c->d64.sigt, &c->d2.sigt, nx}, {c->d64.sse, &c->d2.sse, nx}, {c->d64.q, &c->d2.q, nq},
      {c->d64.alpha, &c->d2.alpha, nal}, {c->p1ra64, &c->p1ra2, 3 * nx}, {c->coef, &c->coef2, ntab}};
  // a failed allocation leaves the arrays made so far in place (freed by lmdg_destroy) for the next attempt
  for (auto &it : items) {
    if (it.n == 0 || it.src == nullptr) continue;
    if (*it.dst == nullptr && lmdg::dmalloc(it.dst, sizeof(f2) * it.n) != cudaSuccess) {
      *it.dst = nullptr;
      return LMDG_ERR_NOMEM;
    }
    CK(convert_to_f2(it.src, *it.dst, it.n, s));
  }
  c->f2_ready = true;
  return 0;
}

// Angle sharding: the 4 * groups partial sets of a launch shape are split into nshards contiguous chunks of
// ceil(4 * groups / nshards) sets; shard r sweeps the directions of chunk r (empty for r beyond the sets).
struct ShardRange { int sets, chunk, pq0, npq; };
ShardRange shard_range(const SweepGeom &g, int shard, int nshards) {
  ShardRange r{};
  r.sets = 4 * g.groups;
  r.chunk = (r.sets + nshards - 1) / nshards;
  r.pq0 = std::min(r.sets, shard * r.chunk);
  r.npq = std::min(r.sets, (shard + 1) * r.chunk) - r.pq0;
  return r;
}

// One transport sweep with its angular reduction.  mode 0: sweep and epilogue (y = K x or K x - b).  mode 1: sweep
// the partial sets of chunk `shard` of nshards into ext (the full [chunks * chunk][nx][NR] layout, only this chunk
// written), no epilogue.  mode 2: epilogue only, from the partial sets in ext.
template <typename T>
int do_sweep(lmdg_ctx *c, const double *X, double *y, int source, bool store, int bf16, cudaStream_t s,
             int mode = 0, int shard = 0, int nshards = 1, void *ext = nullptr) {
  SweepArgs<T> a{};
  constexpr int P = prec_of<T>();
  const bool f64 = P == 0;
  if constexpr (P == 2) {
    if (store) return LMDG_ERR_ARG;   // float-float sweeps feed residuals only
    if (int e = ensure_f2(c, s)) return e;
  }
  a.ni = c->ni; a.nj = c->nj; a.nq = c->nq; a.nang = c->nang; a.nx = c->nx;
  a.h = (T)c->h; a.eps = (T)c->eps;
  a.g = P == 0 ? c->g64 : (P == 1 ? c->g32 : c->g2);
  if constexpr (P == 0) { a.pd = c->d64; a.p1ra = c->p1ra64; }
  else if constexpr (P == 1) { a.pd = c->d32; a.p1ra = c->p1ra32; }
  else { a.pd = c->d2; a.p1ra = c->p1ra2; }
  a.q_per_angle = c->q_layout == 2;
  a.X = X;
  a.source = source;
  const ShardRange sr = shard_range(a.g, shard, nshards);
  const size_t set_bytes = (size_t)c->nx * nr_of(c->kvar) * sizeof(T);
  a.pq0 = sr.pq0;
  a.npq = sr.npq;
  if (mode == 0) {
    // partial reductions of this launch shape and arithmetic: the buffer grows to the largest one used
    const size_t pbytes = (size_t)sr.sets * set_bytes;
    if (c->part_bytes < pbytes) {
      lmdg::dfree(c->part);
      c->part = nullptr;
      c->part_bytes = 0;
      if (lmdg::dmalloc(&c->part, pbytes) != cudaSuccess) { c->part = nullptr; return LMDG_ERR_NOMEM; }
      c->part_bytes = pbytes;
    }
  }
  a.part = reinterpret_cast<T *>(mode == 0 ? c->part : ext);
  a.perm = c->perm;
  a.ytr = reinterpret_cast<T *>(c->ytr);
  a.ctrl = c->ctrl;
  a.spin_limit = c->opt.spin_limit;
  a.cellsrc = reinterpret_cast<const T *>(c->cellsrc);
  a.cellsh = reinterpret_cast<const T *>(c->cellsh);
  a.corr = nullptr;
  a.rev = c->rev;
  if (c->use_adj) {
    if constexpr (P == 0) a.pd.q = c->qadj64;
    else if constexpr (P == 1) a.pd.q = c->qadj32;
    else a.pd.q = c->qadj2;
    a.pd.alpha = nullptr;
    a.q_per_angle = 0;
    a.p1ra = nullptr;
  }
  if constexpr (P == 0) a.corr = c->corr;
  a.supp = c->supp;
  if constexpr (P == 0) a.local = c->local_mode;
  a.coef = nullptr; a.ncoef = 0; a.ncls = 0; a.cls = nullptr; a.matsh = nullptr; a.mat = nullptr;
  // coefficient tables for the FP64 and float-float sweeps, where they replace reciprocals and Schur products;
  // the FP32 sweeps form the coefficients with the hardware reciprocal as fast as they would load them
  // (measured at 1024^2 S16)
  if (c->coef) {
    if constexpr (P == 0) a.coef = c->coef;
    else if constexpr (P == 2) a.coef = c->coef2;
    if (a.coef) { a.ncoef = c->ncoef; a.ncls = c->ncls; a.cls = c->cls; a.matsh = c->matsh; a.mat = c->mat; }
  }
  a.psi = nullptr;
  a.psi_bf16 = 0;
  if (c->no_store) store = false;
  if (store) {
    int kind = f64 ? 0 : (bf16 && c->variant != LMDG_STD ? 2 : 1);
    size_t per = c->variant == LMDG_STD ? 4 : 1;
    size_t elems = (size_t)c->nang * c->nx * per;   // user layout
    // storage: one plane of wavefront-ordered slots per direction (lmdg::psi_plane)
    const size_t bytes = (size_t)c->nang * lmdg::psi_plane(c->ni, c->nj) * per * (kind == 0 ? 8 : (kind == 1 ? 4 : 2));
    if (c->psi_bytes < bytes) {   // grown to the widest kind stored so far (cudaFree waits for earlier use)
      lmdg::dfree(c->psi);
      c->psi = nullptr;
      c->psi_bytes = 0;
      c->psi_kind = -1;
      if (lmdg::dmalloc(&c->psi, bytes) != cudaSuccess) { c->psi = nullptr; return LMDG_ERR_NOMEM; }
      c->psi_bytes = bytes;
    }
    c->psi_kind = kind;
    c->psi_elems = elems;
    a.psi = c->psi;
    a.psi_bf16 = kind == 2;
  }
  if (mode == 2) {
    // epilogue from the caller's partial sets
    CK(launch_epilogue<T>(c->kvar, c->nx, sr.sets, c->h, a.part, X, c->d64.sse, c->d64.sigt, c->qmom,
                          c->use_adj ? nullptr : c->p1ra64, c->use_adj ? nullptr : c->sq1, source, y, s));
    return 0;
  }
  if (!c->ev0) {
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
  }
  if (c->ev_pending >= 0) harvest(c, true);
  // the strip traces must hold the empty pattern: initially, after a change of precision (float words sit at
  // other offsets than double and float-float words) and after a sweep that stopped early
  const int want = P == 1 ? 1 : 0;
  if (c->ytr_dirty || c->ytr_prec != want) {
    if (fill_u32(reinterpret_cast<unsigned *>(c->ytr), kTraceEmpty, c->ytr_words, s) != cudaSuccess)
      return LMDG_ERR_CUDA;
    c->ytr_dirty = false;
    c->ytr_prec = want;
  }
  CK(cudaEventRecord(c->ev0, s));
  // a shard beyond the last set sweeps nothing; its error word is cleared all the same, so that the check after the
  // call does not report an earlier sweep's error
  if (a.npq > 0) CK(launch_sweep<T>(c->kvar, a, s));
  else CK(cudaMemsetAsync(c->ctrl, 0, 2 * sizeof(unsigned), s));
  CK(cudaEventRecord(c->ev1, s));
  c->ev_pending = P;
  c->part_prec = P;
  if (mode == 0) {
    // the adjoint problem has its own source (q_adj, vacuum inflow): no slope moments, no boundary terms
    CK(launch_epilogue<T>(c->kvar, c->nx, sr.sets, c->h, a.part, X, c->d64.sse, c->d64.sigt, c->qmom,
                          c->use_adj ? nullptr : c->p1ra64, c->use_adj ? nullptr : c->sq1, source, y, s));
  }
  if (P == 0) c->sweeps64++;
  else if (P == 1) c->sweeps32++;
  else c->sweeps2++;
  return 0;
}

// prec: 0 FP64, 1 FP32, 2 float-float
int sweep_prec(lmdg_ctx *c, int prec, const double *X, double *y, int source, bool store, int bf16,
               cudaStream_t s) {
  if (prec == 1) return do_sweep<float>(c, X, y, source, store, bf16, s);
  if (prec == 2) return do_sweep<f2>(c, X, y, source, store, 0, s);
  return do_sweep<double>(c, X, y, source, store, 0, s);
}

int check_error_word(lmdg_ctx *c, cudaStream_t s) {
  unsigned err = 0;
  CK(cudaMemcpyAsync(&err, c->ctrl + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  harvest(c, false);
  if (err) c->ytr_dirty = true;
  return err ? LMDG_ERR_TIMEOUT : 0;
}

// phi = scalar-flux moments from the partial reductions of the last sweep at X (low-memory variants):
// phi0 = P0 psi0, phi_r = -W_r + (P1 R psi0)_r (RLMDG, alpha part removed), W = X1 - z the GMRES unknown;
// P0-DG: phi0 only (no slopes).
template <typename T, int VAR>
__global__ void phi_kernel(int nx, int P, const T *__restrict__ part, const double *__restrict__ X,
                           const double *__restrict__ p1ra, double *__restrict__ phi) {
  constexpr int NR = nr_of(VAR);
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  double s[NR];
  for (int r = 0; r < NR; ++r) s[r] = 0;
  for (int p = 0; p < P; ++p)
    for (int r = 0; r < NR; ++r) s[r] += (double)part[((size_t)p * nx + K) * NR + r];
  const double *x = X + 4 * (size_t)K;
  double *o = phi + 4 * (size_t)K;
  o[0] = s[0];
  if (VAR == kP0) { o[1] = 0; o[2] = 0; o[3] = 0; return; }
  o[1] = -x[1]; o[2] = -x[2]; o[3] = -x[3];
  if (VAR == 2 || VAR == kRlmQ1) {
    o[1] += s[4] - (p1ra ? p1ra[3 * (size_t)K] : 0.0);
    o[2] += s[5] - (p1ra ? p1ra[3 * (size_t)K + 1] : 0.0);
  }
  if (VAR == kRlmQ1) o[3] += s[6] - (p1ra ? p1ra[3 * (size_t)K + 2] : 0.0);
}

template <typename T>
cudaError_t launch_phi(lmdg_ctx *c, const T *part, int Pn, const double *X, double *P, cudaStream_t s) {
  const int bs = 256, gs = (c->nx + bs - 1) / bs;
  add_launches(1);
  if (c->variant == LMDG_LM) phi_kernel<T, 1><<<gs, bs, 0, s>>>(c->nx, Pn, part, X, c->p1ra64, P);
  else if (c->variant == LMDG_P0) phi_kernel<T, kP0><<<gs, bs, 0, s>>>(c->nx, Pn, part, X, nullptr, P);
  else if (c->kvar == kRlmQ1) phi_kernel<T, kRlmQ1><<<gs, bs, 0, s>>>(c->nx, Pn, part, X, c->p1ra64, P);
  else phi_kernel<T, 2><<<gs, bs, 0, s>>>(c->nx, Pn, part, X, c->p1ra64, P);
  return cudaGetLastError();
}

int ensure_krylov(lmdg_ctx *c, int m) {
  const size_t N = 4 * (size_t)c->nx;
  if (c->V && c->red_len >= m + 2) return 0;
  lmdg::dfree(c->V);
  for (auto &v : c->vec) { lmdg::dfree(v); v = nullptr; }
  lmdg::dfree(c->red);
  if (c->red_h) cudaFreeHost(c->red_h);
  c->V = nullptr; c->red = nullptr; c->red_h = nullptr;
  if (lmdg::dmalloc(&c->V, sizeof(double) * N * (m + 1)) != cudaSuccess) return LMDG_ERR_NOMEM;
  for (auto &v : c->vec)
    if (lmdg::dmalloc(&v, sizeof(double) * N) != cudaSuccess) return LMDG_ERR_NOMEM;
  size_t rl = mdot_partial_len(m + 2) + 4 * (size_t)(m + 2);
  if (lmdg::dmalloc(&c->red, sizeof(double) * rl) != cudaSuccess) return LMDG_ERR_NOMEM;
  if (cudaMallocHost(&c->red_h, sizeof(double) * 4 * (m + 2)) != cudaSuccess) return LMDG_ERR_NOMEM;
  c->red_len = m + 2;
  return 0;
}

// ||v||^2 into *out_h (synchronises)
int norm2(lmdg_ctx *c, const double *v, double *out_h, cudaStream_t s) {
  const size_t N = 4 * (size_t)c->nx;
  double *partial = c->red, *out = c->red + mdot_partial_len(c->red_len);
  CK(mdot(v, N, 1, v, N, partial, out, 0, s));
  CK(cudaMemcpyAsync(out_h, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return 0;
}

// Per-cell tables of a problem, one thread per cell: sigma_t = sigma_s/eps + eps sigma_a and sigma_s/eps (FP64
// and FP32); the source moments (q_layout 0: qin [N] expanded to q64 [N][4]; FP32 copy for layouts 0 and 1, layout
// 2's is converted separately); the source part of Sigma Q1, eps h^2 D_r sum_l w_l q_l,r (layout 2: over the
// sorted directions); P1 r_alpha = 0 (the inflow terms are added per boundary face afterwards); and the reciprocal
// diagonal of B11, eps sigma_a h^2 D_r + (sum w |Omega_x|) h fx_r + (sum w |Omega_y|) h fy_r (the Jacobi scaling).
__global__ void cell_tables_kernel(size_t nx, double eps, double h, const double *__restrict__ ss,
                                   const double *__restrict__ sa, const double *qin, int q_layout, int nang,
                                   const double *__restrict__ w, double Axs, double Ays, double *__restrict__ sigt64,
                                   double *__restrict__ sse64, float *__restrict__ sigt32, float *__restrict__ sse32,
                                   double *q64, float *__restrict__ q32, double *__restrict__ sq1,
                                   double *__restrict__ p1ra, double *__restrict__ bdinv) {
  const size_t K = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double D[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0};
  const double fx[3] = {1.0, 1.0 / 3.0, 1.0 / 3.0}, fy[3] = {1.0 / 3.0, 1.0, 1.0 / 3.0};
  const double se = ss[K] / eps, st = se + eps * sa[K];
  sigt64[K] = st; sse64[K] = se; sigt32[K] = (float)st; sse32[K] = (float)se;
  double qs[3] = {0, 0, 0};
  if (q_layout == 0) {
    const double q0 = qin[K];
    q64[4 * K] = q0; q64[4 * K + 1] = 0; q64[4 * K + 2] = 0; q64[4 * K + 3] = 0;
    q32[4 * K] = (float)q0; q32[4 * K + 1] = 0; q32[4 * K + 2] = 0; q32[4 * K + 3] = 0;
  } else if (q_layout == 1) {
    for (int r = 0; r < 4; ++r) q32[4 * K + r] = (float)q64[4 * K + r];
    for (int r = 0; r < 3; ++r) qs[r] = q64[4 * K + 1 + r];
  } else {
    for (int l = 0; l < nang; ++l)
      for (int r = 0; r < 3; ++r) qs[r] += w[l] * q64[((size_t)l * nx + K) * 4 + 1 + r];
  }
  for (int r = 0; r < 3; ++r) {
    sq1[3 * K + r] = eps * h * h * D[r] * qs[r];
    p1ra[3 * K + r] = 0.0;
    bdinv[3 * K + r] = 1.0 / (eps * sa[K] * h * h * D[r] + Axs * h * fx[r] + Ays * h * fy[r]);
  }
}

// Adds the inflow terms summed per boundary face (bnd[face][6]: Sigma Q1 r = 1..3, P1 r_alpha r = 1..3; faces
// west, east by row, south, north by column) to the face's cell, for one side
__global__ void boundary_terms_kernel(int ni, int nj, int side, const double *__restrict__ bnd,
                                      double *__restrict__ sq1, double *__restrict__ p1ra) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int count = side < 2 ? nj : ni;
  if (f >= count) return;
  const int off = side == 0 ? 0 : (side == 1 ? nj : (side == 2 ? 2 * nj : 2 * nj + ni));
  const size_t K = side == 0 ? (size_t)f * ni : (side == 1 ? (size_t)f * ni + ni - 1
                                                            : (side == 2 ? (size_t)f : (size_t)(nj - 1) * ni + f));
  const double *b = bnd + (size_t)(off + f) * 6;
  for (int r = 0; r < 3; ++r) {
    sq1[3 * K + r] += b[r];
    p1ra[3 * K + r] += b[3 + r];
  }
}

// Material index of every cell: the entry of the sorted distinct values matsh[0..nmat) nearest to sigma_t h
// (the host formed matsh from the same formula; nearest rather than equal absorbs a last-bit difference between
// host and device arithmetic)
__global__ void material_kernel(size_t nx, double h, const double *__restrict__ sigt, const double *__restrict__ matsh,
                                int nmat, int *__restrict__ mat) {
  const size_t K = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double v = sigt[K] * h;
  int lo = 0, hi = nmat;                  // first entry >= v
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (matsh[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  int m = lo < nmat ? lo : nmat - 1;
  if (lo > 0 && (lo == nmat || fabs(matsh[lo - 1] - v) <= fabs(matsh[lo] - v))) m = lo - 1;
  mat[K] = m;
}

__global__ void to_float_kernel(size_t n, const double *__restrict__ x, float *__restrict__ y) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    y[k] = (float)x[k];
}

cudaError_t to_float(const double *x, float *y, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  add_launches(1);
  const size_t g = std::min<size_t>((n + 255) / 256, 4096);
  to_float_kernel<<<(unsigned)g, 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

// y = Minv x: the right preconditioner of GMRES -- J = diag(I, diag(B11))^-1 for the low-memory schemes
// (precond >= 1), then with precond = 2 the vertex diffusion correction y += I_h D_a^-1 R_h (sigma_s/eps) y (one
// V-cycle); precond = 3 replaces the J x term by the cell-block Jacobi step: y = B^-1 x + C(J x), B the diagonal
// blocks of K
int apply_minv(lmdg_ctx *c, double *y, const double *x, cudaStream_t s) {
  const bool lowmem = c->variant == LMDG_LM || c->variant == LMDG_RLM;
  const int pmode = (lowmem && c->opt.precond) ? 1 : 0;
  CK(precond(y, x, c->b11dinv, c->nx, pmode, s));
  if (c->opt.precond >= 2) CK(dsa_apply(c->dsa, c->ni, c->nj, c->h, c->d64.sse, lowmem ? 1 : 0, y, s));
  if (c->opt.precond == 3) CK(block_step(y, x, c->binv, c->b11dinv, c->nx, pmode, s));
  return 0;
}

struct GmresOut {
  int iters = 0;
  double est = 0;
  bool breakdown = false;
  double kappa = 0;   // condition number of the cycle's Hessenberg matrix (0: no column)
};

// Condition number sigma_max / sigma_min of the k x k upper-triangular factor R (column-major, leading dimension
// ld) that the Givens rotations leave of a GMRES cycle's (k+1) x k Hessenberg matrix (same singular values), by
// one-sided Jacobi (Hestenes): plane rotations of column pairs until every pair is orthogonal to working
// precision; the column norms are then the singular values.  Host arithmetic, k <= 120.
double triangular_cond(const std::vector<double> &Rm, int ld, int k) {
  if (k <= 0) return 0.0;
  std::vector<double> A((size_t)k * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) A[(size_t)j * k + i] = i <= j ? Rm[(size_t)j * ld + i] : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int i = 0; i < k; ++i) {
          const double ap = A[(size_t)p * k + i], aq = A[(size_t)q * k + i];
          al += ap * ap; be += aq * aq; ga += ap * aq;
        }
        if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
        off = std::max(off, std::fabs(ga) / std::sqrt(al * be));
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cth = 1.0 / std::sqrt(1.0 + t * t), sth = cth * t;
        for (int i = 0; i < k; ++i) {
          const double ap = A[(size_t)p * k + i], aq = A[(size_t)q * k + i];
          A[(size_t)p * k + i] = cth * ap - sth * aq;
          A[(size_t)q * k + i] = sth * ap + cth * aq;
        }
      }
    if (off <= 1e-15) break;
  }
  double smax = 0, smin = HUGE_VAL;
  for (int j = 0; j < k; ++j) {
    double nn = 0;
    for (int i = 0; i < k; ++i) nn += A[(size_t)j * k + i] * A[(size_t)j * k + i];
    smax = std::max(smax, std::sqrt(nn));
    smin = std::min(smin, std::sqrt(nn));
  }
  return smin > 0 ? smax / smin : HUGE_VAL;
}

// One GMRES(m) cycle from a zero initial guess for K d = r, ||r|| = rnorm: d (device) receives the
// correction Minv V y.  Stops early when the least-squares residual reaches target.
int gmres_cycle(lmdg_ctx *c, int fp32, const double *r, double rnorm, double *d, int m, double target,
                int max_it, GmresOut *go, cudaStream_t s) {
  const size_t N = 4 * (size_t)c->nx;
  double *V = c->V;
  double *z = c->vec[0], *w = c->vec[1];
  double *partial = c->red;
  double *hdev = c->red + mdot_partial_len(c->red_len);          // [m+2]
  double *h2dev = hdev + (m + 2);
  double *ydev = h2dev + (m + 2);
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
  g[0] = rnorm;
  CK(axpby(V, 1.0 / rnorm, r, 0.0, N, s));
  int k = 0;
  go->breakdown = false;
  for (int j = 0; j < m && j < max_it; ++j) {
    double *vj = V + (size_t)j * N;
    if (int e = apply_minv(c, z, vj, s)) return e;
    if (int e = sweep_prec(c, fp32, z, w, 0, false, 0, s)) return e;
    // classical Gram-Schmidt, twice in FP64 solves; once in the FP32 inner cycles of the refinement, whose
    // operator is exact to FP32 only and whose target (inner_tol, 1e-4) lies far above the orthogonality a
    // single pass keeps -- the FP64 or float-float residual that follows each cycle is exact regardless
    const bool twice = !fp32;
    CK(mdot(V, N, j + 1, w, N, partial, hdev, 0, s));
    CK(maxpy(w, V, N, j + 1, hdev, N, s));
    if (twice) {
      CK(mdot(V, N, j + 1, w, N, partial, h2dev, 0, s));
      CK(maxpy(w, V, N, j + 1, h2dev, N, s));
    }
    CK(mdot(w, N, 1, w, N, partial, h2dev + j + 1, 0, s));
    CK(cudaMemcpyAsync(c->red_h, hdev, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
    if (twice)
      CK(cudaMemcpyAsync(c->red_h + (m + 2), h2dev, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
    else
      CK(cudaMemcpyAsync(c->red_h + (m + 2) + j + 1, h2dev + j + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (int e = check_error_word(c, s)) return e;   // synchronises
    double *col = &H[(size_t)j * (m + 1)];
    for (int i = 0; i <= j; ++i) col[i] = c->red_h[i] + (twice ? c->red_h[m + 2 + i] : 0.0);
    const double hn = std::sqrt(std::max(0.0, c->red_h[m + 2 + j + 1]));
    col[j + 1] = hn;
    if (!std::isfinite(hn)) return LMDG_ERR_BREAKDOWN;
    const bool invariant = hn <= 1e-14 * std::fabs(rnorm) || hn == 0.0;
    if (!invariant) CK(scale_by_inv(V + (size_t)(j + 1) * N, w, h2dev + j + 1, N, s));
    for (int i = 0; i < j; ++i) {
      const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t0;
    }
    const double den = std::hypot(col[j], col[j + 1]);
    cs[j] = den == 0 ? 1.0 : col[j] / den;
    sn[j] = den == 0 ? 0.0 : col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    go->est = std::fabs(g[j + 1]);
    if (go->est <= target || invariant) { go->breakdown = invariant; break; }
  }
  go->kappa = triangular_cond(H, m + 1, k);
  // back substitution H y = g
  std::vector<double> yv(k, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double sacc = g[i];
    for (int l = i + 1; l < k; ++l) sacc -= H[(size_t)l * (m + 1) + i] * yv[l];
    yv[i] = sacc / H[(size_t)i * (m + 1) + i];
  }
  for (int i = 0; i < k; ++i) c->red_h[i] = -yv[i];
  CK(cudaMemcpyAsync(ydev, c->red_h, sizeof(double) * k, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(z, 0, sizeof(double) * N, s));
  CK(maxpy(z, V, N, k, ydev, N, s));
  if (int e = apply_minv(c, d, z, s)) return e;
  CK(cudaStreamSynchronize(s));
  go->iters = k;
  return 0;
}

}  // namespace

extern "C" {

int lmdg_default_options(lmdg_options *o) {
  if (!o) return LMDG_ERR_ARG;
  o->precision = LMDG_FP64;
  o->restart = 30;
  o->max_iters = 5000;
  o->tol = 1e-8;
  o->inner_tol = 1e-4;
  o->max_refine = 50;
  o->precond = 1;
  o->spin_limit = 1LL << 26;
  o->device = 0;
  o->suppress = 0;
  o->recon = 0;
  o->resid = LMDG_RESID_FP64;
  return 0;
}

const char *lmdg_strerror(int code) {
  switch (code) {
    case LMDG_OK: return "success";
    case LMDG_ERR_ARG: return "invalid argument";
    case LMDG_ERR_QUAD: return "invalid quadrature (weights must be positive and sum to 1, no direction on an "
                               "axis, equal number of directions per quadrant)";
    case LMDG_ERR_NOMEM: return "device allocation failed";
    case LMDG_ERR_CUDA: return "CUDA call failed";
    case LMDG_ERR_NOTCONV: return "iteration limit reached before the tolerance";
    case LMDG_ERR_TIMEOUT: return "sweep gave up waiting for an upstream strip (spin limit)";
    case LMDG_ERR_BREAKDOWN: return "non-finite residual or Krylov breakdown";
    case LMDG_ERR_STATE: return "call out of order";
    default: return "unknown error";
  }
}

int lmdg_info(const lmdg_ctx *c, int *nx, int *ny, int *nang, int *variant) {
  if (!c) return LMDG_ERR_ARG;
  if (nx) *nx = c->ni;
  if (ny) *ny = c->nj;
  if (nang) *nang = c->nang;
  if (variant) *variant = c->variant;
  return 0;
}

void lmdg_destroy(lmdg_ctx *c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->dev);
  free_pd(c->d64);
  free_pd(c->d32);
  free_pd(c->d2);
  lmdg::dfree(c->p1ra2); lmdg::dfree(c->coef2); lmdg::dfree(c->qadj2);
  lmdg::dfree(c->perm); lmdg::dfree(c->p1ra64); lmdg::dfree(c->p1ra32); lmdg::dfree(c->sq1); lmdg::dfree(c->b11dinv);
  lmdg::dfree(c->sigma_a); lmdg::dfree(c->qmom); lmdg::dfree(c->part); lmdg::dfree(c->ytr); lmdg::dfree(c->ctrl);
  lmdg::dfree(c->psi); lmdg::dfree(c->binv);
  lmdg::dfree(c->cellsrc); lmdg::dfree(c->cellsh);
  lmdg::dfree(c->rev); lmdg::dfree(c->qadj64); lmdg::dfree(c->qadj32); lmdg::dfree(c->adj_buf);
  lmdg::dfree(c->mat); lmdg::dfree(c->cls); lmdg::dfree(c->matsh); lmdg::dfree(c->coef); lmdg::dfree(c->supp);
  lmdg::dsa_free(c->dsa);
  lmdg::dfree(c->V);
  for (auto &v : c->vec) lmdg::dfree(v);
  lmdg::dfree(c->red);
  if (c->red_h) cudaFreeHost(c->red_h);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete[] c->perm_h;
  delete c;
  cudaSetDevice(prev);
}

int lmdg_setup(lmdg_ctx **out, const lmdg_mesh *mesh, const lmdg_quadrature *quad, const double *sigma_s,
               const double *sigma_a, const double *q, int q_layout, const double *alpha, int alpha_layout,
               double eps, int variant, const lmdg_options *opt) {
  // LMDG_VERBOSE: the setup's phase times on stderr (each taken after a device synchronisation)
  const bool verbose = std::getenv("LMDG_VERBOSE") != nullptr;
  auto tphase = std::chrono::steady_clock::now();
  auto phase = [&](const char *name) {
    if (!verbose) return;
    cudaDeviceSynchronize();
    const auto t = std::chrono::steady_clock::now();
    std::fprintf(stderr, "lmdg_setup %-22s %8.3f ms\n", name,
                 std::chrono::duration<double, std::milli>(t - tphase).count());
    tphase = t;
  };
  if (!out || !mesh || !quad || !sigma_s || !sigma_a || !q) return LMDG_ERR_ARG;
  *out = nullptr;
  const int ni = mesh->nx, nj = mesh->ny;
  if (ni < 1 || nj < 1 || ni > 65536 || nj > 65536 || (long long)ni * nj > (1LL << 30) || !(mesh->h > 0) ||
      !std::isfinite(mesh->h))
    return LMDG_ERR_ARG;
  if (alpha && alpha_layout != 0 && alpha_layout != 1) return LMDG_ERR_ARG;
  if (alpha && alpha_layout == 0 && !std::isfinite(alpha[0])) return LMDG_ERR_ARG;
  if (!(eps > 1e-12) || !std::isfinite(eps)) return LMDG_ERR_ARG;
  if (variant < LMDG_STD || variant > LMDG_P0 || q_layout < 0 || q_layout > 2) return LMDG_ERR_ARG;
  const int na = quad->n;
  if (na < 4 || na > 1024 || na % 4 || !quad->ox || !quad->oy || !quad->w) return LMDG_ERR_QUAD;
  double wsum = 0;
  int cnt[4] = {0, 0, 0, 0};
  for (int l = 0; l < na; ++l) {
    const double a = quad->ox[l], b = quad->oy[l], w = quad->w[l];
    if (!(w > 0) || a == 0 || b == 0 || !std::isfinite(a) || !std::isfinite(b) || a * a + b * b > 1.0 + 1e-12)
      return LMDG_ERR_QUAD;
    wsum += w;
    cnt[quadrant(a, b)]++;
  }
  if (std::fabs(wsum - 1.0) > 1e-12) return LMDG_ERR_QUAD;
  if (cnt[0] != na / 4 || cnt[1] != na / 4 || cnt[2] != na / 4 || cnt[3] != na / 4) return LMDG_ERR_QUAD;
  const size_t nx = (size_t)ni * nj;
  // a cell with the cross sections of the cell before it (piecewise-constant media) passed the same test
  for (size_t K = 0; K < nx; ++K) {
    const double ss = sigma_s[K], sa = sigma_a[K];
    if (K > 0 && ss == sigma_s[K - 1] && sa == sigma_a[K - 1]) continue;
    if (!(ss >= 0) || !(sa >= 0) || !std::isfinite(ss) || !std::isfinite(sa) || !(ss / eps + eps * sa > 0))
      return LMDG_ERR_ARG;
  }
  lmdg_options o;
  lmdg_default_options(&o);
  if (opt) o = *opt;
  if (o.restart < 1 || o.restart > 120 || o.max_iters < 1 || !(o.tol > 0) || o.spin_limit < 1 ||
      (o.suppress != 0 && o.suppress != 1) || (o.suppress && variant != LMDG_RLM) || o.recon < 0 || o.recon > 2 ||
      (o.recon && (variant != LMDG_RLM || o.suppress)) ||
      (o.resid != LMDG_RESID_FP64 && o.resid != LMDG_RESID_F32X2) || o.precond < 0 || o.precond > 3 ||
      (o.precond >= 2 && variant == LMDG_P0))
    return LMDG_ERR_ARG;
  phase("validation");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) return LMDG_ERR_CUDA;
  CK(cudaSetDevice(o.device));

  lmdg_ctx *c = new (std::nothrow) lmdg_ctx();
  if (!c) return LMDG_ERR_NOMEM;
  c->ni = ni; c->nj = nj; c->nx = (int)nx; c->nang = na; c->nq = na / 4; c->variant = variant; c->q_layout = q_layout;
  c->kvar = variant == LMDG_P0 ? kP0 : variant;
  if (variant == LMDG_RLM && o.recon == 1) c->kvar = kRlmStar;
  if (variant == LMDG_RLM && o.recon == 2) c->kvar = kRlmQ1;
  c->has_alpha = alpha != nullptr; c->dev = o.device; c->h = mesh->h; c->eps = eps;
  c->x0 = mesh->x0; c->y0 = mesh->y0; c->opt = o;
  auto fail = [&](int e) { lmdg_destroy(c); return e; };

  // directions sorted by quadrant, stable within a quadrant
  std::vector<int> perm(na);
  for (int l = 0; l < na; ++l) perm[l] = l;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    return quadrant(quad->ox[a], quad->oy[a]) < quadrant(quad->ox[b], quad->oy[b]);
  });
  c->perm_h = new int[na];
  std::copy(perm.begin(), perm.end(), c->perm_h);
  std::vector<double> ox(na), oy(na), w(na);
  for (int k = 0; k < na; ++k) { ox[k] = quad->ox[perm[k]]; oy[k] = quad->oy[perm[k]]; w[k] = quad->w[perm[k]]; }
  // angle-dependent sources are reordered to the sorted directions on the host; constant and per-cell sources go
  // up as given and the device forms the rest of the per-cell tables (cell_tables_kernel)
  std::vector<double> qv;
  if (q_layout == 2) {
    qv.resize((size_t)na * nx * 4);
    for (int k = 0; k < na; ++k)
      std::memcpy(&qv[(size_t)k * nx * 4], q + (size_t)perm[k] * nx * 4, sizeof(double) * nx * 4);
  }
  const double *qsrc = q_layout == 2 ? qv.data() : q;
  const size_t qn = q_layout == 0 ? nx : (q_layout == 1 ? nx * 4 : qv.size());
  // inflow data per direction: [2 nj + 2 ni][2] (west and east faces by row, south and north faces by column);
  // alpha_layout 0 expands the single value given to every face and direction (a0 = value, a1 = 0)
  const size_t per = (size_t)2 * (ni + nj) * 2;
  std::vector<double> afull;
  if (alpha && alpha_layout == 0) {
    afull.assign((size_t)na * per, 0.0);
    for (size_t f = 0; f < afull.size(); f += 2) afull[f] = alpha[0];
    alpha = afull.data();
  }
  std::vector<double> av;
  if (alpha) {
    av.resize((size_t)na * per);
    for (int k = 0; k < na; ++k) std::memcpy(&av[(size_t)k * per], alpha + (size_t)perm[k] * per, sizeof(double) * per);
  }

  // Sigma Q1 = sum_l w_l (eps int q_l b_r + inflow-boundary terms), r = 1..3 (low-memory right-hand sides) and
  // P1 r_alpha = angular average of the boundary part of the reconstruction (RLMDG): the device forms the source
  // part of Sigma Q1; the inflow terms live on the boundary faces and are summed here per face, in the face order
  // of the inflow data (west and east by row, south and north by column), [face][sigma Q1 r = 1..3, P1 r_alpha
  // r = 1..3], and added to the face's cell on the device
  const double h = mesh->h;
  const int nfaces = 2 * (ni + nj);
  std::vector<double> bnd(alpha ? (size_t)nfaces * 6 : 0, 0.0);
  const bool kvar_q1 = c->kvar == kRlmQ1;
  double Ax[2] = {0, 0}, Ay[2] = {0, 0};
  for (int l = 0; l < na; ++l) {
    const double a = quad->ox[l], b = quad->oy[l], wl = quad->w[l];
    Ax[a > 0 ? 0 : 1] += wl * std::fabs(a);
    Ay[b > 0 ? 0 : 1] += wl * std::fabs(b);
    if (!alpha) continue;
    const double sx = a > 0 ? 1 : -1, sy = b > 0 ? 1 : -1, aa = std::fabs(a), bb = std::fabs(b);
    const double *al = alpha + (size_t)l * per;
    const int i0 = a > 0 ? 0 : ni - 1, offx = a > 0 ? 0 : nj;           // west / east faces
    for (int j = 0; j < nj; ++j) {
      const double a0 = al[((size_t)offx + j) * 2], a1 = al[((size_t)offx + j) * 2 + 1];
      double *f = &bnd[((size_t)offx + j) * 6];
      f[0] += wl * (-sx * aa * h * a0);
      f[1] += wl * (aa * h / 3.0 * a1);
      f[2] += wl * (-sx * aa * h / 3.0 * a1);
      f[3] += wl * sx * (-a0);
    }
    const int j0 = b > 0 ? 0 : nj - 1, offy = 2 * nj + (b > 0 ? 0 : ni);   // south / north faces
    for (int i = 0; i < ni; ++i) {
      const double a0 = al[((size_t)offy + i) * 2], a1 = al[((size_t)offy + i) * 2 + 1];
      double *f = &bnd[((size_t)offy + i) * 6];
      f[0] += wl * (bb * h / 3.0 * a1);
      f[1] += wl * (-sy * bb * h * a0);
      f[2] += wl * (-sy * bb * h / 3.0 * a1);
      f[4] += wl * sy * (-a0);
    }
    if (kvar_q1) {
      // Q1-type reconstruction: the xi eta coefficient of r_alpha (zero cell averages), in the direction's local
      // frame rec3 = rec1 - a1 on the y-inflow row (a1 the along-face coefficient there, times sx) and
      // (rec1 - rec1 of the cell below) / 2 above it, with rec1 = -a0 of the x-inflow face on the x-inflow
      // column and 0 elsewhere; the global coefficient is sx sy rec3.  The corner cell's term goes with its
      // y-inflow face, the rest of the x-inflow column's with their x-inflow faces
      auto rec1_loc = [&](int jr) { return -al[((size_t)offx + jr) * 2]; };
      for (int i = 0; i < ni; ++i) {
        const double a1 = sx * al[((size_t)offy + i) * 2 + 1];
        bnd[((size_t)offy + i) * 6 + 5] += wl * sx * sy * ((i == i0 ? rec1_loc(j0) : 0.0) - a1);
      }
      for (int r = 1; r < nj; ++r) {
        const int jr = b > 0 ? r : nj - 1 - r, jb = b > 0 ? r - 1 : nj - r;
        bnd[((size_t)offx + jr) * 6 + 5] += wl * sx * sy * 0.5 * (rec1_loc(jr) - rec1_loc(jb));
      }
    }
  }
  c->Ax[0] = Ax[0]; c->Ax[1] = Ax[1]; c->Ay[0] = Ay[0]; c->Ay[1] = Ay[1];
  // quadrature moments of the epilogue: sum w, sum w |Omega_x|, sum w |Omega_y|, sum w Omega_x, sum w Omega_y
  std::vector<double> qm(5, 0.0);
  for (int l = 0; l < na; ++l) {
    qm[0] += w[l]; qm[1] += w[l] * std::fabs(ox[l]); qm[2] += w[l] * std::fabs(oy[l]);
    qm[3] += w[l] * ox[l]; qm[4] += w[l] * oy[l];
  }
  // opposite direction of every sorted direction (central symmetry, needed by the adjoint)
  std::vector<int> rev(na, 0);
  bool rev_ok = true;
  for (int k = 0; k < na && rev_ok; ++k) {
    int found = -1;
    for (int l = 0; l < na; ++l)
      if (std::fabs(quad->ox[l] + ox[k]) <= 1e-12 && std::fabs(quad->oy[l] + oy[k]) <= 1e-12 &&
          std::fabs(quad->w[l] - w[k]) <= 1e-14 * w[k]) { found = l; break; }
    if (found < 0) rev_ok = false;
    else rev[k] = found;
  }
  c->rev_ok = rev_ok;
  phase("host tables");
  int e = 0;
  if (lmdg::dmalloc(&c->perm, sizeof(int) * na) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  if (lmdg::dmalloc(&c->rev, sizeof(int) * na) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  if (cudaMemcpy(c->rev, rev.data(), sizeof(int) * na, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LMDG_ERR_CUDA);
  if (cudaMemcpy(c->perm, perm.data(), sizeof(int) * na, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LMDG_ERR_CUDA);
  // the problem data goes up as given (cross sections, source) and the device forms the per-cell tables
  double *ss_dev = nullptr, *q0_dev = nullptr;
  const size_t nq4 = q_layout == 2 ? qn : nx * 4;
  if ((e = upload(&c->d64.ox, ox)) || (e = upload(&c->d64.oy, oy)) || (e = upload(&c->d64.w, w)) ||
      (e = upload(&c->d32.ox, ox)) || (e = upload(&c->d32.oy, oy)) || (e = upload(&c->d32.w, w)) ||
      (e = upload(&ss_dev, sigma_s, nx)) || (e = upload(&c->sigma_a, sigma_a, nx)) || (e = upload(&c->qmom, qm)) ||
      (q_layout == 0 && (e = upload(&q0_dev, qsrc, qn)))) {
    lmdg::dfree(ss_dev);
    lmdg::dfree(q0_dev);
    return fail(e);
  }
  if ((q_layout == 0 && lmdg::dmalloc(&c->d64.q, sizeof(double) * nq4) != cudaSuccess) ||
      (q_layout != 0 && (e = upload(&c->d64.q, qsrc, qn)))) {
    lmdg::dfree(ss_dev);
    lmdg::dfree(q0_dev);
    return fail(e ? e : LMDG_ERR_NOMEM);
  }
  bool ok = lmdg::dmalloc(&c->d64.sigt, sizeof(double) * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->d64.sse, sizeof(double) * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->d32.sigt, sizeof(float) * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->d32.sse, sizeof(float) * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->d32.q, sizeof(float) * nq4) == cudaSuccess &&
            lmdg::dmalloc(&c->sq1, sizeof(double) * 3 * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->p1ra64, sizeof(double) * 3 * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->p1ra32, sizeof(float) * 3 * nx) == cudaSuccess &&
            lmdg::dmalloc(&c->b11dinv, sizeof(double) * 3 * nx) == cudaSuccess;
  if (ok) {
    add_launches(1);
    cell_tables_kernel<<<(unsigned)((nx + 255) / 256), 256>>>(
        nx, eps, h, ss_dev, c->sigma_a, q_layout == 0 ? q0_dev : c->d64.q, q_layout, na, c->d64.w, Ax[0] + Ax[1],
        Ay[0] + Ay[1], c->d64.sigt, c->d64.sse, c->d32.sigt, c->d32.sse, c->d64.q, c->d32.q, c->sq1, c->p1ra64,
        c->b11dinv);
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (ok && q_layout == 2) ok = to_float(c->d64.q, c->d32.q, nq4, 0) == cudaSuccess;
  if (ok && alpha) {
    double *bnd_dev = nullptr;
    if ((e = upload(&bnd_dev, bnd))) { lmdg::dfree(ss_dev); lmdg::dfree(q0_dev); return fail(e); }
    for (int side = 0; side < 4 && ok; ++side) {   // one side per launch: a corner cell has faces on two sides
      const int count = side < 2 ? nj : ni;
      add_launches(1);
      boundary_terms_kernel<<<(count + 255) / 256, 256>>>(ni, nj, side, bnd_dev, c->sq1, c->p1ra64);
      ok = cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    lmdg::dfree(bnd_dev);
  }
  if (ok) ok = to_float(c->p1ra64, c->p1ra32, 3 * nx, 0) == cudaSuccess;
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  lmdg::dfree(ss_dev);
  lmdg::dfree(q0_dev);
  if (!ok) return fail(LMDG_ERR_CUDA);
  if (alpha) {
    if ((e = upload(&c->d64.alpha, av)) || (e = upload(&c->d32.alpha, av))) return fail(e);
  }
  if (o.suppress) {
    // interior faces across which (sigma_s, sigma_a) changes: no RLMDG reconstruction there
    std::vector<double> bits(nx, 0.0);
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        const size_t K = (size_t)j * ni + i;
        unsigned m = 0;
        const int fi[4] = {i - 1, i + 1, i, i}, fj[4] = {j, j, j - 1, j + 1};
        for (int f = 0; f < 4; ++f) {
          if (fi[f] < 0 || fi[f] >= ni || fj[f] < 0 || fj[f] >= nj) continue;
          const size_t Kn = (size_t)fj[f] * ni + fi[f];
          if (sigma_s[Kn] != sigma_s[K] || sigma_a[Kn] != sigma_a[K]) m |= 1u << f;
        }
        bits[K] = m;
      }
    if ((e = upload(&c->supp, bits))) return fail(e);
  }
  phase("uploads");
  c->g64 = choose_geom(c->kvar, nj, c->nq, 0);
  c->g32 = choose_geom(c->kvar, nj, c->nq, 1);
  c->g2 = choose_geom(c->kvar, nj, c->nq, 2);
  if (c->g64.units() == 0 || c->g32.units() == 0 || c->g2.units() == 0) return fail(LMDG_ERR_CUDA);
  if (std::getenv("LMDG_VERBOSE"))
    std::fprintf(stderr, "lmdg: %dx%d cells n_omega=%d variant=%d fp64 shape groups=%d warps=%d apw=%d | fp32 "
                 "groups=%d warps=%d apw=%d | f32x2 groups=%d warps=%d apw=%d\n", ni, nj, na, variant, c->g64.groups,
                 c->g64.warps, c->g64.apw, c->g32.groups, c->g32.warps, c->g32.apw, c->g2.groups, c->g2.warps,
                 c->g2.apw);
  const int strips = (nj + 31) / 32;
  const size_t ytr_elems = (size_t)na * strips * ni * kTraceStride;
  if (lmdg::dmalloc(&c->ytr, sizeof(double) * ytr_elems) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  c->ytr_words = 2 * ytr_elems;
  c->ytr_dirty = true;
  if (lmdg::dmalloc(&c->cellsrc, sizeof(double) * 4 * nx) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  if (lmdg::dmalloc(&c->cellsh, sizeof(double) * nx) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  c->ctrl_words = 2 + (size_t)std::max({c->g64.units(), c->g32.units(), c->g2.units()});
  if (lmdg::dmalloc(&c->ctrl, sizeof(unsigned) * c->ctrl_words) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
  if (cudaMemset(c->ctrl, 0, sizeof(unsigned) * c->ctrl_words) != cudaSuccess) return fail(LMDG_ERR_CUDA);
  phase("work buffers");
  // FP64 element-solve coefficient tables per (material = distinct sigma_t h, direction class = distinct
  // (|Omega_x|, |Omega_y|)); the FP64 sweeps read them instead of forming the reciprocals and Schur products
  {
    // distinct values of sigma_t h, sorted (runs of equal neighbours -- piecewise-constant media -- are skipped
    // before the sort); each cell's material index is then found on the device (material_kernel)
    std::vector<double> uniq;
    double prev = 0.0;
    for (size_t K = 0; K < nx; ++K) {
      if (K > 0 && sigma_s[K] == sigma_s[K - 1] && sigma_a[K] == sigma_a[K - 1]) continue;   // same sigma_t h
      const double shK = (sigma_s[K] / eps + eps * sigma_a[K]) * h;
      if (K == 0 || shK != prev) uniq.push_back(shK);
      prev = shK;
    }
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<double> cab;
    std::vector<int> clsv(na);
    for (int k = 0; k < na; ++k) {
      const double aa = std::fabs(ox[k]), bb = std::fabs(oy[k]);
      int f = -1;
      for (size_t q = 0; q < cab.size() / 2; ++q)
        if (cab[2 * q] == aa && cab[2 * q + 1] == bb) { f = (int)q; break; }
      if (f < 0) { f = (int)(cab.size() / 2); cab.push_back(aa); cab.push_back(bb); }
      clsv[k] = f;
    }
    c->nmat = (int)uniq.size();
    c->ncls = (int)(cab.size() / 2);
    c->ncoef = coef_count(c->kvar);
    const size_t tbytes = sizeof(double) * (size_t)c->nmat * c->ncls * c->ncoef;
    double *cabd = nullptr;
    bool ok = lmdg::dmalloc(&c->coef, tbytes) == cudaSuccess &&
              lmdg::dmalloc(&c->mat, sizeof(int) * nx) == cudaSuccess &&
              lmdg::dmalloc(&c->cls, sizeof(int) * na) == cudaSuccess &&
              lmdg::dmalloc(&c->matsh, sizeof(double) * c->nmat) == cudaSuccess &&
              lmdg::dmalloc(&cabd, sizeof(double) * cab.size()) == cudaSuccess;
    ok = ok && cudaMemcpy(c->cls, clsv.data(), sizeof(int) * na, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->matsh, uniq.data(), sizeof(double) * c->nmat, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(cabd, cab.data(), sizeof(double) * cab.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         build_coef_tables(c->kvar, c->nmat, c->ncls, c->matsh, cabd, c->coef, 0) == cudaSuccess;
    if (ok) {
      add_launches(1);
      material_kernel<<<(unsigned)((nx + 255) / 256), 256>>>(nx, h, c->d64.sigt, c->matsh, c->nmat, c->mat);
      ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    }
    lmdg::dfree(cabd);
    if (!ok) {   // no tables: the FP64 sweeps compute the coefficients themselves
      cudaGetLastError();
      lmdg::dfree(c->coef); lmdg::dfree(c->mat); lmdg::dfree(c->cls); lmdg::dfree(c->matsh);
      c->coef = nullptr; c->mat = nullptr; c->cls = nullptr; c->matsh = nullptr;
    }
  }
  phase("coefficient tables");
  if (o.precond >= 2) {
    // vertex diffusion correction of the scheme's own diffusion limit (full gradient for Q1-DG, cell-averaged
    // gradient for the low-memory schemes), multigrid hierarchy built on the device
    if (int e2 = dsa_build(c->dsa, variant == LMDG_STD ? 0 : 1, ni, nj, h, eps, c->d64.sigt, c->sigma_a, Ax[0], Ay[0],
                           0))
      return fail(e2);
  }
  phase("diffusion correction");
  if (o.precond == 3) {
    // the cell-diagonal blocks of K: four FP64 sweeps with the upwind coupling cut, of x = e_r in every cell
    // (column r of every block), then one 4 x 4 inverse per cell
    if (lmdg::dmalloc(&c->binv, sizeof(double) * 16 * nx) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
    double *tmp = nullptr;   // x = e_r, then the four columns
    if (lmdg::dmalloc(&tmp, sizeof(double) * 20 * nx) != cudaSuccess) return fail(LMDG_ERR_NOMEM);
    double *ycol = tmp + 4 * (size_t)nx;
    c->local_mode = 1;
    int e2 = 0;
    for (int r = 0; r < 4 && !e2; ++r) {
      if (unit_vectors(tmp, nx, r, nullptr) != cudaSuccess) e2 = LMDG_ERR_CUDA;
      else e2 = do_sweep<double>(c, tmp, ycol + 4 * (size_t)nx * r, 0, false, 0, nullptr);
    }
    c->local_mode = 0;
    if (!e2) e2 = check_error_word(c, nullptr);
    unsigned *bad = c->ctrl + 2;
    unsigned nbad = 0;
    if (!e2 && (block_inverses(ycol, ycol + 4 * (size_t)nx, ycol + 8 * (size_t)nx, ycol + 12 * (size_t)nx, nx,
                               c->binv, bad, nullptr) != cudaSuccess ||
                cudaMemcpy(&nbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess))
      e2 = LMDG_ERR_CUDA;
    lmdg::dfree(tmp);
    if (!e2 && nbad) e2 = LMDG_ERR_BREAKDOWN;
    if (e2) return fail(e2);
  }
  phase("cell blocks");
  *out = c;
  return 0;
}

int lmdg_sweep(lmdg_ctx *c, const double *x, double *y, int flags, void *stream) {
  if (!c || !x || !y) return LMDG_ERR_ARG;
  if ((flags & LMDG_SWEEP_F32X2) && (flags & (LMDG_SWEEP_FP32 | LMDG_SWEEP_STORE))) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const size_t N = 4 * (size_t)c->nx;
  const double *xd = x;
  double *yd = y;
  if (flags & LMDG_HOST_PTRS) {
    if (int e = ensure_krylov(c, c->opt.restart)) return e;
    CK(cudaMemcpyAsync(c->vec[4], x, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    xd = c->vec[4];
    yd = c->vec[5];
  }
  const int prec = (flags & LMDG_SWEEP_FP32) ? 1 : ((flags & LMDG_SWEEP_F32X2) ? 2 : 0);
  // FP32 storing sweeps of an LMDG_FP32_BF16STORE context keep the low-memory unknowns in bfloat16
  const int bf16 = (prec == 1 && c->opt.precision == LMDG_FP32_BF16STORE) ? 1 : 0;
  if (int e = sweep_prec(c, prec, xd, yd, (flags & LMDG_SWEEP_SOURCE) ? 1 : 0, (flags & LMDG_SWEEP_STORE) != 0, bf16,
                         s))
    return e;
  if (flags & LMDG_HOST_PTRS) CK(cudaMemcpyAsync(y, yd, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  return check_error_word(c, s);
}

int lmdg_shard_layout(const lmdg_ctx *c, int flags, int nshards, int *sets, int *chunk_sets, size_t *chunk_bytes) {
  if (!c || nshards < 1 || nshards > 4096) return LMDG_ERR_ARG;
  if ((flags & LMDG_SWEEP_FP32) && (flags & LMDG_SWEEP_F32X2)) return LMDG_ERR_ARG;
  const int prec = (flags & LMDG_SWEEP_FP32) ? 1 : ((flags & LMDG_SWEEP_F32X2) ? 2 : 0);
  const SweepGeom &g = prec == 0 ? c->g64 : (prec == 1 ? c->g32 : c->g2);
  const ShardRange r = shard_range(g, 0, nshards);
  const size_t word = prec == 1 ? sizeof(float) : (prec == 2 ? sizeof(f2) : sizeof(double));
  if (sets) *sets = r.sets;
  if (chunk_sets) *chunk_sets = r.chunk;
  if (chunk_bytes) *chunk_bytes = (size_t)r.chunk * c->nx * nr_of(c->kvar) * word;
  return 0;
}

int lmdg_sweep_shard(lmdg_ctx *c, const double *x, void *parts, int shard, int nshards, int flags, void *stream) {
  if (!c || !x || !parts || nshards < 1 || nshards > 4096 || shard < 0 || shard >= nshards) return LMDG_ERR_ARG;
  if (flags & (LMDG_HOST_PTRS | LMDG_SOLVE_EXACT_REF)) return LMDG_ERR_ARG;
  if ((flags & LMDG_SWEEP_F32X2) && (flags & (LMDG_SWEEP_FP32 | LMDG_SWEEP_STORE))) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const int prec = (flags & LMDG_SWEEP_FP32) ? 1 : ((flags & LMDG_SWEEP_F32X2) ? 2 : 0);
  const int bf16 = (prec == 1 && c->opt.precision == LMDG_FP32_BF16STORE) ? 1 : 0;
  const int src = (flags & LMDG_SWEEP_SOURCE) ? 1 : 0;
  const bool store = (flags & LMDG_SWEEP_STORE) != 0;
  int e = prec == 1 ? do_sweep<float>(c, x, nullptr, src, store, bf16, s, 1, shard, nshards, parts)
        : prec == 2 ? do_sweep<f2>(c, x, nullptr, src, false, 0, s, 1, shard, nshards, parts)
                    : do_sweep<double>(c, x, nullptr, src, store, 0, s, 1, shard, nshards, parts);
  if (e) return e;
  return check_error_word(c, s);
}

int lmdg_sweep_combine(lmdg_ctx *c, const double *x, const void *parts, double *y, int flags, void *stream) {
  if (!c || !x || !parts || !y) return LMDG_ERR_ARG;
  if (flags & (LMDG_HOST_PTRS | LMDG_SWEEP_STORE | LMDG_SOLVE_EXACT_REF)) return LMDG_ERR_ARG;
  if ((flags & LMDG_SWEEP_F32X2) && (flags & LMDG_SWEEP_FP32)) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const int prec = (flags & LMDG_SWEEP_FP32) ? 1 : ((flags & LMDG_SWEEP_F32X2) ? 2 : 0);
  const int src = (flags & LMDG_SWEEP_SOURCE) ? 1 : 0;
  void *pp = const_cast<void *>(parts);
  if (prec == 1) return do_sweep<float>(c, x, y, src, false, 0, s, 2, 0, 1, pp);
  if (prec == 2) {
    if (int e = ensure_f2(c, s)) return e;
    return do_sweep<f2>(c, x, y, src, false, 0, s, 2, 0, 1, pp);
  }
  return do_sweep<double>(c, x, y, src, false, 0, s, 2, 0, 1, pp);
}

int lmdg_get_psi(lmdg_ctx *c, double *psi, int flags, void *stream) {
  if (!c || !psi) return LMDG_ERR_ARG;
  if (c->psi_kind < 0) return LMDG_ERR_STATE;
  const int per = c->variant == LMDG_STD ? 4 : 1;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  if (flags & LMDG_HOST_PTRS) {
    double *tmp = nullptr;
    if (lmdg::dmalloc(&tmp, sizeof(double) * c->psi_elems) != cudaSuccess) return LMDG_ERR_NOMEM;
    cudaError_t e1 = lmdg::psi_to_user(tmp, c->psi, c->psi_kind, per, c->ni, c->nj, c->nang, c->nq, c->perm, s);
    cudaError_t e2 = cudaMemcpyAsync(psi, tmp, sizeof(double) * c->psi_elems, cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    lmdg::dfree(tmp);
    return (e1 || e2 || e3) ? LMDG_ERR_CUDA : 0;
  }
  CK(lmdg::psi_to_user(psi, c->psi, c->psi_kind, per, c->ni, c->nj, c->nang, c->nq, c->perm, s));
  return 0;
}

int lmdg_solve(lmdg_ctx *c, const double *x0, double *x, double *phi, lmdg_stats *st, int flags, void *stream) {
  if (!c) return LMDG_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const int m = c->opt.restart;
  if (int e = ensure_krylov(c, m)) return e;
  const size_t N = 4 * (size_t)c->nx;
  const int fp32 = c->opt.precision != LMDG_FP64;
  const int bf16 = c->opt.precision == LMDG_FP32_BF16STORE;
  // residual sweeps: FP64, or float-float in the FP32 modes when asked for
  const int rprec = (fp32 && c->opt.resid == LMDG_RESID_F32X2) ? 2 : 0;
  double *X = c->vec[2], *R = c->vec[3], *D = c->vec[4];
  c->sweeps64 = c->sweeps32 = c->sweeps2 = 0;
  harvest(c, true);
  c->sweep_ms[0] = c->sweep_ms[1] = c->sweep_ms[2] = 0;
  const long long launches0 = launch_count();
  if (x0) CK(cudaMemcpyAsync(X, x0, sizeof(double) * N,
                             (flags & LMDG_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(X, 0, sizeof(double) * N, s));
  // r = -(K x - b), storing in FP64 mode (the last one is then the recovery sweep)
  auto residual = [&](double *rn2) -> int {
    if (int e = sweep_prec(c, rprec, X, R, 1, !fp32, 0, s)) return e;
    CK(axpby(R, -1.0, R, 0.0, N, s));
    if (int e = check_error_word(c, s)) return e;
    return norm2(c, R, rn2, s);
  };
  double rn2 = 0;
  int iters = 0, refine = 0, status = 0;
  double r0 = 0, kappa = 0;
  if (fp32 && !x0) {
    // FP32 start from zero: b from an FP32 source sweep (or, with LMDG_SOLVE_EXACT_REF, from a sweep in the
    // residual arithmetic, so that the tolerance reference ||b|| carries no FP32 error) and an FP32 GMRES cycle
    // for the first iterate; the residual-arithmetic sweeps are then spent only on residuals at iterates
    if (flags & LMDG_SOLVE_EXACT_REF) {
      if (int e = residual(&rn2)) return e;                          // X = 0: R = b
    } else {
      if (int e = sweep_prec(c, 1, X, R, 1, false, 0, s)) return e;   // X = 0: R = K 0 - b = -b
      CK(axpby(R, -1.0, R, 0.0, N, s));
      if (int e = check_error_word(c, s)) return e;
      if (int e = norm2(c, R, &rn2, s)) return e;
    }
    r0 = std::sqrt(rn2);
    if (!std::isfinite(r0)) return LMDG_ERR_BREAKDOWN;
    if (r0 > 0) {
      GmresOut go;
      const double target = std::max(c->opt.inner_tol * r0, 0.5 * c->opt.tol * r0);
      if (int e = gmres_cycle(c, 1, R, r0, D, m, target, c->opt.max_iters, &go, s)) return e;
      iters += go.iters;
      kappa = std::max(kappa, go.kappa);
      CK(axpby(X, 1.0, D, 1.0, N, s));
    }
    if (int e = residual(&rn2)) return e;
  } else {
    if (int e = residual(&rn2)) return e;
    r0 = std::sqrt(rn2);
  }
  if (!std::isfinite(r0)) return LMDG_ERR_BREAKDOWN;
  double rn = std::sqrt(rn2);
  if (!std::isfinite(rn)) return LMDG_ERR_BREAKDOWN;
  while (rn > c->opt.tol * r0) {
    if (iters >= c->opt.max_iters || (fp32 && refine >= c->opt.max_refine)) { status = LMDG_ERR_NOTCONV; break; }
    const double target = fp32 ? std::max(c->opt.inner_tol * rn, 0.5 * c->opt.tol * r0) : c->opt.tol * r0;
    GmresOut go;
    if (int e = gmres_cycle(c, fp32, R, rn, D, m, target, c->opt.max_iters - iters, &go, s)) return e;
    iters += go.iters;
    kappa = std::max(kappa, go.kappa);
    refine++;
    CK(axpby(X, 1.0, D, 1.0, N, s));
    if (int e = residual(&rn2)) return e;
    const double rnew = std::sqrt(rn2);
    if (!std::isfinite(rnew)) return LMDG_ERR_BREAKDOWN;
    if (go.breakdown && rnew > c->opt.tol * r0 && rnew >= rn) { rn = rnew; status = LMDG_ERR_BREAKDOWN; break; }
    rn = rnew;
  }
  // outputs: phi from the partial reductions of the last residual sweep (at the final x)
  if (phi) {
    double *P = (flags & LMDG_HOST_PTRS) ? c->vec[5] : phi;
    if (c->variant == LMDG_STD) {
      CK(cudaMemcpyAsync(P, X, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    } else if (rprec == 2) {
      CK(launch_phi(c, reinterpret_cast<const f2 *>(c->part), 4 * c->g2.groups, X, P, s));
    } else {
      CK(launch_phi(c, reinterpret_cast<const double *>(c->part), 4 * c->g64.groups, X, P, s));
    }
    if (flags & LMDG_HOST_PTRS) CK(cudaMemcpyAsync(phi, P, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  }
  if (x) CK(cudaMemcpyAsync(x, X, sizeof(double) * N,
                            (flags & LMDG_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  if (fp32) {
    // recovery sweep in the working precision: angular unknowns stored as float (or bfloat16)
    if (int e = sweep_prec(c, 1, X, c->vec[1], 1, true, bf16, s)) return e;
  }
  if (int e = check_error_word(c, s)) return e;
  if (st) {
    st->iters = iters;
    st->refinements = fp32 ? refine : 0;
    st->sweeps_fp64 = c->sweeps64;
    st->sweeps_fp32 = c->sweeps32;
    st->sweeps_f32x2 = c->sweeps2;
    st->resid0 = r0;
    st->resid = rn;
    st->kappa_est = kappa;
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    harvest(c, true);
    st->sweep_ms_fp64 = c->sweep_ms[0];
    st->sweep_ms_fp32 = c->sweep_ms[1];
    st->sweep_ms_f32x2 = c->sweep_ms[2];
    st->launches = launch_count() - launches0;
  }
  return status;
}

int lmdg_b11_apply(lmdg_ctx *c, const double *x, double *y, int flags, void *stream) {
  if (!c || !x || !y) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const size_t N3 = 3 * (size_t)c->nx;
  const double A4[4] = {c->Ax[0], c->Ax[1], c->Ay[0], c->Ay[1]};
  if (flags & LMDG_HOST_PTRS) {
    if (int e = ensure_krylov(c, c->opt.restart)) return e;
    CK(cudaMemcpyAsync(c->vec[4], x, sizeof(double) * N3, cudaMemcpyHostToDevice, s));
    CK(b11_apply(c->ni, c->nj, c->h, c->eps, c->sigma_a, A4, c->vec[4], c->vec[5], s));
    CK(cudaMemcpyAsync(y, c->vec[5], sizeof(double) * N3, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return 0;
  }
  CK(b11_apply(c->ni, c->nj, c->h, c->eps, c->sigma_a, A4, x, y, s));
  return 0;
}

int lmdg_b11_solve(lmdg_ctx *c, const double *r, double *z, double tol, int *iters, int flags, void *stream) {
  if (!c || !r || !z || !(tol > 0)) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  if (int e = ensure_krylov(c, c->opt.restart)) return e;
  const size_t N3 = 3 * (size_t)c->nx;
  const double A4[4] = {c->Ax[0], c->Ax[1], c->Ay[0], c->Ay[1]};
  double *Z = c->vec[0], *Rr = c->vec[1], *Pp = c->vec[2], *Ap = c->vec[3];
  double *partial = c->red, *out = c->red + mdot_partial_len(c->red_len);
  CK(cudaMemcpyAsync(Rr, r, sizeof(double) * N3,
                     (flags & LMDG_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(Z, 0, sizeof(double) * N3, s));
  CK(cudaMemcpyAsync(Pp, Rr, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s));
  auto dot = [&](const double *a, const double *b, double *res) -> int {
    CK(mdot(a, N3, 1, b, N3, partial, out, 0, s));
    CK(cudaMemcpyAsync(c->red_h, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *res = c->red_h[0];
    return 0;
  };
  double rr = 0;
  if (int e = dot(Rr, Rr, &rr)) return e;
  const double stop = tol * tol * rr;
  int it = 0;
  const int maxit = 100000;
  while (rr > stop && it < maxit) {
    CK(b11_apply(c->ni, c->nj, c->h, c->eps, c->sigma_a, A4, Pp, Ap, s));
    double pap = 0;
    if (int e = dot(Pp, Ap, &pap)) return e;
    if (!(pap > 0)) return LMDG_ERR_BREAKDOWN;
    const double alpha = rr / pap;
    CK(axpby(Z, alpha, Pp, 1.0, N3, s));
    CK(axpby(Rr, -alpha, Ap, 1.0, N3, s));
    double rr2 = 0;
    if (int e = dot(Rr, Rr, &rr2)) return e;
    CK(axpby(Pp, 1.0, Rr, rr2 / rr, N3, s));
    rr = rr2;
    ++it;
  }
  if (iters) *iters = it;
  CK(cudaMemcpyAsync(z, Z, sizeof(double) * N3,
                     (flags & LMDG_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return rr > stop ? LMDG_ERR_NOTCONV : 0;
}

int lmdg_precond_apply(lmdg_ctx *c, const double *x, double *y, int flags, void *stream) {
  if (!c || !x || !y) return LMDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const size_t N = 4 * (size_t)c->nx;
  if (flags & LMDG_HOST_PTRS) {
    if (int e = ensure_krylov(c, c->opt.restart)) return e;
    CK(cudaMemcpyAsync(c->vec[4], x, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    if (int e = apply_minv(c, c->vec[5], c->vec[4], s)) return e;
    CK(cudaMemcpyAsync(y, c->vec[5], sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return 0;
  }
  return apply_minv(c, y, x, s);
}

int lmdg_adjoint(lmdg_ctx *c, const double *g, double *dss, double *dsa, double *dq, double *J, lmdg_stats *st,
                 int flags, void *stream) {
  if (!c || !g) return LMDG_ERR_ARG;
  if (c->variant == LMDG_RLM || c->variant == LMDG_P0 || c->q_layout == 2) return LMDG_ERR_ARG;
  if (!c->rev_ok) return LMDG_ERR_QUAD;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(c->dev));
  const size_t nx = (size_t)c->nx, N = 4 * nx;
  const bool host = (flags & LMDG_HOST_PTRS) != 0;
  if (!c->adj_buf) {
    if (lmdg::dmalloc(&c->adj_buf, sizeof(double) * (5 * N + 4 * nx)) != cudaSuccess) return LMDG_ERR_NOMEM;
    if (lmdg::dmalloc(&c->qadj64, sizeof(double) * N) != cudaSuccess) return LMDG_ERR_NOMEM;
    if (lmdg::dmalloc(&c->qadj32, sizeof(float) * N) != cudaSuccess) return LMDG_ERR_NOMEM;
    if (lmdg::dmalloc(&c->qadj2, sizeof(f2) * N) != cudaSuccess) return LMDG_ERR_NOMEM;
  }
  double *Xf = c->adj_buf, *Lam = c->adj_buf + N, *Y = c->adj_buf + 2 * N, *G = c->adj_buf + 3 * N;
  double *PhiF = c->adj_buf + 3 * N + 4 * nx, *PhiA = PhiF + N;   // scalar-flux moments (low-memory)
  // detector source: eps h^2 q_adj = g h^2  ->  q_adj = g / eps on the cell-average moment
  std::vector<double> qa(N, 0.0), gh(nx);
  if (host) std::memcpy(gh.data(), g, sizeof(double) * nx);
  else CK(cudaMemcpy(gh.data(), g, sizeof(double) * nx, cudaMemcpyDeviceToHost));
  for (size_t K = 0; K < nx; ++K) qa[4 * K] = gh[K] / c->eps;
  std::vector<float> qa32(qa.begin(), qa.end());
  CK(cudaMemcpyAsync(c->qadj64, qa.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->qadj32, qa32.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s));
  CK(convert_to_f2(c->qadj64, c->qadj2, N, s));
  CK(cudaMemcpyAsync(G, gh.data(), sizeof(double) * nx, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  lmdg_stats s1{}, s2{};
  // 1. forward solve and the forward angular flux in FP64
  c->use_adj = false; c->no_store = false;
  int st1 = lmdg_solve(c, nullptr, Xf, PhiF, &s1, 0, stream);
  if (st1 != 0 && st1 != LMDG_ERR_NOTCONV) return st1;
  if (c->psi_kind != 0)
    if (int e = do_sweep<double>(c, Xf, Y, 1, true, 0, s)) return e;
  // 2. adjoint solve: for a centrally symmetric quadrature Lhat_l^T = Lhat_{-l} and S is symmetric, so with angle
  //    reversal Pi, B^T = Pi B Pi; the standard and V_h^lm bases are closed under Pi, hence the adjoint system is the
  //    forward one with the directions reversed and the detector response g as an isotropic source
  c->use_adj = true; c->no_store = true;
  int st2 = lmdg_solve(c, nullptr, Lam, PhiA, &s2, 0, stream);
  if (st2 != 0 && st2 != LMDG_ERR_NOTCONV) { c->use_adj = false; c->no_store = false; return st2; }
  // 3. correlation sweep at the multiplier: per cell sum_l w_l lam_l,r psi_l,r (lam_l = psi_adj of -Omega_l;
  //    cell averages only for the low-memory scheme, whose slopes are isotropic)
  c->corr = reinterpret_cast<const double *>(c->psi);
  int e3 = do_sweep<double>(c, Lam, Y, 1, false, 0, s);
  c->corr = nullptr; c->use_adj = false; c->no_store = false;
  if (e3) return e3;
  if (int e = check_error_word(c, s)) return e;
  // 4. per-cell gradients
  double *out = Y;   // [3][nx] reuse of the scratch vector (4 nx doubles)
  const bool lowmem = c->variant != LMDG_STD;
  CK(lmdg::adjoint_gradients(c->variant, c->nx, 4 * c->g64.groups, c->h, c->eps,
                             reinterpret_cast<const double *>(c->part), lowmem ? PhiF : Xf, lowmem ? PhiA : Lam, out,
                             s));
  std::vector<double> xf_h(N);
  CK(cudaMemcpyAsync(xf_h.data(), lowmem ? PhiF : Xf, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  double *dsts[3] = {dss, dsa, dq};
  for (int f = 0; f < 3; ++f)
    if (dsts[f]) CK(cudaMemcpyAsync(dsts[f], out + f * nx, sizeof(double) * nx,
                                    host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (J) {
    double acc = 0;
    for (size_t K = 0; K < nx; ++K) acc += gh[K] * c->h * c->h * xf_h[4 * K];
    *J = acc;
  }
  if (st) {
    *st = s1;
    st->iters += s2.iters;
    st->refinements += s2.refinements;
    st->sweeps_fp64 = s1.sweeps_fp64 + s2.sweeps_fp64 + 1 + (c->opt.precision != LMDG_FP64 ? 1 : 0);
    st->sweeps_fp32 = s1.sweeps_fp32 + s2.sweeps_fp32;
    st->sweeps_f32x2 = s1.sweeps_f32x2 + s2.sweeps_f32x2;
    st->resid = std::max(s1.resid / std::max(s1.resid0, 1e-300), s2.resid / std::max(s2.resid0, 1e-300));
    st->kappa_est = std::max(s1.kappa_est, s2.kappa_est);
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return (st1 == LMDG_ERR_NOTCONV || st2 == LMDG_ERR_NOTCONV) ? LMDG_ERR_NOTCONV : 0;
}

}  // extern "C"
