// Internal declarations of liblmdg (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <type_traits>
#include "../../include/lmdg.h"
#include "f32x2.cuh"

namespace lmdg {

// Per-precision copies of the problem data, directions sorted by quadrant (+,+), (-,+), (-,-), (+,-).
template <typename T>
struct ProblemData {
  T *ox = nullptr, *oy = nullptr, *w = nullptr;  // [nang] sorted
  T *sigt = nullptr;                              // [nx] sigma_s/eps + eps sigma_a
  T *sse = nullptr;                               // [nx] sigma_s/eps
  T *q = nullptr;                                 // [nx][4] or [nang(sorted)][nx][4]
  T *alpha = nullptr;                             // [nang(sorted)][2 nj + 2 ni][2] or null (faces: west, east,
                                                  // south, north)
};

// Sweep launch geometry: one CTA per (quadrant, angle group, strip of 32 rows); warps of a CTA hold
// disjoint angles of the group, each warp up to kMaxA angles processed per step.
struct SweepGeom {
  int groups;      // angle groups per quadrant
  int warps;       // warps per CTA
  int apw;         // angles per warp (<= kMaxA)
  int strips;      // ceil(nj / 32): strips of 32 rows
  int units() const { return 4 * groups * strips; }
};

constexpr int kMaxA = 4;        // cap on directions per warp (template instances 1..4)

// Stored angular unknowns of one direction are kept in its sweep's wavefront order: the cell in local column x
// and local row r (the quadrant's mirrored frame) sits at slot ((r / 32) (ni + 31) + x + r % 32) 32 + r % 32, so
// the 32 lanes of a warp, which solve the cells (t - k, 32 s + k) of strip s at step t, store to 32 consecutive
// slots.  A plane holds strips x (ni + 31) x 32 slots, the ones outside the mesh unused.
__host__ __device__ inline size_t psi_plane(int ni, int nj) { return (size_t)((nj + 31) / 32) * (ni + 31) * 32; }
__host__ __device__ inline size_t psi_slot(int ni, int x, int r) {
  const int l = r & 31;
  return ((size_t)(r >> 5) * (ni + 31) + x + l) * 32 + l;
}
#ifndef LMDG_CHUNK
#define LMDG_CHUNK 8
#endif
constexpr int kChunk = LMDG_CHUNK;   // steps per chunk: cell staging, inflow staging, one CTA barrier
constexpr unsigned kTraceEmpty = 0xFFF7FFF7u;   // 32-bit pattern of a strip trace not yet written (a NaN)
constexpr int kTraceStride = 4;      // trace values stored per (direction, strip boundary, column)
constexpr int kRlmStar = 3;          // kernel variant of RLMDG* (LMDG_RLM with the three-cell reconstruction)
constexpr int kP0 = 4;               // kernel variant of P0-DG (LMDG_P0)
constexpr int kRlmQ1 = 5;            // kernel variant of RLMDG with the Q1-type reconstruction (also the xi eta term)
// reduced values per cell (partial reductions; even, for paired moves) and trace values passed downwind per face
constexpr int nr_of(int var) { return var == kP0 ? 2 : (var == kRlmQ1 ? 8 : (var >= 2 ? 6 : 4)); }
constexpr int ns_of(int var) {
  return var == kP0 ? 1 : ((var == kRlmStar || var == kRlmQ1) ? 4 : (var == 2 ? 3 : 2));
}

// Arguments of one sweep launch (everything a kernel reads or writes).
template <typename T>
struct SweepArgs {
  int ni, nj, nq, nang, nx;   // cells along x, along y; directions per quadrant, directions; cells
  T h, eps;
  SweepGeom g;
  ProblemData<T> pd;
  int q_per_angle;
  const double *X;     // [nx][4] input vector (always double)
  const T *p1ra;       // [nx][3] P1 r_alpha (RLMDG, source sweeps) or null
  int source;          // 1: add eps q and the inflow data alpha
  T *part;             // [4*groups][nx][NR] partial reductions, written once each
  int pq0, npq;        // the launch sweeps the partial sets [pq0, pq0 + npq) (quadrant * groups + group): all
                       // 4*groups of them, or one shard's range when the directions are split across GPUs
  void *psi;           // storing sweep output or null: [nang (user order, through perm)][psi_plane slots in the
                       // direction's wavefront order, psi_slot][4 standard, 1 low-memory], so a warp's stores coalesce
  int psi_bf16;        // psi is __nv_bfloat16 (low-memory variants only)
  const int *perm;     // [nang] sorted index -> user index
  T *ytr;              // [nang][strips][ni][kTraceStride] strip-boundary traces, kTraceEmpty when unwritten
  unsigned *ctrl;      // [0] ticket, [1] error
  long long spin_limit;
  const T *cellsrc;    // [nx][4] per-cell source moments / isotropic slopes of this sweep (prep_kernel)
  const T *cellsh;     // [nx] sigma_t h
  const double *corr;  // adjoint correlation mode: stored forward psi (layout of psi, double; each plane in the
                       // wavefront order of its own, the opposite, quadrant); the reduction
                       // becomes sum_l w_l u_l,r psi_rev(l),r (r = 0 only for LMDG)
  const int *rev;      // [nang] sorted index -> user index of the opposite direction (corr mode)
  // Coefficient tables (FP64 sweeps; null: coefficients computed in the kernel).  With them, cellsh carries the
  // cell's material index and coef[(material * ncls + class) * ncoef + c] the solve coefficients of that
  // material (sigma_t h) and direction class (|Omega_x|, |Omega_y|).
  const T *coef;
  int ncoef, ncls;
  const int *cls;      // [nang] sorted index -> direction class
  const double *matsh; // [materials] sigma_t h of each material
  const int *mat;      // [nx] material of each cell (prep_kernel writes it into the cellsh slot)
  const unsigned *supp;  // RLMDG: [nx] faces without reconstruction (1 west, 2 east, 4 south, 8 north) or null
  int local;           // FP64 only: every cell's solve sees zero upwind data (the traces from its left and lower
                       // neighbours, the slope traces of LMDG, the upwind values of the reconstruction), so that
                       // y = K x returns the cell-diagonal blocks of K applied to x
};

// Vertex diffusion correction (dsa.cu): one multigrid level, nine-point stencils of bs x bs blocks on the
// (ni + 1) x (nj + 1) vertices of ni x nj cells, with its block-diagonal inverse and work vectors.
struct MgLevel {
  int ni = 0, nj = 0, bs = 1;
  double *A = nullptr;     // [vertices][9][bs][bs]
  double *dinv = nullptr;  // [vertices][bs][bs]
  double *x = nullptr, *y = nullptr, *b = nullptr, *r = nullptr;   // [vertices][bs]
};
constexpr int kMaxMgLevels = 24;
constexpr int kMaxDense = 1156;   // largest coarsest level solved with a dense inverse (unknowns)
struct VertexDsa {
  int avg = 0;                     // 1: cell-average gradient (low-memory schemes), 0: full gradient (Q1-DG)
  int nlev = -1;                   // levels with a coarser one below; lev[nlev] is the coarsest (-1: not built)
  MgLevel lev[kMaxMgLevels];
  double *cinv = nullptr;          // dense inverse of the coarsest matrix, or null (then coarse_sweeps Jacobi steps)
  int nu = 2, coarse_sweeps = 50;  // smoothing steps before and after the coarse correction; coarsest fallback
  double omega = 0.7;              // damping of the block-Jacobi smoother
  cudaGraphExec_t vcycle_graph = nullptr;   // the V-cycle's launches captured once (null: launched one by one)
  long long vcycle_launches = 0;   // kernels in the captured V-cycle
};
// Build the hierarchy for ni x nj cells (sigt, sigma_a per cell, device; Ax, Ay the half-range outflow weights):
// 0 or an LMDG_ERR_* code.  Synchronises s.
int dsa_build(VertexDsa &d, int avg, int ni, int nj, double h, double eps, const double *sigt, const double *sigma_a,
              double Ax, double Ay, cudaStream_t s);
void dsa_free(VertexDsa &d);
// u += I_h D_a^-1 R_h (sigma_s/eps) u~ with one V-cycle, u [ni*nj][4]; lowmem: u holds (X0, X1) and the
// scalar-flux slopes are -X1 (u~ = (u0, -u1), correction (c0, -c1))
cudaError_t dsa_apply(const VertexDsa &d, int ni, int nj, double h, const double *sse, int lowmem, double *u,
                      cudaStream_t s);

// Device memory of the contexts (mem.cu): allocations from a per-device pool that keeps freed memory mapped for the
// next context; dalloc returns memory usable on any stream, dfree waits for the device before returning it.
cudaError_t dalloc(void **p, size_t bytes);
template <typename T>
cudaError_t dmalloc(T **p, size_t bytes) {
  return dalloc(reinterpret_cast<void **>(p), bytes);
}
void dfree(void *p);

// Number of kernels launched by this library (all host wrappers add to it).
long long launch_count();
void add_launches(long long k);

// FP64 coefficient tables of the element solves (sweep.cu)
cudaError_t build_coef_tables(int variant, int nmat, int ncls, const double *matsh, const double *cls_ab,
                              double *coef, cudaStream_t s);
int coef_count(int variant);

// Host-side launchers (sweep.cu)
template <typename T>
cudaError_t launch_sweep(int variant, const SweepArgs<T> &a, cudaStream_t s);
template <typename T>
size_t sweep_smem_bytes(int variant, int warps, int apw);
template <typename T>
int sweep_blocks_per_sm(int variant, int warps, int apw);
// Sweep arithmetic: 0 double, 1 float, 2 float-float (f2)
template <typename T>
constexpr int prec_of() { return std::is_same<T, double>::value ? 0 : (std::is_same<T, float>::value ? 1 : 2); }

// launch shape for nj rows and sweep arithmetic prec; LMDG_SWEEP_GEOM="groups,warps,apw" overrides
SweepGeom choose_geom(int variant, int nj, int nq, int prec);
// y[i] = x[i] rounded to float-float
cudaError_t convert_to_f2(const double *x, f2 *y, size_t n, cudaStream_t s);

// y = K x - source * b  from the partial reductions (sweep.cu); sigt = sigma_t per cell, qm = the quadrature
// moments written by quad_moments
template <typename T>
cudaError_t launch_epilogue(int variant, int nx, int P, double h, const T *part, const double *X,
                            const double *sse, const double *sigt, const double *qm, const double *p1ra,
                            const double *sq1, int source, double *y, cudaStream_t s);
// qm[0..4] = sum w, sum w |Omega_x|, sum w |Omega_y|, sum w Omega_x, sum w Omega_y over all directions
cudaError_t quad_moments(int nang, const double *ox, const double *oy, const double *w, double *qm, cudaStream_t s);

}  // namespace lmdg

// Context
struct lmdg_ctx {
  int ni = 0, nj = 0, nx = 0, nang = 0, nq = 0, variant = 0, q_layout = 0, has_alpha = 0, dev = 0;
  int kvar = 0;                            // kernel variant: the scheme, kRlmStar for RLMDG*, kRlmQ1 for the
                                           // Q1-type reconstruction, kP0 for P0-DG
  double h = 0, eps = 0, x0 = 0, y0 = 0;
  lmdg_options opt{};
  int *perm = nullptr;                     // device [nang]
  int *perm_h = nullptr;                   // host copy
  lmdg::ProblemData<double> d64;
  lmdg::ProblemData<float> d32;
  lmdg::ProblemData<lmdg::f2> d2;          // float-float copies (residual sweeps of the mixed-precision solve)
  bool f2_ready = false;                   // d2, p1ra2 and coef2 hold the converted data
  double *p1ra64 = nullptr;                // [nx][3]
  float *p1ra32 = nullptr;
  lmdg::f2 *p1ra2 = nullptr;
  double *sq1 = nullptr;                   // [nx][3] Sigma Q1
  double *b11dinv = nullptr;               // [nx][3] reciprocal diagonal of B11 (Jacobi preconditioner)
  double *sigma_a = nullptr;               // [nx] (B11 stencil)
  double Ax[2] = {0, 0}, Ay[2] = {0, 0};   // sum of w |Omega_x| over Omega_x > 0 / < 0, likewise y
  double *qmom = nullptr;                  // device [5] quadrature moments (epilogue)
  lmdg::SweepGeom g64{}, g32{}, g2{};
  void *part = nullptr;                    // partial reductions, grown to the largest launch shape used
  size_t part_bytes = 0;
  void *ytr = nullptr;                     // inter-strip traces (double-sized)
  void *cellsrc = nullptr;                 // [nx][4] per-sweep cell inputs (double-sized)
  void *cellsh = nullptr;                  // [nx]
  unsigned *ctrl = nullptr;
  size_t ctrl_words = 0;
  size_t ytr_words = 0;                    // 32-bit words of ytr
  bool ytr_dirty = true;                   // ytr must be refilled with kTraceEmpty before the next sweep
  int ytr_prec = -1;                       // trace layout of the last sweep using ytr (0: 8-byte, 1: 4-byte)
  int part_prec = -1;                      // arithmetic (0 double, 1 float, 2 float-float) of the last partials
  void *psi = nullptr;                     // stored angular unknowns, grown to the widest kind stored
  size_t psi_bytes = 0;
  int psi_kind = -1;                       // -1 none, 0 double, 1 float, 2 bf16
  size_t psi_elems = 0;
  // Krylov workspace
  double *V = nullptr;                     // (m+1) x N basis
  double *vec[6] = {nullptr};              // scratch vectors of length N
  double *red = nullptr;                   // reduction scratch
  double *red_h = nullptr;                 // pinned host mirror
  int red_len = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int ev_pending = -1;                     // arithmetic of a recorded, not yet harvested sweep (-1 none)
  double sweep_ms[3] = {0, 0, 0};          // device time in FP64 / FP32 / float-float sweep kernels
  long long launches = 0;
  int sweeps64 = 0, sweeps32 = 0, sweeps2 = 0;
  // adjoint (standard scheme): opposite directions, detector source, solve-time switches
  int *rev = nullptr;                      // device [nang] sorted -> user index of -Omega
  bool rev_ok = false;                     // the quadrature is centrally symmetric
  double *qadj64 = nullptr;                // [nx][4] detector source g/eps (r = 0)
  float *qadj32 = nullptr;
  lmdg::f2 *qadj2 = nullptr;
  double *adj_buf = nullptr;               // [3][N] forward solution, multiplier, scratch
  bool use_adj = false;                    // sweeps take the detector source and vacuum inflow
  bool no_store = false;                   // solve keeps the stored psi untouched
  const double *corr = nullptr;            // correlation sweep input (forward psi, double)
  // FP64 coefficient tables
  int nmat = 0, ncls = 0, ncoef = 0;
  int *mat = nullptr;                      // [nx] material index
  int *cls = nullptr;                      // [nang] sorted index -> direction class
  double *matsh = nullptr;                 // [nmat] sigma_t h
  double *coef = nullptr;                  // [nmat][ncls][ncoef]
  lmdg::f2 *coef2 = nullptr;               // the same, float-float
  unsigned *supp = nullptr;                // RLMDG suppression bits per cell, or null
  lmdg::VertexDsa dsa;                     // vertex diffusion correction (precond = 2, 3)
  double *binv = nullptr;                  // precond = 3: [nx][4][4] inverses of K's cell-diagonal blocks
  int local_mode = 0;                      // FP64 sweeps cut the upwind coupling (SweepArgs::local)
};
