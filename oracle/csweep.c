/* FP64 sweep oracle for the S_N-DG transport operator L (Sun & Hauck, arXiv 1907.01027).
 *
 * TEST INFRASTRUCTURE ONLY: called from oracle/sweeps.py through ctypes; never linked into the product.
 *
 * Every routine handles ONE discrete ordinate Omega_l = (ox, oy) on a uniform ni x nj Cartesian mesh of square
 * cells of side h (ni cells along x, nj along y; cell (i, j) has index K = j*ni + i) with the Legendre Q1 basis
 * b = (1, xi, eta, xi*eta).  The
 * operator is the unweighted per-angle block of L in Appendix A (the factor w_l is applied by the caller):
 *
 *   L_{l,K}(u, b_r) = -int_K u Omega.grad b_r + int_{dK} u_hat Omega.nu_K b_r + int_K sigma_t u b_r   (eq-Ljk)
 *
 * with the upwind trace u_hat: the interior trace on outflow faces (Omega.nu > 0), the neighbour's trace on
 * inflow faces, and zero on inflow faces that lie on the domain boundary (alpha enters through Q).
 *
 * The cell and face integrals are computed once from the basis functions with 3-point Gauss-Legendre rules
 * (exact for these polynomial integrands); no closed forms are used.  Sweeps solve L_l u = b by forward
 * substitution in upwind order (Section 2.1.1: each block of L is block lower triangular in that order):
 * rows are visited with the loop directions set by the signs of Omega, which is a topological order of
 * the upwind dependency graph on a Cartesian mesh.
 */
#include <math.h>
#include <string.h>

typedef struct {
  double mass[4][4];
  double vol[2][4][4];     /* vol[d][r][s] = int_K b_s d_d b_r */
  double selff[4][4][4];   /* face f: int_F b_s^K b_r^K */
  double nbrf[4][4][4];    /* face f: int_F b_s^{K'} b_r^K, K' across f */
  double nrm[4][2];        /* outward normals: W, E, S, N */
} elem_t;

static const double GP[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};
static const double GW[3] = {0.5555555555555556, 0.8888888888888888, 0.5555555555555556};

static void basis(double xi, double eta, double b[4]) {
  b[0] = 1.0; b[1] = xi; b[2] = eta; b[3] = xi * eta;
}
static void dbasis(double xi, double eta, double h, double dx[4], double dy[4]) {
  double s = 2.0 / h;
  dx[0] = 0; dx[1] = s; dx[2] = 0; dx[3] = s * eta;
  dy[0] = 0; dy[1] = 0; dy[2] = s; dy[3] = s * xi;
}

static void build_elem(double h, elem_t *e) {
  memset(e, 0, sizeof(*e));
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double w = GW[a] * GW[c] * h * h / 4.0, b[4], dx[4], dy[4];
      basis(GP[a], GP[c], b);
      dbasis(GP[a], GP[c], h, dx, dy);
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) {
          e->mass[r][s] += w * b[s] * b[r];
          e->vol[0][r][s] += w * b[s] * dx[r];
          e->vol[1][r][s] += w * b[s] * dy[r];
        }
    }
  /* own / neighbour reference coordinates of the face points */
  for (int f = 0; f < 4; ++f)
    for (int a = 0; a < 3; ++a) {
      double oxi, oeta, nxi, neta;
      switch (f) {
        case 0: oxi = -1; oeta = GP[a]; nxi = 1; neta = GP[a]; break;
        case 1: oxi = 1; oeta = GP[a]; nxi = -1; neta = GP[a]; break;
        case 2: oxi = GP[a]; oeta = -1; nxi = GP[a]; neta = 1; break;
        default: oxi = GP[a]; oeta = 1; nxi = GP[a]; neta = -1; break;
      }
      double bo[4], bn[4], w = GW[a] * h / 2.0;
      basis(oxi, oeta, bo);
      basis(nxi, neta, bn);
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) {
          e->selff[f][r][s] += w * bo[s] * bo[r];
          e->nbrf[f][r][s] += w * bn[s] * bo[r];
        }
    }
  double nr[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  memcpy(e->nrm, nr, sizeof(nr));
}

/* neighbour index across face f of cell (i, j), or -1 on the boundary */
static int nbr(int ni, int nj, int i, int j, int f) {
  switch (f) {
    case 0: return i > 0 ? j * ni + i - 1 : -1;
    case 1: return i < ni - 1 ? j * ni + i + 1 : -1;
    case 2: return j > 0 ? (j - 1) * ni + i : -1;
    default: return j < nj - 1 ? (j + 1) * ni + i : -1;
  }
}

/* diagonal 4x4 block of L_l at cell K */
static void diag_block(const elem_t *e, double ox, double oy, double sigt, double A[4][4]) {
  for (int r = 0; r < 4; ++r)
    for (int s = 0; s < 4; ++s)
      A[r][s] = -(ox * e->vol[0][r][s] + oy * e->vol[1][r][s]) + sigt * e->mass[r][s];
  for (int f = 0; f < 4; ++f) {
    double on = ox * e->nrm[f][0] + oy * e->nrm[f][1];
    if (on > 0)
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) A[r][s] += on * e->selff[f][r][s];
  }
}

/* coupling of row block K to the upwind neighbours: out[r] = sum over inflow faces of
 * (Omega.nu) int_F u_{K'} b_r (K' interior neighbour) */
static void inflow_terms(const elem_t *e, int ni, int nj, int i, int j, double ox, double oy, const double *u,
                         double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int f = 0; f < 4; ++f) {
    double on = ox * e->nrm[f][0] + oy * e->nrm[f][1];
    int k = nbr(ni, nj, i, j, f);
    if (on < 0 && k >= 0)
      for (int r = 0; r < 4; ++r)
        for (int s = 0; s < 4; ++s) out[r] += on * e->nbrf[f][r][s] * u[4 * k + s];
  }
}

/* out = L_l u for one angle (unweighted); u, out: [ni*nj][4] */
void osw_apply_L(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *u, double *out) {
  elem_t e;
  build_elem(h, &e);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      int K = j * ni + i;
      double A[4][4], c[4];
      diag_block(&e, ox, oy, sigt[K], A);
      inflow_terms(&e, ni, nj, i, j, ox, oy, u, c);
      for (int r = 0; r < 4; ++r) {
        double s = c[r];
        for (int q = 0; q < 4; ++q) s += A[r][q] * u[4 * K + q];
        out[4 * K + r] = s;
      }
    }
}

/* Gaussian elimination with partial pivoting on a 4x4 system (A destroyed). */
static void solve4(double A[4][4], double b[4], double x[4]) {
  int p[4] = {0, 1, 2, 3};
  for (int c = 0; c < 4; ++c) {
    int m = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(A[p[r]][c]) > fabs(A[p[m]][c])) m = r;
    int t = p[c]; p[c] = p[m]; p[m] = t;
    for (int r = c + 1; r < 4; ++r) {
      double f = A[p[r]][c] / A[p[c]][c];
      for (int k = c; k < 4; ++k) A[p[r]][k] -= f * A[p[c]][k];
      b[p[r]] -= f * b[p[c]];
    }
  }
  for (int c = 3; c >= 0; --c) {
    double s = b[p[c]];
    for (int k = c + 1; k < 4; ++k) s -= A[p[c]][k] * x[k];
    x[c] = s / A[p[c]][c];
  }
}

/* Solve L_l u = b (unweighted block) by an upwind sweep.  b, u: [ni*nj][4]. */
void osw_sweep_L(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *b, double *u) {
  elem_t e;
  build_elem(h, &e);
  memset(u, 0, sizeof(double) * 4 * (size_t)ni * nj);
  for (int jj = 0; jj < nj; ++jj) {
    int j = oy > 0 ? jj : nj - 1 - jj;
    for (int ii = 0; ii < ni; ++ii) {
      int i = ox > 0 ? ii : ni - 1 - ii;
      int K = j * ni + i;
      double A[4][4], c[4], rhs[4];
      diag_block(&e, ox, oy, sigt[K], A);
      inflow_terms(&e, ni, nj, i, j, ox, oy, u, c);
      for (int r = 0; r < 4; ++r) rhs[r] = b[4 * K + r] - c[r];
      solve4(A, rhs, &u[4 * K]);
    }
  }
}

/* Solve L00 u0 = b0 for one angle: the rows and columns of L restricted to the piecewise constants
 * (V_{h,0}, Section 3.2).  b0, u0: [ni*nj]. */
void osw_sweep_L00(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *b0,
                   double *u0) {
  elem_t e;
  build_elem(h, &e);
  memset(u0, 0, sizeof(double) * (size_t)ni * nj);
  for (int jj = 0; jj < nj; ++jj) {
    int j = oy > 0 ? jj : nj - 1 - jj;
    for (int ii = 0; ii < ni; ++ii) {
      int i = ox > 0 ? ii : ni - 1 - ii;
      int K = j * ni + i;
      double A[4][4];
      diag_block(&e, ox, oy, sigt[K], A);
      double c = 0.0;
      for (int f = 0; f < 4; ++f) {
        double on = ox * e.nrm[f][0] + oy * e.nrm[f][1];
        int k = nbr(ni, nj, i, j, f);
        if (on < 0 && k >= 0) c += on * e.nbrf[f][0][0] * u0[k];
      }
      u0[K] = (b0[K] - c) / A[0][0];
    }
  }
}

/* Upwind reconstruction of one angle at cell (i, j) from cell averages u0 with alpha = 0
 * (R Pi_0, Section 3.3.1): Legendre coefficients of the P1 slopes, (h/2) delta_x on b1 and (h/2) delta_y on
 * b2, using the upwind difference (s_x = -sign(Omega_x)) and spacing h/2 against the zero boundary value.
 * supp (may be NULL): per-cell face bits (1 west, 2 east, 4 south, 8 north) of interior faces across which
 * the reconstruction is suppressed (Section 4, the discontinuous cross-section examples): the difference
 * across such a face is taken as zero.  star (RLMDG*, Section 4.1): from the third cell on the difference is
 * the centre slope of the quadratic through the cell and its two upwind neighbours, (3u_i - 4u_{i-1} +
 * u_{i-2}) / (2h); the second cell keeps the two-cell difference. */
static void recon0(int ni, int nj, double h, double ox, double oy, const double *u0, const unsigned char *supp,
                   int star, int i, int j, double sl[2]) {
  int K = j * ni + i;
  unsigned m = supp ? supp[K] : 0u;
  double dx, dy;
  if (ox > 0) {
    if (i == 0) dx = (u0[K] - 0.0) / (h / 2);
    else if (m & 1u) dx = 0.0;
    else if (star && i >= 2) dx = (3 * u0[K] - 4 * u0[K - 1] + u0[K - 2]) / (2 * h);
    else dx = (u0[K] - u0[K - 1]) / h;
  } else {
    if (i == ni - 1) dx = (0.0 - u0[K]) / (h / 2);
    else if (m & 2u) dx = 0.0;
    else if (star && i <= ni - 3) dx = -(3 * u0[K] - 4 * u0[K + 1] + u0[K + 2]) / (2 * h);
    else dx = (u0[K + 1] - u0[K]) / h;
  }
  if (oy > 0) {
    if (j == 0) dy = (u0[K] - 0.0) / (h / 2);
    else if (m & 4u) dy = 0.0;
    else if (star && j >= 2) dy = (3 * u0[K] - 4 * u0[K - ni] + u0[K - 2 * ni]) / (2 * h);
    else dy = (u0[K] - u0[K - ni]) / h;
  } else {
    if (j == nj - 1) dy = (0.0 - u0[K]) / (h / 2);
    else if (m & 8u) dy = 0.0;
    else if (star && j <= nj - 3) dy = -(3 * u0[K] - 4 * u0[K + ni] + u0[K + 2 * ni]) / (2 * h);
    else dy = (u0[K + ni] - u0[K]) / h;
  }
  sl[0] = 0.5 * h * dx;
  sl[1] = 0.5 * h * dy;
}

/* row 0 of L_l applied to the trial function u0 b0 + R u0 at cell (i, j), given u0 on K and upwind cells */
static double row0_rec(const elem_t *e, int ni, int nj, double h, double ox, double oy, double sigt,
                       const double *u0, const unsigned char *supp, int star, int i, int j) {
  int K = j * ni + i;
  double A[4][4], uK[4], sl[2];
  diag_block(e, ox, oy, sigt, A);
  recon0(ni, nj, h, ox, oy, u0, supp, star, i, j, sl);
  uK[0] = u0[K]; uK[1] = sl[0]; uK[2] = sl[1]; uK[3] = 0.0;
  double s = 0.0;
  for (int q = 0; q < 4; ++q) s += A[0][q] * uK[q];
  for (int f = 0; f < 4; ++f) {
    double on = ox * e->nrm[f][0] + oy * e->nrm[f][1];
    int k = nbr(ni, nj, i, j, f);
    if (on < 0 && k >= 0) {
      int ki = k % ni, kj = k / ni;
      double uk[4], sk[2];
      recon0(ni, nj, h, ox, oy, u0, supp, star, ki, kj, sk);
      uk[0] = u0[k]; uk[1] = sk[0]; uk[2] = sk[1]; uk[3] = 0.0;
      for (int q = 0; q < 4; ++q) s += on * e->nbrf[f][0][q] * uk[q];
    }
  }
  return s;
}

/* Solve Ltilde00 u0 = b0 for one angle, Ltilde00 = L00 + L01 R (Section 3.3.2): row 0 of L applied to the
 * reconstructed trial function.  The reconstruction at K uses only K and its upwind neighbours, so the
 * system is lower triangular in sweep order; each cell's equation is affine in u0[K] and is solved from two
 * evaluations (u0[K] = 0 and u0[K] = 1).  b0, u0: [ni*nj]; supp: suppression bits as in recon0, or NULL;
 * star: the three-cell reconstruction. */
void osw_sweep_Lt00(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *b0,
                    double *u0, const unsigned char *supp, int star) {
  elem_t e;
  build_elem(h, &e);
  memset(u0, 0, sizeof(double) * (size_t)ni * nj);
  for (int jj = 0; jj < nj; ++jj) {
    int j = oy > 0 ? jj : nj - 1 - jj;
    for (int ii = 0; ii < ni; ++ii) {
      int i = ox > 0 ? ii : ni - 1 - ii;
      int K = j * ni + i;
      u0[K] = 0.0;
      double r0 = row0_rec(&e, ni, nj, h, ox, oy, sigt[K], u0, supp, star, i, j);
      u0[K] = 1.0;
      double r1 = row0_rec(&e, ni, nj, h, ox, oy, sigt[K], u0, supp, star, i, j);
      u0[K] = (b0[K] - r0) / (r1 - r0);
    }
  }
}

/* Cell and face integral tables, exported for the closed-form pin test:
 * out = mass(16) vol_x(16) vol_y(16) self(64) nbr(64). */
void osw_elem_tables(double h, double *out) {
  elem_t e;
  build_elem(h, &e);
  memcpy(out, e.mass, sizeof(e.mass));
  memcpy(out + 16, e.vol, sizeof(e.vol));
  memcpy(out + 48, e.selff, sizeof(e.selff));
  memcpy(out + 112, e.nbrf, sizeof(e.nbrf));
}

/* out = L_l^T u for one angle (transpose of the unweighted block of Appendix A).  Row block K of L^T collects
 * the transposed diagonal block of K and the transposed coupling blocks L[K', K] of every cell K' that takes
 * its inflow from K (the downwind neighbours of K). */
void osw_apply_LT(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *u,
                  double *out) {
  elem_t e;
  build_elem(h, &e);
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      int K = j * ni + i;
      double A[4][4];
      diag_block(&e, ox, oy, sigt[K], A);
      double s[4] = {0, 0, 0, 0};
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) s[r] += A[q][r] * u[4 * K + q];
      /* K' = neighbour across face f of K; K is K''s inflow neighbour across the opposite face g of K' */
      for (int f = 0; f < 4; ++f) {
        int k2 = nbr(ni, nj, i, j, f);
        if (k2 < 0) continue;
        int g = f ^ 1;                       /* W<->E, S<->N */
        double on = ox * e.nrm[g][0] + oy * e.nrm[g][1];
        if (on < 0)                          /* inflow face of K' */
          for (int r = 0; r < 4; ++r)
            for (int q = 0; q < 4; ++q) s[r] += on * e.nbrf[g][q][r] * u[4 * k2 + q];
      }
      for (int r = 0; r < 4; ++r) out[4 * K + r] = s[r];
    }
}

/* Solve L_l^T u = b (unweighted block) by back substitution: L_l is block lower triangular in upwind order, so
 * its transpose is solved in the reverse order, each cell's transposed diagonal block against b minus the
 * transposed couplings to its (already solved) downwind neighbours. */
void osw_sweep_LT(int ni, int nj, double h, double ox, double oy, const double *sigt, const double *b, double *u) {
  elem_t e;
  build_elem(h, &e);
  memset(u, 0, sizeof(double) * 4 * (size_t)ni * nj);
  for (int jj = nj - 1; jj >= 0; --jj) {
    int j = oy > 0 ? jj : nj - 1 - jj;
    for (int ii = ni - 1; ii >= 0; --ii) {
      int i = ox > 0 ? ii : ni - 1 - ii;
      int K = j * ni + i;
      double A[4][4], At[4][4], rhs[4];
      diag_block(&e, ox, oy, sigt[K], A);
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) At[r][q] = A[q][r];
      for (int r = 0; r < 4; ++r) rhs[r] = b[4 * K + r];
      for (int f = 0; f < 4; ++f) {
        int k2 = nbr(ni, nj, i, j, f);
        if (k2 < 0) continue;
        int g = f ^ 1;
        double on = ox * e.nrm[g][0] + oy * e.nrm[g][1];
        if (on < 0)
          for (int r = 0; r < 4; ++r)
            for (int q = 0; q < 4; ++q) rhs[r] -= on * e.nbrf[g][q][r] * u[4 * k2 + q];
      }
      solve4(At, rhs, &u[4 * K]);
    }
  }
}
