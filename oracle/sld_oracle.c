/*
 * sld_oracle.c -- plain, slow CPU FP64 oracle for subdomain-levelset (SLD)
 * deflated Jacobi-preconditioned CG on the cell-centred two-point-flux
 * pressure matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both only consume the same
 * seeded inputs.
 *
 * Everything is written from the definitions, in the most direct form:
 *   - the matrix is assembled cell by cell into a CSR matrix (diagonal plus
 *     up to six neighbours), never as face arrays;
 *   - the deflation matrix Z is held explicitly (a CSR indicator part plus an
 *     optional dense part), AZ is formed by sparse products and
 *     E = Z^T (A Z) by a second product (Def. 3.1, eq. (E));
 *   - E is factorised by an unpivoted Cholesky that fails on a pivot <= 0;
 *   - the deflated system P A xhat = P b (eq. (defsys)) is solved by
 *     Jacobi-preconditioned CG with the projection applied explicitly,
 *     w = A p - AZ E^{-1} Z^T A p (eq. (deflops), P = P_1);
 *   - the solution is recovered by eq. (projectback):
 *     x = Z E^{-1} Z^T b + P_2 xhat with P_2 = P_1^T for symmetric A.
 *
 * Paper: van der Linden, Jonsthovel, Lukyanov, Vuik, "The parallel
 * subdomain-levelset deflation method in reservoir simulation",
 * arXiv:1510.02148.  Section 2 (pressure equation), Section 3.1
 * (Def. 3.1, eqs. (E), (deflops), (defsplit), (defsys), (projectback)),
 * Section 3.2.2 (eq. (domdefl), subdomain-levelset deflation).
 * The discretisation (TPFA, harmonic mean), the CG form of the iteration and
 * the Dirichlet-cell treatment are readings: the paper only says
 * "finite-volume" and uses GMRES.
 *
 * Parity pins (checked by tests, not by this file): closed-form linear
 * pressure, series-resistance flux of a 1-D column, dense direct solves on
 * tiny grids, dense Z^T A Z, the invariants P A Z = 0 and Z^T r_k = 0, SciPy
 * CG for d = 0, and dense eigenvalue counts (Theorem 3.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_CONVERGED 3
#define OR_ERR_BREAKDOWN 4
#define OR_ERR_SINGULAR 5
#define OR_ERR_OOM 7

/* Boundary faces of the box, in this order: -x, +x, -y, +y, -z, +z. */
#define BC_NOFLOW 0
#define BC_DIRICHLET 1

/* Parallel loops only above this size, so small cases run serially. */
#define PAR_MIN 65536

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Dirichlet cells (a reading: the paper gives no boundary treatment).       */
/* A cell lying on a box face marked Dirichlet is a fixed-value cell.  When a */
/* cell lies on several such faces the first one in the order above wins.   */
/* ------------------------------------------------------------------------ */
static int dirichlet_face_of(int nx, int ny, int nz, int ix, int iy, int iz, const int* bct) {
  if (bct[0] == BC_DIRICHLET && ix == 0) return 0;
  if (bct[1] == BC_DIRICHLET && ix == nx - 1) return 1;
  if (bct[2] == BC_DIRICHLET && iy == 0) return 2;
  if (bct[3] == BC_DIRICHLET && iy == ny - 1) return 3;
  if (bct[4] == BC_DIRICHLET && iz == 0) return 4;
  if (bct[5] == BC_DIRICHLET && iz == nz - 1) return 5;
  return -1;
}

/*
 * Assemble A and b for -div(K grad p) = q (Section 2, eq. (pressure) with the
 * mobility lambda := K) on unit cells.  Two-point flux: the transmissibility
 * between neighbouring cells i and j is the harmonic mean 2 K_i K_j / (K_i+K_j).
 *
 * Free cell i:   A_ii = sum of the transmissibilities of all its faces
 *                A_ij = -T_ij for free neighbours j
 *                b_i  = q_i + sum over Dirichlet neighbours j of T_ij g_j
 * Dirichlet cell: identity row, b_i = g_i.
 *
 * CSR output, columns ascending.  rowptr has n+1 entries, col/val at most 7n.
 */
int oracle_assemble(int nx, int ny, int nz, const double* K, const double* q, const int* bct,
                    const double* bcv, int64_t* rowptr, int32_t* col, double* val, double* b,
                    uint8_t* is_dirichlet) {
  if (nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < n; ++i)
    if (!(K[i] > 0.0) || !isfinite(K[i])) return OR_ERR_ARG;
  int64_t nnz = 0;
  rowptr[0] = 0;
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        const int64_t i = ((int64_t)iz * ny + iy) * nx + ix;
        const int fi = dirichlet_face_of(nx, ny, nz, ix, iy, iz, bct);
        is_dirichlet[i] = (uint8_t)(fi >= 0);
        if (fi >= 0) {
          col[nnz] = (int32_t)i;
          val[nnz] = 1.0;
          ++nnz;
          b[i] = bcv[fi];
          rowptr[i + 1] = nnz;
          continue;
        }
        /* Neighbours in ascending index order: -z, -y, -x, (self), +x, +y, +z. */
        int jx[6] = {ix, ix, ix - 1, ix + 1, ix, ix};
        int jy[6] = {iy, iy - 1, iy, iy, iy + 1, iy};
        int jz[6] = {iz - 1, iz, iz, iz, iz, iz + 1};
        double diag = 0.0;
        double rhs = q ? q[i] : 0.0;
        int64_t self_pos = -1;
        for (int m = 0; m < 6; ++m) {
          if (m == 3) { /* the diagonal sits between -x and +x */
            self_pos = nnz;
            col[nnz] = (int32_t)i;
            val[nnz] = 0.0;
            ++nnz;
          }
          if (jx[m] < 0 || jx[m] >= nx || jy[m] < 0 || jy[m] >= ny || jz[m] < 0 || jz[m] >= nz)
            continue; /* no-flow (or absent) box face: no flux */
          const int64_t j = ((int64_t)jz[m] * ny + jy[m]) * nx + jx[m];
          const double Ki = K[i], Kj = K[j];
          const double T = (2.0 * Ki * Kj) / (Ki + Kj);
          diag += T;
          const int fj = dirichlet_face_of(nx, ny, nz, jx[m], jy[m], jz[m], bct);
          if (fj >= 0) {
            rhs += T * bcv[fj]; /* coupling to a fixed value moves to the rhs */
          } else {
            col[nnz] = (int32_t)j;
            val[nnz] = -T;
            ++nnz;
          }
        }
        val[self_pos] = diag;
        b[i] = rhs;
        rowptr[i + 1] = nnz;
      }
  return OR_OK;
}

/* y = A x (CSR). */
void oracle_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static) if (n > PAR_MIN)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/*
 * Subdomain-levelset labels (Section 3.2.2, eq. (domdefl) applied per
 * (subdomain, levelset) region; the parallel form gives every subdomain its
 * own vectors).  Subdomain index from integer division of the cell
 * coordinates; levelset class = number of thresholds tau_m with K_i >= tau_m.
 * label = subdomain * L + class.
 */
int oracle_labels(int nx, int ny, int nz, const double* K, int Sx, int Sy, int Sz,
                  const double* tau, int L, int32_t* label) {
  if (Sx < 1 || Sy < 1 || Sz < 1 || L < 1 || Sx > nx || Sy > ny || Sz > nz) return OR_ERR_ARG;
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        const int64_t i = ((int64_t)iz * ny + iy) * nx + ix;
        const int64_t sx = ((int64_t)ix * Sx) / nx;
        const int64_t sy = ((int64_t)iy * Sy) / ny;
        const int64_t sz = ((int64_t)iz * Sz) / nz;
        int cls = 0;
        for (int m = 0; m < L - 1; ++m)
          if (K[i] >= tau[m]) ++cls;
        label[i] = (int32_t)(((sz * Sy + sy) * Sx + sx) * L + cls);
      }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Deflation space Z = [Z_lab, Z_dense]:                                     */
/*   Z_lab  : n x d indicator matrix, column label[i] has a 1 in row i       */
/*   Z_dense: n x k dense (row-major, k values per cell), may be absent      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n;
  int d, k, dt;          /* dt = d + k */
  const int32_t* label;  /* may be NULL when d == 0 */
  const double* Zd;      /* n*k, may be NULL when k == 0 */
  /* AZ in CSR over the dt columns (the indicator part is sparse) */
  int64_t* az_ptr;
  int32_t* az_col;
  double* az_val;
  double* E;             /* dt x dt */
  double* Lc;            /* Cholesky factor, lower, dt x dt */
} defl_t;

/* s = Z^T v */
static void Zt_apply(const defl_t* D, const double* v, double* s) {
  for (int c = 0; c < D->dt; ++c) s[c] = 0.0;
  for (int64_t i = 0; i < D->n; ++i) {
    if (D->d > 0) s[D->label[i]] += v[i];
    for (int c = 0; c < D->k; ++c) s[D->d + c] += D->Zd[i * D->k + c] * v[i];
  }
}

/* v = Z y */
static void Z_apply(const defl_t* D, const double* y, double* v) {
#pragma omp parallel for schedule(static) if (D->n > PAR_MIN)
  for (int64_t i = 0; i < D->n; ++i) {
    double s = 0.0;
    if (D->d > 0) s += y[D->label[i]];
    for (int c = 0; c < D->k; ++c) s += D->Zd[i * D->k + c] * y[D->d + c];
    v[i] = s;
  }
}

/* v = (AZ) y */
static void AZ_apply(const defl_t* D, const double* y, double* v) {
#pragma omp parallel for schedule(static) if (D->n > PAR_MIN)
  for (int64_t i = 0; i < D->n; ++i) {
    double s = 0.0;
    for (int64_t e = D->az_ptr[i]; e < D->az_ptr[i + 1]; ++e) s += D->az_val[e] * y[D->az_col[e]];
    v[i] = s;
  }
}

/* Solve E y = s with the Cholesky factor (forward then backward). */
static void coarse_solve(const defl_t* D, const double* s, double* y) {
  const int m = D->dt;
  const double* L = D->Lc;
  for (int i = 0; i < m; ++i) {
    double t = s[i];
    for (int j = 0; j < i; ++j) t -= L[(int64_t)i * m + j] * y[j];
    y[i] = t / L[(int64_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double t = y[i];
    for (int j = i + 1; j < m; ++j) t -= L[(int64_t)j * m + i] * y[j];
    y[i] = t / L[(int64_t)i * m + i];
  }
}

/* Unpivoted Cholesky E = L L^T; fails on a pivot <= 0 (E not SPD). */
int oracle_cholesky(int m, const double* E, double* L) {
  memset(L, 0, sizeof(double) * (size_t)m * m);
  for (int j = 0; j < m; ++j) {
    double s = E[(int64_t)j * m + j];
    for (int p = 0; p < j; ++p) s -= L[(int64_t)j * m + p] * L[(int64_t)j * m + p];
    if (!(s > 0.0)) return OR_ERR_SINGULAR;
    const double ljj = sqrt(s);
    L[(int64_t)j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double t = E[(int64_t)i * m + j];
      for (int p = 0; p < j; ++p) t -= L[(int64_t)i * m + p] * L[(int64_t)j * m + p];
      L[(int64_t)i * m + j] = t / ljj;
    }
  }
  return OR_OK;
}

/*
 * Build AZ (sparse, by the product of the CSR matrix with the explicit Z) and
 * E = Z^T (AZ) (Def. 3.1, eq. (E)).  A column of Z that is empty (no cell
 * carries that label) would make E singular; its diagonal entry is set to 1,
 * which leaves the deflated operator unchanged since that column of Z is 0.
 */
static int build_defl(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                      defl_t* D) {
  const int dt = D->dt;
  /* per-row AZ: at most 7 distinct label columns plus k dense columns */
  const int maxrow = 7 + D->k;
  D->az_ptr = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  D->az_col = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * maxrow);
  D->az_val = (double*)malloc(sizeof(double) * (size_t)n * maxrow);
  D->E = (double*)calloc((size_t)dt * dt, sizeof(double));
  D->Lc = (double*)calloc((size_t)dt * dt, sizeof(double));
  if (!D->az_ptr || !D->az_col || !D->az_val || !D->E || !D->Lc) return OR_ERR_OOM;
  /* dense part of AZ: A applied to each dense column */
  double* AZd = NULL;
  if (D->k > 0) {
    AZd = (double*)malloc(sizeof(double) * (size_t)n * D->k);
    double* colv = (double*)malloc(sizeof(double) * n);
    double* outv = (double*)malloc(sizeof(double) * n);
    if (!AZd || !colv || !outv) return OR_ERR_OOM;
    for (int c = 0; c < D->k; ++c) {
      for (int64_t i = 0; i < n; ++i) colv[i] = D->Zd[i * D->k + c];
      oracle_spmv(n, rp, ci, va, colv, outv);
      for (int64_t i = 0; i < n; ++i) AZd[i * D->k + c] = outv[i];
    }
    free(colv);
    free(outv);
  }
  int64_t pos = 0;
  D->az_ptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t start = pos;
    if (D->d > 0) {
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int32_t c = D->label[ci[e]];
        int64_t f = start;
        while (f < pos && D->az_col[f] != c) ++f;
        if (f == pos) {
          D->az_col[pos] = c;
          D->az_val[pos] = 0.0;
          ++pos;
        }
        D->az_val[f] += va[e];
      }
    }
    for (int c = 0; c < D->k; ++c) {
      D->az_col[pos] = D->d + c;
      D->az_val[pos] = AZd[i * D->k + c];
      ++pos;
    }
    D->az_ptr[i + 1] = pos;
  }
  free(AZd);
  /* E = Z^T (AZ): row i of AZ is added into row label[i] of E, and
     Zd[i][c] times row i of AZ into row d+c. */
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = D->az_ptr[i]; e < D->az_ptr[i + 1]; ++e) {
      const int32_t c = D->az_col[e];
      if (D->d > 0) D->E[(int64_t)D->label[i] * dt + c] += D->az_val[e];
      for (int r = 0; r < D->k; ++r) D->E[(int64_t)(D->d + r) * dt + c] += D->Zd[i * D->k + r] * D->az_val[e];
    }
  }
  if (D->d > 0) {
    int64_t* cnt = (int64_t*)calloc(D->d, sizeof(int64_t));
    if (!cnt) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) cnt[D->label[i]]++;
    for (int c = 0; c < D->d; ++c)
      if (cnt[c] == 0) D->E[(int64_t)c * dt + c] = 1.0;
    free(cnt);
  }
  return oracle_cholesky(dt, D->E, D->Lc);
}

static void free_defl(defl_t* D) {
  free(D->az_ptr);
  free(D->az_col);
  free(D->az_val);
  free(D->E);
  free(D->Lc);
}

static int check_labels(int64_t n, const int32_t* label, int d) {
  for (int64_t i = 0; i < n; ++i)
    if (label[i] < 0 || label[i] >= d) return OR_ERR_ARG;
  return OR_OK;
}

/* E = Z^T A Z (and its Cholesky factor) for the given Z; E_out and L_out are
   (d+k)^2, either may be NULL. */
int oracle_coarse(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                  const int32_t* label, int d, const double* Zd, int k, double* E_out,
                  double* L_out) {
  if (d < 0 || k < 0 || d + k < 1) return OR_ERR_ARG;
  if (d > 0 && check_labels(n, label, d) != OR_OK) return OR_ERR_ARG;
  defl_t D;
  memset(&D, 0, sizeof(D));
  D.n = n; D.d = d; D.k = k; D.dt = d + k; D.label = label; D.Zd = Zd;
  int st = build_defl(n, rp, ci, va, &D);
  if (D.E && E_out) memcpy(E_out, D.E, sizeof(double) * (size_t)D.dt * D.dt);
  if (st == OR_OK && L_out) memcpy(L_out, D.Lc, sizeof(double) * (size_t)D.dt * D.dt);
  free_defl(&D);
  return st;
}

/* s = Z^T v (d + k values) */
int oracle_restrict(int64_t n, const int32_t* label, int d, const double* Zd, int k,
                    const double* v, double* s) {
  if (d > 0 && check_labels(n, label, d) != OR_OK) return OR_ERR_ARG;
  defl_t D;
  memset(&D, 0, sizeof(D));
  D.n = n; D.d = d; D.k = k; D.dt = d + k; D.label = label; D.Zd = Zd;
  Zt_apply(&D, v, s);
  return OR_OK;
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static) if (n > PAR_MIN)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/*
 * Deflated Jacobi-PCG (the CG form of the deflated solve of Section 3.1).
 *
 * Input: CSR A (SPD), b, labels (d columns of Z_lab, d may be 0), optional
 * dense columns Zd (k), tolerance tol on ||rhat||_2 / ||b||_2, maxiter.
 * Output: x (full solution), iterations, true relative residual
 * ||b - A x|| / ||b||, and optionally per-iteration ||rhat_k|| / ||b||
 * (hist, maxiter+1 entries) and max_k ||Z^T rhat_k|| / ||b|| (ztr_max), a
 * check of the projection: Z^T P = 0, so in exact arithmetic Z^T rhat_k = 0;
 * in floating point it stays at roundoff relative to ||b||.
 *
 *   P   = I - AZ E^{-1} Z^T            (eq. (deflops), P_1)
 *   rhat_0 = P b, xhat_0 = 0           (deflated system, eq. (defsys))
 *   z = M^{-1} rhat, M = diag(A);  p = z;  rho = rhat^T z
 *   loop:  w = P A p;  alpha = rho / p^T w
 *          xhat += alpha p;  rhat -= alpha w;  stop if ||rhat|| <= tol ||b||
 *          z = M^{-1} rhat;  rho' = rhat^T z;  p = z + (rho'/rho) p
 *   x = Z E^{-1} Z^T b + P^T xhat      (eq. (projectback), P_2 = P_1^T)
 */
int oracle_dpcg(int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                const double* b, const int32_t* label, int d, const double* Zd, int k,
                double tol, int maxiter, double* x, int* iterations, double* true_relres,
                double* hist, double* ztr_max) {
  if (d < 0 || k < 0) return OR_ERR_ARG;
  if (d > 0 && check_labels(n, label, d) != OR_OK) return OR_ERR_ARG;
  const int dt = d + k;
  defl_t D;
  memset(&D, 0, sizeof(D));
  D.n = n; D.d = d; D.k = k; D.dt = dt; D.label = label; D.Zd = Zd;
  int st = OR_OK;
  if (dt > 0) {
    st = build_defl(n, rp, ci, va, &D);
    if (st != OR_OK) {
      free_defl(&D);
      return st;
    }
  }
  double* diag = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* xh = (double*)calloc(n, sizeof(double));
  double* z = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* s = (double*)malloc(sizeof(double) * (dt > 0 ? dt : 1));
  double* y = (double*)malloc(sizeof(double) * (dt > 0 ? dt : 1));
  double* yb = (double*)malloc(sizeof(double) * (dt > 0 ? dt : 1));
  if (!diag || !r || !xh || !z || !p || !v || !w || !s || !y || !yb) {
    st = OR_ERR_OOM;
    goto done;
  }
  for (int64_t i = 0; i < n; ++i) {
    diag[i] = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) diag[i] = va[e];
  }
  const double bnorm = sqrt(dot(n, b, b));
  double ztr = 0.0;
  /* rhat_0 = P b */
  if (dt > 0) {
    Zt_apply(&D, b, s);
    coarse_solve(&D, s, yb); /* E^{-1} Z^T b, reused for x* below */
    AZ_apply(&D, yb, v);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - v[i];
  } else {
    memcpy(r, b, sizeof(double) * n);
  }
  double rr = dot(n, r, r);
  if (hist) hist[0] = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
  if (dt > 0 && bnorm > 0) {
    Zt_apply(&D, r, s);
    double m = 0;
    for (int c = 0; c < dt; ++c) m += s[c] * s[c];
    ztr = sqrt(m) / bnorm;
  }
  int it = 0;
  int converged = (sqrt(rr) <= tol * bnorm);
  if (!converged) {
    for (int64_t i = 0; i < n; ++i) z[i] = r[i] / diag[i];
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot(n, r, z);
    while (it < maxiter) {
      ++it;
      oracle_spmv(n, rp, ci, va, p, v); /* v = A p */
      if (dt > 0) {                     /* w = P v = v - AZ E^{-1} Z^T v */
        Zt_apply(&D, v, s);
        coarse_solve(&D, s, y);
        AZ_apply(&D, y, w);
        for (int64_t i = 0; i < n; ++i) w[i] = v[i] - w[i];
      } else {
        memcpy(w, v, sizeof(double) * n);
      }
      const double pw = dot(n, p, w);
      if (!(pw > 0.0) || !isfinite(rho)) {
        st = OR_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rho / pw;
      for (int64_t i = 0; i < n; ++i) {
        xh[i] += alpha * p[i];
        r[i] -= alpha * w[i];
      }
      rr = dot(n, r, r);
      if (hist) hist[it] = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
      if (dt > 0 && bnorm > 0) {
        Zt_apply(&D, r, s);
        double m = 0;
        for (int c = 0; c < dt; ++c) m += s[c] * s[c];
        const double q = sqrt(m) / bnorm;
        if (q > ztr) ztr = q;
      }
      if (sqrt(rr) <= tol * bnorm) {
        converged = 1;
        break;
      }
      for (int64_t i = 0; i < n; ++i) z[i] = r[i] / diag[i];
      const double rho_new = dot(n, r, z);
      const double beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rho = rho_new;
    }
  }
  /* x = Z E^{-1} Z^T b + P^T xhat,  P^T xhat = xhat - Z E^{-1} Z^T A xhat */
  if (dt > 0) {
    oracle_spmv(n, rp, ci, va, xh, v);
    Zt_apply(&D, v, s);
    coarse_solve(&D, s, y);
    for (int c = 0; c < dt; ++c) y[c] = yb[c] - y[c];
    Z_apply(&D, y, w);
    for (int64_t i = 0; i < n; ++i) x[i] = xh[i] + w[i];
  } else {
    memcpy(x, xh, sizeof(double) * n);
  }
  oracle_spmv(n, rp, ci, va, x, v);
  for (int64_t i = 0; i < n; ++i) v[i] = b[i] - v[i];
  if (true_relres) *true_relres = bnorm > 0 ? sqrt(dot(n, v, v)) / bnorm : 0.0;
  if (iterations) *iterations = it;
  if (ztr_max) *ztr_max = ztr;
  if (st == OR_OK && !converged) st = OR_ERR_NOT_CONVERGED;
done:
  free(diag); free(r); free(xh); free(z); free(p); free(v); free(w);
  free(s); free(y); free(yb);
  if (dt > 0) free_defl(&D);
  return st;
}
