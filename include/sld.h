/*
 * sld.h -- C ABI of libsld: subdomain-levelset (SLD) deflated
 * Jacobi-preconditioned CG for the cell-centred two-point-flux pressure matrix
 * on a structured 3-D grid, on one GB300 GPU.
 *
 * Paper: J.H. van der Linden, T.B. Jonsthovel, A.A. Lukyanov, C. Vuik,
 * "The parallel subdomain-levelset deflation method in reservoir simulation",
 * arXiv:1510.02148.
 *   - pressure equation -div(lambda grad p) = q ............ Section 2, eq. (pressure)
 *   - linear system A x = b ................................ Section 2, eq. (coupledsys)
 *   - E = Z^T A Z, P_1 = I - A Z E^{-1} Z^T, P_2 = I - Z E^{-1} Z^T A
 *                                                     ...... Section 3.1, Def. 3.1, eqs. (E), (deflops)
 *   - x = Z E^{-1} Z^T b + P_2 xhat with P_1 A xhat = P_1 b
 *                                                     ...... Section 3.1, eqs. (defsplit), (defsys), (projectback)
 *   - subdomain / levelset / subdomain-levelset vectors .... Section 3.2.2, eq. (domdefl)
 *   - one subdomain per processor, vectors zero outside it . Section 3.2.2 (parallel SLD)
 *
 * Conventions
 *   Grid: nx * ny * nz unit cells, cell (ix, iy, iz) has index
 *         i = (iz * ny + iy) * nx + ix  (x fastest).  n = nx * ny * nz.
 *   Pointers: every array argument may be host memory or device memory of the
 *         handle's device; the library tells them apart with
 *         cudaPointerGetAttributes.  Inputs are copied into buffers the handle
 *         owns; outputs are written into the caller's memory.  Nothing is
 *         returned that the caller frees, except the handle (sld_destroy).
 *   Streams: all device work of a handle runs on the stream given to
 *         sld_build_system (NULL = the legacy default stream).  Calls that
 *         return data to host memory synchronise that stream.
 *   Errors: every call returns an sld_status; sld_last_error() gives a
 *         message (thread-local).  No call traps or asserts on the device;
 *         every device-side wait is bounded and reports SLD_ERR_TIMEOUT.
 *   Precision: the assembled operator, E, its factor and inverse, and the
 *         refinement residual are FP64.  SLD_FP32_IR runs the inner deflated
 *         iteration in FP32 (FP32 faces and vectors, FP64 coarse solve);
 *         SLD_BF16COEF_IR stores the inner stencil coefficients in BF16 with
 *         an FP32 per-cell inverse diagonal.
 *   The GPU must be sm_103 (GB300); there is no CPU fallback.
 */
#ifndef SLD_H
#define SLD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sld_system_s* sld_system; /* opaque; owns its device buffers */

typedef enum {
  SLD_OK = 0,
  SLD_ERR_INVALID_ARG = 1,      /* bad size, pointer, label, K <= 0 or not finite */
  SLD_ERR_CUDA = 2,             /* a CUDA runtime call failed (message has the CUDA error) */
  SLD_ERR_NOT_CONVERGED = 3,    /* maxiter / max_outer reached; x holds the last iterate */
  SLD_ERR_BREAKDOWN = 4,        /* p^T P A p <= 0 or a non-finite scalar in the iteration */
  SLD_ERR_COARSE_SINGULAR = 5,  /* E = Z^T A Z not SPD (Cholesky pivot <= 0) */
  SLD_ERR_TIMEOUT = 6,          /* a device-side wait ran out; the context stays usable */
  SLD_ERR_OOM = 7,              /* device allocation failed */
  SLD_ERR_STATE = 8             /* call out of order (e.g. solve before build_deflation) */
} sld_status;

/* Boundary faces, in this order: -x, +x, -y, +y, -z, +z. */
enum { SLD_BC_NOFLOW = 0, SLD_BC_DIRICHLET = 1 };

/* Inner precision of the solve. */
enum { SLD_FP64 = 0, SLD_FP32_IR = 1, SLD_BF16COEF_IR = 2 };

/* Element type of the extra dense deflation vectors given to sld_build_deflation. */
enum { SLD_ZEXTRA_F64 = 0, SLD_ZEXTRA_F32 = 1 };

typedef struct {
  int nx, ny, nz; /* cells per axis, each >= 1; unit cell size */
} sld_grid;

/*
 * type[f] = SLD_BC_NOFLOW: no flux through box face f.
 * type[f] = SLD_BC_DIRICHLET: the cells on box face f are fixed-value cells
 *   holding value[f] (identity rows; their couplings move into b, so A stays
 *   symmetric positive definite).  A cell on several Dirichlet faces takes
 *   the value of the first one in the order above.
 * At least one face must be Dirichlet for A to be nonsingular.
 */
typedef struct {
  int type[6];
  double value[6];
} sld_bc;

typedef struct {
  int precision;          /* SLD_FP64 (default), SLD_FP32_IR, SLD_BF16COEF_IR */
  double tol;             /* stop when ||b - A x||_2 <= tol * ||b||_2 (default 1e-9) */
  double inner_tol;       /* mixed modes: residual reduction per inner solve (default 1e-5) */
  int maxiter;            /* cap on iterations summed over inner solves (default 20000) */
  int max_outer;          /* mixed modes: cap on refinement steps (default 40) */
  int ctas_per_sm;        /* persistent-kernel CTAs per SM; 0 = as many as fit */
  double timeout_s;       /* bound on every device-side wait, seconds (default 2.0) */
  int debug_skip_barrier; /* test hook: CTA 0 skips the k-th barrier arrival of the
                             solve so that the other CTAs' bounded waits run out
                             (SLD_ERR_TIMEOUT); -1 = off (default) */
  double fwd_tol;         /* mixed modes: a forward-error test on top of the residual
                             test.  The refinement stops only after a step whose
                             inner solve had a relative target (a cut of at least
                             10x, not the 0.3 tol floor), reached it, and changed
                             x by at most fwd_tol * ||x||: that change estimates
                             the error of the previous iterate, which the step
                             does not increase.  A step that cut the residual
                             and shrank the correction each at least 1e3-fold
                             is also accepted when |d_k|^2 / |d_{k-1}| (its
                             error at that contraction) is <= fwd_tol / 10.
                             Where the inner precision cannot
                             resolve the slowest modes the corrections stop
                             shrinking: the test then gives up (the residual test
                             stands) once a verified correction fails to halve
                             the previous one, or after 4 steps past the residual
                             test.  With SLD_BF16COEF_IR a test that gave up
                             above fwd_tol hands the solve on: sld_solve goes on
                             from its x with SLD_FP32_IR refinement steps (FP32
                             faces made on first use), and sld_result counts
                             both parts (iterations, outer steps, solve_ms; the
                             estimate is the FP32 part's).  Without device
                             memory for the FP32 faces the BF16 result stands.
                             0 = 100 * tol (the default); < 0 = off (the
                             residual test alone: fewer steps on high-contrast
                             fields, larger error along the smallest
                             eigenvalues). */
} sld_options;

typedef struct {
  int iterations;          /* deflated-CG iterations (steps a4-a6), summed over inner solves */
  int outer_steps;         /* refinement steps; 1 for SLD_FP64 */
  double true_relres;      /* ||b - A x||_2 / ||b||_2, recomputed in FP64 after the solve */
  double recursive_relres; /* the iteration's own deflated residual at exit, / ||b|| */
  double solve_ms;         /* device time of the persistent solve kernel (CUDA events) */
  int kernel_path;         /* 1: TMA-pipelined sweeps (nx % 8 == 0), 0: register/shuffle sweeps,
                              2: batched launch (register/shuffle sweeps) */
  double fwd_err_estimate; /* mixed modes: the forward-error test's last estimate (see
                              fwd_tol): |d| / |x| of a verified step, or the
                              contraction estimate of an accepted fast step; -1 =
                              none (SLD_FP64, or the test off and never met) */
} sld_result;

/* Fill *o with the defaults listed above. */
void sld_default_options(sld_options* o);

/*
 * Assemble A and b for -div(K grad p) = q (Section 2, eq. (pressure) with
 * the total mobility lambda := K, single phase).  Two-point flux: the
 * transmissibility of the face between cells i and j is the harmonic mean
 * (2 K_i K_j) / (K_i + K_j), evaluated in that order in FP64.
 *   K: n values > 0 and finite.  q: n values or NULL (= 0).
 *   stream: a cudaStream_t (NULL = default stream).
 * On success *out is a new handle.  Errors: SLD_ERR_INVALID_ARG (sizes,
 * K <= 0 or non-finite, no Dirichlet face), SLD_ERR_OOM, SLD_ERR_CUDA.
 */
sld_status sld_build_system(const double* K, const double* q, sld_grid g, sld_bc bc,
                            void* stream, sld_system* out);

/*
 * Subdomain-levelset labels (Section 3.2.2, eq. (domdefl) per
 * (subdomain, levelset) region; one set of vectors per subdomain as in the
 * parallel form).  Subdomain of cell i: sx = floor(ix * Sx / nx) (likewise
 * y, z), s = (sz * Sy + sy) * Sx + sx.  Levelset class: the number of
 * thresholds tau[m] (m < L-1, ascending) with K_i >= tau[m].
 * label_i = s * L + class_i, so d = Sx * Sy * Sz * L.
 *   tau: L-1 values (host or device; may be NULL when L == 1).
 *   labels_out: n int32 (host or device) or NULL.
 * The labels stay on the device for sld_build_deflation(s, NULL, d, ...).
 * Errors: SLD_ERR_INVALID_ARG (S < 1 or S > grid size, L < 1, d > 65535).
 */
sld_status sld_make_labels(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L,
                           int32_t* labels_out);

/*
 * Automatic subdomain-levelset labels: the regions of sld_make_labels (one
 * per subdomain and levelset class) split into their face-connected
 * components (6-neighbour, inside the subdomain), one label per component --
 * Section 3.2.2's vectors built without manual input, the way the
 * physics-based vectors of Section 4 take one vector per layer.  Numbering:
 * components ordered by (sld_make_labels label, smallest cell index x-fastest
 * of the component), labelled 0 .. d-1.
 *   Sx, Sy, Sz, tau, L: as sld_make_labels (Sx*Sy*Sz*L <= 2^20).
 *   labels_out: n int32 (host or device) or NULL.  d_out: the number of
 *   components (host; also set when there are too many).
 * The labels stay on the device for sld_build_deflation(s, NULL, *d_out, ...).
 * Errors: SLD_ERR_INVALID_ARG (arguments; more than 4096 components, in which
 * case the handle keeps the sld_make_labels labels), SLD_ERR_OOM,
 * SLD_ERR_CUDA.
 */
sld_status sld_make_labels_cc(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L,
                              int32_t* labels_out, int* d_out);

/*
 * Deflation space Z = [Z_lab, Z_extra] (Section 3.1, Def. 3.1): Z_lab has d
 * indicator columns (column labels[i] is 1 in row i), Z_extra k dense columns.
 * Builds E = Z^T A Z (eq. (E)) on the device, pins E_cc = 1 for an empty
 * label column c, factors E = L L^T (FP64 Cholesky) and forms E^{-1}.
 *   labels: n int32 in [0, d), or NULL to use those of sld_make_labels.
 *   d: 1 .. 4096.
 *   Zextra: n x k values, row-major (the k values of cell i contiguous), host
 *     or device memory, FP64 or FP32 as zextra_dtype says (SLD_ZEXTRA_F64,
 *     SLD_ZEXTRA_F32); NULL when k == 0.  k: 0 .. 8.  The values are rounded
 *     to FP32 and those rounded vectors are the extra columns.  The solver
 *     keeps them with W = A Z_extra (FP64 and FP32): k * 20 bytes per cell.
 *     The Cholesky factorisation bounds the extra columns' pivots relative
 *     to their diagonal (1e-10); if that fails (a column numerically in the
 *     span of the others), the extra columns are dropped and the label
 *     deflation alone is built -- sld_deflation_info reports k_used = 0.
 *     Extra columns need the TMA solve path (nx % 8 == 0), SLD_FP64 or
 *     SLD_FP32_IR, and a single (not batched) solve.
 * Errors: SLD_ERR_INVALID_ARG (label out of range, k out of range, Zextra
 * NULL with k > 0 or non-finite), SLD_ERR_COARSE_SINGULAR (a label pivot
 * <= 0), SLD_ERR_TIMEOUT, SLD_ERR_CUDA.
 */
sld_status sld_build_deflation(sld_system s, const int32_t* labels, int d, const void* Zextra,
                               int k, int zextra_dtype);

/* The deflation last built: d label columns, the k extra columns asked
 * for, and k_used (k, or 0 if they were dropped).  Any pointer may be NULL.
 * Errors: SLD_ERR_STATE (no deflation built). */
sld_status sld_deflation_info(sld_system s, int* d, int* k_requested, int* k_used);

/*
 * Solve A x = b by SLD-deflated Jacobi-PCG (the CG form of the deflated
 * solve of Section 3.1: iterate on P_1 A xhat = P_1 b, M = diag(A), then
 * x = Z E^{-1} Z^T b + P_2 xhat, eq. (projectback)).  One cooperative
 * persistent kernel runs every iteration; in the mixed modes an FP64
 * refinement loop (residual, coarse correction, x update) wraps FP32 inner
 * solves inside the same launch.
 *   b: n values, or NULL for the assembled right-hand side.
 *   o: options or NULL for the defaults.
 *   x: n values (output).  res: may be NULL.
 * With the environment variable SLD_TRACE_REFINEMENT set, a mixed-mode
 * solve prints |d_k| / |x_k| and ||r_k|| / ||b|| of its first 16
 * refinement steps to stderr.
 * Errors: SLD_ERR_STATE (no deflation built), SLD_ERR_NOT_CONVERGED (x and
 * res still written), SLD_ERR_BREAKDOWN (with SLD_FP64 and finite scalars x
 * and res are still written: x = x* + P_2 xhat of the last iterate before
 * p^T P A p <= 0, the progress made), SLD_ERR_TIMEOUT, SLD_ERR_CUDA.
 */
sld_status sld_solve(sld_system s, const double* b, const sld_options* o, double* x,
                     sld_result* res);

/*
 * PDGMRES: restarted GMRES(m), right-preconditioned with Jacobi (M = diag A),
 * deflated with the system's label columns Z (Section 3.2, the deflated
 * GMRES of the paper with the physics-based vectors of Section 3.2.2 fixed
 * before the iteration; its remark on right preconditioning: the deflation
 * operators use A, not A M^{-1}):
 *   E = Z^T A Z, P1 = I - A Z E^{-1} Z^T, P2 = I - Z E^{-1} Z^T A,
 *   x* = Z E^{-1} Z^T b,  GMRES(m) on P1 A M^{-1} u = P1 b,
 *   x = P2 M^{-1} u + x*   (b - A x = P1 (b - A M^{-1} u): the GMRES
 *   residual is the residual of x).
 * FP64 throughout; Arnoldi by classical Gram-Schmidt with one
 * reorthogonalisation; the Givens least-squares problem on the host.  Each
 * cycle starts from the recomputed residual; a cycle ends after m steps, or
 * when ||b - A x|| <= tol ||b|| by the Givens estimate, or at maxiter steps.
 *   b: n values (host or device), or NULL for the assembled rhs.
 *   m: 1 .. 31 (cycle length).  deflate: 1 = use the label columns (needs
 *   sld_build_deflation, label columns only), 0 = plain GMRES(m).
 *   tol: in (0, 1).  maxiter >= 1: Arnoldi steps over all cycles.
 *   x: n values (output, host or device).  info: may be NULL.
 * Work space: (m + 4) n FP64 on the device, allocated per call.
 * Errors: SLD_ERR_INVALID_ARG, SLD_ERR_STATE, SLD_ERR_OOM, SLD_ERR_CUDA,
 * SLD_ERR_NOT_CONVERGED (x and info still written).
 */
typedef struct {
  int iterations;          /* Arnoldi steps over all cycles */
  int cycles;              /* restart cycles */
  double relres_estimate;  /* ||b - A x|| / ||b|| from the Givens recurrence at exit */
  double true_relres;      /* ||b - A x|| / ||b||, recomputed in FP64 from x */
  double solve_ms;         /* device time of the whole solve (CUDA events) */
} sld_gmres_info;

sld_status sld_solve_gmres(sld_system s, const double* b, int m, int deflate, double tol, int maxiter,
                           double* x, sld_gmres_info* info);

/*
 * RDGMRES: restarted GMRES(m) with harmonic-Ritz deflation (Section 3.2.1 and
 * its algorithm).  The first cycle is plain right-preconditioned GMRES(m)
 * (M = diag A) in the preconditioned variable u (x = M^{-1} u); its d
 * harmonic Ritz vectors of smallest |theta| (sld_harmonic_ritz) give
 * Z = V_m Y, and with B = A M^{-1}, E = Z^T B Z, P1 = I - B Z E^{-1} Z^T,
 * P2 = I - Z E^{-1} Z^T B the remaining cycles solve P1 B t = P1 r1
 * (r1 = b - B u1); x = M^{-1} (u1 + P2 t + Z E^{-1} Z^T r1).  FP64; the
 * kernels of sld_solve_gmres.  Needs no label deflation.
 *   b: n values (host or device) or NULL (the assembled rhs).  2 <= m <= 31,
 *   1 <= d <= min(8, m), tol in (0, 1), maxiter >= 1.  x: n values (output).
 * Work space: (m + 2 d + 7) n FP64 on the device, per call.
 * Errors: SLD_ERR_INVALID_ARG, SLD_ERR_OOM, SLD_ERR_CUDA, SLD_ERR_BREAKDOWN
 * (harmonic Ritz pairs), SLD_ERR_COARSE_SINGULAR (E singular),
 * SLD_ERR_NOT_CONVERGED (x and info still written).
 */
sld_status sld_solve_rdgmres(sld_system s, const double* b, int m, int d, double tol, int maxiter, double* x,
                             sld_gmres_info* info);

/*
 * Harmonic Ritz pairs of an Arnoldi cycle (host computation; Section 3.2.1,
 * eq. (defleig) form (a)): with the (m+1) x m Hessenberg matrix Hbar of m
 * Arnoldi steps, F = H_m + h_{m+1,m}^2 H_m^{-T} e_m e_m^T, F y = theta y;
 * the d pairs of smallest |theta| (a complex-conjugate pair as the real and
 * imaginary parts of y, the next two columns).  The deflation vectors are
 * z = V_m y.  Eigenvalues by the Francis double-shift QR iteration, vectors
 * by inverse iteration.
 *   Hbar: (m+1) x m, row-major, host.  2 <= m <= 64, 1 <= d <= m.
 *   Y: m x d row-major (host, output); theta_re, theta_im: d values (host).
 * Errors: SLD_ERR_INVALID_ARG, SLD_ERR_BREAKDOWN (singular H_m or no
 * convergence of the QR iteration).
 */
sld_status sld_harmonic_ritz(const double* Hbar, int m, int d, double* Y, double* theta_re, double* theta_im);

/* Release the handle and its device memory.  NULL is ignored. */
void sld_destroy(sld_system s);

/* ---------------------------------------------------------------------- */
/* Batched solves: many independent systems in one persistent launch.     */
/* ---------------------------------------------------------------------- */

typedef struct sld_batch_s* sld_batch; /* opaque plan; does not own the systems */

/*
 * Plan a batched solve of `count` systems (each built up to
 * sld_build_deflation, all on one device; the stream of systems[0] is used).
 * Every system gets its own team of CTAs in one cooperative launch -- a
 * share proportional to n^e with e in {1, 4/3} -- with its own barriers and
 * reductions; teams never wait on each other and leave as soon as their
 * system is solved.  The launch and the resets of every system's state are
 * captured in one CUDA graph.  With o->ctas_per_sm == 0 the plan is tuned:
 * each candidate launch shape (team exponent, cells per lane) solves the
 * batch once with the assembled right-hand sides and the fastest is kept
 * (sld_batch_describe lists them).  This is the parallel subdomain idea of
 * Section 3.2.2 applied across systems: independent problems share the GPU.
 *   o: SLD_FP64 or SLD_FP32_IR; NULL = defaults.
 * Errors: SLD_ERR_INVALID_ARG (count > co-resident CTAs, mixed devices,
 * a system twice), SLD_ERR_STATE (no deflation), SLD_ERR_CUDA.
 */
sld_status sld_batch_create(sld_system* systems, int count, const sld_options* o, sld_batch* out);

/*
 * Run the plan: b[k] (n_k values, host or device; b or b[k] NULL = the
 * assembled right-hand side) -> x[k] (n_k values, host or device; x or x[k]
 * may be NULL).  res (count entries, may be NULL) gets each system's
 * iterations, refinement steps and FP64 true residual; solve_ms is the time
 * of the whole batched launch; kernel_path = 2.  Returns the first failing
 * system's status (the others are still solved and reported).
 */
sld_status sld_batch_solve(sld_batch bt, const double* const* b, double* const* x, sld_result* res);

/* Text description of the plan (CTAs, teams, tuning times). */
const char* sld_batch_describe(sld_batch bt);

/* Release the plan (not the systems).  NULL is ignored. */
void sld_batch_destroy(sld_batch bt);

/* sld_batch_create + sld_batch_solve + sld_batch_destroy. */
sld_status sld_solve_batched(sld_system* systems, int count, const double* const* b, const sld_options* o,
                             double* const* x, sld_result* res);

/* Message of the last failed call on this thread ("" if none). */
const char* sld_last_error(void);

/* ---------------------------------------------------------------------- */
/* Per-step access, for parity tests of the individual steps.             */
/* ---------------------------------------------------------------------- */

/*
 * Copy out the assembled FP64 operator: face transmissibilities Tx, Ty, Tz
 * (face between cell i and its +x / +y / +z neighbour, stored at i; 0 on the
 * box boundary; couplings to Dirichlet cells included), the diagonal A_ii and
 * the right-hand side b.  Any pointer may be NULL.  n values each.
 */
sld_status sld_get_operator(sld_system s, double* Tx, double* Ty, double* Tz, double* diag,
                            double* b);

/* y = A x with the FP64 operator (n values each). */
sld_status sld_apply_A(sld_system s, const double* x, double* y);

/* out = Z^T v (d values; the segmented sum over labels), FP64. */
sld_status sld_restrict(sld_system s, const double* v, double* out);

/* Copy out E (D*D, row-major, D = d + k_used: label columns first, then the
 * extra columns) and E^{-1} (D*D); either may be NULL. */
sld_status sld_get_coarse(sld_system s, double* E, double* Einv);

/* ---------------------------------------------------------------------- */
/* Allocation-free variant.                                               */
/* ---------------------------------------------------------------------- */

/*
 * out = Z^T v, like sld_restrict, but without allocating any device memory
 * (no cudaMalloc, cudaFree or allocating library call).  The paper has no
 * counterpart: this exists for callers that cannot allocate -- processes
 * whose device memory is already handed to another allocator (a framework's
 * pool or arena, a hard memory cap) and loops that must not pay for
 * cudaMalloc / cudaFree, which can block and (cudaFree) synchronise the
 * device.
 *   v: n values in device memory; out: d values in device memory (host
 *   pointers are rejected: staging them would need a buffer).  d <= 1024.
 *   The handle's device must be the current device, and v and out must be
 *   memory of that same GPU (or managed memory): device memory of another
 *   GPU is rejected, since the kernels would read it directly.
 * Work runs on the handle's stream and is asynchronous: out is valid once
 * that stream has reached the call.  The partial sums go to a fixed 1 MiB
 * __device__ array (128 CTAs x 1024 labels) that every GPU loading the
 * library keeps until the process exits.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  Every call
 * shares the array and overwrites what it reads, so calls whose kernels
 * overlap on the GPU (other streams, other host threads) race.
 * Errors: SLD_ERR_INVALID_ARG (d > 1024, host pointer, another GPU's
 * memory, wrong current device), SLD_ERR_STATE (no deflation built), SLD_ERR_CUDA.
 */
sld_status sld_restrict_noalloc(sld_system s, const double* v, double* out);

#ifdef __cplusplus
}
#endif
#endif /* SLD_H */
