// sld_internal.h -- internal types of libsld: the handle, launch arguments,
// and the launchers each translation unit provides.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sld.h"

namespace sld {

// Tile of the persistent sweeps: each warp owns one grid row of TX cells
// (32 lanes x CX cells), a CTA owns TY consecutive rows plus two halo rows
// (one warp each) and marches through a range of z planes.
constexpr int kTY = 8;                  // rows per tile
constexpr int kWarps = kTY + 2;         // + two halo-row warps
constexpr int kThreads = kWarps * 32;   // 320
constexpr int kMaxD = 4096;             // largest d (labels) the kernels take
constexpr int kWarpAccMaxD = 256;       // per-warp label rows in shared memory up to this d (global above)
constexpr int kGaccRows = kWarps > 8 ? kWarps : 8;  // warp rows per CTA in the global label-sum rows
constexpr int kPartScalars = 8;         // scalar slots after the dk coarse sums
constexpr int kMaxL = 8;                // extra dense deflation vectors (slots per cell)

struct SyncArgs {
  unsigned* count;                // arrival counter of the team, zeroed before the launch
  int cta0, ncta;                 // the team: CTAs cta0 .. cta0+ncta-1 of the launch
  int* status;                    // 0 or an sld_status, written on error
  unsigned long long timeout_ns;  // bound on every wait
  int skip_epoch;                 // test hook: CTA 0 does not arrive at this barrier (0 = off)
};

struct Geo {
  int nx, ny, nz;
  int64_t nxy, n;
  unsigned dlo_x, dhi_x, dlo_y, dhi_y, dlo_z, dhi_z;  // Dirichlet faces
};

// Everything the persistent solve kernel reads and writes for one system.
// The system is solved by a team of CTAs (all of them for a single solve,
// a share of them in a batched solve): sy.cta0 .. sy.cta0 + sy.ncta - 1.
struct SolveArgs {
  Geo g;
  int cx;                 // cells per lane in x (1 or 4)
  int vp;                 // row pitch (cells) of the inner vectors and inner faces
  int64_t vpxy;           // vp * ny: plane pitch
  int ntx, nty;           // column tiles in x and y
  int64_t ntiles;         // ntx * nty * nz plane-tiles
  int d;                  // label columns of Z
  int kL;                 // extra dense columns of Z (0 .. kMaxL)
  int dk;                 // coarse dimension d + kL
  const int32_t* label;
  const uint16_t* label16;  // the same labels as 16-bit (streamed by the TMA sweeps)
  int lab_L;                // labels are subdomain * lab_L + class (1..4), or 0: any labels
  const double* Einv;     // d x d, E = Z^T A Z of the FP64 operator (refinement steps)
  const double* Einv_inner;  // the inverse used by the inner iterations (E of their operator)
  const float* invdi;     // BF16 form: FP32 inverse diagonal of the quantized operator
  // extra dense columns: Z_L (FP32 values, kMaxL per cell), W_L = A Z_L in
  // FP64 (refinement steps) and in the inner precision (double or float)
  const float* ZL32;
  const double* WL64;
  const void* WLi;
  // FP64 operator
  const double *Tx64, *Ty64, *Tz64, *diag64, *invdiag64, *b;
  double* x;              // solution (FP64)
  double* r64;            // FP64 refinement residual
  // inner operator and state, element type per mode (double or float)
  const void *Txi, *Tyi, *Tzi;
  void *z, *p0, *p1, *xh;
  // per-warp label-sum rows in global memory (d > kWarpAccMaxD): CTA c owns
  // gacc[c * gacc_stride .. + rows * d), indexed by blockIdx.x
  double* gacc;
  int64_t gacc_stride;
  // reductions
  double* part;           // [grid][pstride]
  int pstride;
  double* s_glob;         // dk
  double* y_glob;         // dk
  double* out;            // results: see kOut*
  SyncArgs sy;
  double tol, inner_tol;
  double fwd_tol;         // mixed forms: forward-error bound of the refinement (< 0: off)
  int maxiter, max_outer;
  int fp64;               // 1: inner in FP64, single inner solve + finalisation
  int bf16;               // 1: inner faces stored as BF16
  int warm;               // 1: x holds an earlier solve's result, refined further
};

enum {
  kOutIters = 0, kOutOuter, kOutRR, kOutBB, kOutStatus, kOutRecRR, kOutFwd,
  kOutStartNs, kOutEndNs,  // the team's first and last moment in the kernel (%globaltimer, ns)
  // refinement trace (mixed forms): for outer step k < kTraceSteps, the
  // squared norm of its correction at kOutTrace + 2k, its residual at +2k+1
  kOutTrace = 10, kTraceSteps = 16, kOutCount = kOutTrace + 2 * kTraceSteps
};

}  // namespace sld

struct sld_system_s {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  sld::Geo g{};
  int nxp = 0;  // nx rounded up to 8: row pitch of the FP32/BF16 inner arrays and 16-bit labels
  int64_t np = 0;  // nxp * ny * nz
  int64_t nvec = 0;  // doubles allocated for each inner vector (z, p0, p1, xhat)
  int bc_type[6]{};
  double bc_value[6]{};
  // FP64 operator (assembled) and the permeability
  double *K = nullptr, *Tx = nullptr, *Ty = nullptr, *Tz = nullptr;
  double *diag = nullptr, *invdiag = nullptr, *b = nullptr;
  // FP32 inner operator (lazily made)
  float *Tx32 = nullptr, *Ty32 = nullptr, *Tz32 = nullptr;
  // BF16 inner operator, its FP32 inverse diagonal and coarse inverse (lazily made)
  __nv_bfloat16 *Tx16 = nullptr, *Ty16 = nullptr, *Tz16 = nullptr;
  float* invd16 = nullptr;
  double *E16 = nullptr, *Einv16 = nullptr;
  bool bf16_ready = false;
  // deflation
  int32_t* label = nullptr;
  uint16_t* label16 = nullptr;
  int d = 0, have_labels_d = 0;
  int labels_L = 0;  // L of labels made by sld_make_labels (0 after user labels)
  double *E = nullptr, *Einv = nullptr;  // dk x dk, dk = d + kL
  bool deflation_ready = false;
  // extra dense deflation vectors (kMaxL slots per cell, zero past kL)
  int kL = 0, kL_requested = 0;
  float* ZL32 = nullptr;   // Z_L, FP32
  double* WL64 = nullptr;  // A Z_L, FP64
  float* WL32 = nullptr;   // A Z_L rounded to FP32
  int dk() const { return d + kL; }
  // solve work space (lazily made)
  double *x = nullptr, *r64 = nullptr, *bwork = nullptr;
  void *z = nullptr, *p0 = nullptr, *p1 = nullptr, *xh = nullptr;  // sized for FP64
  double *part = nullptr, *s_glob = nullptr, *y_glob = nullptr, *out = nullptr;
  unsigned* bar = nullptr;
  int* status = nullptr;
  int part_rows = 0;
  double* gacc = nullptr;  // global per-warp label-sum rows (d > kWarpAccMaxD), grown on demand
  size_t gacc_cap = 0;     // doubles
  double* gm_ws = nullptr;  // PDGMRES work space (basis, vectors, scalars), grown on demand
  size_t gm_ws_cap = 0;     // doubles
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace sld {
// sld_setup.cu
cudaError_t launch_assemble(sld_system s, const double* q);
cudaError_t launch_labels(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L);
cudaError_t launch_coarse_E(sld_system s, const double* Tx, const double* Ty, const double* Tz, double* E,
                            int* bad_label);
// E (dim x dim) = L L^T and Einv.  Pivots k >= rel_from must also exceed
// rel_tol times their original diagonal (else SLD_ERR_COARSE_SINGULAR).
int coarse_factor(sld_system s, int dim, const double* E, double* Einv, double timeout_s, std::string* msg,
                  int rel_from = 1 << 30, double rel_tol = 0.0);  // returns sld_status
// Z_L from n x k user values (row-major, FP64 or FP32), W_L = A Z_L, and the
// blocks Z_lab^T W_L (d x k) and Z_L^T W_L (k x k) written into Efull
// (dk x dk) next to the label block E (d x d).  *bad: non-finite inputs.
cudaError_t launch_learned_setup(sld_system s, const void* Zextra_dev, int k, int f32, const double* E,
                                 double* Efull, int* bad);
cudaError_t launch_quantize_bf16(sld_system s);
cudaError_t launch_widen_bf16(sld_system s, double* Tx, double* Ty, double* Tz);
cudaError_t launch_quantize_fp32(sld_system s);
cudaError_t launch_labels16(sld_system s);
cudaError_t launch_apply_A(sld_system s, const double* x, double* y);
cudaError_t launch_restrict(sld_system s, const double* v, double* out);
cudaError_t launch_residual(sld_system s, const double* b, const double* x, double* partial_out,
                            double* rr_host, double* bb_host);
// s->gacc with room for `doubles` values (kept, grown on demand)
cudaError_t ensure_gacc(sld_system s, size_t doubles);
// s->gm_ws with room for `doubles` values (kept, grown on demand)
cudaError_t ensure_gmres_ws(sld_system s, size_t doubles);
// sld_solve_tma.cu
bool tma_eligible(const Geo& g, bool fp64);
int launch_solve_tma(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg);
// batched FP32-inner solve on the TMA sweeps
unsigned tma_batch_args_off(int dmax, bool wacc);
size_t tma_batch_smem(int dmax, bool wacc);
int tma_batch_occupancy(bool wacc, size_t smem);
void tma_batch_tiles(SolveArgs* a);
size_t tma_maps_bytes();
bool tma_batch_maps(const SolveArgs& a, void* out);  // host memory, tma_maps_bytes() bytes
// h_args (count systems, host): when count <= tma_batch_param_max(), every
// system's arguments go into one kernel parameter; else the kernel copies
// its system's arguments from d_args into shared memory
cudaError_t tma_batch_launch(int G, size_t smem, unsigned args_off, bool wacc, const SolveArgs* d_args,
                             const SolveArgs* h_args, int count, const void* d_maps, const int* d_cta,
                             cudaStream_t st);
int tma_batch_param_max();
// sld_solve_tma_learned.cu (extra dense deflation columns)
int launch_solve_tma_learned(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg);
// sld_api.cu: the thread-local message returned by sld_last_error()
void set_last_error(const std::string& msg);
// sld_cc.cu: split the plain labels in s->label (d0 values) into connected
// components, renumbered canonically in place; *d_out = component count (the
// labels are left unchanged when it exceeds maxd).  Returns an sld_status.
int run_cc_labels(sld_system s, int d0, int maxd, int* d_out, std::string* msg);
// sld_hritz.cu: harmonic Ritz pairs (host); returns an sld_status
int harmonic_ritz(const double* Hbar, int m, int d, double* Y, double* theta_re, double* theta_im);
// sld_gmres.cu: PDGMRES (deflated right-Jacobi restarted GMRES, FP64);
// b: device.  Writes the solution to s->x.  Returns an sld_status.
int run_gmres(sld_system s, const double* b, int m, int deflate, double tol, int maxiter, sld_gmres_info* info,
              std::string* msg);
// RDGMRES (harmonic-Ritz deflation from the first cycle, nd vectors); b: device
int run_rdgmres(sld_system s, const double* b, int m, int nd, double tol, int maxiter, sld_gmres_info* info,
                std::string* msg);
// sld_solve.cu
void fill_args(sld_system s, const double* b_dev, const sld_options& o, SolveArgs* a);
// warm: keep x and refine it (no zeroing, and the first refinement step is
// not taken as the exact coarse solution by the forward-error test)
int run_solve(sld_system s, const double* b_dev, const sld_options& o, sld_result* res,
              std::string* msg, bool warm = false);  // returns sld_status

// A batched solve: one cooperative launch over all systems, each solved by
// its own team of CTAs, captured with its state resets in a CUDA graph.
struct BatchPlan {
  int count = 0, G = 0, cx = 1, per_sm = 0;
  double expo = 1.0;
  bool fp64 = false, wacc = true;
  bool tma = false;        // TMA sweeps (FP32 inner), else the register/shuffle sweeps
  unsigned args_off = 0;   // TMA: shared-memory offset of the copied arguments
  void* d_maps = nullptr;  // TMA: one set of tensor maps per system (device)
  size_t smem = 0;
  SolveArgs* d_args = nullptr;
  int* d_cta = nullptr;
  double* d_gacc = nullptr;  // global per-warp label-sum rows (dmax > kWarpAccMaxD)
  SolveArgs* h_args = nullptr;  // host copy of the systems' arguments (new[], count)
  cudaStream_t stream = nullptr;  // the batch's own stream (capture and launch), not owned here
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int teams[4096];
};
// cost: modelled CTA-time per system (count values; teams by min-max of
// cost / team + fixed, fixed = the part of a system's time that more CTAs do
// not shorten, nullptr = 0), or nullptr for teams proportional to n^expo
int batch_build(sld_system* sys, int count, const sld_options& o, int per_sm, double expo, const double* cost,
                int cx, cudaStream_t stream, BatchPlan* plan, std::string* msg, const double* fixed = nullptr);
void batch_free(BatchPlan* plan);
}  // namespace sld
