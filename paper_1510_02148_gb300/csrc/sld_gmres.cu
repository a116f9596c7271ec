// sld_gmres.cu -- PDGMRES: restarted GMRES(m), right-preconditioned with
// Jacobi, deflated with the subdomain-levelset columns (Section 3.2, with the
// physics-based vectors of Section 3.2.2 built before the iteration):
//
//   E = Z^T A Z,  P1 = I - A Z E^{-1} Z^T,  P2 = I - Z E^{-1} Z^T A,
//   x* = Z E^{-1} Z^T b;  GMRES(m) on P1 A M^{-1} u = P1 b,  M = diag A;
//   x = P2 x~ + x*,  x~ = M^{-1} u   (b - A x = P1 (b - A x~)).
//
// One Arnoldi step, FP64, stream-ordered kernels over all cells:
//   k_gm_apply     w = A M^{-1} v_j, v_j = raw / |raw| written to the basis,
//                  and this CTA's Z^T w (fixed-order label sums)
//   k_gm_colsum    s = the column sums of those rows;  k_gm_gemv  y = E^{-1} s
//   k_gm_defl      w -= A Z y   (the 7-point stencil on y[label])
//   k_gm_dots      h1 = V^T w   (8 basis vectors per CTA row of the grid)
//   k_gm_orth      w -= V h1
//   k_gm_dots      h2 = V^T w
//   k_gm_orth      raw = w - V h2, |raw|^2
//   k_gm_givens    the Hessenberg column, the Givens rotations, the test
// Classical Gram-Schmidt with one reorthogonalisation (two passes over the
// basis, each fully parallel) stands in for the sequential modified
// Gram-Schmidt; the Hessenberg column is h1 + h2 and h_{j+1,j} = |raw|.  The
// rotations and the residual test run on the device (k_gm_givens), so a
// cycle's steps are launched without host round trips; once the test stops
// the cycle, the kernels of the remaining steps return at once.  The host
// reads the rotated Hessenberg matrix once per cycle and solves the small
// triangular system.  Every sum is a per-CTA partial row reduced in a fixed
// order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "sld_solve_common.cuh"

namespace sld {
namespace {

constexpr int kGT = 256;         // threads per CTA
constexpr int kGMaxBasis = 32;   // basis vectors (m + 1)
constexpr int kGDots = 8;        // basis vectors per CTA in k_gm_dots

enum { GM_PRECOND = 0, GM_RESID = 1, GM_APPLY = 2, GM_COPY = 3, GM_BAPPLY = 4 };

// w = op(v) at every cell, and this CTA's row of Z^T w.
//   GM_PRECOND: v is the raw next basis vector; v_j = v / sqrt(*norm2) is
//               written to vout and w = A M^{-1} v_j (with u = M^{-1} v given:
//               w = A u / sqrt(*norm2), the scaling applied once per cell)
//   GM_RESID:   w = b - A v        GM_APPLY: w = A v        GM_COPY: w = v (not stored)
//   GM_BAPPLY:  w = A M^{-1} v (the right-preconditioned operator B)
template <int MODE, bool WACC>
__global__ void __launch_bounds__(kGT) k_gm_apply(SolveArgs a, const double* __restrict__ v,
                                                  const double* __restrict__ norm2, double* __restrict__ vout,
                                                  double* __restrict__ w, double* __restrict__ part,
                                                  const int* __restrict__ stop = nullptr,
                                                  const double* __restrict__ u = nullptr) {
  if (stop && *stop) return;  // the device Givens step ended the cycle
  extern __shared__ double sacc[];
  const int d = a.d;
  const int warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < (WACC ? acc_rows() : 1) * d; k += blockDim.x) sacc[k] = 0.0;
  __syncthreads();
  double sc = 1.0;
  if constexpr (MODE == GM_PRECOND) sc = 1.0 / sqrt(*norm2);
  // each CTA takes one contiguous chunk of cells (a multiple of its size), so
  // that a lane's label stays the same over many rounds and the label sums
  // are flushed rarely
  const int64_t chunk = ((a.g.n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t i_end = min(a.g.n, (int64_t)(blockIdx.x + 1) * chunk);
  const int64_t nround = chunk / blockDim.x;
  CellWalk c;
  c.init(a, (int64_t)blockIdx.x * chunk + threadIdx.x, blockDim.x);
  LabelAcc<double, WACC> la;
  la.init(a.lab_L);
  auto cell = [&](const CellWalk& cw, double& wv, int& l) {
    const int64_t i = cw.i;
    if constexpr (MODE == GM_PRECOND) {
      if (u) wv = sc * apply64(a, cw, [&](int64_t j, int64_t) { return u[j]; });
      else wv = apply64(a, cw, [&](int64_t j, int64_t) { return (v[j] * sc) * a.invdiag64[j]; });
      vout[i] = v[i] * sc;
    } else if constexpr (MODE == GM_RESID) {
      wv = a.b[i] - apply64(a, cw, [&](int64_t j, int64_t) { return v[j]; });
    } else if constexpr (MODE == GM_APPLY) {
      wv = apply64(a, cw, [&](int64_t j, int64_t) { return v[j]; });
    } else if constexpr (MODE == GM_BAPPLY) {
      wv = apply64(a, cw, [&](int64_t j, int64_t) { return v[j] * a.invdiag64[j]; });
    } else {
      wv = v[i];
    }
    if constexpr (MODE != GM_COPY) w[i] = wv;
    if (d > 0) l = a.label[i];
  };
  // two rounds at a time (this round's cell and the next round's): more
  // loads in flight; the label sums still take the cells in round order
  for (int64_t rnd = 0; rnd < nround; rnd += 2) {
    CellWalk c2 = c;
    c2.next();
    const bool ok0 = c.i < i_end, ok1 = rnd + 1 < nround && c2.i < i_end;
    double w0 = 0.0, w1 = 0.0;
    int l0 = -1, l1 = -1;
    if (ok0) cell(c, w0, l0);
    if (ok1) cell(c2, w1, l1);
    if (d > 0) {
      la.add(ok0, l0, w0, sacc, d, warp);
      if (rnd + 1 < nround) la.add(ok1, l1, w1, sacc, d, warp);
    }
    c = c2;
    c.next();
  }
  if (d > 0) {
    la.flush(sacc, d, warp);
    __syncthreads();
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
      double t = 0.0;
      if constexpr (WACC) {
        for (int r = 0; r < acc_rows(); ++r) t += sacc[r * d + k];
      } else {
        t = sacc[k];
      }
      part[(int64_t)k * a.pstride + blockIdx.x] = t;
    }
  }
}

// out[k] = sum of column k of the partial rows (G CTAs), k < ncol; one warp
// per column, the same order every time.
__global__ void k_gm_colsum(const double* __restrict__ part, int pstride, int G, int ncol, double* __restrict__ out,
                            const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  const int col = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (col >= ncol) return;
  double t = ordered_sum(part + (int64_t)col * pstride, 1, lane, G, 32);
  t = warp_sum(t);
  if (lane == 0) out[col] = t;
}

// y = E^{-1} s, one warp per row.
__global__ void k_gm_gemv(int d, const double* __restrict__ Einv, const double* __restrict__ s, double* __restrict__ y,
                          const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  const int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= d) return;
  double t = 0.0;
  for (int k = lane; k < d; k += 32) t += Einv[(int64_t)row * d + k] * s[k];
  t = warp_sum(t);
  if (lane == 0) y[row] = t;
}

// w -= A Z y  ((A Z y)_i: the stencil applied to the cellwise y[label]).
__global__ void __launch_bounds__(kGT) k_gm_defl(SolveArgs a, const double* __restrict__ y, double* __restrict__ w,
                                                 const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  CellWalk c;
  c.init(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride);
  while (c.ok()) {  // two cells per pass: more loads in flight
    CellWalk c2 = c;
    c2.next();
    const double u0 = apply64(a, c, [&](int64_t j, int64_t) { return y[__ldg(a.label + j)]; });
    double u1 = 0.0;
    if (c2.ok()) u1 = apply64(a, c2, [&](int64_t j, int64_t) { return y[__ldg(a.label + j)]; });
    w[c.i] -= u0;
    if (c2.ok()) w[c2.i] -= u1;
    c = c2;
    c.next();
  }
}

// Partial rows of V_k . w for the kGDots basis vectors k0 = blockIdx.y * kGDots ..
__global__ void __launch_bounds__(kGT) k_gm_dots(int64_t n, const double* __restrict__ V, int nv,
                                                 const double* __restrict__ w, double* __restrict__ part,
                                                 int pstride, const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  __shared__ double red[kGDots][kGT / 32];
  const int k0 = blockIdx.y * kGDots;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc[kGDots];
#pragma unroll
  for (int k = 0; k < kGDots; ++k) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < kGDots; ++k)
      if (k0 + k < nv) acc[k] += V[(int64_t)(k0 + k) * n + i] * wi;
  }
#pragma unroll
  for (int k = 0; k < kGDots; ++k) {
    const double t = warp_sum(acc[k]);
    if (lane == 0) red[k][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < kGDots && k0 + (int)threadIdx.x < nv) {
    double t = 0.0;
    for (int q = 0; q < kGT / 32; ++q) t += red[threadIdx.x][q];
    part[(int64_t)(k0 + threadIdx.x) * pstride + blockIdx.x] = t;
  }
}

// out = w - sum_{k < nv} h[k] V_k (out may be w); with norm_col >= 0 also the
// partial row of |out|^2 in that column.
__global__ void __launch_bounds__(kGT) k_gm_orth(int64_t n, const double* __restrict__ V, int nv,
                                                 const double* __restrict__ h, const double* w, double* out,
                                                 double* __restrict__ part, int pstride, int norm_col,
                                                 const int* __restrict__ stop = nullptr,
                                                 const double* __restrict__ invd = nullptr,
                                                 double* __restrict__ uout = nullptr) {
  if (stop && *stop) return;
  __shared__ double hs[kGMaxBasis];
  __shared__ double red[kGT / 32];
  if (threadIdx.x < kGMaxBasis) hs[threadIdx.x] = (int)threadIdx.x < nv ? h[threadIdx.x] : 0.0;
  __syncthreads();
  double nn = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double t = w[i];
#pragma unroll 4
    for (int k = 0; k < nv; ++k) t -= hs[k] * V[(int64_t)k * n + i];
    out[i] = t;
    if (uout) uout[i] = t * invd[i];  // M^{-1} of the next raw vector, for its apply
    nn += t * t;
  }
  if (norm_col < 0) return;
  nn = warp_sum(nn);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kGT / 32; ++q) t += red[q];
    part[(int64_t)norm_col * pstride + blockIdx.x] = t;
  }
}

// The Givens step of GMRES on the device (one thread): Hessenberg column j =
// h1 + h2 with h_{j+1,j} = |raw|, the earlier rotations applied, a new one
// for row j+1, the rotated right-hand side g; the cycle stops (later kernels
// of the cycle return at once) when |g_{j+1}| <= tol_abs, at a breakdown
// (h_{j+1,j} = 0) or at the cycle's last step.
struct GivensState {
  double R[kGMaxBasis * kGMaxBasis];  // (m + 1) x m, row-major, pitch kGMaxBasis
  double cs[kGMaxBasis], sn[kGMaxBasis], g[kGMaxBasis + 1];
  double est;  // |g_k| after the last step
  int k;       // steps done in this cycle
  int stop;    // 1: the cycle is over
};

__global__ void k_gm_givens(const double* __restrict__ h1, const double* __restrict__ h2, const double* __restrict__ nn,
                            GivensState* __restrict__ gs, int j, double tol_abs, int last) {
  if (threadIdx.x != 0 || gs->stop) return;
  double col[kGMaxBasis + 1];
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  const double hn = sqrt(*nn);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = gs->cs[i] * col[i] + gs->sn[i] * col[i + 1];
    col[i + 1] = -gs->sn[i] * col[i] + gs->cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rho = hypot(col[j], col[j + 1]);
  const double c = rho == 0.0 ? 1.0 : col[j] / rho, sv = rho == 0.0 ? 0.0 : col[j + 1] / rho;
  gs->cs[j] = c;
  gs->sn[j] = sv;
  col[j] = rho;
  col[j + 1] = 0.0;
  for (int i = 0; i <= j + 1; ++i) gs->R[i * kGMaxBasis + j] = col[i];
  gs->g[j + 1] = -sv * gs->g[j];
  gs->g[j] = c * gs->g[j];
  gs->k = j + 1;
  gs->est = fabs(gs->g[j + 1]);
  if (gs->est <= tol_abs || hn == 0.0 || last) gs->stop = 1;
}

// x~ += M^{-1} sum_{k < nv} u[k] V_k
__global__ void __launch_bounds__(kGT) k_gm_update(int64_t n, const double* __restrict__ V, int nv,
                                                   const double* __restrict__ u, const double* __restrict__ invdiag,
                                                   double* __restrict__ xt) {
  __shared__ double us[kGMaxBasis];
  if (threadIdx.x < kGMaxBasis) us[threadIdx.x] = (int)threadIdx.x < nv ? u[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
#pragma unroll 4
    for (int k = 0; k < nv; ++k) t += us[k] * V[(int64_t)k * n + i];
    xt[i] += invdiag[i] * t;
  }
}

// x = M^{-1} (u1 + delta)
__global__ void k_rd_final(int64_t n, const double* __restrict__ invdiag, const double* __restrict__ u1,
                           const double* __restrict__ delta, double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = invdiag[i] * (u1[i] + delta[i]);
}

// x = x~ - Z y1 + Z y0   (P2 x~ + x*, y1 = E^{-1} Z^T A x~, y0 = E^{-1} Z^T b)
__global__ void k_gm_final(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ xt,
                           const double* __restrict__ y1, const double* __restrict__ y0, double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int l = label[i];
    x[i] = xt[i] - y1[l] + y0[l];
  }
}

// Device scalars of the solve (one block, copied to the host once per step).
struct Scal {
  double h1[kGMaxBasis];
  double h2[kGMaxBasis];
  double nn;  // |raw|^2 of the vector the next step normalises
  double pad[7];
};

}  // namespace

int run_gmres(sld_system s, const double* b, int m, int deflate, double tol, int maxiter, sld_gmres_info* info,
              std::string* msg) {
  const int64_t n = s->g.n;
  cudaStream_t st = s->stream;
  sld_options o;
  sld_default_options(&o);
  o.precision = SLD_FP64;
  SolveArgs a;
  fill_args(s, b, o, &a);
  const int d = deflate ? s->d : 0;
  a.d = d;
  a.dk = d;
  a.kL = 0;
  const bool wacc = d <= kWarpAccMaxD;
  const int G = std::min(s->nsm * 4, s->part_rows);
  a.sy.ncta = G;
  a.sy.cta0 = 0;
  const int ps = a.pstride;
  double* part = a.part;
  // work space, kept by the handle between calls: the basis (m + 1) n, w,
  // raw, x~, M^{-1} raw (n each), small vectors, the device scalars and
  // Givens state
  const size_t small = (size_t)4 * (d + 1) + kGMaxBasis;
  const size_t scal_off = ((size_t)(m + 5) * n + small + 31) / 32 * 32;  // doubles, 256-byte aligned
  const size_t gs_off = scal_off + (sizeof(Scal) + 255) / 256 * 32;
  const size_t need = gs_off + (sizeof(GivensState) + 255) / 256 * 32;
  cudaError_t e = ensure_gmres_ws(s, need);
  if (e != cudaSuccess) {
    *msg = std::string("GMRES work space: ") + cudaGetErrorString(e);
    return SLD_ERR_OOM;
  }
  auto release = [&]() {};
  double* V = s->gm_ws;
  double* work = V + (size_t)(m + 1) * n;
  Scal* sc = reinterpret_cast<Scal*>(s->gm_ws + scal_off);
  GivensState* gs = reinterpret_cast<GivensState*>(s->gm_ws + gs_off);
  std::unique_ptr<GivensState> hgs_own(new GivensState());
  GivensState* hgs = hgs_own.get();
  double *w = work, *raw = w + n, *xt = raw + n, *um = xt + n;  // um = M^{-1} raw
  double *sv = um + n, *y = sv + (d + 1), *y0 = y + (d + 1), *y1 = y0 + (d + 1), *ud = y1 + (d + 1);
  const size_t smem = sizeof(double) * (size_t)(wacc ? kGT / 32 : 1) * (size_t)std::max(d, 1);
  // colsum / gemv: one warp per column (row), 8 warps per block
  auto cols = [&](int ncol) { return dim3((unsigned)((ncol + 7) / 8)); };
  auto colsum = [&](int ncol, double* out, const int* stp = nullptr) {
    k_gm_colsum<<<cols(ncol), 256, 0, st>>>(part, ps, G, ncol, out, stp);
  };
  // s = Z^T (partials from the last k_gm_apply), y = E^{-1} s
  auto coarse = [&](double* yout) {
    colsum(d, sv);
    k_gm_gemv<<<cols(d), 256, 0, st>>>(d, a.Einv, sv, yout);
  };
  auto apply = [&](int mode, const double* v, const double* nrm2, double* vout, double* wout,
                   const int* stp = nullptr, const double* uin = nullptr) {
#define GM_LAUNCH(MODE)                                                                              \
  (wacc ? k_gm_apply<MODE, true><<<G, kGT, smem, st>>>(a, v, nrm2, vout, wout, part, stp, uin)        \
        : k_gm_apply<MODE, false><<<G, kGT, smem, st>>>(a, v, nrm2, vout, wout, part, stp, uin))
    switch (mode) {
      case GM_PRECOND: GM_LAUNCH(GM_PRECOND); break;
      case GM_RESID: GM_LAUNCH(GM_RESID); break;
      case GM_APPLY: GM_LAUNCH(GM_APPLY); break;
      default: GM_LAUNCH(GM_COPY); break;
    }
#undef GM_LAUNCH
  };
  auto dots = [&](int nv, double* out) {
    k_gm_dots<<<dim3(G, (nv + kGDots - 1) / kGDots), kGT, 0, st>>>(n, V, nv, w, part, ps);
    colsum(nv, out);
  };
  // R: the Hessenberg matrix with the rotations applied (upper triangular part used)
  std::vector<double> u(m);
  cudaEventRecord(s->ev0, st);
  // ||b||, and x* = Z y0 with y0 = E^{-1} Z^T b
  k_gm_orth<<<G, kGT, 0, st>>>(n, V, 0, sc->h1, b, raw, part, ps, 0);
  colsum(1, &sc->nn);
  double bb = 0.0;
  if ((e = cudaMemcpyAsync(&bb, &sc->nn, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    release();
    *msg = std::string("GMRES: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  const double bnorm = std::sqrt(bb);
  if (d > 0) {
    apply(GM_COPY, b, nullptr, nullptr, nullptr);
    coarse(y0);
  }
  cudaMemsetAsync(xt, 0, sizeof(double) * n, st);
  int its = 0, cycles = 0;
  bool converged = bnorm == 0.0;
  double est = 0.0;
  Scal hs;
  auto fetch = [&]() -> bool {
    if ((e = cudaMemcpyAsync(&hs, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return false;
    return (e = cudaStreamSynchronize(st)) == cudaSuccess;
  };
  while (!converged) {
    // r = P1 (b - A x~): raw, |raw|^2
    apply(GM_RESID, xt, nullptr, nullptr, w);
    if (d > 0) {
      coarse(y);
      k_gm_defl<<<G, kGT, 0, st>>>(a, y, w);
    }
    k_gm_orth<<<G, kGT, 0, st>>>(n, V, 0, sc->h1, w, raw, part, ps, 0, nullptr, a.invdiag64, um);
    colsum(1, &sc->nn);
    if (!fetch()) break;
    const double beta = std::sqrt(hs.nn);
    est = bnorm > 0 ? beta / bnorm : 0.0;
    if (beta <= tol * bnorm) {
      converged = true;
      break;
    }
    if (its >= maxiter) break;
    ++cycles;
    // the cycle's steps run stream-ordered without host round trips: the
    // Givens rotations and the residual test are a one-thread kernel per
    // step, and once it stops the cycle the remaining kernels return at once
    const int steps = std::min(m, maxiter - its);
    hgs->k = 0;
    hgs->stop = 0;
    hgs->est = beta;
    std::fill(hgs->g, hgs->g + kGMaxBasis + 1, 0.0);
    hgs->g[0] = beta;
    cudaMemcpyAsync(gs, hgs, sizeof(GivensState), cudaMemcpyHostToDevice, st);
    const int* stp = &gs->stop;
    for (int j = 0; j < steps; ++j) {
      const int nv = j + 1;
      // v_j = raw / |raw|, w = P1 A M^{-1} v_j, h1 = V^T w
      apply(GM_PRECOND, raw, &sc->nn, V + (size_t)j * n, w, stp, um);
      if (d > 0) {
        colsum(d, sv, stp);
        k_gm_gemv<<<cols(d), 256, 0, st>>>(d, a.Einv, sv, y, stp);
        k_gm_defl<<<G, kGT, 0, st>>>(a, y, w, stp);
      }
      k_gm_dots<<<dim3(G, (nv + kGDots - 1) / kGDots), kGT, 0, st>>>(n, V, nv, w, part, ps, stp);
      colsum(nv, sc->h1, stp);
      // classical Gram-Schmidt, twice: w -= V h1, h2 = V^T w, raw = w - V h2 and |raw|^2
      k_gm_orth<<<G, kGT, 0, st>>>(n, V, nv, sc->h1, w, w, part, ps, -1, stp);
      k_gm_dots<<<dim3(G, (nv + kGDots - 1) / kGDots), kGT, 0, st>>>(n, V, nv, w, part, ps, stp);
      colsum(nv, sc->h2, stp);
      k_gm_orth<<<G, kGT, 0, st>>>(n, V, nv, sc->h2, w, raw, part, ps, 0, stp, a.invdiag64, um);
      colsum(1, &sc->nn, stp);
      k_gm_givens<<<1, 32, 0, st>>>(sc->h1, sc->h2, &sc->nn, gs, j, tol * bnorm, j + 1 == steps ? 1 : 0);
    }
    if ((e = cudaMemcpyAsync(hgs, gs, sizeof(GivensState), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      break;
    const int k = hgs->k;
    its += k;
    est = bnorm > 0 ? hgs->est / bnorm : 0.0;
    // R u = g (upper triangular, k x k), then x~ += M^{-1} V u
    for (int i = k - 1; i >= 0; --i) {
      double t = hgs->g[i];
      for (int q = i + 1; q < k; ++q) t -= hgs->R[i * kGMaxBasis + q] * u[q];
      u[i] = hgs->R[i * kGMaxBasis + i] != 0.0 ? t / hgs->R[i * kGMaxBasis + i] : 0.0;
    }
    if (k > 0) {
      cudaMemcpyAsync(ud, u.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st);
      k_gm_update<<<G, kGT, 0, st>>>(n, V, k, ud, a.invdiag64, xt);
    }
    if (its >= maxiter) {
      // one more residual evaluation decides convergence at the cap
      apply(GM_RESID, xt, nullptr, nullptr, w);
      if (d > 0) {
        coarse(y);
        k_gm_defl<<<G, kGT, 0, st>>>(a, y, w);
      }
      k_gm_orth<<<G, kGT, 0, st>>>(n, V, 0, sc->h1, w, raw, part, ps, 0);
      colsum(1, &sc->nn);
      if (!fetch()) break;
      est = bnorm > 0 ? std::sqrt(hs.nn) / bnorm : 0.0;
      converged = std::sqrt(hs.nn) <= tol * bnorm;
      break;
    }
  }
  if (e != cudaSuccess) {
    release();
    *msg = std::string("GMRES: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  // x = P2 x~ + x*
  if (d > 0) {
    apply(GM_APPLY, xt, nullptr, nullptr, w);
    coarse(y1);
    k_gm_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a.label, xt, y1, y0, a.x);
  } else {
    cudaMemcpyAsync(a.x, xt, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  }
  cudaEventRecord(s->ev1, st);
  e = cudaEventSynchronize(s->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  release();
  if (e != cudaSuccess) {
    *msg = std::string("GMRES: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  info->iterations = its;
  info->cycles = cycles;
  info->relres_estimate = est;
  info->solve_ms = ms;
  if (!converged) {
    *msg = "GMRES did not reach the tolerance within maxiter steps";
    return SLD_ERR_NOT_CONVERGED;
  }
  return SLD_OK;
}

// RDGMRES (Section 3.2.1): the first cycle is plain right-preconditioned
// GMRES(m) in the preconditioned variable u (x = M^{-1} u, B = A M^{-1});
// from its Arnoldi data the d harmonic Ritz vectors of smallest |theta|
// (harmonic_ritz) give Z = V_m Y; with E = Z^T B Z, P1 = I - B Z E^{-1} Z^T
// and P2 = I - Z E^{-1} Z^T B, the correction delta (B delta = r1 = b - B u1)
// is P2 t + Z E^{-1} Z^T r1 with t from GMRES(m) on P1 B t = P1 r1, and
// x = M^{-1} (u1 + delta).  b - A x = P1 (r1 - B t): the GMRES residual is
// the residual of x.  The kernels are PDGMRES's, with no label columns.
int run_rdgmres(sld_system s, const double* b, int m, int nd, double tol, int maxiter, sld_gmres_info* info,
                std::string* msg) {
  const int64_t n = s->g.n;
  cudaStream_t st = s->stream;
  sld_options o;
  sld_default_options(&o);
  o.precision = SLD_FP64;
  SolveArgs a;
  fill_args(s, b, o, &a);
  a.d = 0;
  a.dk = 0;
  a.kL = 0;
  const int G = std::min(s->nsm * 4, s->part_rows);
  a.sy.ncta = G;
  a.sy.cta0 = 0;
  const int ps = a.pstride;
  double* part = a.part;
  // device: basis V (m+1) n; Z, BZ (nd n each); w, raw, u1, r1, t, tmp (n each); small
  double *V = nullptr, *work = nullptr;
  Scal* sc = nullptr;
  const size_t nsmall = (size_t)nd * nd + 3 * (size_t)nd + 2 * (size_t)kGMaxBasis + 8;
  auto release = [&]() {
    cudaFree(V);
    cudaFree(work);
    cudaFree(sc);
  };
  cudaError_t e = cudaMalloc(&V, sizeof(double) * (size_t)(m + 1) * n);
  if (e == cudaSuccess) e = cudaMalloc(&work, sizeof(double) * ((size_t)(2 * nd + 6) * n + nsmall));
  if (e == cudaSuccess) e = cudaMalloc(&sc, sizeof(Scal));
  if (e != cudaSuccess) {
    release();
    *msg = std::string("RDGMRES work space: ") + cudaGetErrorString(e);
    return SLD_ERR_OOM;
  }
  double *Z = work, *BZ = Z + (size_t)nd * n, *w = BZ + (size_t)nd * n, *raw = w + n, *u1 = raw + n, *r1 = u1 + n,
         *t = r1 + n, *tmp = t + n;
  double *Einv = tmp + n, *sv = Einv + (size_t)nd * nd, *cv = sv + nd, *one = cv + nd, *coef = one + nd;
  const size_t smem = sizeof(double);  // no label sums
  auto cols = [&](int ncol) { return dim3((unsigned)((ncol + 7) / 8)); };
  auto colsum = [&](int ncol, double* out) { k_gm_colsum<<<cols(ncol), 256, 0, st>>>(part, ps, G, ncol, out); };
  auto Bapply = [&](const double* v, double* out) {
    k_gm_apply<GM_BAPPLY, true><<<G, kGT, smem, st>>>(a, v, nullptr, nullptr, out, part);
  };
  auto precond = [&](const double* rawv, double* vj, double* out) {
    k_gm_apply<GM_PRECOND, true><<<G, kGT, smem, st>>>(a, rawv, &sc->nn, vj, out, part);
  };
  auto dots_of = [&](const double* basis, int nv, const double* vec, double* out) {
    k_gm_dots<<<dim3(G, (nv + kGDots - 1) / kGDots), kGT, 0, st>>>(n, basis, nv, vec, part, ps);
    colsum(nv, out);
  };
  // out = vec - sum_k h_k basis_k (|out|^2 into sc->nn when want_norm)
  auto minus_comb = [&](const double* basis, int nv, const double* h, const double* vec, double* out,
                        bool want_norm) {
    k_gm_orth<<<G, kGT, 0, st>>>(n, basis, nv, h, vec, out, part, ps, want_norm ? 0 : -1);
    if (want_norm) colsum(1, &sc->nn);
  };
  Scal hs;
  auto fetch = [&]() -> bool {
    if ((e = cudaMemcpyAsync(&hs, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return false;
    return (e = cudaStreamSynchronize(st)) == cudaSuccess;
  };
  auto fail_cuda = [&]() {
    release();
    *msg = std::string("RDGMRES: ") + cudaGetErrorString(e);
    return (int)SLD_ERR_CUDA;
  };
  // host-side GMRES(m) cycle state
  std::vector<double> R((size_t)(m + 1) * m), Hb((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), u(m);
  int its = 0, cycles = 0;
  double est = 0.0;
  cudaEventRecord(s->ev0, st);
  // ||b||; raw = b, sc->nn = ||b||^2
  minus_comb(V, 0, sc->h1, b, raw, true);
  if (!fetch()) return fail_cuda();
  const double bnorm = std::sqrt(hs.nn);
  {
    const double h1 = 1.0;
    cudaMemcpyAsync(one, &h1, sizeof(double), cudaMemcpyHostToDevice, st);
  }
  cudaMemsetAsync(u1, 0, sizeof(double) * n, st);
  cudaMemsetAsync(t, 0, sizeof(double) * n, st);
  // One GMRES(m) cycle from raw (|raw|^2 in sc->nn); `deflated` applies P1
  // after B.  The solution of the least-squares problem is added to `acc`.
  // Returns the steps taken, or -1 on a CUDA error.
  bool converged = bnorm == 0.0;
  auto cycle = [&](bool deflated, double* acc) -> int {
    const double beta = std::sqrt(hs.nn);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      precond(raw, V + (size_t)j * n, w);  // v_j = raw / |raw|, w = B v_j
      if (deflated) {                      // w -= B Z E^{-1} Z^T w
        dots_of(Z, nd, w, sv);
        k_gm_gemv<<<cols(nd), 256, 0, st>>>(nd, Einv, sv, cv);
        minus_comb(BZ, nd, cv, w, w, false);
      }
      dots_of(V, j + 1, w, sc->h1);
      minus_comb(V, j + 1, sc->h1, w, w, false);
      dots_of(V, j + 1, w, sc->h2);
      minus_comb(V, j + 1, sc->h2, w, raw, true);
      if (!fetch()) return -1;
      std::vector<double> col(j + 2);
      for (int i = 0; i <= j; ++i) col[i] = Hb[(size_t)i * m + j] = hs.h1[i] + hs.h2[i];
      const double hn = std::sqrt(hs.nn);
      col[j + 1] = Hb[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double tt = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = tt;
      }
      const double rho = std::hypot(col[j], col[j + 1]);
      cs[j] = rho == 0.0 ? 1.0 : col[j] / rho;
      sn[j] = rho == 0.0 ? 0.0 : col[j + 1] / rho;
      col[j] = rho;
      col[j + 1] = 0.0;
      for (int i = 0; i <= j + 1; ++i) R[(size_t)i * m + j] = col[i];
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      est = std::fabs(g[j + 1]) / bnorm;
      if (std::fabs(g[j + 1]) <= tol * bnorm || hn == 0.0 || its >= maxiter) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double tt = g[i];
      for (int q = i + 1; q < k; ++q) tt -= R[(size_t)i * m + q] * u[q];
      u[i] = R[(size_t)i * m + i] != 0.0 ? tt / R[(size_t)i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) u[i] = -u[i];  // acc -= sum (-u_i) V_i
    cudaMemcpyAsync(coef, u.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st);
    minus_comb(V, k, coef, acc, acc, false);
    ++cycles;
    return k;
  };
  int k1 = 0;
  if (!converged) {
    k1 = cycle(false, u1);
    if (k1 < 0) return fail_cuda();
  }
  // residual after the first cycle: r1 = b - B u1
  Bapply(u1, w);
  minus_comb(w, 1, one, b, r1, true);
  if (!fetch()) return fail_cuda();
  est = bnorm > 0 ? std::sqrt(hs.nn) / bnorm : 0.0;
  if (!converged && std::sqrt(hs.nn) > tol * bnorm && its < maxiter && k1 == m) {
    // harmonic Ritz vectors of the first cycle: Z = V_m Y, BZ = B Z, E = Z^T B Z
    std::vector<double> Y((size_t)m * nd), tr(nd), ti(nd);
    if (harmonic_ritz(Hb.data(), m, nd, Y.data(), tr.data(), ti.data()) != SLD_OK) {
      release();
      *msg = "RDGMRES: harmonic Ritz pairs failed";
      return SLD_ERR_BREAKDOWN;
    }
    std::vector<double> ycol(m);
    for (int kz = 0; kz < nd; ++kz) {
      for (int j = 0; j < m; ++j) ycol[j] = -Y[(size_t)j * nd + kz];
      cudaMemcpyAsync(coef, ycol.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(Z + (size_t)kz * n, 0, sizeof(double) * n, st);
      minus_comb(V, m, coef, Z + (size_t)kz * n, Z + (size_t)kz * n, false);
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail_cuda();  // coef is reused
      Bapply(Z + (size_t)kz * n, BZ + (size_t)kz * n);
    }
    std::vector<double> E((size_t)nd * nd), col(nd);
    for (int kz = 0; kz < nd; ++kz) {
      dots_of(Z, nd, BZ + (size_t)kz * n, sv);  // column kz: Z_i . B Z_kz
      if ((e = cudaMemcpyAsync(col.data(), sv, sizeof(double) * nd, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_cuda();
      for (int i = 0; i < nd; ++i) E[(size_t)i * nd + kz] = col[i];
    }
    // E^{-1} by Gauss-Jordan with partial pivoting
    std::vector<double> Mx = E, Inv((size_t)nd * nd, 0.0);
    for (int i = 0; i < nd; ++i) Inv[(size_t)i * nd + i] = 1.0;
    double emax = 0.0;
    for (double vv : E) emax = std::max(emax, std::fabs(vv));
    for (int c = 0; c < nd; ++c) {
      int p = c;
      for (int r = c + 1; r < nd; ++r)
        if (std::fabs(Mx[(size_t)r * nd + c]) > std::fabs(Mx[(size_t)p * nd + c])) p = r;
      if (!(std::fabs(Mx[(size_t)p * nd + c]) > 1e-14 * emax)) {
        release();
        *msg = "RDGMRES: the coarse matrix of the harmonic Ritz vectors is singular";
        return SLD_ERR_COARSE_SINGULAR;
      }
      for (int j = 0; j < nd; ++j) {
        std::swap(Mx[(size_t)c * nd + j], Mx[(size_t)p * nd + j]);
        std::swap(Inv[(size_t)c * nd + j], Inv[(size_t)p * nd + j]);
      }
      const double piv = Mx[(size_t)c * nd + c];
      for (int j = 0; j < nd; ++j) {
        Mx[(size_t)c * nd + j] /= piv;
        Inv[(size_t)c * nd + j] /= piv;
      }
      for (int r = 0; r < nd; ++r) {
        if (r == c) continue;
        const double f = Mx[(size_t)r * nd + c];
        for (int j = 0; j < nd; ++j) {
          Mx[(size_t)r * nd + j] -= f * Mx[(size_t)c * nd + j];
          Inv[(size_t)r * nd + j] -= f * Inv[(size_t)c * nd + j];
        }
      }
    }
    cudaMemcpyAsync(Einv, Inv.data(), sizeof(double) * nd * nd, cudaMemcpyHostToDevice, st);
    // deflated cycles on P1 B t = P1 r1
    for (;;) {
      // raw = P1 (r1 - B t), |raw|^2
      Bapply(t, w);
      minus_comb(w, 1, one, r1, tmp, false);
      dots_of(Z, nd, tmp, sv);
      k_gm_gemv<<<cols(nd), 256, 0, st>>>(nd, Einv, sv, cv);
      minus_comb(BZ, nd, cv, tmp, raw, true);
      if (!fetch()) return fail_cuda();
      est = std::sqrt(hs.nn) / bnorm;
      if (std::sqrt(hs.nn) <= tol * bnorm) {
        converged = true;
        break;
      }
      if (its >= maxiter) break;
      if (cycle(true, t) < 0) return fail_cuda();
    }
    // delta = t + Z E^{-1} Z^T (r1 - B t); x = M^{-1} (u1 + delta)
    Bapply(t, w);
    minus_comb(w, 1, one, r1, tmp, false);
    dots_of(Z, nd, tmp, sv);
    k_gm_gemv<<<cols(nd), 256, 0, st>>>(nd, Einv, sv, cv);
    // tmp = t + Z cv: negate cv on the device side by combining with -1
    {
      std::vector<double> c_h(nd);
      if ((e = cudaMemcpyAsync(c_h.data(), cv, sizeof(double) * nd, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_cuda();
      for (double& vv : c_h) vv = -vv;
      cudaMemcpyAsync(coef, c_h.data(), sizeof(double) * nd, cudaMemcpyHostToDevice, st);
    }
    minus_comb(Z, nd, coef, t, tmp, false);
    k_rd_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a.invdiag64, u1, tmp, a.x);
  } else {
    converged = converged || std::sqrt(hs.nn) <= tol * bnorm;
    cudaMemsetAsync(tmp, 0, sizeof(double) * n, st);
    k_rd_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a.invdiag64, u1, tmp, a.x);
  }
  cudaEventRecord(s->ev1, st);
  e = cudaEventSynchronize(s->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  release();
  if (e != cudaSuccess) {
    *msg = std::string("RDGMRES: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  info->iterations = its;
  info->cycles = cycles;
  info->relres_estimate = est;
  info->solve_ms = ms;
  if (!converged) {
    *msg = "RDGMRES did not reach the tolerance within maxiter steps";
    return SLD_ERR_NOT_CONVERGED;
  }
  return SLD_OK;
}

}  // namespace sld
