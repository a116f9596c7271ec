// sld_solve_common.cuh -- device code shared by the two implementations of
// the persistent SLD-DPCG solve (sld_solve.cu: register/shuffle z-march for
// any grid; sld_solve_tma.cu: TMA-pipelined z-march for aligned grids): the
// FP64 refinement sweeps, the grid-wide reduction and coarse-solve phases, the
// 7-point operator, the label accumulators and the solve's control flow.
//
// Control flow (the CG form of the deflated solve of Section 3.1, Def. 3.1,
// with P = I - A Z E^{-1} Z^T and M = diag A):
//   refinement step  O1: r' = b - A (x + xhat), s = Z^T r'
//                    y = E^{-1} s
//                    O2: x += xhat + Z y, rhat = r' - A Z y (= P r'), z = M^{-1} rhat
//   With x = 0 this gives x = Z E^{-1} Z^T b (x*) and rhat_0 = P b; after an
//   inner solve it gives x = x* + P^T xhat (eq. (projectback)).
//   inner iteration  A : p = z + beta p, v = A p, s = Z^T v, gamma = p.v
//                    y = E^{-1} s, delta = gamma - s.y (= p.P A p), alpha = rho/delta
//                    B : w = A (p - Z y) (= P A p), xhat += alpha p,
//                        r = diag z - alpha w, z = r / diag, rho' = r.z, rr = r.r
#pragma once
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "sld_device.cuh"
#include "sld_internal.h"

namespace sld {
namespace {

// The plane-tiles [*t0, *t1) of team rank tr.  Tiles run column by column
// (nz planes per column), and a rank reads two halo planes more for every
// column it touches, so the split balances plane loads, nz + 2 per column,
// rather than tiles: a rank whose range crosses a column boundary gets two
// tiles fewer.  With fewer than four tiles per rank the split is by tiles
// (it keeps every range non-empty).
__device__ __forceinline__ void tile_range(const SolveArgs& a, int tr, int64_t* t0, int64_t* t1) {
  const int64_t G = a.sy.ncta, nz = a.g.nz;
  if (a.ntiles < 4 * G || a.ntiles % nz != 0) {
    *t0 = a.ntiles * tr / G;
    *t1 = a.ntiles * (tr + 1) / G;
    return;
  }
  const int64_t per = nz + 2, units = a.ntiles / nz * per;
  auto bound = [&](int64_t r) {
    const int64_t p = units * r / G;  // position in plane loads
    const int64_t j = p / per, q = p - j * per;
    return j * nz + (q < 1 ? 0 : (q - 1 < nz ? q - 1 : nz));
  };
  *t0 = bound(tr);
  *t1 = bound(tr + 1);
}

// Block-wide sum of one double per thread (fixed order); result to all threads.
__device__ double block_sum(double v, double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  v = warp_sum(v);
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

// Per-lane accumulation of v into the label sums s = Z^T v.  Each lane keeps
// a run sum for its current label; a change of label is a vote of the warp.
//   L == 0 (labels of any form): every change flushes the runs warp-wide.
//   1 <= L <= 4 (labels made by the subdomain-levelset rule, label =
//     subdomain * L + class): a lane whose label changes banks its run in one
//     of L class slots of its current subdomain, without touching the other
//     lanes; only a change of some lane's subdomain flushes warp-wide --
//     rare, since tiles follow the grid and subdomains are boxes of it.
// A flush groups the lanes with __match_any_sync and sums each group in lane
// order by its lowest lane, so no two lanes of a warp write one slot.
template <typename T, bool WACC>
struct LabelAcc {
  int L;
  float invL;
  int curl;  // current label, -1 = none
  int curs;  // current subdomain (L > 0), -1 = none
  T run, a0, a1, a2, a3;
  __device__ __forceinline__ void init(int L_) {
    L = L_;
    invL = L_ > 0 ? 1.0f / (float)L_ : 0.0f;
    curl = curs = -1;
    run = a0 = a1 = a2 = a3 = T(0);
  }
  __device__ __forceinline__ int sub_of(int lab) const { return __float2int_rz(((float)lab + 0.5f) * invL); }
  // add the run into the class slot of the current label
  __device__ __forceinline__ void bank() {
    if (curl >= 0) {
      const int cls = curl - curs * L;
      a0 += (cls == 0) ? run : T(0);
      a1 += (cls == 1) ? run : T(0);
      a2 += (cls == 2) ? run : T(0);
      a3 += (cls == 3) ? run : T(0);
    }
    run = T(0);
  }
  // The group sums are formed in the inner precision T (FP32 in the mixed
  // solve: the run sums already are), in a fixed order: a 5-step butterfly
  // when the whole warp is one group (the usual case), else lane order.
  __device__ __forceinline__ void flush_group(int key, int nk, double* sacc, int d, int warp) {
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(kFull, key);
    for (int k = 0; k < nk; ++k) {
      const T mine = L == 0 ? run : (k == 0 ? a0 : k == 1 ? a1 : k == 2 ? a2 : a3);
      T sum = T(0);
      if (grp == kFull) {
        sum = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
      } else {
#pragma unroll 4
        for (int src = 0; src < 32; ++src) {
          const T v = __shfl_sync(kFull, mine, src);
          if ((grp >> src) & 1u) sum += v;
        }
      }
      if (key >= 0 && lane == __ffs(grp) - 1) {
        const int slot = L > 0 ? key * L + k : key;
        if constexpr (WACC) sacc[warp * d + slot] += sum;
        else atomicAdd(&sacc[slot], sum);
      }
    }
  }
  // everything accumulated so far into the shared sums (warp-wide)
  __device__ __forceinline__ void flush(double* sacc, int d, int warp) {
    if (L == 0) {
      flush_group(curl, 1, sacc, d, warp);
      run = T(0);
    } else {
      bank();
      flush_group(curs, L, sacc, d, warp);
      a0 = a1 = a2 = a3 = T(0);
    }
  }
  // one cell; every lane of the warp calls this together
  __device__ __forceinline__ void add(bool valid, int lab, T v, double* sacc, int d, int warp) {
    const int l = valid ? lab : curl;
    if (__any_sync(kFull, l != curl)) {
      if (L == 0) {
        flush(sacc, d, warp);
      } else {
        const bool ch = l != curl;
        if (ch) bank();
        const int ns = ch ? sub_of(l) : curs;
        if (__any_sync(kFull, ns != curs)) {
          flush_group(curs, L, sacc, d, warp);
          a0 = a1 = a2 = a3 = T(0);
          curs = ns;
        }
      }
      curl = l;
    }
    if (valid) run += v;
  }
  // four consecutive cells of a lane (the first nv valid): the same as four
  // add() calls, with one vote when every lane stays on its current label
  __device__ __forceinline__ void add4(int nv, const int (&lab)[4], const T (&v)[4], double* sacc, int d, int warp) {
    bool same = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) same = same && (c >= nv || lab[c] == curl);
    if (__all_sync(kFull, same)) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < nv) run += v[c];
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) add(c < nv, lab[c], v[c], sacc, d, warp);
    }
  }
};

// The 7-point operator at one free or Dirichlet cell.
//   FP32 inner form: sum over faces T (u_i - m_j u_j)  (m_j = 0 for a Dirichlet
//   neighbour), exact zero row sums, no cancellation of diag * u against the
//   neighbour sum.  FP64 form: diag u_i - sum m_j T u_j with the stored diagonal.
template <typename T>
__device__ __forceinline__ T stencil(bool dirc, T u, T dg, T fxm, T xm, bool mxm, T fxp, T xp, bool mxp, T fym,
                                     T ym, bool mym, T fyp, T yp, bool myp, T fzm, T zm, bool mzm, T fzp, T zp,
                                     bool mzp) {
  if (dirc) return u;
  if constexpr (sizeof(T) == 8) {
    T s = dg * u;
    s -= fxm * (mxm ? xm : T(0));
    s -= fxp * (mxp ? xp : T(0));
    s -= fym * (mym ? ym : T(0));
    s -= fyp * (myp ? yp : T(0));
    s -= fzm * (mzm ? zm : T(0));
    s -= fzp * (mzp ? zp : T(0));
    return s;
  } else {
    T s = fxm * (u - (mxm ? xm : T(0)));
    s += fxp * (u - (mxp ? xp : T(0)));
    s += fym * (u - (mym ? ym : T(0)));
    s += fyp * (u - (myp ? yp : T(0)));
    s += fzm * (u - (mzm ? zm : T(0)));
    s += fzp * (u - (mzp ? zp : T(0)));
    return s;
  }
}

// ---------------------------------------------------------------------------
// Refinement sweeps (FP64, one thread per cell).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_dir_cell(const Geo& g, int ix, int iy, int iz) {
  return dir_axis(ix, g.nx, g.dlo_x, g.dhi_x) || dir_axis(iy, g.ny, g.dlo_y, g.dhi_y) ||
         dir_axis(iz, g.nz, g.dlo_z, g.dhi_z);
}

// Cells i0, i0 + stride, i0 + 2 stride, ... with their grid coordinates and
// their index in the padded inner vectors, stepped by carries (one division
// per thread and sweep instead of several per cell).
struct CellWalk {
  int64_t i, ip, stride, n;
  int ix, iy, iz, sx, sy, sz, nx, ny, vp;
  int64_t vpxy;
  __device__ void init(const SolveArgs& a, int64_t i0, int64_t st) {
    const Geo& g = a.g;
    i = i0;
    stride = st;
    n = g.n;
    nx = g.nx;
    ny = g.ny;
    vp = a.vp;
    vpxy = a.vpxy;
    ix = (int)(i0 % g.nx);
    iy = (int)((i0 / g.nx) % g.ny);
    iz = (int)(i0 / g.nxy);
    sx = (int)(st % g.nx);
    sy = (int)((st / g.nx) % g.ny);
    sz = (int)(st / g.nxy);
    ip = (int64_t)iz * vpxy + (int64_t)iy * vp + ix;
  }
  __device__ bool ok() const { return i < n; }
  __device__ void next() {
    i += stride;
    ix += sx;
    int c = 0;
    if (ix >= nx) { ix -= nx; c = 1; }
    iy += sy + c;
    c = 0;
    if (iy >= ny) { iy -= ny; c = 1; }
    iz += sz + c;
    ip = (int64_t)iz * vpxy + (int64_t)iy * vp + ix;
  }
};

// (A w)_i in FP64 for the vector given by `val(j, jp)` (j: cell index, jp:
// its index in the padded inner vectors) at the walk's cell.
template <typename F>
__device__ __forceinline__ double apply64(const SolveArgs& a, const CellWalk& c, F val) {
  const Geo& g = a.g;
  const int64_t i = c.i, ip = c.ip;
  const int ix = c.ix, iy = c.iy, iz = c.iz;
  if (is_dir_cell(g, ix, iy, iz)) return val(i, ip);
  double v = a.diag64[i] * val(i, ip);
  if (ix > 0 && !dir_axis(ix - 1, g.nx, g.dlo_x, g.dhi_x)) v -= a.Tx64[i - 1] * val(i - 1, ip - 1);
  if (ix + 1 < g.nx && !dir_axis(ix + 1, g.nx, g.dlo_x, g.dhi_x)) v -= a.Tx64[i] * val(i + 1, ip + 1);
  if (iy > 0 && !dir_axis(iy - 1, g.ny, g.dlo_y, g.dhi_y)) v -= a.Ty64[i - g.nx] * val(i - g.nx, ip - a.vp);
  if (iy + 1 < g.ny && !dir_axis(iy + 1, g.ny, g.dlo_y, g.dhi_y)) v -= a.Ty64[i] * val(i + g.nx, ip + a.vp);
  if (iz > 0 && !dir_axis(iz - 1, g.nz, g.dlo_z, g.dhi_z)) v -= a.Tz64[i - g.nxy] * val(i - g.nxy, ip - a.vpxy);
  if (iz + 1 < g.nz && !dir_axis(iz + 1, g.nz, g.dlo_z, g.dhi_z)) v -= a.Tz64[i] * val(i + g.nxy, ip + a.vpxy);
  return v;
}

// Rows of per-warp label accumulators: one per warp of the launch.
__device__ __forceinline__ int acc_rows() { return (int)(blockDim.x >> 5); }

// O1: r' = b - A (x + xhat), s = Z^T r', ||b||^2
// The label sums use the run-sum accumulator below (FP64): groups summed in a
// fixed order and added into the warp's own row of accumulators (shared
// memory for d <= kWarpAccMaxD, the CTA's global rows above), so the result
// does not depend on warp scheduling.

template <typename T, bool WACC>
__device__ void sweep_O1(const SolveArgs& a, double* sacc, double* red, double* part_row) {
  const Geo& g = a.g;
  const int d = a.d;
  const int warp = threadIdx.x >> 5;
  const T* xh = static_cast<const T*>(a.xh);
  for (int k = threadIdx.x; k < acc_rows() * d; k += blockDim.x) sacc[k] = 0.0;
  __syncthreads();
  double bb = 0.0;
  double sl[kMaxL] = {};  // Z_L^T r' (extra columns)
  // each CTA takes one contiguous chunk of cells (a multiple of its size):
  // a lane's label then stays the same over many rounds, and the label sums
  // are flushed rarely
  const int64_t chunk = ((g.n + a.sy.ncta - 1) / a.sy.ncta + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t i_end = min(g.n, (int64_t)(team_rank(a.sy) + 1) * chunk);
  const int64_t nround = chunk / blockDim.x;
  CellWalk c;
  c.init(a, (int64_t)team_rank(a.sy) * chunk + threadIdx.x, blockDim.x);
  LabelAcc<double, true> la;
  la.init(a.lab_L);
  for (int64_t rnd = 0; rnd < nround; ++rnd, c.next()) {
    const int64_t i = c.i;
    const bool ok = i < i_end;
    double r = 0.0;
    int l = -1;
    if (ok) {
      const double Aw = apply64(a, c, [&](int64_t j, int64_t jp) { return a.x[j] + (double)xh[jp]; });
      const double bi = a.b[i];
      r = bi - Aw;
      a.r64[i] = r;
      bb += bi * bi;
      l = a.label[i];
      if (a.kL > 0) {
#pragma unroll
        for (int j = 0; j < kMaxL; ++j) sl[j] += (double)a.ZL32[i * kMaxL + j] * r;
      }
    }
    la.add(ok, l, r, sacc, d, warp);
  }
  la.flush(sacc, d, warp);
#pragma unroll
  for (int j = 0; j < kMaxL; ++j) {
    if (j < a.kL) {
      const double t = block_sum(sl[j], red);
      if (threadIdx.x == 0) part_row[(int64_t)(d + j) * a.pstride] = t;
    }
  }
  const double bsum = block_sum(bb, red);
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < acc_rows(); ++w) t += sacc[w * d + k];  // warp order: deterministic
    part_row[(int64_t)(k) * a.pstride] = t;
  }
  if (threadIdx.x == 0) part_row[(int64_t)(a.dk + 3) * a.pstride] = bsum;
}

// O2: x += xhat + Z y, rhat = r' - A Z y, z = M^{-1} rhat, xhat = p = 0;
// also ||x_new - x||^2 and ||x_new||^2 for the refinement's forward-error test
template <typename T>
__device__ void sweep_O2(const SolveArgs& a, const double* Yd, double* red, double* part_row) {
  T* xh = static_cast<T*>(a.xh);
  T* zb = static_cast<T*>(a.z);
  T* p0 = static_cast<T*>(a.p0);
  T* p1 = static_cast<T*>(a.p1);
  double rr = 0.0, rho = 0.0, dd = 0.0, xx = 0.0;
  const int64_t stride = (int64_t)a.sy.ncta * blockDim.x;
  CellWalk c;
  for (c.init(a, (int64_t)team_rank(a.sy) * blockDim.x + threadIdx.x, stride); c.ok(); c.next()) {
    const int64_t i = c.i, ip = c.ip;
    double AZy = apply64(a, c, [&](int64_t j, int64_t) { return Yd[__ldg(a.label + j)]; });
    double Zy = Yd[__ldg(a.label + i)];
    for (int j = 0; j < a.kL; ++j) {  // extra columns: (A Z_L y_L)_i = (W_L y_L)_i, (Z_L y_L)_i
      const double yj = Yd[a.d + j];
      AZy += a.WL64[i * kMaxL + j] * yj;
      Zy += (double)a.ZL32[i * kMaxL + j] * yj;
    }
    const double rh = a.r64[i] - AZy;
    const double xo = a.x[i];
    const double xn = xo + (double)xh[ip] + Zy;
    a.x[i] = xn;
    dd += (xn - xo) * (xn - xo);  // the change this step applies to x
    xx += xn * xn;
    const T zt = (T)(rh * (a.invdi ? (double)a.invdi[ip] : a.invdiag64[i]));
    zb[ip] = zt;
    xh[ip] = T(0);
    p0[ip] = T(0);
    p1[ip] = T(0);
    rr += rh * rh;
    rho += rh * (double)zt;
  }
  fence_proxy_async();  // z, xhat, p stores before the next sweep's TMA reads
  const double s1 = block_sum(rho, red);
  const double s2 = block_sum(rr, red);
  const double s4 = block_sum(dd, red);
  const double s5 = block_sum(xx, red);
  if (threadIdx.x == 0) {
    part_row[(int64_t)(a.dk + 1) * a.pstride] = s1;
    part_row[(int64_t)(a.dk + 2) * a.pstride] = s2;
    part_row[(int64_t)(a.dk + 4) * a.pstride] = s4;
    part_row[(int64_t)(a.dk + 5) * a.pstride] = s5;
  }
}

// ---------------------------------------------------------------------------
// Grid-wide phases on the partial sums.
// ---------------------------------------------------------------------------
// Partial sums are stored column-major: part[k * pstride + c] is CTA c's
// contribution to column k (coarse sums k < dk, then the scalar slots), so a
// column is one contiguous run.
// s_k = sum over CTAs of column k, one warp per column, fixed order; columns
// k < dk + extra (extra = 1: the scalar slot dk + 0 as well, into s_glob[dk]).
__device__ void phase_reduce_s(const SolveArgs& a, int extra = 0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int G = a.sy.ncta;
  for (int k = team_rank(a.sy) * nw + warp; k < a.dk + extra; k += G * nw) {
    double t = ordered_sum(a.part + (int64_t)k * a.pstride, 1, lane, G, 32);
    t = warp_sum(t);
    if (lane == 0) a.s_glob[k] = t;
  }
}

// y = E^{-1} s, one warp per row.
__device__ void phase_coarse(const SolveArgs& a, const double* Einv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int j = team_rank(a.sy) * nw + warp; j < a.dk; j += a.sy.ncta * nw) {
    const double* row = Einv + (int64_t)j * a.dk;
    double t = 0.0;
    for (int k0 = lane; k0 < a.dk; k0 += 4 * 32) {  // four products' loads at a time
      double e[4], v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + 32 * u;
        e[u] = k < a.dk ? __ldg(row + k) : 0.0;
        v[u] = k < a.dk ? a.s_glob[k] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) t += e[u] * v[u];
    }
    t = warp_sum(t);
    if (lane == 0) a.y_glob[j] = t;
  }
}

// Sums of two scalar slots over all CTAs (same order in every CTA), by
// warps 0 and 1 at once.
__device__ void cta_scalar2(const SolveArgs& a, int slot0, int slot1, double* red, double* v0, double* v1) {
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2) {
    const double* col = a.part + (int64_t)(a.dk + (warp ? slot1 : slot0)) * a.pstride;
    double t = ordered_sum(col, 1, lane, a.sy.ncta, 32);
    t = warp_sum(t);
    if (lane == 0) red[40 + warp] = t;
  }
  __syncthreads();
  *v0 = red[40];
  *v1 = red[41];
}

__device__ double cta_scalar(const SolveArgs& a, int slot, double* red) {
  double v0, v1;
  cta_scalar2(a, slot, slot, red, &v0, &v1);
  return v0;
}

// This CTA's copy Y = y (in the sweep type) and s . y, in one pass over the
// coarse vectors (s . y summed in the same order in every CTA).  Ends with a
// CTA barrier: Y is complete.
template <typename T>
__device__ double cta_take_y(const SolveArgs& a, T* Y, double* red) {
  double t = 0.0;
  for (int k = threadIdx.x; k < a.dk; k += blockDim.x) {
    const double yk = a.y_glob[k];
    Y[k] = (T)yk;
    t += a.s_glob[k] * yk;
  }
  return block_sum(t, red);
}


// ---------------------------------------------------------------------------
// The solve's control flow, shared by the sweep implementations.
//   sweepA(pold, beta, part) : p_new = z + beta p[pold] into p[pold ^ 1],
//                              v = A p_new, s = Z^T v, gamma   (part row)
//   sweepB(pnew, alpha, part): u = p[pnew] - Z y, w = A u, xhat, z, rho', rr
// Each returns false if a bounded wait inside it gave up.
// All decisions use scalars every CTA reduces in the same order, so every
// CTA takes the same branches.
// ---------------------------------------------------------------------------
// Squared least residual cut of an inner solve in the mixed forms (10x).
constexpr double kMinCut2 = 0.01;
// Most refinement steps taken for the forward-error test after the residual
// test has passed.
constexpr int kMaxFwdSteps = 4;

template <typename T, bool WACC, class SweepA, class SweepB>
__device__ void solve_body(const SolveArgs& a, double* acc, double* Yd, T* Y, double* red, SweepA&& sweepA,
                           SweepB&& sweepB) {
  double* my_part = a.part + team_rank(a.sy);  // column-major: stride a.pstride
  unsigned epoch = 0;
  const double tol2 = a.tol * a.tol;
  double bb = 0.0, rr_outer = 0.0, rho = 0.0, rec_rr = 0.0;
  // Refinement state of the forward-error test (mixed forms), in shared
  // memory so that it holds no registers during the sweeps: the inner
  // target of the last step, whether it was relative (not the 0.3 tol
  // floor), the last verified |d| / |x| (reported at exit).  Every thread
  // reads it after a CTA barrier; thread 0 writes it after another one.
  // kEst: the estimate reported at exit (the last verified |d| / |x|, or the
  // contraction estimate of a step the fast rule accepted).
  enum { kTgtPrev = 0, kRelPrev, kFwdRel, kFwdSteps, kDdPrev, kRrPrev, kEst, kFsCount };
  __shared__ double fs[kFsCount];
  if (threadIdx.x == 0) {
    for (int k = 0; k < kFsCount; ++k) fs[k] = 0.0;
    fs[kFwdRel] = -1.0;
    fs[kEst] = -1.0;
  }
  int its = 0, outer = 0, status = 0;
  bool fin_ok = false;  // a breakdown with finite scalars (see the inner loop)
  bool converged = false;
  bool failed = false;
  if (team_rank(a.sy) == 0 && threadIdx.x == 0) a.out[kOutStartNs] = (double)global_ns();
  for (;;) {
    // ---- refinement step: residual, coarse correction, projection ----
    sweep_O1<T, WACC>(a, acc, red, my_part);
    if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
    phase_reduce_s(a);
    if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
    phase_coarse(a, a.Einv);
    if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
    if (outer == 0) bb = cta_scalar(a, 3, red);
    for (int k = threadIdx.x; k < a.dk; k += blockDim.x) Yd[k] = a.y_glob[k];
    __syncthreads();
    sweep_O2<T>(a, Yd, red, my_part);
    if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
    cta_scalar2(a, 1, 2, red, &rho, &rr_outer);
    ++outer;
    if (!isfinite(rr_outer) || !isfinite(rho)) { status = SLD_ERR_BREAKDOWN; break; }
    if (a.fp64) {
      if (outer == 1 && rr_outer <= tol2 * bb) { converged = true; rec_rr = rr_outer; break; }
      if (outer >= 2) break;  // x = x* + P^T xhat written: done
    } else {
      rec_rr = rr_outer;
      double dd, xx;
      cta_scalar2(a, 4, 5, red, &dd, &xx);
      if (team_rank(a.sy) == 0 && threadIdx.x == 0 && outer <= kTraceSteps) {
        a.out[kOutTrace + 2 * (outer - 1)] = dd / fmax(xx, 1e-300);
        a.out[kOutTrace + 2 * (outer - 1) + 1] = rr_outer / fmax(bb, 1e-300);
      }
      const bool res_ok = rr_outer <= tol2 * bb;
      // The residual test alone lets errors along the smallest eigenvalues
      // of the deflated operator through (their residual is tiny), and
      // restarted low-precision inner solves resolve those modes less well
      // than one long FP64 CG run.  So the refinement also checks its
      // forward error: a step whose inner solve had a relative target (a
      // residual cut, not the 0.3 tol floor) and reached it applies a
      // correction d_k ~ the previous error e_{k-1}, and e_k <= e_{k-1}
      // (the refinement contracts the energy norm).  Accept once such a
      // step has |d_k| <= fwd_tol |x|.  Step 1 is the FP64 coarse solution
      // x* (exact to rounding): no low-precision step has touched x yet.
      // Where the inner precision cannot resolve the slowest modes (fields
      // spanning more decades than FP32 does) the corrections stop
      // shrinking: the test then ends at the residual test's result once a
      // verified correction fails to halve the previous verified one, or
      // after kMaxFwdSteps steps past the residual test (the reported
      // estimate keeps the last verified correction).  A warm start (x
      // refined further) has no exact first step.
      const bool verified = outer >= 3 && fs[kRelPrev] != 0.0 && rr_outer <= 4.0 * fs[kTgtPrev];
      const double drel = xx > 0.0 ? sqrt(dd / xx) : 0.0;
      // A step that cut the residual at least 1e3-fold and shrank the
      // correction at least 1e3-fold contracts fast: its error is then
      // estimated as |d_k|^2 / |d_{k-1}| and accepted at a tenth of fwd_tol.
      const bool strong = outer >= 3 && fs[kDdPrev] > 0.0 && rr_outer <= 1e-6 * fs[kRrPrev] &&
                          dd <= 1e-6 * fs[kDdPrev] && xx > 0.0 &&
                          dd / sqrt(fs[kDdPrev] * xx) <= 0.1 * a.fwd_tol;
      const bool fwd_ok = a.fwd_tol < 0.0 || (outer == 1 && !a.warm) || (verified && drel <= a.fwd_tol) || strong;
      const bool stalled = res_ok && ((verified && fs[kFwdRel] >= 0.0 && drel > 0.5 * fs[kFwdRel]) ||
                                      fs[kFwdSteps] >= (double)kMaxFwdSteps);
      // next inner target: inner_tol relative, floored at 0.3 tol ||b||, and
      // at least a 10x cut of the residual (so that the steps after the
      // residual test has passed are relative ones)
      const double floor2 = 0.09 * tol2 * bb;
      const double tgt2n = fmin(fmax(a.inner_tol * a.inner_tol * rr_outer, floor2), kMinCut2 * rr_outer);
      __syncthreads();  // every thread has read fs
      if (threadIdx.x == 0) {
        if (verified) fs[kFwdRel] = fs[kEst] = drel;
        if (res_ok) fs[kFwdSteps] += 1.0;
        if (strong) {
          const double est = dd / sqrt(fs[kDdPrev] * xx);
          if (!verified) fs[kFwdRel] = est;
          fs[kEst] = est;
        }
        fs[kDdPrev] = dd;
        fs[kRrPrev] = rr_outer;
        fs[kTgtPrev] = tgt2n;
        fs[kRelPrev] = (tgt2n < floor2 || a.inner_tol * a.inner_tol * rr_outer > floor2) ? 1.0 : 0.0;
      }
      if (res_ok && (fwd_ok || stalled)) { converged = true; break; }
      if (outer > a.max_outer || its >= a.maxiter) { converged = res_ok; break; }
    }
    const double tgt2 = a.fp64 ? tol2 * bb
                               : fmin(fmax(a.inner_tol * a.inner_tol * rr_outer, 0.09 * tol2 * bb), kMinCut2 * rr_outer);
    // ---- inner deflated CG ----
    double beta = 0.0;
    int pold = 0;
    for (;;) {
      if (!sweepA(pold, (T)beta, my_part)) { failed = true; break; }
      if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
      phase_reduce_s(a, 1);  // and gamma into s_glob[dk]
      if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
      phase_coarse(a, a.Einv_inner);
      if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
      const double gamma = a.s_glob[a.dk];
      const double delta = gamma - cta_take_y(a, Y, red);
      if (!(delta > 0.0) || !isfinite(delta) || !isfinite(rho)) {
        if (a.fp64) status = SLD_ERR_BREAKDOWN;
        fin_ok = isfinite(delta) && isfinite(rho);
        break;
      }
      const double alpha = rho / delta;
      if (!sweepB(pold ^ 1, (T)alpha, my_part)) { failed = true; break; }
      if (!grid_barrier(a.sy, epoch)) { failed = true; break; }
      double rho_new, rr;
      cta_scalar2(a, 1, 2, red, &rho_new, &rr);
      ++its;
      if (a.fp64) rec_rr = rr;
      if (rr <= tgt2) {
        if (a.fp64) converged = true;
        break;
      }
      if (its >= a.maxiter) break;
      beta = rho_new / rho;
      rho = rho_new;
      pold ^= 1;
    }
    // a plain FP64 solve that broke down with finite scalars still takes
    // its finalisation step: x = x* + P^T xhat keeps the iterations' progress
    // (xhat is the last consistent iterate); the status stays BREAKDOWN
    if (failed || (status && !(a.fp64 && fin_ok && outer == 1))) break;
  }
  if (team_rank(a.sy) == 0 && threadIdx.x == 0) {
    a.out[kOutIters] = its;
    a.out[kOutOuter] = outer;
    a.out[kOutRR] = rr_outer;
    a.out[kOutBB] = bb;
    a.out[kOutStatus] = failed ? -1.0 : (status ? (double)status : (converged ? 0.0 : (double)SLD_ERR_NOT_CONVERGED));
    a.out[kOutRecRR] = rec_rr;
    a.out[kOutFwd] = fs[kEst];
    a.out[kOutEndNs] = (double)global_ns();
  }
}

}  // namespace
}  // namespace sld
