// sld_solve.cu -- the persistent SLD-deflated Jacobi-PCG solve (steps a4-a8).
//
// One cooperative launch runs the whole solve.  Each CTA owns a fixed range
// of "plane tiles" (a TX x 8 patch of one z plane); the ranges are contiguous
// in (column tile, z), so a CTA marches up a column of the grid, keeping the
// z-1, z, z+1 values of its rows in registers, exchanging the y neighbours
// through shared memory and the x neighbours through warp shuffles.
//
// Per deflated-CG iteration (the CG form of the deflated solve of
// Section 3.1, Def. 3.1: iterate on P A xhat = P b with P = I - A Z E^{-1} Z^T,
// M = diag A):
//   sweep A : p = z + beta p (also at halo cells), v = A p,
//             s = Z^T v (segmented sum over labels), gamma = p.v
//   barrier, s reduced column-wise; barrier, y = E^{-1} s row-wise; barrier
//   every CTA: delta = p.P A p = gamma - s.y (A symmetric), alpha = rho/delta
//   sweep B : u = p - Z y, w = A u (= P A p), xhat += alpha p,
//             r = diag z - alpha w, z = r / diag, rho' = r.z, rr = r.r
//   barrier, every CTA reduces rho', rr in the same order and takes the same
//   branch.  The residual r is kept as z = M^{-1} r; r = diag * z.
//
// Refinement step (FP64, once per inner solve; also the initial projection
// and the final back-projection, eq. (projectback)):
//   O1: r' = b - A (x + xhat), s = Z^T r'
//   barrier, reduce, barrier, y = E^{-1} s, barrier
//   O2: x += xhat + Z y, rhat = r' - A Z y (= P r'), z = M^{-1} rhat, xhat = p = 0
// With x = 0 this is x = Z E^{-1} Z^T b and rhat_0 = P b; after an inner solve
// it is x = x + xhat + Z E^{-1} Z^T (b - A (x + xhat)), i.e. x* + P^T xhat.
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sld_solve_common.cuh"

namespace sld {
namespace {

template <typename T, int CX, bool WACC>
struct Cfg {
  static constexpr int TX = 32 * CX;
  static constexpr int HOFF = (CX == 4) ? int(16 / sizeof(T)) : 1;
  static constexpr int RS = TX + 2 * HOFF;  // shared row stride (with x halo)
};

template <typename T>
struct Sm {
  T* P;        // [2][kTY+2][RS]   published neighbour values
  T* Ty;       // [2][kTY+1][TX]   Ty of rows y0-1 .. y0+kTY-1
  T* Txh;      // [2][kTY]         Tx of the face left of the tile
  double* acc; // [kWarps][d] label sums: shared memory, or the CTA's global rows (d > kWarpAccMaxD)
  double* Yd;  // [d] coarse correction, FP64
  T* Y;        // [d] coarse correction, inner precision
  double* red; // [64] block reduction scratch
};

template <typename T, int CX, bool WACC>
__host__ __device__ constexpr size_t smem_bytes(int d, int dk) {
  using C = Cfg<T, CX, WACC>;
  size_t b = 0;
  b += sizeof(T) * 2 * (kTY + 2) * C::RS;
  b += sizeof(T) * 2 * (kTY + 1) * C::TX;
  b += sizeof(T) * 2 * kTY;
  b = (b + 15) / 16 * 16;
  b += sizeof(double) * (size_t)(WACC ? kWarps : 0) * d;
  b += sizeof(double) * dk;
  b += sizeof(T) * dk;
  b = (b + 15) / 16 * 16;
  b += sizeof(double) * 64;
  return b;
}

template <typename T, int CX, bool WACC>
__device__ Sm<T> carve(unsigned char* base, int d, int dk) {
  using C = Cfg<T, CX, WACC>;
  Sm<T> s;
  size_t o = 0;
  s.P = reinterpret_cast<T*>(base + o);
  o += sizeof(T) * 2 * (kTY + 2) * C::RS;
  s.Ty = reinterpret_cast<T*>(base + o);
  o += sizeof(T) * 2 * (kTY + 1) * C::TX;
  s.Txh = reinterpret_cast<T*>(base + o);
  o += sizeof(T) * 2 * kTY;
  o = (o + 15) / 16 * 16;
  s.acc = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * (size_t)(WACC ? kWarps : 0) * d;
  s.Yd = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * dk;
  s.Y = reinterpret_cast<T*>(base + o);
  o += sizeof(T) * dk;
  o = (o + 15) / 16 * 16;
  s.red = reinterpret_cast<double*>(base + o);
  return s;
}

// Reads of CX consecutive T from shared memory (16-byte aligned when CX == 4).
template <typename T, int CX>
__device__ __forceinline__ void sm_ld(const T* p, T (&v)[CX]) {
  if constexpr (CX == 4) {
    if constexpr (sizeof(T) == 4) {
      float4 q = *reinterpret_cast<const float4*>(p);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
      double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
      v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < CX; ++c) v[c] = p[c];
  }
}
template <typename T, int CX>
__device__ __forceinline__ void sm_st(T* p, const T (&v)[CX]) {
  if constexpr (CX == 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
      reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < CX; ++c) p[c] = v[c];
  }
}

// Where this thread sits for a segment (column tile, z range).
struct Seg {
  int x0, y0, z0, z1;
  int y;      // the grid row this warp handles
  bool own;   // an interior row (else a halo row)
  int xl;     // first cell of this lane
  int nv;     // valid cells of this lane (0 if the row is outside the grid)
  int64_t rowbase;  // row start in cell order (labels, FP64 arrays)
  int64_t rowp;     // row start at the inner arrays' pitch (vectors, inner faces)
};

template <int TX>
__device__ __forceinline__ Seg make_seg(const SolveArgs& a, int64_t ct, int z0, int z1, int cx) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Seg s;
  const int tx = (int)(ct % a.ntx), ty = (int)(ct / a.ntx);
  s.x0 = tx * TX;
  s.y0 = ty * kTY;
  s.z0 = z0;
  s.z1 = z1;
  s.own = warp < kTY;
  s.y = s.own ? s.y0 + warp : (warp == kTY ? s.y0 - 1 : s.y0 + kTY);
  s.xl = s.x0 + lane * cx;
  const bool rowok = s.y >= 0 && s.y < a.g.ny;
  s.nv = rowok ? max(0, min(cx, a.g.nx - s.xl)) : 0;
  s.rowbase = (int64_t)s.y * a.g.nx + s.xl;
  s.rowp = (int64_t)s.y * a.vp + s.xl;
  return s;
}

// ---------------------------------------------------------------------------
// Sweep A: p = z + beta p_old, v = A p, s = Z^T v, gamma = p . v
//
// Software pipeline: at step z a lane issues the loads of plane z+2's z and
// p_old (its z+1 neighbour one step later), plane z+1's faces and labels,
// and its x-halo values of plane z+1, and consumes them a step later; the
// halo-row warps likewise load plane z+1 while publishing plane z.
// ---------------------------------------------------------------------------
template <typename T, int CX>
struct FacesA {
  T fx[CX], fy[CX], fz[CX], dg[CX];
  int lb[CX];
};

template <typename T, int CX, bool WACC>
__device__ void sweep_A(const SolveArgs& a, const Sm<T>& sm, const T* zb, const T* pold, T* pnew, T beta,
                        const T* __restrict__ Fx, const T* __restrict__ Fy, const T* __restrict__ Fz,
                        double* part_row) {
  using C = Cfg<T, CX, WACC>;
  constexpr int TX = C::TX, RS = C::RS, HOFF = C::HOFF;
  const Geo& g = a.g;
  const int d = a.d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < kTY * d; k += blockDim.x) sm.acc[k] = 0.0;
  __syncthreads();
  LabelAcc<T, true> la;
  la.init(a.lab_L);
  double dgam = 0.0;
  const int tr = team_rank(a.sy);
  int64_t t0, t1;
  tile_range(a, tr, &t0, &t1);
  for (int64_t t = t0; t < t1;) {
    const int64_t ct = t / g.nz;
    const int z0 = (int)(t % g.nz);
    const int z1 = (int)((int64_t)g.nz < (int64_t)z0 + (t1 - t) ? (int64_t)g.nz : (int64_t)z0 + (t1 - t));
    t += z1 - z0;
    const Seg sg = make_seg<TX>(a, ct, z0, z1, CX);
    // raw z and p_old of this lane's cells of plane zz (0 outside the grid)
    auto ld_raw = [&](int zz, T(&zv)[CX], T(&po)[CX]) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) zv[c] = po[c] = T(0);
        return;
      }
      const int64_t i = (int64_t)zz * a.vpxy + sg.rowp;
      ld_cells<T, CX, false>(zb, i, sg.nv, zv);
      ld_cells<T, CX, false>(pold, i, sg.nv, po);
    };
    auto ld_faces = [&](int zz, FacesA<T, CX>& f) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          f.fx[c] = f.fy[c] = f.fz[c] = f.dg[c] = T(0);
          f.lb[c] = -1;
        }
        return;
      }
      const int64_t i = (int64_t)zz * g.nxy + sg.rowbase, ip = (int64_t)zz * a.vpxy + sg.rowp;
      ld_cells<T, CX, true>(Fx, ip, sg.nv, f.fx);
      ld_cells<T, CX, true>(Fy, ip, sg.nv, f.fy);
      ld_cells<T, CX, true>(Fz, ip, sg.nv, f.fz);
      ld_labels<CX>(a.label, i, sg.nv, f.lb);
      if constexpr (sizeof(T) == 8) {
        ld_cells<T, CX, true>(a.diag64, i, sg.nv, f.dg);
      } else {
#pragma unroll
        for (int c = 0; c < CX; ++c) f.dg[c] = T(0);
      }
    };
    auto ld_fy = [&](int zz, T(&o)[CX]) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) o[c] = T(0);
        return;
      }
      ld_cells<T, CX, true>(Fy, (int64_t)zz * a.vpxy + sg.rowp, sg.nv, o);
    };
    // x-halo values of plane zz: lane 0 the cell left of the tile (z, p_old,
    // and the face between), lane 31 the cell right of it
    const bool hl_ok = sg.own && lane == 0 && sg.x0 - 1 >= 0 && sg.y < g.ny;
    const bool hr_ok = sg.own && lane == 31 && sg.x0 + TX < g.nx && sg.y < g.ny;
    auto ld_xh = [&](int zz, T& zx, T& px, T& fxl) {
      zx = px = fxl = T(0);
      if (zz < 0 || zz >= g.nz) return;
      const int64_t row = (int64_t)zz * a.vpxy + (int64_t)sg.y * a.vp;
      if (hl_ok) {
        zx = zb[row + sg.x0 - 1];
        px = pold[row + sg.x0 - 1];
        fxl = __ldg(Fx + row + sg.x0 - 1);
      } else if (hr_ok) {
        zx = zb[row + sg.x0 + TX];
        px = pold[row + sg.x0 + TX];
      }
    };
    T pm[CX], pc[CX], pn[CX], tzm[CX], zv2[CX], po2[CX];
    FacesA<T, CX> F, F1;
    T xz0 = T(0), xp0 = T(0), xf0 = T(0), xz1 = T(0), xp1 = T(0), xf1 = T(0);
    bool dxc[CX], dxm[CX], dxp[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) {
      const int x = sg.xl + c;
      dxc[c] = dir_axis(x, g.nx, g.dlo_x, g.dhi_x);
      dxm[c] = dir_axis(x - 1, g.nx, g.dlo_x, g.dhi_x);
      dxp[c] = dir_axis(x + 1, g.nx, g.dlo_x, g.dhi_x);
    }
    const bool dyc = dir_axis(sg.y, g.ny, g.dlo_y, g.dhi_y);
    const bool dym = dir_axis(sg.y - 1, g.ny, g.dlo_y, g.dhi_y);
    const bool dyp = dir_axis(sg.y + 1, g.ny, g.dlo_y, g.dhi_y);
    if (sg.own) {
      T zv[CX], po[CX];
      ld_raw(z0 - 1, zv, po);
#pragma unroll
      for (int c = 0; c < CX; ++c) pm[c] = zv[c] + beta * po[c];
      ld_raw(z0, zv, po);
#pragma unroll
      for (int c = 0; c < CX; ++c) pc[c] = zv[c] + beta * po[c];
      ld_raw(z0 + 1, zv, po);
#pragma unroll
      for (int c = 0; c < CX; ++c) pn[c] = zv[c] + beta * po[c];
      ld_faces(z0, F);
      FacesA<T, CX> Fm;
      ld_faces(z0 - 1, Fm);
#pragma unroll
      for (int c = 0; c < CX; ++c) tzm[c] = Fm.fz[c];
      ld_xh(z0, xz0, xp0, xf0);
    } else {
      ld_raw(z0, zv2, po2);  // halo rows: plane z0 in (zv2, po2)
      if (warp == kTY) ld_fy(z0, F.fy);
    }
    T gam = T(0);
    for (int z = z0; z < z1; ++z) {
      const int buf = z & 1;
      T* sP = sm.P + buf * (kTY + 2) * RS;
      T* sTy = sm.Ty + buf * (kTY + 1) * TX;
      T* sTxh = sm.Txh + buf * kTY;
      const int64_t iz = (int64_t)z * a.vpxy + sg.rowp;
      if (sg.own) {
        // prefetch: plane z+2 vectors, plane z+1 faces and x-halo values
        ld_raw(z + 2, zv2, po2);
        ld_faces(z + 1, F1);
        ld_xh(z + 1, xz1, xp1, xf1);
        sm_st<T, CX>(sP + (warp + 1) * RS + HOFF + lane * CX, pc);
        sm_st<T, CX>(sTy + (warp + 1) * TX + lane * CX, F.fy);
        if (lane == 0) {
          sP[(warp + 1) * RS + HOFF - 1] = xz0 + beta * xp0;
          sTxh[warp] = xf0;
        }
        if (lane == 31) sP[(warp + 1) * RS + HOFF + TX] = xz0 + beta * xp0;
      } else {
        T ph[CX], zv_n[CX], po_n[CX];
        ld_raw(z + 1, zv_n, po_n);
        T fyn[CX];
        if (warp == kTY) ld_fy(z + 1, fyn);
#pragma unroll
        for (int c = 0; c < CX; ++c) ph[c] = zv2[c] + beta * po2[c];
        const int row = (warp == kTY) ? 0 : kTY + 1;
        sm_st<T, CX>(sP + row * RS + HOFF + lane * CX, ph);
        if (warp == kTY) {
          sm_st<T, CX>(sTy + lane * CX, F.fy);
#pragma unroll
          for (int c = 0; c < CX; ++c) F.fy[c] = fyn[c];
        }
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          zv2[c] = zv_n[c];
          po2[c] = po_n[c];
        }
      }
      __syncthreads();
      if (sg.own) {
        T left = __shfl_up_sync(kFull, pc[CX - 1], 1);
        T right = __shfl_down_sync(kFull, pc[0], 1);
        T txl = __shfl_up_sync(kFull, F.fx[CX - 1], 1);
        if (lane == 0) {
          left = sP[(warp + 1) * RS + HOFF - 1];
          txl = sTxh[warp];
        }
        if (lane == 31) right = sP[(warp + 1) * RS + HOFF + TX];
        T ym[CX], yp[CX], fym[CX];
        sm_ld<T, CX>(sP + warp * RS + HOFF + lane * CX, ym);
        sm_ld<T, CX>(sP + (warp + 2) * RS + HOFF + lane * CX, yp);
        sm_ld<T, CX>(sTy + warp * TX + lane * CX, fym);
        const bool dzc = dir_axis(z, g.nz, g.dlo_z, g.dhi_z);
        const bool dzm = dir_axis(z - 1, g.nz, g.dlo_z, g.dhi_z);
        const bool dzp = dir_axis(z + 1, g.nz, g.dlo_z, g.dhi_z);
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          const bool valid = c < sg.nv;
          const T u = pc[c];
          const T xm = (c > 0) ? pc[(c > 0) ? c - 1 : 0] : left;
          const T xp = (c < CX - 1) ? pc[(c < CX - 1) ? c + 1 : 0] : right;
          const T fxm = (c > 0) ? F.fx[(c > 0) ? c - 1 : 0] : txl;
          const T v = stencil<T>(dxc[c] || dyc || dzc, u, F.dg[c], fxm, xm, !dxm[c], F.fx[c], xp, !dxp[c],
                                 fym[c], ym[c], !dym, F.fy[c], yp[c], !dyp, tzm[c], pm[c], !dzm, F.fz[c], pn[c],
                                 !dzp);
          la.add(valid, F.lb[c], v, sm.acc, d, warp);
          if (valid) gam += u * v;
        }
        st_cells<T, CX>(pnew, iz, sg.nv, pc);
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          pm[c] = pc[c];
          pc[c] = pn[c];
          pn[c] = zv2[c] + beta * po2[c];
          tzm[c] = F.fz[c];
        }
        F = F1;
        xz0 = xz1;
        xp0 = xp1;
        xf0 = xf1;
      }
    }
    dgam += (double)gam;
  }
  if (warp < kTY) la.flush(sm.acc, d, warp);
  const double gsum = block_sum(dgam, sm.red);  // contains __syncthreads
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kTY; ++w) t += sm.acc[w * d + k];  // warp order: deterministic
    part_row[(int64_t)(k) * a.pstride] = t;
  }
  if (threadIdx.x == 0) part_row[(int64_t)(a.dk + 0) * a.pstride] = gsum;
}

// ---------------------------------------------------------------------------
// Sweep B: u = p - Z y, w = A u, xhat += alpha p, r = diag z - alpha w,
// z = r / diag, rho' = r . z, rr = r . r  (pipelined like sweep A)
// ---------------------------------------------------------------------------
template <typename T, int CX>
struct FacesB {
  T fx[CX], fy[CX], fz[CX], dg[CX], idg[CX], zo[CX], xo[CX];
};

template <typename T, int CX, bool WACC>
__device__ void sweep_B(const SolveArgs& a, const Sm<T>& sm, const T* p, T* zb, T* xh, T alpha,
                        const T* __restrict__ Fx, const T* __restrict__ Fy, const T* __restrict__ Fz,
                        double* part_row) {
  using C = Cfg<T, CX, WACC>;
  constexpr int TX = C::TX, RS = C::RS, HOFF = C::HOFF;
  const Geo& g = a.g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* Y = sm.Y;
  double drho = 0.0, drr = 0.0;
  const int tr = team_rank(a.sy);
  int64_t t0, t1;
  tile_range(a, tr, &t0, &t1);
  for (int64_t t = t0; t < t1;) {
    const int64_t ct = t / g.nz;
    const int z0 = (int)(t % g.nz);
    const int z1 = (int)((int64_t)g.nz < (int64_t)z0 + (t1 - t) ? (int64_t)g.nz : (int64_t)z0 + (t1 - t));
    t += z1 - z0;
    const Seg sg = make_seg<TX>(a, ct, z0, z1, CX);
    // raw p and labels of this lane's cells of plane zz
    auto ld_raw = [&](int zz, T(&pv)[CX], int(&lb)[CX]) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          pv[c] = T(0);
          lb[c] = -1;
        }
        return;
      }
      ld_cells<T, CX, false>(p, (int64_t)zz * a.vpxy + sg.rowp, sg.nv, pv);
      ld_labels<CX>(a.label, (int64_t)zz * g.nxy + sg.rowbase, sg.nv, lb);
    };
    auto mk_u = [&](const T(&pv)[CX], const int(&lb)[CX], T(&u)[CX]) {
#pragma unroll
      for (int c = 0; c < CX; ++c) u[c] = (lb[c] >= 0) ? pv[c] - Y[lb[c]] : T(0);
    };
    auto ld_faces = [&](int zz, FacesB<T, CX>& f) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) f.fx[c] = f.fy[c] = f.fz[c] = f.dg[c] = f.idg[c] = f.zo[c] = f.xo[c] = T(0);
        return;
      }
      const int64_t i = (int64_t)zz * g.nxy + sg.rowbase, ip = (int64_t)zz * a.vpxy + sg.rowp;
      ld_cells<T, CX, true>(Fx, ip, sg.nv, f.fx);
      ld_cells<T, CX, true>(Fy, ip, sg.nv, f.fy);
      ld_cells<T, CX, true>(Fz, ip, sg.nv, f.fz);
      if (sg.own) {
        ld_cells<T, CX, false>(zb, ip, sg.nv, f.zo);
        ld_cells<T, CX, false>(xh, ip, sg.nv, f.xo);
      }
      if constexpr (sizeof(T) == 8) {
        ld_cells<T, CX, true>(a.diag64, i, sg.nv, f.dg);
        ld_cells<T, CX, true>(a.invdiag64, i, sg.nv, f.idg);
      } else {
#pragma unroll
        for (int c = 0; c < CX; ++c) f.dg[c] = f.idg[c] = T(0);
      }
    };
    auto ld_fy = [&](int zz, T(&o)[CX]) {
      if (zz < 0 || zz >= g.nz || sg.nv == 0) {
#pragma unroll
        for (int c = 0; c < CX; ++c) o[c] = T(0);
        return;
      }
      ld_cells<T, CX, true>(Fy, (int64_t)zz * a.vpxy + sg.rowp, sg.nv, o);
    };
    const bool hl_ok = sg.own && lane == 0 && sg.x0 - 1 >= 0 && sg.y < g.ny;
    const bool hr_ok = sg.own && lane == 31 && sg.x0 + TX < g.nx && sg.y < g.ny;
    auto ld_xh = [&](int zz, T& px, int& lx, T& fxl) {
      px = T(0);
      lx = -1;
      fxl = T(0);
      if (zz < 0 || zz >= g.nz) return;
      const int64_t row = (int64_t)zz * g.nxy + (int64_t)sg.y * g.nx;
      const int64_t rowp = (int64_t)zz * a.vpxy + (int64_t)sg.y * a.vp;
      if (hl_ok) {
        px = p[rowp + sg.x0 - 1];
        lx = __ldg(a.label + row + sg.x0 - 1);
        fxl = __ldg(Fx + rowp + sg.x0 - 1);
      } else if (hr_ok) {
        px = p[rowp + sg.x0 + TX];
        lx = __ldg(a.label + row + sg.x0 + TX);
      }
    };
    T um[CX], uc[CX], un[CX], pcur[CX], pnx[CX], tzm[CX], p2[CX];
    int l2[CX];
    FacesB<T, CX> F, F1;
    T xp0 = T(0), xf0 = T(0), xp1 = T(0), xf1 = T(0);
    int xl0 = -1, xl1 = -1;
    bool dxc[CX], dxm[CX], dxp[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) {
      const int x = sg.xl + c;
      dxc[c] = dir_axis(x, g.nx, g.dlo_x, g.dhi_x);
      dxm[c] = dir_axis(x - 1, g.nx, g.dlo_x, g.dhi_x);
      dxp[c] = dir_axis(x + 1, g.nx, g.dlo_x, g.dhi_x);
    }
    const bool dyc = dir_axis(sg.y, g.ny, g.dlo_y, g.dhi_y);
    const bool dym = dir_axis(sg.y - 1, g.ny, g.dlo_y, g.dhi_y);
    const bool dyp = dir_axis(sg.y + 1, g.ny, g.dlo_y, g.dhi_y);
    if (sg.own) {
      T pv[CX];
      int lb[CX];
      ld_raw(z0 - 1, pv, lb);
      mk_u(pv, lb, um);
      ld_raw(z0, pcur, lb);
      mk_u(pcur, lb, uc);
      ld_raw(z0 + 1, pnx, lb);
      mk_u(pnx, lb, un);
      ld_faces(z0, F);
      FacesB<T, CX> Fm;
      ld_faces(z0 - 1, Fm);
#pragma unroll
      for (int c = 0; c < CX; ++c) tzm[c] = Fm.fz[c];
      ld_xh(z0, xp0, xl0, xf0);
    } else {
      ld_raw(z0, p2, l2);  // halo rows: plane z0
      if (warp == kTY) ld_fy(z0, F.fy);
    }
    T rho = T(0), rr = T(0);
    for (int z = z0; z < z1; ++z) {
      const int buf = z & 1;
      T* sP = sm.P + buf * (kTY + 2) * RS;
      T* sTy = sm.Ty + buf * (kTY + 1) * TX;
      T* sTxh = sm.Txh + buf * kTY;
      const int64_t iz = (int64_t)z * a.vpxy + sg.rowp;
      if (sg.own) {
        ld_raw(z + 2, p2, l2);
        ld_faces(z + 1, F1);
        ld_xh(z + 1, xp1, xl1, xf1);
        sm_st<T, CX>(sP + (warp + 1) * RS + HOFF + lane * CX, uc);
        sm_st<T, CX>(sTy + (warp + 1) * TX + lane * CX, F.fy);
        if (lane == 0) {
          sP[(warp + 1) * RS + HOFF - 1] = xl0 >= 0 ? xp0 - Y[xl0] : T(0);
          sTxh[warp] = xf0;
        }
        if (lane == 31) sP[(warp + 1) * RS + HOFF + TX] = xl0 >= 0 ? xp0 - Y[xl0] : T(0);
      } else {
        T uh[CX], pv[CX];
        int lb[CX];
        ld_raw(z + 1, pv, lb);
        T fyn[CX];
        if (warp == kTY) ld_fy(z + 1, fyn);
        mk_u(p2, l2, uh);
        const int row = (warp == kTY) ? 0 : kTY + 1;
        sm_st<T, CX>(sP + row * RS + HOFF + lane * CX, uh);
        if (warp == kTY) {
          sm_st<T, CX>(sTy + lane * CX, F.fy);
#pragma unroll
          for (int c = 0; c < CX; ++c) F.fy[c] = fyn[c];
        }
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          p2[c] = pv[c];
          l2[c] = lb[c];
        }
      }
      __syncthreads();
      if (sg.own) {
        T left = __shfl_up_sync(kFull, uc[CX - 1], 1);
        T right = __shfl_down_sync(kFull, uc[0], 1);
        T txl = __shfl_up_sync(kFull, F.fx[CX - 1], 1);
        if (lane == 0) {
          left = sP[(warp + 1) * RS + HOFF - 1];
          txl = sTxh[warp];
        }
        if (lane == 31) right = sP[(warp + 1) * RS + HOFF + TX];
        T ym[CX], yp[CX], fym[CX];
        sm_ld<T, CX>(sP + warp * RS + HOFF + lane * CX, ym);
        sm_ld<T, CX>(sP + (warp + 2) * RS + HOFF + lane * CX, yp);
        sm_ld<T, CX>(sTy + warp * TX + lane * CX, fym);
        const bool dzc = dir_axis(z, g.nz, g.dlo_z, g.dhi_z);
        const bool dzm = dir_axis(z - 1, g.nz, g.dlo_z, g.dhi_z);
        const bool dzp = dir_axis(z + 1, g.nz, g.dlo_z, g.dhi_z);
        T zn[CX], xn[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          const T u = uc[c];
          const T xm = (c > 0) ? uc[(c > 0) ? c - 1 : 0] : left;
          const T xp = (c < CX - 1) ? uc[(c < CX - 1) ? c + 1 : 0] : right;
          const T fxm = (c > 0) ? F.fx[(c > 0) ? c - 1 : 0] : txl;
          const bool dirc = dxc[c] || dyc || dzc;
          T dgi;
          if constexpr (sizeof(T) == 8) dgi = F.dg[c];
          else dgi = dirc ? T(1) : (((((tzm[c] + fym[c]) + fxm) + F.fx[c]) + F.fy[c]) + F.fz[c]);
          const T w = stencil<T>(dirc, u, dgi, fxm, xm, !dxm[c], F.fx[c], xp, !dxp[c], fym[c], ym[c], !dym,
                                 F.fy[c], yp[c], !dyp, tzm[c], um[c], !dzm, F.fz[c], un[c], !dzp);
          const T r = dgi * F.zo[c] - alpha * w;
          T znew;
          if constexpr (sizeof(T) == 8) znew = r * F.idg[c];
          else znew = __fdividef(r, dgi);  // FP32 inner: 2-ulp division
          zn[c] = znew;
          xn[c] = F.xo[c] + alpha * pcur[c];
          if (c < sg.nv) {
            rho += r * znew;
            rr += r * r;
          }
        }
        st_cells<T, CX>(zb, iz, sg.nv, zn);
        st_cells<T, CX>(xh, iz, sg.nv, xn);
        T u2[CX];
        mk_u(p2, l2, u2);
#pragma unroll
        for (int c = 0; c < CX; ++c) {
          um[c] = uc[c];
          uc[c] = un[c];
          un[c] = u2[c];
          pcur[c] = pnx[c];
          pnx[c] = p2[c];
          tzm[c] = F.fz[c];
        }
        F = F1;
        xp0 = xp1;
        xl0 = xl1;
        xf0 = xf1;
      }
    }
    drho += (double)rho;
    drr += (double)rr;
  }
  const double s1 = block_sum(drho, sm.red);
  const double s2 = block_sum(drr, sm.red);
  if (threadIdx.x == 0) {
    part_row[(int64_t)(a.dk + 1) * a.pstride] = s1;
    part_row[(int64_t)(a.dk + 2) * a.pstride] = s2;
  }
}

template <typename T, int CX, bool WACC>
__device__ __forceinline__ void solve_generic(const SolveArgs& a, unsigned char* smem_raw) {
  Sm<T> sm = carve<T, CX, WACC>(smem_raw, a.d, a.dk);
  if (!WACC) sm.acc = a.gacc + (int64_t)blockIdx.x * a.gacc_stride;
  const T* Fx = static_cast<const T*>(a.Txi);
  const T* Fy = static_cast<const T*>(a.Tyi);
  const T* Fz = static_cast<const T*>(a.Tzi);
  T* zb = static_cast<T*>(a.z);
  T* xh = static_cast<T*>(a.xh);
  T* pb[2] = {static_cast<T*>(a.p0), static_cast<T*>(a.p1)};
  solve_body<T, WACC>(
      a, sm.acc, sm.Yd, sm.Y, sm.red,
      [&](int po, T beta, double* part) {
        sweep_A<T, CX, WACC>(a, sm, zb, pb[po], pb[po ^ 1], beta, Fx, Fy, Fz, part);
        return true;
      },
      [&](int pn, T alpha, double* part) {
        sweep_B<T, CX, WACC>(a, sm, pb[pn], zb, xh, alpha, Fx, Fy, Fz, part);
        return true;
      });
}

template <typename T, int CX, bool WACC>
__global__ void __launch_bounds__(kThreads, 1) k_solve(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  solve_generic<T, CX, WACC>(a, smem_raw);
}

// Batched solve: CTA c works on system cta_sys[c] with the team of CTAs the
// host assigned to it (its barriers, reductions and partial sums are the
// team's own); teams never wait on each other, and a team leaves the kernel
// as soon as its system is solved.
template <typename T, int CX, bool WACC>
__global__ void __launch_bounds__(kThreads, 1) k_solve_batch(const SolveArgs* __restrict__ all,
                                                         const int* __restrict__ cta_sys) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SolveArgs a;
  if (threadIdx.x == 0) a = all[cta_sys[blockIdx.x]];
  __syncthreads();
  solve_generic<T, CX, WACC>(a, smem_raw);
}

template <typename T, int CX, bool WACC>
int launch(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg) {
  const size_t smem = smem_bytes<T, CX, WACC>(a.d, a.dk);
  auto kern = k_solve<T, CX, WACC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    *msg = std::string("solve kernel attribute: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
  if (per < 1) {
    *msg = "solve kernel does not fit on an SM";
    return SLD_ERR_CUDA;
  }
  if (o.ctas_per_sm > 0) per = std::min(per, o.ctas_per_sm);
  int G = s->nsm * per;
  G = (int)std::max<int64_t>(1, std::min<int64_t>(G, a.ntiles));
  if (G > s->part_rows) G = s->part_rows;
  a.sy.cta0 = 0;
  a.sy.ncta = G;
  if (!WACC) {
    a.gacc_stride = (int64_t)kGaccRows * a.d;
    e = ensure_gacc(s, (size_t)G * a.gacc_stride);
    if (e != cudaSuccess) {
      *msg = std::string("label-sum rows: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? SLD_ERR_OOM : SLD_ERR_CUDA;
    }
    a.gacc = s->gacc;
  }
  void* args[] = {&a};
  cudaEventRecord(s->ev0, s->stream);
  e = cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(kThreads), args, smem, s->stream);
  cudaEventRecord(s->ev1, s->stream);
  if (e != cudaSuccess) {
    *msg = std::string("solve launch: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  e = cudaEventSynchronize(s->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    *msg = std::string("solve kernel: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  cudaEventElapsedTime(ms, s->ev0, s->ev1);
  return SLD_OK;
}

}  // namespace

void fill_args(sld_system s, const double* b_dev, const sld_options& o, SolveArgs* ap) {
  SolveArgs& a = *ap;
  a = SolveArgs{};
  const bool fp64 = o.precision == SLD_FP64;
  a.g = s->g;
  a.cx = (s->g.nx % 4 == 0 && s->g.nx >= 96) ? 4 : 1;
  const int TX = 32 * a.cx;
  a.ntx = (s->g.nx + TX - 1) / TX;
  a.nty = (s->g.ny + kTY - 1) / kTY;
  a.ntiles = (int64_t)a.ntx * a.nty * s->g.nz;
  // inner vectors and inner faces: rows padded to s->nxp cells in the FP32
  // and BF16 forms (TMA boxes need 16-byte row strides); FP64 form unpadded
  a.vp = fp64 ? s->g.nx : s->nxp;
  a.vpxy = (int64_t)a.vp * s->g.ny;
  a.d = s->d;
  a.kL = s->kL;
  a.dk = s->d + s->kL;
  a.ZL32 = s->ZL32;
  a.WL64 = s->WL64;
  a.WLi = fp64 ? (const void*)s->WL64 : (const void*)s->WL32;
  a.label = s->label;
  a.label16 = s->label16;
  // labels from the subdomain-levelset rule with d = S * L keep that structure
  a.lab_L = (s->labels_L >= 1 && s->labels_L <= 4 && s->d == s->have_labels_d) ? s->labels_L : 0;
  const char* lmode = std::getenv("SLD_LABEL_MODE");  // "general": treat labels as unstructured
  if (lmode && std::strcmp(lmode, "general") == 0) a.lab_L = 0;
  a.Einv = s->Einv;
  const bool bf16 = o.precision == SLD_BF16COEF_IR;
  a.Einv_inner = bf16 ? s->Einv16 : s->Einv;
  a.invdi = bf16 ? s->invd16 : nullptr;
  a.bf16 = bf16 ? 1 : 0;
  a.Tx64 = s->Tx;
  a.Ty64 = s->Ty;
  a.Tz64 = s->Tz;
  a.diag64 = s->diag;
  a.invdiag64 = s->invdiag;
  a.b = b_dev;
  a.x = s->x;
  a.r64 = s->r64;
  if (fp64) {
    a.Txi = s->Tx;
    a.Tyi = s->Ty;
    a.Tzi = s->Tz;
  } else if (bf16) {
    a.Txi = s->Tx16;
    a.Tyi = s->Ty16;
    a.Tzi = s->Tz16;
  } else {
    a.Txi = s->Tx32;
    a.Tyi = s->Ty32;
    a.Tzi = s->Tz32;
  }
  a.z = s->z;
  a.p0 = s->p0;
  a.p1 = s->p1;
  a.xh = s->xh;
  a.part = s->part;
  a.pstride = s->part_rows;  // column-major partials: one slot per CTA
  a.gacc = nullptr;          // set at launch when d > kWarpAccMaxD
  a.gacc_stride = 0;
  a.s_glob = s->s_glob;
  a.y_glob = s->y_glob;
  a.out = s->out;
  a.sy.count = s->bar;
  a.sy.status = s->status;
  a.sy.timeout_ns = (unsigned long long)((o.timeout_s > 0 ? o.timeout_s : 2.0) * 1e9);
  a.sy.skip_epoch = o.debug_skip_barrier >= 0 ? o.debug_skip_barrier + 1 : 0;
  a.tol = o.tol;
  a.inner_tol = o.inner_tol;
  a.fwd_tol = o.fwd_tol == 0.0 ? 100.0 * o.tol : o.fwd_tol;
  a.maxiter = o.maxiter;
  a.max_outer = fp64 ? 1 : o.max_outer;
  a.fp64 = fp64 ? 1 : 0;
  a.warm = 0;
}

int run_solve(sld_system s, const double* b_dev, const sld_options& o, sld_result* res, std::string* msg,
              bool warm) {
  const int64_t n = s->g.n;
  const bool fp64 = o.precision == SLD_FP64;
  const bool bf16 = o.precision == SLD_BF16COEF_IR;
  SolveArgs a;
  fill_args(s, b_dev, o, &a);
  a.warm = warm && !fp64 ? 1 : 0;
  // x = 0 (unless warm); the inner state is set by the first refinement step
  if (!a.warm) cudaMemsetAsync(s->x, 0, sizeof(double) * n, s->stream);
  cudaMemsetAsync(s->xh, 0, sizeof(double) * s->nvec, s->stream);
  cudaMemsetAsync(s->bar, 0, 64, s->stream);
  cudaMemsetAsync(s->out, 0, sizeof(double) * kOutCount, s->stream);
  float ms = 0.f;
  int st;
  const bool wacc = s->d <= kWarpAccMaxD;
  const char* force = std::getenv("SLD_SOLVER_PATH");
  const bool use_tma = tma_eligible(s->g, fp64) && !(force && std::strcmp(force, "generic") == 0);
  if (bf16 && !use_tma) {
    *msg = "BF16 coefficients are streamed by the TMA sweeps only";
    return SLD_ERR_INVALID_ARG;
  }
  if (s->kL > 0 && (!use_tma || bf16 || s->g.nx % 8 != 0)) {
    *msg = "extra dense deflation vectors need the TMA sweeps (nx % 8 == 0) and SLD_FP64 or SLD_FP32_IR";
    return SLD_ERR_INVALID_ARG;
  }
  res->kernel_path = use_tma ? 1 : 0;
  if (use_tma) {
    st = launch_solve_tma(s, a, o, &ms, msg);
  } else if (fp64) {
    if (a.cx == 4) st = wacc ? launch<double, 4, true>(s, a, o, &ms, msg) : launch<double, 4, false>(s, a, o, &ms, msg);
    else st = wacc ? launch<double, 1, true>(s, a, o, &ms, msg) : launch<double, 1, false>(s, a, o, &ms, msg);
  } else {
    if (a.cx == 4) st = wacc ? launch<float, 4, true>(s, a, o, &ms, msg) : launch<float, 4, false>(s, a, o, &ms, msg);
    else st = wacc ? launch<float, 1, true>(s, a, o, &ms, msg) : launch<float, 1, false>(s, a, o, &ms, msg);
  }
  if (st != SLD_OK) return st;
  double out[kOutCount];
  int dev_status = 0;
  cudaMemcpyAsync(out, s->out, sizeof(out), cudaMemcpyDeviceToHost, s->stream);
  cudaMemcpyAsync(&dev_status, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    *msg = std::string("solve readback: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  res->iterations = (int)out[kOutIters];
  res->outer_steps = (int)out[kOutOuter];
  res->recursive_relres = out[kOutBB] > 0 ? std::sqrt(out[kOutRecRR] / out[kOutBB]) : 0.0;
  res->fwd_err_estimate = out[kOutFwd];
  if (!fp64 && std::getenv("SLD_TRACE_REFINEMENT")) {
    // |d_k| / |x_k| and ||r_k|| / ||b|| per refinement step, to stderr
    std::fprintf(stderr, "sld refinement: %d steps, %d iterations, estimate %.3e\n", res->outer_steps,
                 res->iterations, res->fwd_err_estimate);
    for (int k = 0; k < res->outer_steps && k < kTraceSteps; ++k)
      std::fprintf(stderr, "  step %2d  |d|/|x| %.3e  |r|/|b| %.3e\n", k + 1, std::sqrt(out[kOutTrace + 2 * k]),
                   std::sqrt(out[kOutTrace + 2 * k + 1]));
  }
  res->solve_ms = ms;
  if (dev_status != 0) {
    *msg = dev_status == SLD_ERR_TIMEOUT ? "a device-side wait timed out (grid barrier)" : "device error";
    return dev_status;
  }
  const int code = (int)out[kOutStatus];
  if (code == SLD_ERR_NOT_CONVERGED) *msg = "not converged within maxiter / max_outer";
  if (code == SLD_ERR_BREAKDOWN) *msg = "breakdown: p^T P A p <= 0 or a non-finite scalar";
  return code;
}


// ---------------------------------------------------------------------------
// Batched solve plan.
// ---------------------------------------------------------------------------
namespace {

template <typename T, int CX, bool WACC>
int batch_capture(sld_system s0, BatchPlan* p, sld_system* sys, std::string* msg) {
  auto kern = k_solve_batch<T, CX, WACC>;
  cudaError_t e = p->tma ? cudaSuccess
                         : cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
  if (e != cudaSuccess) {
    *msg = std::string("batch kernel attribute: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  (void)s0;
  cudaStream_t st = p->stream;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    *msg = std::string("graph capture: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  for (int k = 0; k < p->count; ++k) {
    sld_system s = sys[k];
    cudaMemsetAsync(s->x, 0, sizeof(double) * s->g.n, st);
    cudaMemsetAsync(s->xh, 0, sizeof(double) * s->nvec, st);
    cudaMemsetAsync(s->bar, 0, 64, st);
    cudaMemsetAsync(s->out, 0, sizeof(double) * kOutCount, st);
    cudaMemsetAsync(s->status, 0, sizeof(int) * 4, st);
  }
  cudaError_t el;
  if (p->tma) {
    el = tma_batch_launch(p->G, p->smem, p->args_off, p->wacc, p->d_args, p->h_args, p->count, p->d_maps, p->d_cta,
                          st);
  } else {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(p->G);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = p->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const SolveArgs* da = p->d_args;
    const int* dc = p->d_cta;
    el = cudaLaunchKernelEx(&cfg, kern, da, dc);
  }
  e = cudaStreamEndCapture(st, &p->graph);
  if (el != cudaSuccess || e != cudaSuccess) {
    *msg = std::string("batch capture: ") + cudaGetErrorString(el != cudaSuccess ? el : e);
    return SLD_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) {
    *msg = std::string("graph instantiate: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  return SLD_OK;
}

template <typename T, int CX, bool WACC>
int batch_occupancy(size_t smem) {
  auto kern = k_solve_batch<T, CX, WACC>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
  return per;
}

template <typename T, int CX, bool WACC>
size_t batch_smem(int dmax) {
  return smem_bytes<T, CX, WACC>(dmax, dmax);
}

}  // namespace

void batch_free(BatchPlan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_args) cudaFree(p->d_args);
  if (p->d_cta) cudaFree(p->d_cta);
  if (p->d_maps) cudaFree(p->d_maps);
  if (p->d_gacc) cudaFree(p->d_gacc);
  delete[] p->h_args;
  p->d_maps = nullptr;
  p->d_gacc = nullptr;
  p->h_args = nullptr;
  p->exec = nullptr;
  p->graph = nullptr;
  p->d_args = nullptr;
  p->d_cta = nullptr;
}

// Teams: at least one CTA per system, at most one per plane tile and per
// partial-sum row.  Without a measurement, system k's share is proportional
// to n_k^expo.  With one (cost: the CTA-time each system took in an earlier
// launch, its team's CTAs x its time in the kernel), the CTAs are dealt out
// to minimise the slowest system's modelled time
// T_k(t) = cost_k / t + fixed_k: every system starts with one CTA and each
// further CTA goes to the currently slowest system (optimal for these
// decreasing convex times).
int batch_build(sld_system* sys, int count, const sld_options& o, int per_sm, double expo, const double* cost,
                int cx, cudaStream_t stream, BatchPlan* p, std::string* msg, const double* fixed) {
  sld_system s0 = sys[0];
  p->stream = stream;
  p->count = count;
  p->fp64 = o.precision == SLD_FP64;
  p->cx = cx;
  p->expo = expo;
  int dmax = 1;
  for (int k = 0; k < count; ++k) dmax = std::max(dmax, sys[k]->d);
  p->wacc = dmax <= kWarpAccMaxD;
#define SLD_BATCH_DISPATCH(FN, ...)                                                              \
  (p->fp64 ? (cx == 4 ? (p->wacc ? FN<double, 4, true>(__VA_ARGS__) : FN<double, 4, false>(__VA_ARGS__)) \
                      : (p->wacc ? FN<double, 1, true>(__VA_ARGS__) : FN<double, 1, false>(__VA_ARGS__))) \
           : (cx == 4 ? (p->wacc ? FN<float, 4, true>(__VA_ARGS__) : FN<float, 4, false>(__VA_ARGS__))   \
                      : (p->wacc ? FN<float, 1, true>(__VA_ARGS__) : FN<float, 1, false>(__VA_ARGS__))))
  // the FP32-inner batch runs on the TMA sweeps; the FP64 one on the
  // register/shuffle sweeps (the FP64 operator's rows are not padded)
  p->tma = !p->fp64 && tma_eligible(s0->g, false);
  int occ;
  if (p->tma) {
    p->args_off = tma_batch_args_off(dmax, p->wacc);
    p->smem = tma_batch_smem(dmax, p->wacc);
    occ = tma_batch_occupancy(p->wacc, p->smem);
  } else {
    p->smem = SLD_BATCH_DISPATCH(batch_smem, dmax);
    occ = SLD_BATCH_DISPATCH(batch_occupancy, p->smem);
  }
  if (occ < 1) {
    *msg = "batch kernel does not fit on an SM";
    return SLD_ERR_CUDA;
  }
  p->per_sm = per_sm > 0 ? std::min(per_sm, occ) : occ;
  int G = s0->nsm * p->per_sm;
  if (count > G) {
    *msg = "more systems (" + std::to_string(count) + ") than co-resident CTAs (" + std::to_string(G) + ")";
    return SLD_ERR_INVALID_ARG;
  }
  std::vector<SolveArgs> args(count);
  std::vector<double> w(count), ideal(count);
  std::vector<int> cap(count);
  double wsum = 0.0;
  for (int k = 0; k < count; ++k) {
    fill_args(sys[k], sys[k]->bwork, o, &args[k]);
    SolveArgs& a = args[k];
    if (p->tma) {
      tma_batch_tiles(&a);
    } else {
      a.cx = cx;
      const int TX = 32 * cx;
      a.ntx = (a.g.nx + TX - 1) / TX;
      a.nty = (a.g.ny + kTY - 1) / kTY;
      a.ntiles = (int64_t)a.ntx * a.nty * a.g.nz;
    }
    cap[k] = (int)std::min<int64_t>(std::min<int64_t>(a.ntiles, sys[k]->part_rows), G);
    w[k] = std::pow((double)a.g.n, expo);
    wsum += w[k];
  }
  int used = 0;
  if (cost) {  // min-max over the modelled times, greedy
    for (int k = 0; k < count; ++k) p->teams[k] = 1;
    used = count;
    auto T = [&](int k, int t) { return std::max(cost[k], 1e-9) / t + (fixed ? fixed[k] : 0.0); };
    std::vector<std::pair<double, int>> heap;
    for (int k = 0; k < count; ++k) heap.push_back({T(k, 1), k});
    std::make_heap(heap.begin(), heap.end());
    while (used < G && !heap.empty()) {
      std::pop_heap(heap.begin(), heap.end());
      const int k = heap.back().second;
      heap.pop_back();
      if (p->teams[k] >= cap[k]) break;  // the slowest system cannot be sped up: stop
      ++p->teams[k];
      ++used;
      heap.push_back({T(k, p->teams[k]), k});
      std::push_heap(heap.begin(), heap.end());
    }
  } else {
    for (int k = 0; k < count; ++k) {
      ideal[k] = G * w[k] / wsum;
      p->teams[k] = std::max(1, std::min(cap[k], (int)ideal[k]));
      used += p->teams[k];
    }
    while (used > G) {  // give back from the largest teams
      int j = 0;
      for (int k = 1; k < count; ++k)
        if (p->teams[k] > p->teams[j]) j = k;
      if (p->teams[j] <= 1) break;
      --p->teams[j];
      --used;
    }
    while (used < G) {  // hand out the rest where the share is most short
      int j = -1;
      double best = -1e300;
      for (int k = 0; k < count; ++k)
        if (p->teams[k] < cap[k] && ideal[k] - p->teams[k] > best) {
          best = ideal[k] - p->teams[k];
          j = k;
        }
      if (j < 0) break;
      ++p->teams[j];
      ++used;
    }
  }
  p->G = used;
  std::vector<int> cta_sys;
  cta_sys.reserve(used);
  for (int k = 0; k < count; ++k) {
    args[k].sy.cta0 = (int)cta_sys.size();
    args[k].sy.ncta = p->teams[k];
    for (int c = 0; c < p->teams[k]; ++c) cta_sys.push_back(k);
  }
  cudaError_t e = cudaSuccess;
  if (!p->wacc) {  // the CTAs' global label-sum rows, one slice per CTA of the launch
    const int64_t stride = (int64_t)kGaccRows * dmax;
    e = cudaMalloc(&p->d_gacc, sizeof(double) * (size_t)used * stride);
    for (int k = 0; k < count; ++k) {
      args[k].gacc = p->d_gacc;
      args[k].gacc_stride = stride;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->d_args, sizeof(SolveArgs) * count);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_cta, sizeof(int) * used);
  if (e == cudaSuccess && p->tma) {
    std::vector<unsigned char> maps(tma_maps_bytes() * count);
    for (int k = 0; k < count; ++k)
      if (!tma_batch_maps(args[k], maps.data() + tma_maps_bytes() * k)) {
        *msg = "batch: tensor map creation failed";
        return SLD_ERR_CUDA;
      }
    e = cudaMalloc(&p->d_maps, maps.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice);
  }
  p->h_args = new SolveArgs[count];
  std::memcpy(p->h_args, args.data(), sizeof(SolveArgs) * count);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_args, args.data(), sizeof(SolveArgs) * count, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_cta, cta_sys.data(), sizeof(int) * used, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    *msg = std::string("batch plan: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SLD_ERR_OOM : SLD_ERR_CUDA;
  }
  return SLD_BATCH_DISPATCH(batch_capture, s0, p, sys, msg);
#undef SLD_BATCH_DISPATCH
}

}  // namespace sld
