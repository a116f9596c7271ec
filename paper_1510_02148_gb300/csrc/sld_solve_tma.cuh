// sld_solve_tma.cuh -- the persistent SLD-DPCG solve with TMA-pipelined sweeps
// (grids with nx % 8 == 0): kernel templates, tensor maps and the launch;
// sld_solve_tma.cu and sld_solve_tma_learned.cu instantiate them.
//
// Each CTA owns a contiguous range of plane tiles (kTX x TY cells of one z
// plane) in (column tile, z) order and walks it plane by plane.  For every
// plane one elected thread issues cp.async.bulk.tensor loads of all boxes the
// plane needs -- the vectors with a one-cell halo in x and y (the x halo
// rounded out to 16 bytes), the three face arrays, the labels -- into one
// slot of an S-deep shared-memory ring; an mbarrier per slot counts the
// bytes in.  Boxes that reach past the grid are zero-filled by the TMA unit,
// and the face coefficients on the boundary are 0, so no edge code is needed.
// While plane z is computed, plane z+1 (its +z neighbour, already resident)
// and planes z+2 .. z+S-1 (in flight) occupy the other slots; a slot is refilled right after
// the __syncthreads that ends the step that last read it.  Thread (r, c) of a
// CTA computes the four cells x0+4c .. x0+4c+3 of row y0+r.
//
// The control flow, refinement sweeps and reductions are those of
// sld_solve_common.cuh.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "sld_solve_common.cuh"

namespace sld {
namespace {

constexpr int kTX = 64;  // cells per tile row

// T: vector type (double, or float for the inner iteration of the mixed
// solve); F: stored face type (T, or bf16 for the BF16-coefficient form).
template <typename T, typename F, int TY>
struct TCfg {
  static constexpr int H = 16 / (int)sizeof(T);  // x halo so that boxes start on 16 bytes
  static constexpr int HF = 16 / (int)sizeof(F);  // the same for the Fx box
  static constexpr int WF = kTX + 2 * HF;
  static constexpr int HL = 8;                   // x halo of the (16-bit) label box
  static constexpr int WH = kTX + 2 * H;         // halo box width
  static constexpr int WL = kTX + 2 * HL;
  static constexpr bool kDiag = sizeof(T) == 8;  // FP64 form uses the stored diagonal and inverse
  static constexpr bool kScale = sizeof(F) == 2;  // BF16 form: FP32 per-cell inverse diagonal
  static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr size_t bH = sizeof(T) * (TY + 2) * WH;   // vector with halo
  static constexpr size_t bX = sizeof(F) * TY * WF;         // Fx with the face left of the tile
  static constexpr size_t bY = sizeof(F) * (TY + 1) * kTX;  // Fy with the face below the tile
  static constexpr size_t bOF = sizeof(F) * TY * kTX;       // Fz, own cells
  static constexpr size_t bO = sizeof(T) * TY * kTX;        // own cells
  static constexpr size_t bOS = 4 * TY * kTX;               // FP32 per-cell scale, own cells
  static constexpr size_t bLO = 2 * TY * kTX;               // labels, own cells
  static constexpr size_t bLH = 2 * (TY + 2) * WL;          // labels with halo
  // sweep A slot: z(h) p_old(h) Fx Fy Fz labels [diag]
  static constexpr size_t A_ZB = 0, A_PO = al(bH), A_FX = A_PO + al(bH), A_FY = A_FX + al(bX),
                          A_FZ = A_FY + al(bY), A_LB = A_FZ + al(bOF), A_DG = A_LB + al(bLO),
                          A_END = A_DG + (kDiag ? al(bO) : 0);
  static constexpr unsigned TX_A = unsigned(2 * bH + bX + bY + bOF + bLO + (kDiag ? bO : 0));
  // sweep B slot: p(h) labels(h) Fx Fy Fz z xhat [diag, 1/diag].  In the FP64
  // form the own z and xhat are read straight from global memory instead, so
  // that three slots of the wider FP64 boxes fit two CTAs per SM.
  static constexpr bool kOwnRing = !kDiag;  // own z, xhat through the ring
  static constexpr size_t B_P = 0, B_LB = al(bH), B_FX = B_LB + al(bLH), B_FY = B_FX + al(bX),
                          B_FZ = B_FY + al(bY), B_ZO = B_FZ + al(bOF), B_XO = B_ZO + (kOwnRing ? al(bO) : 0),
                          B_DG = B_XO + (kOwnRing ? al(bO) : 0), B_IDG = B_DG + (kDiag ? al(bO) : 0),
                          B_SC = B_IDG + (kDiag ? al(bO) : 0), B_END = B_SC + (kScale ? al(bOS) : 0);
  static constexpr unsigned TX_B = unsigned(bH + bLH + bX + bY + bOF + (kOwnRing ? 2 * bO : 0) +
                                            (kDiag ? 2 * bO : 0) + (kScale ? bOS : 0));
  static constexpr size_t SLOT = A_END > B_END ? A_END : B_END;
  static constexpr int kAcc = TY / 2;  // warps = rows of label accumulators (acc_rows())
};

// Tensor maps (3-D: x, y, z), built on the host for this handle's buffers.
struct Maps {
  CUtensorMap zb_h;     // z with halo          box (WH, TY+2)
  CUtensorMap p_h[2];   // p buffers with halo  box (WH, TY+2)
  CUtensorMap fx;       // Fx                   box (WF, TY)
  CUtensorMap fy;       // Fy                   box (kTX, TY+1)
  CUtensorMap fz;       // Fz                   box (kTX, TY)
  CUtensorMap lb_o;     // labels               box (kTX, TY)
  CUtensorMap lb_h;     // labels with halo     box (WL, TY+2)
  CUtensorMap zb_o;     // z                    box (kTX, TY)
  CUtensorMap xh_o;     // xhat                 box (kTX, TY)
  CUtensorMap dg_o;     // diag (FP64 form)     box (kTX, TY)
  CUtensorMap idg_o;    // 1/diag (FP64 form)   box (kTX, TY)
  CUtensorMap sc_o;     // FP32 1/diag (BF16)   box (kTX, TY)
};

// The CTA's sequence of planes to load: for every segment (column tile ct,
// planes z0 .. z1-1) the planes z0-1 .. z1 (the z neighbours included); the
// tile origin (x0, y0) is computed once per segment.
struct Walk {
  int64_t t, t1;
  int nz, ntx, ty, z0, z1, k, kn, x0, y0;
  __device__ void begin(int64_t a, int64_t b, int nz_, int ntx_, int ty_) {
    t = a;
    t1 = b;
    nz = nz_;
    ntx = ntx_;
    ty = ty_;
    load();
  }
  __device__ void load() {
    if (t < t1) {
      const int64_t ct = t / nz;
      z0 = (int)(t % nz);
      z1 = (int)((int64_t)nz < z0 + (t1 - t) ? (int64_t)nz : z0 + (t1 - t));
      k = 0;
      kn = z1 - z0 + 2;
      x0 = (int)(ct % ntx) * kTX;
      y0 = (int)(ct / ntx) * ty;
    }
  }
  __device__ bool more() const { return t < t1; }
  __device__ int plane() const { return z0 - 1 + k; }
  __device__ void next() {
    if (++k == kn) {
      t += z1 - z0;
      load();
    }
  }
};

template <typename T>
__device__ __forceinline__ void ld4s(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
}

// Four stored faces (F = T, or bf16 widened exactly to float).
template <typename F, typename T>
__device__ __forceinline__ void ld4f(const F* p, T (&v)[4]) {
  if constexpr (sizeof(F) == 2) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(q.x << 16);
    v[1] = __uint_as_float(q.x & 0xffff0000u);
    v[2] = __uint_as_float(q.y << 16);
    v[3] = __uint_as_float(q.y & 0xffff0000u);
  } else {
    ld4s(reinterpret_cast<const T*>(p), v);
  }
}

template <typename T>
__device__ __forceinline__ void st4s(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

__device__ __forceinline__ void ld4i(const uint16_t* p, int (&v)[4]) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  v[0] = (int)(q.x & 0xffffu); v[1] = (int)(q.x >> 16); v[2] = (int)(q.y & 0xffffu); v[3] = (int)(q.y >> 16);
}

// Ring state: item i of the CTA's load sequence lives in slot i % S and
// completes phase (i / S) & 1 of that slot's mbarrier.
template <int S>
struct Ring {
  unsigned char* slots;
  uint64_t* full;
  size_t slot_bytes;
  unsigned long long timeout_ns;
  __device__ unsigned char* slot(uint64_t i) const { return slots + (i % S) * slot_bytes; }
  __device__ bool wait(uint64_t i) const {
    return mbar_wait_bounded(full + (i % S), (unsigned)((i / S) & 1ull), timeout_ns);
  }
};

// After a failed wait: record the timeout and let the copies already issued
// land (each wait bounded) before the CTA leaves, so no TMA write targets
// shared memory of a finished CTA.
template <int S>
__device__ void ring_drain(const Ring<S>& rg, const SyncArgs& sy, uint64_t from, uint64_t to) {
  if (threadIdx.x == 0) {
    atomicCAS(sy.status, 0, (int)SLD_ERR_TIMEOUT);
    for (uint64_t i = from; i < to; ++i) rg.wait(i);
  }
  __syncthreads();
}

// Loads of one plane item into its ring slot (one thread): arm the slot's
// mbarrier with the plane's byte count, then issue every box.
template <typename T, typename F, int TY, int S, bool IS_A>
__device__ __forceinline__ void issue(const Ring<S>& rg, const Maps& mp, uint64_t item, int x0, int y0, int pz,
                                      int pbuf) {
  using C = TCfg<T, F, TY>;
  const unsigned si = (unsigned)(item % S);
  unsigned char* st = rg.slots + (size_t)si * rg.slot_bytes;
  uint64_t* bar = rg.full + si;
  if constexpr (IS_A) {
    mbar_expect_tx(bar, C::TX_A);
    tma_load_3d(st + C::A_ZB, &mp.zb_h, bar, x0 - C::H, y0 - 1, pz);
    tma_load_3d(st + C::A_PO, &mp.p_h[pbuf], bar, x0 - C::H, y0 - 1, pz);
    tma_load_3d(st + C::A_FX, &mp.fx, bar, x0 - C::HF, y0, pz);
    tma_load_3d(st + C::A_FY, &mp.fy, bar, x0, y0 - 1, pz);
    tma_load_3d(st + C::A_FZ, &mp.fz, bar, x0, y0, pz);
    tma_load_3d(st + C::A_LB, &mp.lb_o, bar, x0, y0, pz);
    if constexpr (C::kDiag) tma_load_3d(st + C::A_DG, &mp.dg_o, bar, x0, y0, pz);
  } else {
    mbar_expect_tx(bar, C::TX_B);
    tma_load_3d(st + C::B_P, &mp.p_h[pbuf], bar, x0 - C::H, y0 - 1, pz);
    tma_load_3d(st + C::B_LB, &mp.lb_h, bar, x0 - C::HL, y0 - 1, pz);
    tma_load_3d(st + C::B_FX, &mp.fx, bar, x0 - C::HF, y0, pz);
    tma_load_3d(st + C::B_FY, &mp.fy, bar, x0, y0 - 1, pz);
    tma_load_3d(st + C::B_FZ, &mp.fz, bar, x0, y0, pz);
    if constexpr (C::kOwnRing) {
      tma_load_3d(st + C::B_ZO, &mp.zb_o, bar, x0, y0, pz);
      tma_load_3d(st + C::B_XO, &mp.xh_o, bar, x0, y0, pz);
    }
    if constexpr (C::kDiag) {
      tma_load_3d(st + C::B_DG, &mp.dg_o, bar, x0, y0, pz);
      tma_load_3d(st + C::B_IDG, &mp.idg_o, bar, x0, y0, pz);
    }
    if constexpr (C::kScale) tma_load_3d(st + C::B_SC, &mp.sc_o, bar, x0, y0, pz);
  }
}

// One sweep (A or B) over the CTA's plane tiles.  `gitem` is the CTA's running
// item count (identical in all threads), continued across sweeps.
// LRN: extra dense deflation columns; sweep A adds W_L^T p (= Z_L^T A p) to
// the coarse sums, sweep B subtracts W_L y_L from w (A Z y = A Z_lab y_lab +
// W_L y_L), W_L = A Z_L read per own cell from global memory.
template <typename T>
__device__ __forceinline__ void ld_wl(const T* __restrict__ p, T (&w)[kMaxL]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(p)), q1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    w[0] = q0.x; w[1] = q0.y; w[2] = q0.z; w[3] = q0.w; w[4] = q1.x; w[5] = q1.y; w[6] = q1.z; w[7] = q1.w;
  } else {
#pragma unroll
    for (int h = 0; h < kMaxL / 2; ++h) {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p) + h);
      w[2 * h] = q.x;
      w[2 * h + 1] = q.y;
    }
  }
}

template <typename T, typename F, int TY, int S, bool WACC, bool IS_A, bool LRN>
__device__ bool sweep_tma(const SolveArgs& a, const Maps& mp, const Ring<S>& rg, uint64_t& gitem, int ntx,
                          double* sacc, const T* Y, double* red, double* lsum, int pbuf, T* pnew, T coef,
                          double* part_row) {
  using C = TCfg<T, F, TY>;
  const Geo& g = a.g;
  const int d = a.d;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid >> 4, c4 = tid & 15;
  T* zbw = static_cast<T*>(a.z);
  T* xhw = static_cast<T*>(a.xh);
  if constexpr (IS_A) {
    for (int k = tid; k < C::kAcc * d; k += blockDim.x) sacc[k] = 0.0;
  }
  const int tr = team_rank(a.sy);
  int64_t t0, t1;
  tile_range(a, tr, &t0, &t1);
  const uint64_t first = gitem;
  uint64_t released = gitem;  // items below this are free
  uint64_t issued = gitem;    // thread 0 only
  Walk pw;
  // Global data read by this sweep's TMA loads was written before the last
  // grid barrier (each sweep and refinement step ends with a proxy fence
  // before it); one fence here orders this thread's own earlier writes.  No
  // fence per refill: it would wait for the thread's in-flight stores of the
  // plane just computed, which no TMA load of this sweep reads.
  if (tid == 0) fence_proxy_async();
  auto refill = [&]() {
    if (tid == 0) {
      while (pw.more() && issued < released + S) {
        issue<T, F, TY, S, IS_A>(rg, mp, issued, pw.x0, pw.y0, pw.plane(), pbuf);
        ++issued;
        pw.next();
      }
    }
  };
  if (tid == 0) pw.begin(t0, t1, g.nz, ntx, TY);
  __syncthreads();
  refill();
  uint64_t item = gitem;
  LabelAcc<T, true> la;  // per-warp rows (shared or global): deterministic
  la.init(a.lab_L);
  T acc1 = T(0), acc2 = T(0);
  double dacc1 = 0.0, dacc2 = 0.0;
  bool ok = true;
  const T* WL = static_cast<const T*>(a.WLi);
  T sl[LRN ? kMaxL : 1] = {};  // sweep A: W_L^T p over the current segment, then
                               // per warp into lsum[warp][j] (fixed order)
  T yl[LRN ? kMaxL : 1] = {};  // sweep B: y of the extra columns
  if constexpr (LRN && IS_A) {
    for (int k = tid; k < C::kAcc * kMaxL; k += blockDim.x) lsum[k] = 0.0;
  }
  if constexpr (LRN && !IS_A) {
#pragma unroll
    for (int j = 0; j < kMaxL; ++j) yl[j] = j < a.kL ? Y[a.d + j] : T(0);
  }
  // offsets of this thread's cells in the boxes
  const int hi = (r + 1) * C::WH + C::H + 4 * c4;   // vector halo box
  const int hl = (r + 1) * C::WL + C::HL + 4 * c4;  // label halo box
  const int ox = r * C::WF + C::HF + 4 * c4;        // Fx box
  const int oy = (r + 1) * kTX + 4 * c4;            // Fy box (own row)
  const int oo = r * kTX + 4 * c4;                  // own boxes
  // FP64 form (bound by FP64 arithmetic): the stencil operand of a plane
  // (sweep A: z + coef p_old; sweep B: p - y[label]) is formed once per cell
  // and written over the plane's first vector box in its ring slot
  // ("combined"): each thread its own cells, and the cells of the rows below
  // and above the tile and of the columns left and right of it (2 kTX + 2 TY,
  // the halo the stencil reads) spread over the threads.  Neighbours then are
  // plain loads instead of 3.5 recomputations per cell.  The generic stores
  // precede a later TMA refill of the slot: each writing thread fences the
  // async proxy.  (The FP32 and BF16 forms recompute: there the stores and
  // fences cost more than the FP32 operations they save, 173 vs 169 ms.)
  constexpr bool kCmb = C::kDiag;
  constexpr int kNH = 2 * kTX + 2 * TY;
  constexpr size_t oCmb = IS_A ? C::A_ZB : C::B_P;  // combined values overwrite this box
  auto combine_halo = [&](unsigned char* st) {
    T* V = reinterpret_cast<T*>(st + oCmb);
    for (int e = tid; e < kNH; e += blockDim.x) {
      int row, x;  // box row (0 = the row below the tile), tile-relative x (-1 .. kTX)
      if (e < kTX) { row = 0; x = e; }
      else if (e < 2 * kTX) { row = TY + 1; x = e - kTX; }
      else if (e < 2 * kTX + TY) { row = e - 2 * kTX + 1; x = -1; }
      else { row = e - 2 * kTX - TY + 1; x = kTX; }
      const int bo = row * C::WH + C::H + x;
      if constexpr (IS_A) {
        V[bo] = V[bo] + coef * reinterpret_cast<const T*>(st + C::A_PO)[bo];
      } else {
        V[bo] = V[bo] - Y[reinterpret_cast<const uint16_t*>(st + C::B_LB)[row * C::WL + C::HL + x]];
      }
    }
  };
  for (int64_t t = t0; t < t1;) {
    const int64_t ct = t / g.nz;
    const int z0 = (int)(t % g.nz);
    const int z1 = (int)((int64_t)g.nz < z0 + (t1 - t) ? (int64_t)g.nz : z0 + (t1 - t));
    t += z1 - z0;
    const int x0 = (int)(ct % ntx) * kTX, y0 = (int)(ct / ntx) * TY;
    const int xl = x0 + 4 * c4, y = y0 + r;
    const int nv = (y < g.ny) ? max(0, min(4, g.nx - xl)) : 0;
    bool dxc[4], dxm[4], dxp[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      dxc[c] = dir_axis(xl + c, g.nx, g.dlo_x, g.dhi_x);
      dxm[c] = dir_axis(xl + c - 1, g.nx, g.dlo_x, g.dhi_x);
      dxp[c] = dir_axis(xl + c + 1, g.nx, g.dlo_x, g.dhi_x);
    }
    const bool dyc = dir_axis(y, g.ny, g.dlo_y, g.dhi_y);
    const bool dym = dir_axis(y - 1, g.ny, g.dlo_y, g.dhi_y);
    const bool dyp = dir_axis(y + 1, g.ny, g.dlo_y, g.dhi_y);
    // z-1 (previous), z (current) values of this thread's cells
    T vm[4], vc[4], pcur[4], tzm[4];
    // prologue: plane z0-1 (its own values and Fz), then plane z0
    ok = rg.wait(item) && ok;
    {
      const unsigned char* st = rg.slot(item);
      if constexpr (IS_A) {
        T zv[4], po[4];
        ld4s(reinterpret_cast<const T*>(st + C::A_ZB) + hi, zv);
        ld4s(reinterpret_cast<const T*>(st + C::A_PO) + hi, po);
#pragma unroll
        for (int c = 0; c < 4; ++c) vm[c] = zv[c] + coef * po[c];
        ld4f(reinterpret_cast<const F*>(st + C::A_FZ) + oo, tzm);
      } else {
        T pv[4];
        int lb[4];
        ld4s(reinterpret_cast<const T*>(st + C::B_P) + hi, pv);
        ld4i(reinterpret_cast<const uint16_t*>(st + C::B_LB) + hl, lb);
#pragma unroll
        for (int c = 0; c < 4; ++c) vm[c] = pv[c] - Y[lb[c]];
        ld4f(reinterpret_cast<const F*>(st + C::B_FZ) + oo, tzm);
      }
    }
    if (!__syncthreads_and(ok)) { ring_drain(rg, a.sy, released, issued); return false; }
    released = item + 1;
    ++item;
    refill();
    ok = rg.wait(item) && ok;
    {
      const unsigned char* st = rg.slot(item);
      if constexpr (IS_A) {
        T zv[4], po[4];
        ld4s(reinterpret_cast<const T*>(st + C::A_ZB) + hi, zv);
        ld4s(reinterpret_cast<const T*>(st + C::A_PO) + hi, po);
#pragma unroll
        for (int c = 0; c < 4; ++c) vc[c] = zv[c] + coef * po[c];
      } else {
        int lb[4];
        ld4s(reinterpret_cast<const T*>(st + C::B_P) + hi, pcur);
        ld4i(reinterpret_cast<const uint16_t*>(st + C::B_LB) + hl, lb);
#pragma unroll
        for (int c = 0; c < 4; ++c) vc[c] = pcur[c] - Y[lb[c]];
      }
      if constexpr (kCmb) {
        unsigned char* stw = rg.slot(item);
        st4s(reinterpret_cast<T*>(stw + oCmb) + hi, vc);
        combine_halo(stw);
        fence_proxy_async_smem();
      }
    }
    if constexpr (kCmb) {
      if (!__syncthreads_and(ok)) { ring_drain(rg, a.sy, released, issued); return false; }
    }
    for (int z = z0; z < z1; ++z) {
      const uint64_t ic = item, in = item + 1;
      ok = rg.wait(in) && ok;
      const unsigned char* sc = rg.slot(ic);
      const unsigned char* sn = rg.slot(in);
      // plane z+1: own values;  plane z: in-plane neighbours, faces, labels
      T vn[4], pnx[4], ym[4], yp[4], left, right;
      T fx[4], fy[4], fz[4], fym[4], fxl, dg[4] = {}, idg[4] = {};
      int lb[4];
      const T* Vc = reinterpret_cast<const T*>(sc + oCmb);  // plane z, combined
      T* Vn = reinterpret_cast<T*>(const_cast<unsigned char*>(sn) + oCmb);
      if constexpr (IS_A) {
        {
          T zv[4], po[4];
          ld4s(reinterpret_cast<const T*>(sn + C::A_ZB) + hi, zv);
          ld4s(reinterpret_cast<const T*>(sn + C::A_PO) + hi, po);
#pragma unroll
          for (int c = 0; c < 4; ++c) vn[c] = zv[c] + coef * po[c];
        }
        if constexpr (!kCmb) {
          const T* ZBc = reinterpret_cast<const T*>(sc + C::A_ZB);
          const T* POc = reinterpret_cast<const T*>(sc + C::A_PO);
          T z1v[4], p1v[4], z2v[4], p2v[4];
          ld4s(ZBc + hi - C::WH, z1v);
          ld4s(POc + hi - C::WH, p1v);
          ld4s(ZBc + hi + C::WH, z2v);
          ld4s(POc + hi + C::WH, p2v);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            ym[c] = z1v[c] + coef * p1v[c];
            yp[c] = z2v[c] + coef * p2v[c];
          }
          left = ZBc[hi - 1] + coef * POc[hi - 1];
          right = ZBc[hi + 4] + coef * POc[hi + 4];
        }
        ld4f(reinterpret_cast<const F*>(sc + C::A_FX) + ox, fx);
        fxl = (T)reinterpret_cast<const F*>(sc + C::A_FX)[ox - 1];
        ld4f(reinterpret_cast<const F*>(sc + C::A_FY) + oy, fy);
        ld4f(reinterpret_cast<const F*>(sc + C::A_FY) + oy - kTX, fym);
        ld4f(reinterpret_cast<const F*>(sc + C::A_FZ) + oo, fz);
        ld4i(reinterpret_cast<const uint16_t*>(sc + C::A_LB) + oo, lb);
        if constexpr (C::kDiag) ld4s(reinterpret_cast<const T*>(sc + C::A_DG) + oo, dg);
      } else {
        {
          int ln[4];
          ld4s(reinterpret_cast<const T*>(sn + C::B_P) + hi, pnx);
          ld4i(reinterpret_cast<const uint16_t*>(sn + C::B_LB) + hl, ln);
#pragma unroll
          for (int c = 0; c < 4; ++c) vn[c] = pnx[c] - Y[ln[c]];
        }
        if constexpr (!kCmb) {
          const T* Pc = reinterpret_cast<const T*>(sc + C::B_P);
          const uint16_t* Lc = reinterpret_cast<const uint16_t*>(sc + C::B_LB);
          T p1v[4], p2v[4];
          int l1[4], l2[4];
          ld4s(Pc + hi - C::WH, p1v);
          ld4i(Lc + hl - C::WL, l1);
          ld4s(Pc + hi + C::WH, p2v);
          ld4i(Lc + hl + C::WL, l2);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            ym[c] = p1v[c] - Y[l1[c]];
            yp[c] = p2v[c] - Y[l2[c]];
          }
          left = Pc[hi - 1] - Y[Lc[hl - 1]];
          right = Pc[hi + 4] - Y[Lc[hl + 4]];
        }
        ld4f(reinterpret_cast<const F*>(sc + C::B_FX) + ox, fx);
        fxl = (T)reinterpret_cast<const F*>(sc + C::B_FX)[ox - 1];
        ld4f(reinterpret_cast<const F*>(sc + C::B_FY) + oy, fy);
        ld4f(reinterpret_cast<const F*>(sc + C::B_FY) + oy - kTX, fym);
        ld4f(reinterpret_cast<const F*>(sc + C::B_FZ) + oo, fz);
        if constexpr (C::kDiag) {
          ld4s(reinterpret_cast<const T*>(sc + C::B_DG) + oo, dg);
          ld4s(reinterpret_cast<const T*>(sc + C::B_IDG) + oo, idg);
        }
      }
      if constexpr (kCmb) {
        // in-plane neighbours from the combined values of plane z
        ld4s(Vc + hi - C::WH, ym);
        ld4s(Vc + hi + C::WH, yp);
        left = Vc[hi - 1];
        right = Vc[hi + 4];
        // plane z+1 combined: own cells; the halo only if it becomes a current plane
        st4s(Vn + hi, vn);
        if (z + 1 < z1) combine_halo(reinterpret_cast<unsigned char*>(Vn) - oCmb);
        fence_proxy_async_smem();
      }
      const bool dzc = dir_axis(z, g.nz, g.dlo_z, g.dhi_z);
      const bool dzm = dir_axis(z - 1, g.nz, g.dlo_z, g.dhi_z);
      const bool dzp = dir_axis(z + 1, g.nz, g.dlo_z, g.dhi_z);
      // this thread's cells in the inner vectors (rows a.vp long; extra
      // deflation columns need a.vp == nx)
      const int64_t iz = (int64_t)z * a.vpxy + (int64_t)y * a.vp + xl;
      if constexpr (IS_A) {
        T av[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool valid = c < nv;
          const T u = vc[c];
          const T xm = (c > 0) ? vc[(c > 0) ? c - 1 : 0] : left;
          const T xp = (c < 3) ? vc[(c < 3) ? c + 1 : 0] : right;
          const T fxm = (c > 0) ? fx[(c > 0) ? c - 1 : 0] : fxl;
          const T v = stencil<T>(dxc[c] || dyc || dzc, u, dg[c], fxm, xm, !dxm[c], fx[c], xp, !dxp[c], fym[c],
                                 ym[c], !dym, fy[c], yp[c], !dyp, tzm[c], vm[c], !dzm, fz[c], vn[c], !dzp);
          av[c] = v;
          if (valid) acc1 += u * v;
          if constexpr (LRN) {
            if (valid) {
              T w[kMaxL];
              ld_wl<T>(WL + (iz + c) * kMaxL, w);
#pragma unroll
              for (int j = 0; j < kMaxL; ++j) sl[j] += w[j] * u;
            }
          }
        }
        la.add4(nv, lb, av, sacc, d, warp);
        st_cells<T, 4>(pnew, iz, nv, vc);
      } else {
        T zo[4], xo[4], zn[4], xn[4], sci[4] = {};
        if constexpr (C::kScale) ld4s(reinterpret_cast<const T*>(sc + C::B_SC) + oo, sci);
        if constexpr (C::kOwnRing) {
          ld4s(reinterpret_cast<const T*>(sc + C::B_ZO) + oo, zo);
          ld4s(reinterpret_cast<const T*>(sc + C::B_XO) + oo, xo);
        } else {
          ld_cells<T, 4, false>(zbw, iz, nv, zo);
          ld_cells<T, 4, false>(xhw, iz, nv, xo);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const T u = vc[c];
          const T xm = (c > 0) ? vc[(c > 0) ? c - 1 : 0] : left;
          const T xp = (c < 3) ? vc[(c < 3) ? c + 1 : 0] : right;
          const T fxm = (c > 0) ? fx[(c > 0) ? c - 1 : 0] : fxl;
          const bool dirc = dxc[c] || dyc || dzc;
          T dgi;
          if constexpr (C::kDiag) dgi = dg[c];
          else dgi = dirc ? T(1) : (((((tzm[c] + fym[c]) + fxm) + fx[c]) + fy[c]) + fz[c]);
          T w = stencil<T>(dirc, u, dgi, fxm, xm, !dxm[c], fx[c], xp, !dxp[c], fym[c], ym[c], !dym, fy[c],
                           yp[c], !dyp, tzm[c], vm[c], !dzm, fz[c], vn[c], !dzp);
          if constexpr (LRN) {
            if (c < nv) {
              T wl[kMaxL];
              ld_wl<T>(WL + (iz + c) * kMaxL, wl);
              T corr = T(0);
#pragma unroll
              for (int j = 0; j < kMaxL; ++j) corr += wl[j] * yl[j];
              w -= corr;
            }
          }
          const T rr = dgi * zo[c] - coef * w;
          T znew;
          if constexpr (C::kDiag) znew = rr * idg[c];
          else if constexpr (C::kScale) znew = rr * sci[c];  // FP32 per-cell inverse diagonal
          else znew = __fdividef(rr, dgi);  // FP32 inner: 2-ulp division
          zn[c] = znew;
          xn[c] = xo[c] + coef * pcur[c];
          if (c < nv) {
            acc1 += rr * znew;
            acc2 += rr * rr;
          }
        }
        st_cells<T, 4>(zbw, iz, nv, zn);
        st_cells<T, 4>(xhw, iz, nv, xn);
#pragma unroll
        for (int c = 0; c < 4; ++c) pcur[c] = pnx[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        vm[c] = vc[c];
        vc[c] = vn[c];
        tzm[c] = fz[c];
      }
      if (!__syncthreads_and(ok)) { ring_drain(rg, a.sy, released, issued); return false; }
      released = ic + 1;
      item = in;
      refill();
    }
    // the segment's last item (plane z1) was read before the last barrier
    released = item + 1;
    ++item;
    refill();
    dacc1 += (double)acc1;
    dacc2 += (double)acc2;
    acc1 = acc2 = T(0);
    if constexpr (LRN && IS_A) {
#pragma unroll
      for (int j = 0; j < kMaxL; ++j) {
        const double t = warp_sum((double)sl[j]);
        if ((tid & 31) == 0) lsum[warp * kMaxL + j] += t;
        sl[j] = T(0);
      }
    }
  }
  gitem = item;
  (void)first;
  fence_proxy_async();  // this sweep's global stores before later TMA reads
  if constexpr (IS_A) {
    la.flush(sacc, d, warp);
    const double gsum = block_sum(dacc1, red);
    for (int k = tid; k < d; k += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sacc[w * d + k];  // warp order: deterministic
      part_row[(int64_t)(k) * a.pstride] = s;
    }
    if (tid == 0) part_row[(int64_t)(a.dk + 0) * a.pstride] = gsum;
    if constexpr (LRN) {
      // block_sum above ended with a CTA barrier: every lsum row is final
      for (int j = tid; j < a.kL; j += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += lsum[w * kMaxL + j];
        part_row[(int64_t)(d + j) * a.pstride] = t;
      }
    }
  } else {
    const double s1 = block_sum(dacc1, red);
    const double s2 = block_sum(dacc2, red);
    if (tid == 0) {
      part_row[(int64_t)(a.dk + 1) * a.pstride] = s1;
      part_row[(int64_t)(a.dk + 2) * a.pstride] = s2;
    }
  }
  return true;
}

// CTAs per SM the register allocation must allow: FP32 forms up to 64K
// registers per SM at 128 per thread; the FP64 form two CTAs (its ring
// slots fit two per SM), i.e. up to 255 registers per thread.
template <typename T, int TY>
constexpr int tma_min_ctas() { return sizeof(T) == 8 ? 2 : (512 / (16 * TY) > 1 ? 512 / (16 * TY) : 1); }

template <typename T, typename F, int TY, int S, bool WACC>
__host__ __device__ constexpr size_t tma_smem_bytes(int d, int dk) {
  using C = TCfg<T, F, TY>;
  size_t b = C::SLOT * S;
  b += 8 * S;
  b = (b + 15) / 16 * 16;
  b += sizeof(double) * (size_t)(WACC ? C::kAcc : 0) * d;
  b += sizeof(double) * dk;
  b += sizeof(T) * dk;
  b = (b + 15) / 16 * 16;
  b += sizeof(double) * 64;
  b += sizeof(double) * C::kAcc * kMaxL;
  return b;
}

template <typename T, typename F, int TY, int S, bool WACC, bool LRN>
__device__ __forceinline__ void tma_body(const SolveArgs& a, const Maps& mp, int ntx, unsigned char* smem_raw) {
  using C = TCfg<T, F, TY>;
  Ring<S> rg;
  rg.slots = smem_raw;
  rg.slot_bytes = C::SLOT;
  rg.timeout_ns = a.sy.timeout_ns;
  size_t o = C::SLOT * S;
  rg.full = reinterpret_cast<uint64_t*>(smem_raw + o);
  o += 8 * S;
  o = (o + 15) / 16 * 16;
  double* acc = WACC ? reinterpret_cast<double*>(smem_raw + o) : a.gacc + (int64_t)blockIdx.x * a.gacc_stride;
  o += sizeof(double) * (size_t)(WACC ? C::kAcc : 0) * a.d;
  double* Yd = reinterpret_cast<double*>(smem_raw + o);
  o += sizeof(double) * a.dk;
  T* Y = reinterpret_cast<T*>(smem_raw + o);
  o += sizeof(T) * a.dk;
  o = (o + 15) / 16 * 16;
  double* red = reinterpret_cast<double*>(smem_raw + o);
  double* lsum = red + 64;
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; ++k) mbar_init(rg.full + k, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < (int)(sizeof(Maps) / sizeof(CUtensorMap)))  // descriptors into the TMA unit's cache
    prefetch_tensormap(reinterpret_cast<const CUtensorMap*>(&mp) + threadIdx.x);
  __syncthreads();
  T* pb[2] = {static_cast<T*>(a.p0), static_cast<T*>(a.p1)};
  uint64_t gitem = 0;
  solve_body<T, WACC>(
      a, acc, Yd, Y, red,
      [&](int po, T beta, double* part) {
        return sweep_tma<T, F, TY, S, WACC, true, LRN>(a, mp, rg, gitem, ntx, acc, Y, red, lsum, po, pb[po ^ 1],
                                                       beta, part);
      },
      [&](int pn, T alpha, double* part) {
        return sweep_tma<T, F, TY, S, WACC, false, LRN>(a, mp, rg, gitem, ntx, acc, Y, red, lsum, pn, nullptr,
                                                        alpha, part);
      });
}

template <typename T, typename F, int TY, int S, bool WACC, bool LRN>
__global__ void __launch_bounds__(16 * TY, tma_min_ctas<T, TY>()) k_solve_tma(SolveArgs a, const __grid_constant__ Maps mp, int ntx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  tma_body<T, F, TY, S, WACC, LRN>(a, mp, ntx, smem_raw);
}

// Batched solve: CTA c works on system cta_sys[c] with the team of CTAs the
// host assigned to it.  Its arguments are copied into shared memory (at
// args_off, past the solve's own layout); its tensor maps stay in global
// memory, where the TMA unit reads them.
template <typename T, typename F, int TY, int S, bool WACC>
__global__ void __launch_bounds__(16 * TY, tma_min_ctas<T, TY>()) k_solve_tma_batch(const SolveArgs* __restrict__ all,
                                                           const Maps* __restrict__ maps,
                                                           const int* __restrict__ cta_sys, unsigned args_off) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SolveArgs* as = reinterpret_cast<SolveArgs*>(smem_raw + args_off);
  const int k = cta_sys[blockIdx.x];
  if (threadIdx.x == 0) *as = all[k];
  __syncthreads();
  tma_body<T, F, TY, S, WACC, false>(*as, maps[k], as->ntx, smem_raw);
}

// Batched solve with every system's arguments in one kernel parameter (up to
// kBatchParamMax systems): a CTA reads its system's arguments from the
// constant bank like the single solve does, instead of from a shared-memory
// copy that the compiler must reload after every shared-memory store.
constexpr int kBatchParamMax = 72;  // 72 x sizeof(SolveArgs) fits the 32 KB parameter space
struct BatchParam {
  SolveArgs a[kBatchParamMax];
};

template <typename T, typename F, int TY, int S, bool WACC>
__global__ void __launch_bounds__(16 * TY, tma_min_ctas<T, TY>())
    k_solve_tma_batch_p(const __grid_constant__ BatchParam P, const Maps* __restrict__ maps,
                        const int* __restrict__ cta_sys) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int k = cta_sys[blockIdx.x];
  const SolveArgs& a = P.a[k];
  tma_body<T, F, TY, S, WACC, false>(a, maps[k], a.ntx, smem_raw);
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and the launch.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A map over nx x ny x nz cells stored with rows of `pitch` cells.
bool make_map(CUtensorMap* m, CUtensorMapDataType dt, size_t es, const void* ptr, const Geo& g, int pitch, int bx,
              int by) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * g.ny * es};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, typename F, int TY>
bool build_maps(const SolveArgs& a, Maps* mp) {
  using C = TCfg<T, F, TY>;
  const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUtensorMapDataType df = sizeof(F) == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : dt;
  const size_t es = sizeof(T), ef = sizeof(F);
  const Geo& g = a.g;
  bool ok = true;
  ok = ok && make_map(&mp->zb_h, dt, es, a.z, g, a.vp, C::WH, TY + 2);
  ok = ok && make_map(&mp->p_h[0], dt, es, a.p0, g, a.vp, C::WH, TY + 2);
  ok = ok && make_map(&mp->p_h[1], dt, es, a.p1, g, a.vp, C::WH, TY + 2);
  ok = ok && make_map(&mp->fx, df, ef, a.Txi, g, a.vp, C::WF, TY);
  ok = ok && make_map(&mp->fy, df, ef, a.Tyi, g, a.vp, kTX, TY + 1);
  ok = ok && make_map(&mp->fz, df, ef, a.Tzi, g, a.vp, kTX, TY);
  ok = ok && make_map(&mp->lb_o, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, a.label16, g, a.vp, kTX, TY);
  ok = ok && make_map(&mp->lb_h, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, a.label16, g, a.vp, C::WL, TY + 2);
  ok = ok && make_map(&mp->zb_o, dt, es, a.z, g, a.vp, kTX, TY);
  ok = ok && make_map(&mp->xh_o, dt, es, a.xh, g, a.vp, kTX, TY);
  if (C::kDiag) {
    ok = ok && make_map(&mp->dg_o, dt, es, a.diag64, g, a.vp, kTX, TY);
    ok = ok && make_map(&mp->idg_o, dt, es, a.invdiag64, g, a.vp, kTX, TY);
  } else {
    mp->dg_o = mp->zb_o;
    mp->idg_o = mp->zb_o;
  }
  if (C::kScale) ok = ok && make_map(&mp->sc_o, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.invdi, g, a.vp, kTX, TY);
  else mp->sc_o = mp->zb_o;
  return ok;
}

template <typename T, typename F, int TY, int S, bool WACC, bool LRN>
int launch_tma(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg) {
  Maps mp;
  if (!build_maps<T, F, TY>(a, &mp)) {
    *msg = "tensor map creation failed";
    return SLD_ERR_CUDA;
  }
  int ntx = (a.g.nx + kTX - 1) / kTX;
  const int nty = (a.g.ny + TY - 1) / TY;
  a.ntiles = (int64_t)ntx * nty * a.g.nz;
  a.ntx = ntx;
  a.nty = nty;
  const size_t smem = tma_smem_bytes<T, F, TY, S, WACC>(a.d, a.dk);
  auto kern = k_solve_tma<T, F, TY, S, WACC, LRN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    *msg = std::string("tma kernel attribute: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 16 * TY, smem);
  if (per < 1) {
    *msg = "tma solve kernel does not fit on an SM";
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
  void* args[] = {&a, &mp, &ntx};
  cudaEventRecord(s->ev0, s->stream);
  e = cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(16 * TY), args, smem, s->stream);
  cudaEventRecord(s->ev1, s->stream);
  if (e != cudaSuccess) {
    *msg = std::string("tma solve launch: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  e = cudaEventSynchronize(s->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    *msg = std::string("tma solve kernel: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  cudaEventElapsedTime(ms, s->ev0, s->ev1);
  return SLD_OK;
}

}  // namespace
}  // namespace sld
