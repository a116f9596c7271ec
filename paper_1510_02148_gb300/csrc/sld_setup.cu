// sld_setup.cu -- setup kernels of libsld: two-point-flux assembly (a1),
// subdomain-levelset labels (a2), E = Z^T A Z with its Cholesky factor and
// inverse (a3), FP32 coefficient copies, and the FP64 diagnostics
// (y = A x, Z^T v, residual norms).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "sld_device.cuh"
#include "sld_internal.h"

namespace sld {

namespace {

struct BcVals {
  int type[6];
  double value[6];
};

__device__ __forceinline__ int dirichlet_face(const Geo& g, const BcVals& bc, int ix, int iy, int iz) {
  if (bc.type[0] && ix == 0) return 0;
  if (bc.type[1] && ix == g.nx - 1) return 1;
  if (bc.type[2] && iy == 0) return 2;
  if (bc.type[3] && iy == g.ny - 1) return 3;
  if (bc.type[4] && iz == 0) return 4;
  if (bc.type[5] && iz == g.nz - 1) return 5;
  return -1;
}

// Harmonic-mean transmissibility of the face between cells with K = a, b
// (unit cells): (2 a b) / (a + b), evaluated in exactly this order.  The
// expression has no multiply-add pair, so no contraction can change it.
__device__ __forceinline__ double harmonic(double a, double b) { return (2.0 * a * b) / (a + b); }

// a1: per cell, the three forward faces, the diagonal, its inverse and the
// right-hand side with the Dirichlet couplings moved into it.
__global__ void k_assemble(Geo g, BcVals bc, const double* __restrict__ K, const double* __restrict__ q,
                           double* __restrict__ Tx, double* __restrict__ Ty, double* __restrict__ Tz,
                           double* __restrict__ diag, double* __restrict__ invdiag, double* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int ix = (int)(i % g.nx);
  const int iy = (int)((i / g.nx) % g.ny);
  const int iz = (int)(i / g.nxy);
  const double Ki = K[i];
  const double tpx = (ix + 1 < g.nx) ? harmonic(Ki, K[i + 1]) : 0.0;
  const double tpy = (iy + 1 < g.ny) ? harmonic(Ki, K[i + g.nx]) : 0.0;
  const double tpz = (iz + 1 < g.nz) ? harmonic(Ki, K[i + g.nxy]) : 0.0;
  Tx[i] = tpx;
  Ty[i] = tpy;
  Tz[i] = tpz;
  const int fi = dirichlet_face(g, bc, ix, iy, iz);
  if (fi >= 0) {
    diag[i] = 1.0;
    invdiag[i] = 1.0;
    b[i] = bc.value[fi];
    return;
  }
  // faces in the order -z, -y, -x, +x, +y, +z
  const double tmz = (iz > 0) ? harmonic(Ki, K[i - g.nxy]) : 0.0;
  const double tmy = (iy > 0) ? harmonic(Ki, K[i - g.nx]) : 0.0;
  const double tmx = (ix > 0) ? harmonic(Ki, K[i - 1]) : 0.0;
  const double T[6] = {tmz, tmy, tmx, tpx, tpy, tpz};
  const int jx[6] = {ix, ix, ix - 1, ix + 1, ix, ix};
  const int jy[6] = {iy, iy - 1, iy, iy, iy + 1, iy};
  const int jz[6] = {iz - 1, iz, iz, iz, iz, iz + 1};
  double dsum = 0.0;
  double rhs = q ? q[i] : 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    if (jx[m] < 0 || jx[m] >= g.nx || jy[m] < 0 || jy[m] >= g.ny || jz[m] < 0 || jz[m] >= g.nz) continue;
    dsum = __dadd_rn(dsum, T[m]);
    const int fj = dirichlet_face(g, bc, jx[m], jy[m], jz[m]);
    if (fj >= 0) rhs = __dadd_rn(rhs, __dmul_rn(T[m], bc.value[fj]));
  }
  diag[i] = dsum;
  invdiag[i] = 1.0 / dsum;
  b[i] = rhs;
}

struct Thresholds {
  double tau[16];
};

// a2: label = subdomain * L + #{m : K >= tau_m}; integer index arithmetic and
// FP64 compares only, so the result is exact.
__global__ void k_labels(Geo g, int Sx, int Sy, int Sz, Thresholds th, int L, const double* __restrict__ K,
                         int32_t* __restrict__ label) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int64_t ix = i % g.nx, iy = (i / g.nx) % g.ny, iz = i / g.nxy;
  const int64_t sx = ix * Sx / g.nx, sy = iy * Sy / g.ny, sz = iz * Sz / g.nz;
  const double k = K[i];
  int cls = 0;
  for (int m = 0; m < L - 1; ++m) cls += (k >= th.tau[m]) ? 1 : 0;
  label[i] = (int32_t)(((sz * Sy + sy) * Sx + sx) * L + cls);
}

// a3: E = Z^T A Z by faces.  A face inside one label adds nothing; a face
// between free cells with labels k != l adds T to E_kk and E_ll and -T to
// E_kl and E_lk; a face between a free and a Dirichlet cell adds T at the
// free cell's label; a Dirichlet cell adds 1 (its identity row) at its own.
// The diagonal and the label counts are gathered per CTA in shared memory.
__global__ void k_coarse_E(Geo g, BcVals bc, int d, const int32_t* __restrict__ label,
                           const double* __restrict__ Tx, const double* __restrict__ Ty,
                           const double* __restrict__ Tz, double* __restrict__ E,
                           unsigned long long* __restrict__ count, int* __restrict__ bad) {
  extern __shared__ double sm[];
  double* sdiag = sm;
  unsigned* scnt = reinterpret_cast<unsigned*>(sm + d);
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    sdiag[k] = 0.0;
    scnt[k] = 0u;
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    const int li = label[i];
    if (li < 0 || li >= d) {
      atomicExch(bad, 1);
      continue;
    }
    const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.nxy);
    atomicAdd(&scnt[li], 1u);
    const bool di = dirichlet_face(g, bc, ix, iy, iz) >= 0;
    if (di) atomicAdd(&sdiag[li], 1.0);
    const double T[3] = {Tx[i], Ty[i], Tz[i]};
    const int jx[3] = {ix + 1, ix, ix};
    const int jy[3] = {iy, iy + 1, iy};
    const int jz[3] = {iz, iz, iz + 1};
    const int64_t off[3] = {1, g.nx, g.nxy};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (jx[m] >= g.nx || jy[m] >= g.ny || jz[m] >= g.nz) continue;
      const int64_t j = i + off[m];
      const int lj = label[j];
      if (lj < 0 || lj >= d) continue;  // reported by its own cell
      const bool dj = dirichlet_face(g, bc, jx[m], jy[m], jz[m]) >= 0;
      const double t = T[m];
      if (!di && !dj) {
        if (li != lj) {
          atomicAdd(&sdiag[li], t);
          atomicAdd(&sdiag[lj], t);
          atomicAdd(&E[(int64_t)li * d + lj], -t);
          atomicAdd(&E[(int64_t)lj * d + li], -t);
        }
      } else if (!di && dj) {
        atomicAdd(&sdiag[li], t);
      } else if (di && !dj) {
        atomicAdd(&sdiag[lj], t);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    if (sdiag[k] != 0.0) atomicAdd(&E[(int64_t)k * d + k], sdiag[k]);
    if (scnt[k]) atomicAdd(&count[k], (unsigned long long)scnt[k]);
  }
}

// An empty column of Z (no cell carries that label) gets E_kk = 1: the
// column is zero, so this changes neither P nor x.
__global__ void k_pin_empty(int d, const unsigned long long* __restrict__ count, double* __restrict__ E) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d && count[k] == 0) E[(int64_t)k * d + k] = 1.0;
}

// Right-looking FP64 Cholesky E = L L^T on a cooperative grid.  Row i is
// owned by CTA i mod G; step k scales column k (kept in shared memory) and
// updates the owned rows of the trailing lower triangle; one bounded grid
// barrier per column.  A pivot <= 0 (E not SPD) sets SLD_ERR_COARSE_SINGULAR;
// every CTA reads the same pivot, so all of them stop at the same step.
// Pivots k >= rel_from must also exceed rel_tol times the original diagonal
// E0_kk: a column that is (nearly) a combination of the earlier ones fails.
__global__ void k_cholesky(int d, double* __restrict__ A, double* __restrict__ Lm, SyncArgs sy,
                           const double* __restrict__ E0, int rel_from, double rel_tol) {
  extern __shared__ double sc[];
  unsigned epoch = 0;
  const int G = gridDim.x;
  for (int k = 0; k < d; ++k) {
    const double akk = A[(int64_t)k * d + k];
    const bool rel_bad = k >= rel_from && !(akk > rel_tol * E0[(int64_t)k * d + k]);
    if (!(akk > 0.0) || !isfinite(akk) || rel_bad) {
      if (threadIdx.x == 0) atomicCAS(sy.status, 0, (int)SLD_ERR_COARSE_SINGULAR);
      return;
    }
    const double lkk = sqrt(akk);
    const double inv = 1.0 / lkk;
    for (int i = k + 1 + threadIdx.x; i < d; i += blockDim.x) sc[i] = A[(int64_t)i * d + k] * inv;
    __syncthreads();
    if ((k % G) == (int)blockIdx.x && threadIdx.x == 0) Lm[(int64_t)k * d + k] = lkk;
    int i0 = k + 1;
    i0 += ((int)blockIdx.x - i0 % G + G) % G;  // first owned row > k
    for (int i = i0; i < d; i += G) {
      const double li = sc[i];
      if (threadIdx.x == 0) Lm[(int64_t)i * d + k] = li;
      double* Ai = A + (int64_t)i * d;
      for (int j = k + 1 + threadIdx.x; j <= i; j += blockDim.x) Ai[j] -= li * sc[j];
    }
    if (!grid_barrier(sy, epoch)) return;
  }
}

// W = L^{-1}, one warp per column: forward substitution L w = e_c with the
// column kept in shared memory.
__global__ void k_tri_inverse(int d, const double* __restrict__ Lm, double* __restrict__ W) {
  extern __shared__ double sw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  double* w = sw + (int64_t)warp * d;
  for (int c = blockIdx.x * nw + warp; c < d; c += gridDim.x * nw) {
    for (int i = lane; i < d; i += 32) w[i] = 0.0;
    __syncwarp();
    if (lane == 0) w[c] = 1.0 / Lm[(int64_t)c * d + c];
    __syncwarp();
    for (int i = c + 1; i < d; ++i) {
      const double* Li = Lm + (int64_t)i * d;
      double t = 0.0;
      for (int m = c + lane; m < i; m += 32) t += Li[m] * w[m];
      t = warp_sum(t);
      if (lane == 0) w[i] = -t / Li[i];
      __syncwarp();
    }
    for (int i = lane; i < d; i += 32) W[(int64_t)i * d + c] = w[i];
    __syncwarp();
  }
}

// Einv = W^T W (W lower triangular): Einv_ij = sum over m of W_mi W_mj.
__global__ void k_wtw(int d, const double* __restrict__ W, double* __restrict__ Einv) {
  __shared__ double sa[16][17], sb[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  const int m0 = max(blockIdx.y * 16, blockIdx.x * 16) / 16 * 16;
  double acc = 0.0;
  for (int mt = m0; mt < d; mt += 16) {
    const int ma = mt + ty, ia = blockIdx.y * 16 + tx, jb = blockIdx.x * 16 + tx;
    sa[ty][tx] = (ma < d && ia < d) ? W[(int64_t)ma * d + ia] : 0.0;  // sa[m][i]
    sb[ty][tx] = (ma < d && jb < d) ? W[(int64_t)ma * d + jb] : 0.0;  // sb[m][j]
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; ++m) acc += sa[m][ty] * sb[m][tx];
    __syncthreads();
  }
  if (i < d && j < d) Einv[(int64_t)i * d + j] = acc;
}

// ---------------------------------------------------------------------------
// Extra dense deflation vectors Z_L (k <= kMaxL columns appended to the label
// columns, Z = [Z_lab, Z_L]; Section 3.1, Def. 3.1 holds for any full-rank
// Z).  Stored cell-major with kMaxL FP32 slots per cell (zero past k): the
// FP32-rounded values are the vectors deflated with.  W_L = A Z_L in FP64
// (refinement steps, coarse matrix) and rounded to FP32 (inner iterations).
// ---------------------------------------------------------------------------
__global__ void k_learned_pack(int64_t n, int k, const void* __restrict__ src, int f32, float* __restrict__ ZL,
                               int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[kMaxL];
#pragma unroll
  for (int j = 0; j < kMaxL; ++j) {
    float t = 0.0f;
    if (j < k) t = f32 ? static_cast<const float*>(src)[i * k + j] : (float)static_cast<const double*>(src)[i * k + j];
    if (!isfinite(t)) {
      atomicExch(bad, 1);
      t = 0.0f;
    }
    v[j] = t;
  }
  float4* o = reinterpret_cast<float4*>(ZL + i * kMaxL);
  o[0] = make_float4(v[0], v[1], v[2], v[3]);
  o[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// W_L = A Z_L column by column, the operator of k_apply_A.
__global__ void k_learned_W(Geo g, const double* __restrict__ Tx, const double* __restrict__ Ty,
                            const double* __restrict__ Tz, const double* __restrict__ diag,
                            const float* __restrict__ ZL, double* __restrict__ W64, float* __restrict__ W32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.nxy);
  const bool dirc = dir_axis(ix, g.nx, g.dlo_x, g.dhi_x) || dir_axis(iy, g.ny, g.dlo_y, g.dhi_y) ||
                    dir_axis(iz, g.nz, g.dlo_z, g.dhi_z);
  double w[kMaxL];
  const double dg = dirc ? 1.0 : diag[i];
#pragma unroll
  for (int j = 0; j < kMaxL; ++j) w[j] = dg * (double)ZL[i * kMaxL + j];
  if (!dirc) {
    auto sub = [&](int64_t jn, double t) {
#pragma unroll
      for (int j = 0; j < kMaxL; ++j) w[j] -= t * (double)ZL[jn * kMaxL + j];
    };
    if (ix > 0 && !dir_axis(ix - 1, g.nx, g.dlo_x, g.dhi_x)) sub(i - 1, Tx[i - 1]);
    if (ix + 1 < g.nx && !dir_axis(ix + 1, g.nx, g.dlo_x, g.dhi_x)) sub(i + 1, Tx[i]);
    if (iy > 0 && !dir_axis(iy - 1, g.ny, g.dlo_y, g.dhi_y)) sub(i - g.nx, Ty[i - g.nx]);
    if (iy + 1 < g.ny && !dir_axis(iy + 1, g.ny, g.dlo_y, g.dhi_y)) sub(i + g.nx, Ty[i]);
    if (iz > 0 && !dir_axis(iz - 1, g.nz, g.dlo_z, g.dhi_z)) sub(i - g.nxy, Tz[i - g.nxy]);
    if (iz + 1 < g.nz && !dir_axis(iz + 1, g.nz, g.dlo_z, g.dhi_z)) sub(i + g.nxy, Tz[i]);
  }
#pragma unroll
  for (int j = 0; j < kMaxL; ++j) {
    W64[i * kMaxL + j] = w[j];
    W32[i * kMaxL + j] = (float)w[j];
  }
}

// Z_lab^T W_L: ESL[a * kMaxL + j] = sum over cells with label a of W_ij.  A
// warp whose 32 cells share one label adds its warp sum once.
__global__ void k_learned_ESL(int64_t n, const int32_t* __restrict__ label, const double* __restrict__ W64,
                              double* __restrict__ ESL) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nround = (n + stride - 1) / stride;
  const int lane = threadIdx.x & 31;
  for (int64_t r = 0; r < nround; ++r) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < n;
    const int l = ok ? label[i] : -1;
    const int l0 = __shfl_sync(kFull, l, 0);
    const bool uniform = __all_sync(kFull, l == l0) && l0 >= 0;
#pragma unroll
    for (int j = 0; j < kMaxL; ++j) {
      const double v = ok ? W64[i * kMaxL + j] : 0.0;
      if (uniform) {
        const double t = warp_sum(v);
        if (lane == 0) atomicAdd(&ESL[(int64_t)l0 * kMaxL + j], t);
      } else if (ok) {
        atomicAdd(&ESL[(int64_t)l * kMaxL + j], v);
      }
    }
  }
}

// Z_L^T W_L: one CTA per entry (j, m), fixed-order block sum.
__global__ void k_learned_ELL(int64_t n, const float* __restrict__ ZL, const double* __restrict__ W64,
                              double* __restrict__ ELL) {
  __shared__ double red[32];
  const int j = blockIdx.x / kMaxL, m = blockIdx.x % kMaxL;
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += (double)ZL[i * kMaxL + j] * W64[i * kMaxL + m];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
    ELL[j * kMaxL + m] = u;
  }
}

// Efull (D x D, D = d + k) = [[E, ESL], [ESL^T, ELL]] restricted to k columns;
// the label block is E (d x d).  ELL is symmetrised, (ELL + ELL^T) / 2.
__global__ void k_learned_Efull(int d, int k, const double* __restrict__ E, const double* __restrict__ ESL,
                                const double* __restrict__ ELL, double* __restrict__ Ef) {
  const int D = d + k;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)D * D) return;
  const int r = (int)(t / D), c = (int)(t % D);
  double v;
  if (r < d && c < d) v = E[(int64_t)r * d + c];
  else if (r < d) v = ESL[(int64_t)r * kMaxL + (c - d)];
  else if (c < d) v = ESL[(int64_t)c * kMaxL + (r - d)];
  else v = 0.5 * (ELL[(r - d) * kMaxL + (c - d)] + ELL[(c - d) * kMaxL + (r - d)]);
  Ef[t] = v;
}

// BF16 inner operator: each face rounded to nearest BF16, and the FP32
// inverse of the quantized operator's diagonal (the sum of the six rounded
// faces, in the order -z, -y, -x, +x, +y, +z, as the sweeps add them), 1 for
// a Dirichlet cell.  The quantized operator is again a weighted Laplacian with
// the Dirichlet couplings, so it stays symmetric positive definite.
// Cell i = (iz * ny + iy) * nx + ix of the padded-row arrays sits at
// (iz * ny + iy) * nxp + ix.
__device__ __forceinline__ int64_t padded(const Geo& g, int nxp, int64_t i) {
  return i + (i / g.nx) * (int64_t)(nxp - g.nx);
}

__global__ void k_quantize_bf16(Geo g, int nxp, const double* __restrict__ Tx, const double* __restrict__ Ty,
                                const double* __restrict__ Tz, __nv_bfloat16* __restrict__ Tx16,
                                __nv_bfloat16* __restrict__ Ty16, __nv_bfloat16* __restrict__ Tz16,
                                float* __restrict__ invd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.nxy);
  const int64_t ip = padded(g, nxp, i);
  auto q = [](double t) { return __double2bfloat16(t); };
  const __nv_bfloat16 px = q(Tx[i]), py = q(Ty[i]), pz = q(Tz[i]);
  Tx16[ip] = px;
  Ty16[ip] = py;
  Tz16[ip] = pz;
  if (dir_axis(ix, g.nx, g.dlo_x, g.dhi_x) || dir_axis(iy, g.ny, g.dlo_y, g.dhi_y) ||
      dir_axis(iz, g.nz, g.dlo_z, g.dhi_z)) {
    invd[ip] = 1.0f;
    return;
  }
  const float mz = iz > 0 ? __bfloat162float(q(Tz[i - g.nxy])) : 0.0f;
  const float my = iy > 0 ? __bfloat162float(q(Ty[i - g.nx])) : 0.0f;
  const float mx = ix > 0 ? __bfloat162float(q(Tx[i - 1])) : 0.0f;
  const float dsum = ((((mz + my) + mx) + __bfloat162float(px)) + __bfloat162float(py)) + __bfloat162float(pz);
  invd[ip] = 1.0f / dsum;
}

__global__ void k_widen_bf16(Geo g, int nxp, const __nv_bfloat16* __restrict__ a, double* __restrict__ o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g.n) o[i] = (double)__bfloat162float(a[padded(g, nxp, i)]);
}

// FP32 inner faces, rounded to nearest, at the padded row pitch.
__global__ void k_to_f32_padded(Geo g, int nxp, const double* __restrict__ a, float* __restrict__ o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g.n) o[padded(g, nxp, i)] = (float)a[i];
}

// 16-bit copy of the labels (d <= 65535), streamed by the TMA sweeps.
__global__ void k_convert_labels(Geo g, int nxp, const int32_t* __restrict__ a, uint16_t* __restrict__ o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g.n) o[padded(g, nxp, i)] = (uint16_t)a[i];
}

// y = A x, FP64, one thread per cell.
__global__ void k_apply_A(Geo g, const double* __restrict__ Tx, const double* __restrict__ Ty,
                          const double* __restrict__ Tz, const double* __restrict__ diag,
                          const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.nxy);
  const bool dx = dir_axis(ix, g.nx, g.dlo_x, g.dhi_x), dy = dir_axis(iy, g.ny, g.dlo_y, g.dhi_y),
             dz = dir_axis(iz, g.nz, g.dlo_z, g.dhi_z);
  if (dx || dy || dz) {
    y[i] = x[i];
    return;
  }
  double v = diag[i] * x[i];
  if (ix > 0 && !dir_axis(ix - 1, g.nx, g.dlo_x, g.dhi_x)) v -= Tx[i - 1] * x[i - 1];
  if (ix + 1 < g.nx && !dir_axis(ix + 1, g.nx, g.dlo_x, g.dhi_x)) v -= Tx[i] * x[i + 1];
  if (iy > 0 && !dir_axis(iy - 1, g.ny, g.dlo_y, g.dhi_y)) v -= Ty[i - g.nx] * x[i - g.nx];
  if (iy + 1 < g.ny && !dir_axis(iy + 1, g.ny, g.dlo_y, g.dhi_y)) v -= Ty[i] * x[i + g.nx];
  if (iz > 0 && !dir_axis(iz - 1, g.nz, g.dlo_z, g.dhi_z)) v -= Tz[i - g.nxy] * x[i - g.nxy];
  if (iz + 1 < g.nz && !dir_axis(iz + 1, g.nz, g.dlo_z, g.dhi_z)) v -= Tz[i] * x[i + g.nxy];
  y[i] = v;
}

// out = Z^T v (segmented sum by label), FP64.
__global__ void k_restrict(int64_t n, int d, const int32_t* __restrict__ label, const double* __restrict__ v,
                           double* __restrict__ out) {
  extern __shared__ double sacc[];
  for (int k = threadIdx.x; k < d; k += blockDim.x) sacc[k] = 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) atomicAdd(&sacc[label[i]], v[i]);
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x)
    if (sacc[k] != 0.0) atomicAdd(&out[k], sacc[k]);
}

// Per-CTA partial sums of ||b - A x||^2 and ||b||^2.
__global__ void k_residual(Geo g, const double* __restrict__ Tx, const double* __restrict__ Ty,
                           const double* __restrict__ Tz, const double* __restrict__ diag,
                           const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sr[32], sb[32];
  double rr = 0.0, bb = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / g.nxy);
    double v;
    if (dir_axis(ix, g.nx, g.dlo_x, g.dhi_x) || dir_axis(iy, g.ny, g.dlo_y, g.dhi_y) ||
        dir_axis(iz, g.nz, g.dlo_z, g.dhi_z)) {
      v = x[i];
    } else {
      v = diag[i] * x[i];
      if (ix > 0 && !dir_axis(ix - 1, g.nx, g.dlo_x, g.dhi_x)) v -= Tx[i - 1] * x[i - 1];
      if (ix + 1 < g.nx && !dir_axis(ix + 1, g.nx, g.dlo_x, g.dhi_x)) v -= Tx[i] * x[i + 1];
      if (iy > 0 && !dir_axis(iy - 1, g.ny, g.dlo_y, g.dhi_y)) v -= Ty[i - g.nx] * x[i - g.nx];
      if (iy + 1 < g.ny && !dir_axis(iy + 1, g.ny, g.dlo_y, g.dhi_y)) v -= Ty[i] * x[i + g.nx];
      if (iz > 0 && !dir_axis(iz - 1, g.nz, g.dlo_z, g.dhi_z)) v -= Tz[i - g.nxy] * x[i - g.nxy];
      if (iz + 1 < g.nz && !dir_axis(iz + 1, g.nz, g.dlo_z, g.dhi_z)) v -= Tz[i] * x[i + g.nxy];
    }
    const double r = b[i] - v;
    rr += r * r;
    bb += b[i] * b[i];
  }
  rr = warp_sum(rr);
  bb = warp_sum(bb);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sr[w] = rr;
    sb[w] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sr[k];
      c += sb[k];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
  }
}

__global__ void k_sum_pairs(int m, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < m; ++k) {
      a += part[2 * k];
      c += part[2 * k + 1];
    }
    out[0] = a;
    out[1] = c;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_assemble(sld_system s, const double* q) {
  BcVals bc;
  for (int f = 0; f < 6; ++f) {
    bc.type[f] = s->bc_type[f] == SLD_BC_DIRICHLET;
    bc.value[f] = s->bc_value[f];
  }
  k_assemble<<<blocks_for(s->g.n, 256), 256, 0, s->stream>>>(s->g, bc, s->K, q, s->Tx, s->Ty, s->Tz, s->diag,
                                                            s->invdiag, s->b);
  return cudaGetLastError();
}

cudaError_t launch_labels(sld_system s, int Sx, int Sy, int Sz, const double* tau, int L) {
  Thresholds th{};
  for (int m = 0; m < L - 1; ++m) th.tau[m] = tau[m];
  k_labels<<<blocks_for(s->g.n, 256), 256, 0, s->stream>>>(s->g, Sx, Sy, Sz, th, L, s->K, s->label);
  return cudaGetLastError();
}

cudaError_t launch_coarse_E(sld_system s, const double* Tx, const double* Ty, const double* Tz, double* E,
                            int* bad_label) {
  const int d = s->d;
  BcVals bc;
  for (int f = 0; f < 6; ++f) {
    bc.type[f] = s->bc_type[f] == SLD_BC_DIRICHLET;
    bc.value[f] = s->bc_value[f];
  }
  unsigned long long* cnt = nullptr;
  int* bad = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&cnt, sizeof(unsigned long long) * d + sizeof(int) * 4, s->stream)) != cudaSuccess) return e;
  bad = reinterpret_cast<int*>(cnt + d);
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * d + sizeof(int) * 4, s->stream);
  cudaMemsetAsync(E, 0, sizeof(double) * d * d, s->stream);
  const size_t smem = sizeof(double) * d + sizeof(unsigned) * d;
  cudaFuncSetAttribute(k_coarse_E, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(s->g.n, 256), (int64_t)s->nsm * 4);
  k_coarse_E<<<grid, 256, smem, s->stream>>>(s->g, bc, d, s->label, Tx, Ty, Tz, E, cnt, bad);
  k_pin_empty<<<blocks_for(d, 128), 128, 0, s->stream>>>(d, cnt, E);
  int hbad = 0;
  cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  e = cudaStreamSynchronize(s->stream);
  cudaFreeAsync(cnt, s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  *bad_label = hbad;
  return e;
}

int coarse_factor(sld_system s, int dim, const double* E, double* Einv, double timeout_s, std::string* msg,
                  int rel_from, double rel_tol) {
  const int d = dim;
  double *A = nullptr, *Lm = nullptr, *W = nullptr;
  unsigned* bar = nullptr;
  int* st = nullptr;
  const size_t mat = sizeof(double) * (size_t)d * d;
  cudaError_t e = cudaMallocAsync(&A, 3 * mat + 256, s->stream);
  if (e != cudaSuccess) {
    *msg = std::string("coarse factor allocation: ") + cudaGetErrorString(e);
    return SLD_ERR_OOM;
  }
  Lm = A + (size_t)d * d;
  W = Lm + (size_t)d * d;
  bar = reinterpret_cast<unsigned*>(W + (size_t)d * d);
  st = reinterpret_cast<int*>(bar + 4);
  cudaMemcpyAsync(A, E, mat, cudaMemcpyDeviceToDevice, s->stream);
  cudaMemsetAsync(Lm, 0, mat, s->stream);
  cudaMemsetAsync(bar, 0, 64, s->stream);
  SyncArgs sy{};
  sy.count = bar;
  sy.status = st;
  sy.timeout_ns = (unsigned long long)(timeout_s * 1e9);
  sy.skip_epoch = 0;
  const size_t smem = sizeof(double) * d;
  cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cholesky, 256, smem);
  int G = std::max(1, std::min(s->nsm * std::max(per, 1), (d + 7) / 8));
  if (per < 1) G = 1;
  sy.cta0 = 0;
  sy.ncta = G;
  void* args[] = {(void*)&d, (void*)&A, (void*)&Lm, (void*)&sy, (void*)&E, (void*)&rel_from, (void*)&rel_tol};
  e = cudaLaunchCooperativeKernel((void*)k_cholesky, dim3(G), dim3(256), args, smem, s->stream);
  int hst = 0;
  if (e == cudaSuccess) {
    cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    e = cudaStreamSynchronize(s->stream);
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(A, s->stream);
    *msg = std::string("coarse Cholesky: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  if (hst != 0) {
    cudaFreeAsync(A, s->stream);
    *msg = hst == SLD_ERR_COARSE_SINGULAR ? "E = Z^T A Z is not SPD (Cholesky pivot <= 0, or below the relative bound)"
                                          : "coarse Cholesky: device wait timed out";
    return hst;
  }
  const int wpb = 4;
  const size_t smem2 = sizeof(double) * d * wpb;
  cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  k_tri_inverse<<<std::max(1, std::min((d + wpb - 1) / wpb, s->nsm * 2)), 32 * wpb, smem2, s->stream>>>(d, Lm, W);
  dim3 tg((d + 15) / 16, (d + 15) / 16);
  k_wtw<<<tg, dim3(16, 16), 0, s->stream>>>(d, W, Einv);
  e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFreeAsync(A, s->stream);
  if (e != cudaSuccess) {
    *msg = std::string("coarse inverse: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  return SLD_OK;
}

cudaError_t launch_learned_setup(sld_system s, const void* Zextra_dev, int k, int f32, const double* E,
                                 double* Efull, int* bad) {
  const int64_t n = s->g.n;
  const int d = s->d;
  double* scratch = nullptr;  // ESL (d x kMaxL), ELL (kMaxL x kMaxL), bad flag
  const size_t nsc = (size_t)d * kMaxL + kMaxL * kMaxL + 2;
  cudaError_t e = cudaMallocAsync(&scratch, sizeof(double) * nsc, s->stream);
  if (e != cudaSuccess) return e;
  double* ESL = scratch;
  double* ELL = ESL + (size_t)d * kMaxL;
  int* dbad = reinterpret_cast<int*>(ELL + kMaxL * kMaxL);
  cudaMemsetAsync(scratch, 0, sizeof(double) * nsc, s->stream);
  k_learned_pack<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, k, Zextra_dev, f32, s->ZL32, dbad);
  k_learned_W<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->Tx, s->Ty, s->Tz, s->diag, s->ZL32, s->WL64,
                                                         s->WL32);
  const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(n, 256), (int64_t)s->nsm * 4);
  k_learned_ESL<<<grid, 256, 0, s->stream>>>(n, s->label, s->WL64, ESL);
  k_learned_ELL<<<kMaxL * kMaxL, 512, 0, s->stream>>>(n, s->ZL32, s->WL64, ELL);
  const int D = d + k;
  k_learned_Efull<<<blocks_for((int64_t)D * D, 256), 256, 0, s->stream>>>(d, k, E, ESL, ELL, Efull);
  int hbad = 0;
  cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  e = cudaStreamSynchronize(s->stream);
  cudaFreeAsync(scratch, s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  *bad = hbad;
  return e;
}

cudaError_t launch_quantize_fp32(sld_system s) {
  const int64_t n = s->g.n;
  k_to_f32_padded<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Tx, s->Tx32);
  k_to_f32_padded<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Ty, s->Ty32);
  k_to_f32_padded<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Tz, s->Tz32);
  return cudaGetLastError();
}

cudaError_t launch_quantize_bf16(sld_system s) {
  k_quantize_bf16<<<blocks_for(s->g.n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Tx, s->Ty, s->Tz, s->Tx16,
                                                                 s->Ty16, s->Tz16, s->invd16);
  return cudaGetLastError();
}

cudaError_t launch_widen_bf16(sld_system s, double* Tx, double* Ty, double* Tz) {
  const int64_t n = s->g.n;
  k_widen_bf16<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Tx16, Tx);
  k_widen_bf16<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Ty16, Ty);
  k_widen_bf16<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->Tz16, Tz);
  return cudaGetLastError();
}

cudaError_t launch_labels16(sld_system s) {
  const int64_t n = s->g.n;
  k_convert_labels<<<blocks_for(n, 256), 256, 0, s->stream>>>(s->g, s->nxp, s->label, s->label16);
  return cudaGetLastError();
}

cudaError_t launch_apply_A(sld_system s, const double* x, double* y) {
  k_apply_A<<<blocks_for(s->g.n, 256), 256, 0, s->stream>>>(s->g, s->Tx, s->Ty, s->Tz, s->diag, x, y);
  return cudaGetLastError();
}

cudaError_t launch_restrict(sld_system s, const double* v, double* out) {
  cudaMemsetAsync(out, 0, sizeof(double) * s->d, s->stream);
  const size_t smem = sizeof(double) * s->d;
  cudaFuncSetAttribute(k_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(s->g.n, 256), (int64_t)s->nsm * 4);
  k_restrict<<<grid, 256, smem, s->stream>>>(s->g.n, s->d, s->label, v, out);
  return cudaGetLastError();
}

cudaError_t launch_residual(sld_system s, const double* b, const double* x, double* part, double* rr_host,
                            double* bb_host) {
  const int grid = s->nsm * 4;
  k_residual<<<grid, 256, 0, s->stream>>>(s->g, s->Tx, s->Ty, s->Tz, s->diag, b, x, part);
  k_sum_pairs<<<1, 32, 0, s->stream>>>(grid, part, part + 2 * grid);
  double h[2] = {0, 0};
  cudaMemcpyAsync(h, part + 2 * grid, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  *rr_host = h[0];
  *bb_host = h[1];
  return e;
}

}  // namespace sld
