// sld_net.cu -- the deflation-vector network: 3x3x3 convolutions as implicit
// GEMMs on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation), their
// data and weight gradients, pooling/upsampling, the subspace loss and Adam.
//
// Activations are channels-last BF16 [cell][C]; gradients of activations are
// FP32.  A forward convolution is, per 3x3x3 tap, a GEMM of the shifted input
// (cells x Cin) with the tap's weights (Cin x Cout): one warp owns 16
// consecutive cells and all Cout columns.  The data gradient is the same
// kernel on the flipped, transposed weights; the weight gradient is a GEMM
// over cells (Cout x cells times cells x Cin per tap).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sld_net.h"
#include "sld_internal.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kL = 9;
constexpr int kCin[kL] = {16, 16, 16, 32, 48, 64, 48, 32, 16};
constexpr int kCout[kL] = {16, 16, 32, 48, 64, 48, 32, 16, 8};
constexpr int kOutC = 8;
constexpr int kInC = 16;

int64_t w_off(int l) {
  int64_t o = 0;
  for (int i = 0; i < l; ++i) o += 27LL * kCin[i] * kCout[i] + kCout[i];
  return o;
}
int64_t b_off(int l) { return w_off(l) + 27LL * kCin[l] * kCout[l]; }
int64_t n_params() { return w_off(kL); }

struct Dims {
  int nx, ny, nz;
  int64_t nxy, n;
};
Dims dims(int nx, int ny, int nz) { return Dims{nx, ny, nz, (int64_t)nx * ny, (int64_t)nx * ny * nz}; }

__device__ __forceinline__ unsigned ld_b32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Linear index of the neighbour of cell r at tap offset, or -1.
__device__ __forceinline__ int64_t nbr(const Dims& d, int64_t r, int dz, int dy, int dx) {
  if (r < 0 || r >= d.n) return -1;
  const int x = (int)(r % d.nx), y = (int)((r / d.nx) % d.ny), z = (int)(r / d.nxy);
  const int xx = x + dx, yy = y + dy, zz = z + dz;
  if (xx < 0 || xx >= d.nx || yy < 0 || yy >= d.ny || zz < 0 || zz >= d.nz) return -1;
  return r + (int64_t)dz * d.nxy + (int64_t)dy * d.nx + dx;
}

// ---------------------------------------------------------------------------
// Convolution: Y[r][co] = epi(sum_t sum_ci W[t][co][ci] X[r + off_t][ci])
// with epi = + bias, + skip, relu as requested.  Cin a multiple of 8, Cout =
// 8 * NT.  One warp: cells m0 .. m0+15 (A rows), all Cout (NT n8 tiles).
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(128) k_conv(Dims d, int Cin, const bf16* __restrict__ X,
                                              const bf16* __restrict__ W, const float* __restrict__ bias,
                                              const bf16* __restrict__ skip, int relu, bf16* __restrict__ Y16,
                                              float* __restrict__ Y32) {
  constexpr int Cout = 8 * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  if (m0 >= d.n) return;
  const int g = lane >> 2, t = lane & 3;
  const int64_t r0 = m0 + g, r1 = m0 + g + 8;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int64_t q0 = nbr(d, r0, dz, dy, dx), q1 = nbr(d, r1, dz, dy, dx);
    const bf16* x0 = X + (q0 < 0 ? 0 : q0) * Cin;
    const bf16* x1 = X + (q1 < 0 ? 0 : q1) * Cin;
    const bf16* wt = W + (int64_t)tap * Cout * Cin;
    for (int c0 = 0; c0 < Cin; c0 += 16) {
      const bool hi = c0 + 8 < Cin;
      const unsigned a0 = q0 >= 0 ? ld_b32(x0 + c0 + 2 * t) : 0u;
      const unsigned a1 = q1 >= 0 ? ld_b32(x1 + c0 + 2 * t) : 0u;
      const unsigned a2 = (q0 >= 0 && hi) ? ld_b32(x0 + c0 + 8 + 2 * t) : 0u;
      const unsigned a3 = (q1 >= 0 && hi) ? ld_b32(x1 + c0 + 8 + 2 * t) : 0u;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const bf16* wr = wt + (int64_t)(j * 8 + g) * Cin + c0 + 2 * t;
        const unsigned b0 = ld_b32(wr);
        const unsigned b1 = hi ? ld_b32(wr + 8) : 0u;
        mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int co = j * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = h ? r1 : r0;
      if (r >= d.n) continue;
      float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
      if (bias) {
        v0 += bias[co];
        v1 += bias[co + 1];
      }
      if (skip) {
        v0 += __bfloat162float(skip[r * Cout + co]);
        v1 += __bfloat162float(skip[r * Cout + co + 1]);
      }
      if (relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      if (Y16) *reinterpret_cast<unsigned*>(Y16 + r * Cout + co) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
      if (Y32) *reinterpret_cast<float2*>(Y32 + r * Cout + co) = make_float2(v0, v1);
    }
  }
}

// Weight gradient: dW[t][co][ci] += sum over cells r of G[r][co] X[r + off_t][ci].
// One warp: one tap, 16 output channels (rows co0 .. co0+15, zero past
// Cout), all Cin (NT n8 tiles), cells [r_beg, r_end) in k-steps of 16.
template <int NT>
__global__ void __launch_bounds__(128) k_wgrad(Dims d, int Cout, const bf16* __restrict__ G,
                                               const bf16* __restrict__ X, float* __restrict__ dW, int64_t chunk) {
  constexpr int Cin = 8 * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.y;
  const int co0 = (blockIdx.z * 4 + warp) * 16;
  if (co0 >= Cout) return;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(rb + chunk, d.n);
  const int coA = co0 + g, coB = co0 + g + 8;
  const bool okA = coA < Cout, okB = coB < Cout;
  const bf16 z = __float2bfloat16(0.f);
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int64_t p0 = rb; p0 < re; p0 += 16) {
    // the four cells this thread touches in this k-step
    const int64_t pc[4] = {p0 + 2 * t, p0 + 2 * t + 1, p0 + 2 * t + 8, p0 + 2 * t + 9};
    bf16 gA[4], gB[4];
    int64_t q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = pc[u] < re;
      gA[u] = (in && okA) ? G[pc[u] * Cout + coA] : z;
      gB[u] = (in && okB) ? G[pc[u] * Cout + coB] : z;
      q[u] = in ? nbr(d, pc[u], dz, dy, dx) : -1;
    }
    const unsigned a0 = pack2(gA[0], gA[1]), a1 = pack2(gB[0], gB[1]);
    const unsigned a2 = pack2(gA[2], gA[3]), a3 = pack2(gB[2], gB[3]);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int ci = j * 8 + g;
      bf16 xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = q[u] >= 0 ? X[q[u] * Cin + ci] : z;
      mma_bf16(acc[j], a0, a1, a2, a3, pack2(xv[0], xv[1]), pack2(xv[2], xv[3]));
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int ci = j * 8 + 2 * t;
    float* base = dW + (int64_t)tap * Cout * Cin;
    if (okA) {
      atomicAdd(base + (int64_t)coA * Cin + ci, acc[j][0]);
      atomicAdd(base + (int64_t)coA * Cin + ci + 1, acc[j][1]);
    }
    if (okB) {
      atomicAdd(base + (int64_t)coB * Cin + ci, acc[j][2]);
      atomicAdd(base + (int64_t)coB * Cin + ci + 1, acc[j][3]);
    }
  }
}

// Wt[26 - t][ci][co] = W[t][co][ci]: the weights of the data-gradient convolution.
__global__ void k_flip_weights(int Cin, int Cout, const bf16* __restrict__ W, bf16* __restrict__ Wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = 27LL * Cin * Cout;
  if (i >= tot) return;
  const int t = (int)(i / ((int64_t)Cout * Cin));
  const int co = (int)((i / Cin) % Cout), ci = (int)(i % Cin);
  Wt[((int64_t)(26 - t) * Cin + ci) * Cout + co] = W[i];
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, bf16* __restrict__ o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = __float2bfloat16(a[i]);
}

// dz = bf16(g * [y > 0]) (no mask when y is NULL); gskip += g * [y > 0];
// dbias[c] += sum over cells of g * [y > 0].
__global__ void k_mask(int64_t n, int C, const float* __restrict__ g, const bf16* __restrict__ y,
                       bf16* __restrict__ dz, float* __restrict__ gskip, float* __restrict__ dbias) {
  __shared__ float sb[64];
  for (int c = threadIdx.x; c < C; c += blockDim.x) sb[c] = 0.f;
  __syncthreads();
  const int64_t tot = n * C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
    float v = g[i];
    if (y && !(__bfloat162float(y[i]) > 0.f)) v = 0.f;
    dz[i] = __float2bfloat16(v);
    if (gskip) gskip[i] += v;
    atomicAdd(&sb[(int)(i % C)], v);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dbias[c], sb[c]);
}

// 2x2x2 mean pooling; fine grid d (coarse nx/2 ...).
__global__ void k_pool(Dims d, int C, const bf16* __restrict__ X, bf16* __restrict__ Y) {
  const int cx = d.nx / 2, cy = d.ny / 2, cz = d.nz / 2;
  const int64_t tot = (int64_t)cx * cy * cz * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  const int64_t p = i / C;
  const int x = (int)(p % cx), y = (int)((p / cx) % cy), z = (int)(p / ((int64_t)cx * cy));
  float s = 0.f;
  for (int k = 0; k < 8; ++k) {
    const int64_t f = (int64_t)(2 * z + (k >> 2)) * d.nxy + (int64_t)(2 * y + ((k >> 1) & 1)) * d.nx + 2 * x + (k & 1);
    s += __bfloat162float(X[f * C + c]);
  }
  Y[i] = __float2bfloat16(s * 0.125f);
}

// gX (fine) += gY (coarse) / 8 at each child.
__global__ void k_pool_bwd(Dims d, int C, const float* __restrict__ gY, float* __restrict__ gX) {
  const int64_t tot = d.n * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  const int64_t f = i / C;
  const int x = (int)(f % d.nx), y = (int)((f / d.nx) % d.ny), z = (int)(f / d.nxy);
  const int cx = d.nx / 2, cy = d.ny / 2;
  const int64_t p = (int64_t)(z / 2) * cx * cy + (int64_t)(y / 2) * cx + x / 2;
  gX[i] += gY[p * C + c] * 0.125f;
}

// Nearest upsampling onto the fine grid d.
__global__ void k_up(Dims d, int C, const bf16* __restrict__ X, bf16* __restrict__ Y) {
  const int64_t tot = d.n * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  const int64_t f = i / C;
  const int x = (int)(f % d.nx), y = (int)((f / d.nx) % d.ny), z = (int)(f / d.nxy);
  const int cx = d.nx / 2, cy = d.ny / 2;
  const int64_t p = (int64_t)(z / 2) * cx * cy + (int64_t)(y / 2) * cx + x / 2;
  Y[i] = X[p * C + c];
}

// gX (coarse) = sum of gY over the 8 children (fine grid d).
__global__ void k_up_bwd(Dims d, int C, const float* __restrict__ gY, float* __restrict__ gX) {
  const int cx = d.nx / 2, cy = d.ny / 2, cz = d.nz / 2;
  const int64_t tot = (int64_t)cx * cy * cz * C;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int c = (int)(i % C);
  const int64_t p = i / C;
  const int x = (int)(p % cx), y = (int)((p / cx) % cy), z = (int)(p / ((int64_t)cx * cy));
  float s = 0.f;
  for (int k = 0; k < 8; ++k) {
    const int64_t f = (int64_t)(2 * z + (k >> 2)) * d.nxy + (int64_t)(2 * y + ((k >> 1) & 1)) * d.nx + 2 * x + (k & 1);
    s += gY[f * C + c];
  }
  gX[i] = s;
}

// Sums of log10 K and its square (FP64), for the input standardisation.
__global__ void k_logk_stats(int64_t n, const double* __restrict__ K, double* __restrict__ out) {
  __shared__ double s1[8], s2[8];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double l = log10(K[i]);
    a += l;
    b += l * l;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = a;
    s2[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      u += s1[w];
      v += s2[w];
    }
    atomicAdd(out, u);
    atomicAdd(out + 1, v);
  }
}

__global__ void k_features(Dims d, const double* __restrict__ K, const double* __restrict__ st, bf16* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const double mean = st[0] / (double)d.n;
  const double var = fmax(st[1] / (double)d.n - mean * mean, 0.0);
  const double sd = var > 1e-24 ? sqrt(var) : 1.0;
  const int x = (int)(i % d.nx), y = (int)((i / d.nx) % d.ny), z = (int)(i / d.nxy);
  float f[kInC];
  f[0] = (float)((log10(K[i]) - mean) / sd);
  f[1] = 2.f * (x + 0.5f) / d.nx - 1.f;
  f[2] = 2.f * (y + 0.5f) / d.ny - 1.f;
  f[3] = 2.f * (z + 0.5f) / d.nz - 1.f;
#pragma unroll
  for (int c = 4; c < kInC; ++c) f[c] = 0.f;
#pragma unroll
  for (int c = 0; c < kInC; c += 2)
    *reinterpret_cast<unsigned*>(F + i * kInC + c) = pack2(__float2bfloat16(f[c]), __float2bfloat16(f[c + 1]));
}

// Loss sums (FP64): S[0..63] = Y^T D Y, S[64 .. 64+8m) = Y^T D V, S[64+8m] =
// tr(V^T D V).  A block stages 128 cells in shared memory; thread k then adds
// sum k over them.
__global__ void __launch_bounds__(160) k_loss_sums(int64_t n, int m, const float* __restrict__ Y,
                                                   const float* __restrict__ V, const double* __restrict__ D,
                                                   double* __restrict__ S) {
  constexpr int kC = 128;
  __shared__ float sy[kC][8], sv[kC][8];
  __shared__ double sd[kC];
  const int nsum = 64 + 8 * m + 1;
  const int k = threadIdx.x;
  double acc = 0.0;
  for (int64_t c0 = (int64_t)blockIdx.x * kC; c0 < n; c0 += (int64_t)gridDim.x * kC) {
    __syncthreads();
    for (int u = threadIdx.x; u < kC * 8; u += blockDim.x) {
      const int c = u / 8, a = u % 8;
      const int64_t i = c0 + c;
      sy[c][a] = i < n ? Y[i * 8 + a] : 0.f;
      sv[c][a] = (i < n && a < m) ? V[i * m + a] : 0.f;
    }
    for (int c = threadIdx.x; c < kC; c += blockDim.x) sd[c] = c0 + c < n ? D[c0 + c] : 0.0;
    __syncthreads();
    if (k < 64) {
      const int a = k / 8, b = k % 8;
      for (int c = 0; c < kC; ++c) acc += sd[c] * (double)sy[c][a] * (double)sy[c][b];
    } else if (k < 64 + 8 * m) {
      const int a = (k - 64) / m, b = (k - 64) % m;
      for (int c = 0; c < kC; ++c) acc += sd[c] * (double)sy[c][a] * (double)sv[c][b];
    } else if (k == 64 + 8 * m) {
      for (int c = 0; c < kC; ++c)
        for (int b = 0; b < m; ++b) acc += sd[c] * (double)sv[c][b] * (double)sv[c][b];
    }
  }
  if (k < nsum) atomicAdd(&S[k], acc);
}

struct Small {
  float M1[64];  // X = G^{-1} C  (8 x m)
  float scale;
  int m;
};

// dY_i = scale * D_i (V_i - Y_i G^{-1}C) (G^{-1}C)^T
__global__ void k_loss_grad(int64_t n, Small sm, const float* __restrict__ Y, const float* __restrict__ V,
                            const double* __restrict__ D, float* __restrict__ dY) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = sm.m;
  float y[8], r[8];
  for (int a = 0; a < 8; ++a) y[a] = Y[i * 8 + a];
  for (int b = 0; b < m; ++b) {
    float s = V[i * m + b];
    for (int a = 0; a < 8; ++a) s -= y[a] * sm.M1[a * m + b];
    r[b] = s;
  }
  const float w = sm.scale * (float)D[i];
  for (int a = 0; a < 8; ++a) {
    float s = 0.f;
    for (int b = 0; b < m; ++b) s += r[b] * sm.M1[a * m + b];
    dY[i * 8 + a] = w * s;
  }
}

__global__ void k_adam(int64_t n, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct sld_net_s {
  Dims d[4];  // levels 0..3
  cudaStream_t stream = nullptr;
  int64_t np = 0;
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  bf16* W16 = nullptr;   // all weights, BF16, same offsets as P (biases unused)
  bf16* Wt16 = nullptr;  // flipped, transposed weights (data gradient)
  double* K = nullptr;   // staged K
  double* stats = nullptr;
  double* S = nullptr;   // loss sums
  // activations (BF16)
  bf16 *f = nullptr, *a0 = nullptr, *e0 = nullptr, *p1 = nullptr, *e1 = nullptr, *p2 = nullptr, *e2 = nullptr,
       *p3 = nullptr, *b3 = nullptr, *u2 = nullptr, *d2 = nullptr, *u1 = nullptr, *d1 = nullptr, *u0 = nullptr,
       *d0 = nullptr;
  float* out = nullptr;  // n x 8
  // gradients (FP32) and the BF16 masked gradient scratch
  float *gout = nullptr, *g0a = nullptr, *g0b = nullptr, *g0c = nullptr, *g1a = nullptr, *g1b = nullptr,
        *g1c = nullptr, *g2a = nullptr, *g2b = nullptr, *g2c = nullptr, *g3 = nullptr;
  bf16* dz = nullptr;
  float* Vst = nullptr;   // staged targets
  double* Dst = nullptr;  // staged weights
  std::vector<void*> allocs;
};

namespace {

sld_status nfail(sld_status st, const std::string& m) {
  sld::set_last_error(m);
  return st;
}
sld_status ncuda(cudaError_t e, const char* what) {
  return nfail(e == cudaErrorMemoryAllocation ? SLD_ERR_OOM : SLD_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}
bool on_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t nalloc(sld_net net, T** p, int64_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  if (e == cudaSuccess) {
    net->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

cudaError_t conv(sld_net net, int level, int l, const bf16* X, const bf16* W, const float* bias, const bf16* skip,
                 int relu, bf16* Y16, float* Y32, int Cin, int Cout) {
  const Dims& d = net->d[level];
  const unsigned grid = blocks(d.n, 64);
  switch (Cout / 8) {
#define CONV_CASE(NT)                                                                                         \
  case NT:                                                                                                    \
    k_conv<NT><<<grid, 128, 0, net->stream>>>(d, Cin, X, W, bias, skip, relu, Y16, Y32);                      \
    break;
    CONV_CASE(1)
    CONV_CASE(2)
    CONV_CASE(4)
    CONV_CASE(6)
    CONV_CASE(8)
#undef CONV_CASE
    default:
      return cudaErrorInvalidValue;
  }
  (void)l;
  return cudaGetLastError();
}

cudaError_t wgrad(sld_net net, int level, int l, const bf16* Gz, const bf16* X) {
  const Dims& d = net->d[level];
  const int Cin = kCin[l], Cout = kCout[l];
  const int64_t chunk = 4096;
  dim3 grid((unsigned)((d.n + chunk - 1) / chunk), 27, (unsigned)((Cout + 63) / 64));
  float* dW = net->G + w_off(l);
  switch (Cin / 8) {
#define WG_CASE(NT)                                                                     \
  case NT:                                                                              \
    k_wgrad<NT><<<grid, 128, 0, net->stream>>>(d, Cout, Gz, X, dW, chunk);              \
    break;
    WG_CASE(2)
    WG_CASE(4)
    WG_CASE(6)
    WG_CASE(8)
#undef WG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// g (FP32 gradient of layer l's output) -> masked BF16 dz, bias grad, skip
// accumulation; then weight grad, and (if gx) the data gradient into gx.
cudaError_t conv_back(sld_net net, int level, int l, const float* g, const bf16* y, float* gskip, const bf16* X,
                      float* gx) {
  const Dims& d = net->d[level];
  const int Cin = kCin[l], Cout = kCout[l];
  const unsigned gb = (unsigned)std::min<int64_t>(blocks(d.n * Cout, 256), 4096);
  k_mask<<<gb, 256, 0, net->stream>>>(d.n, Cout, g, y, net->dz, gskip, net->G + b_off(l));
  cudaError_t e = wgrad(net, level, l, net->dz, X);
  if (e != cudaSuccess || !gx) return e;
  return conv(net, level, l, net->dz, net->Wt16 + w_off(l), nullptr, nullptr, 0, nullptr, gx, Cout, Cin);
}

cudaError_t forward(sld_net net) {
  cudaStream_t s = net->stream;
  // weights: FP32 master -> BF16, and the flipped copy for the data gradient
  k_to_bf16<<<blocks(net->np, 256), 256, 0, s>>>(net->np, net->P, net->W16);
  for (int l = 0; l < kL; ++l)
    k_flip_weights<<<blocks(27LL * kCin[l] * kCout[l], 256), 256, 0, s>>>(kCin[l], kCout[l], net->W16 + w_off(l),
                                                                           net->Wt16 + w_off(l));
  auto W = [&](int l) { return net->W16 + w_off(l); };
  auto B = [&](int l) { return net->P + b_off(l); };
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  C(conv(net, 0, 0, net->f, W(0), B(0), nullptr, 1, net->a0, nullptr, 16, 16));
  C(conv(net, 0, 1, net->a0, W(1), B(1), nullptr, 1, net->e0, nullptr, 16, 16));
  k_pool<<<blocks(net->d[1].n * 16, 256), 256, 0, s>>>(net->d[0], 16, net->e0, net->p1);
  C(conv(net, 1, 2, net->p1, W(2), B(2), nullptr, 1, net->e1, nullptr, 16, 32));
  k_pool<<<blocks(net->d[2].n * 32, 256), 256, 0, s>>>(net->d[1], 32, net->e1, net->p2);
  C(conv(net, 2, 3, net->p2, W(3), B(3), nullptr, 1, net->e2, nullptr, 32, 48));
  k_pool<<<blocks(net->d[3].n * 48, 256), 256, 0, s>>>(net->d[2], 48, net->e2, net->p3);
  C(conv(net, 3, 4, net->p3, W(4), B(4), nullptr, 1, net->b3, nullptr, 48, 64));
  k_up<<<blocks(net->d[2].n * 64, 256), 256, 0, s>>>(net->d[2], 64, net->b3, net->u2);
  C(conv(net, 2, 5, net->u2, W(5), B(5), net->e2, 1, net->d2, nullptr, 64, 48));
  k_up<<<blocks(net->d[1].n * 48, 256), 256, 0, s>>>(net->d[1], 48, net->d2, net->u1);
  C(conv(net, 1, 6, net->u1, W(6), B(6), net->e1, 1, net->d1, nullptr, 48, 32));
  k_up<<<blocks(net->d[0].n * 32, 256), 256, 0, s>>>(net->d[0], 32, net->d1, net->u0);
  C(conv(net, 0, 7, net->u0, W(7), B(7), net->e0, 1, net->d0, nullptr, 32, 16));
  C(conv(net, 0, 8, net->d0, W(8), B(8), nullptr, 0, nullptr, net->out, 16, 8));
  C(cudaGetLastError());
  return e;
}

// Backward from net->gout (d out), mirroring forward().
cudaError_t backward(sld_net net) {
  cudaStream_t s = net->stream;
  cudaMemsetAsync(net->G, 0, sizeof(float) * net->np, s);
  const Dims* d = net->d;
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  // level 0 buffers: g0a = d(d0) [16], g0b = d(e0) [16], g0c = d(u0) [32]
  cudaMemsetAsync(net->g0b, 0, sizeof(float) * d[0].n * 16, s);
  cudaMemsetAsync(net->g1b, 0, sizeof(float) * d[1].n * 32, s);
  cudaMemsetAsync(net->g2b, 0, sizeof(float) * d[2].n * 48, s);
  C(conv_back(net, 0, 8, net->gout, nullptr, nullptr, net->d0, net->g0a));           // out = conv8(d0)
  C(conv_back(net, 0, 7, net->g0a, net->d0, net->g0b, net->u0, net->g0c));          // d0 = relu(conv7(u0) + e0)
  k_up_bwd<<<blocks(d[1].n * 32, 256), 256, 0, s>>>(d[0], 32, net->g0c, net->g1a);   // u0 = up(d1)
  C(conv_back(net, 1, 6, net->g1a, net->d1, net->g1b, net->u1, net->g1c));           // d1 = relu(conv6(u1) + e1)
  k_up_bwd<<<blocks(d[2].n * 48, 256), 256, 0, s>>>(d[1], 48, net->g1c, net->g2a);   // u1 = up(d2)
  C(conv_back(net, 2, 5, net->g2a, net->d2, net->g2b, net->u2, net->g2c));           // d2 = relu(conv5(u2) + e2)
  k_up_bwd<<<blocks(d[3].n * 64, 256), 256, 0, s>>>(d[2], 64, net->g2c, net->g3);    // u2 = up(b3)
  // b3 = relu(conv4(p3)); p3 = pool(e2): d(p3) into g2c's space (N3 x 48), reuse g2a
  C(conv_back(net, 3, 4, net->g3, net->b3, nullptr, net->p3, net->g2a));
  k_pool_bwd<<<blocks(d[2].n * 48, 256), 256, 0, s>>>(d[2], 48, net->g2a, net->g2b);
  // e2 = relu(conv3(p2)); p2 = pool(e1): d(p2) (N2 x 32) into g2c
  C(conv_back(net, 2, 3, net->g2b, net->e2, nullptr, net->p2, net->g2c));
  k_pool_bwd<<<blocks(d[1].n * 32, 256), 256, 0, s>>>(d[1], 32, net->g2c, net->g1b);
  // e1 = relu(conv2(p1)); p1 = pool(e0): d(p1) (N1 x 16) into g1c
  C(conv_back(net, 1, 2, net->g1b, net->e1, nullptr, net->p1, net->g1c));
  k_pool_bwd<<<blocks(d[0].n * 16, 256), 256, 0, s>>>(d[0], 16, net->g1c, net->g0b);
  // e0 = relu(conv1(a0)): d(a0) into g0a
  C(conv_back(net, 0, 1, net->g0b, net->e0, nullptr, net->a0, net->g0a));
  // a0 = relu(conv0(f)): weights only
  C(conv_back(net, 0, 0, net->g0a, net->a0, nullptr, net->f, nullptr));
  C(cudaGetLastError());
  return e;
}

}  // namespace

extern "C" {

int64_t sld_net_num_params(void) { return n_params(); }

sld_status sld_net_create(int nx, int ny, int nz, void* stream, sld_net* out) {
  if (!out) return nfail(SLD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8)
    return nfail(SLD_ERR_INVALID_ARG, "grid sizes must be multiples of 8 (three pooling levels)");
  sld_net net = new sld_net_s();
  net->stream = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < 4; ++l) net->d[l] = dims(nx >> l, ny >> l, nz >> l);
  net->np = n_params();
  const int64_t n0 = net->d[0].n, n1 = net->d[1].n, n2 = net->d[2].n, n3 = net->d[3].n;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  A(nalloc(net, &net->P, net->np));
  A(nalloc(net, &net->G, net->np));
  A(nalloc(net, &net->M, net->np));
  A(nalloc(net, &net->V, net->np));
  A(nalloc(net, &net->W16, net->np));
  A(nalloc(net, &net->Wt16, net->np));
  A(nalloc(net, &net->K, n0));
  A(nalloc(net, &net->stats, 4));
  A(nalloc(net, &net->S, 64 + 64 + 8));
  A(nalloc(net, &net->f, n0 * 16));
  A(nalloc(net, &net->a0, n0 * 16));
  A(nalloc(net, &net->e0, n0 * 16));
  A(nalloc(net, &net->p1, n1 * 16));
  A(nalloc(net, &net->e1, n1 * 32));
  A(nalloc(net, &net->p2, n2 * 32));
  A(nalloc(net, &net->e2, n2 * 48));
  A(nalloc(net, &net->p3, n3 * 48));
  A(nalloc(net, &net->b3, n3 * 64));
  A(nalloc(net, &net->u2, n2 * 64));
  A(nalloc(net, &net->d2, n2 * 48));
  A(nalloc(net, &net->u1, n1 * 48));
  A(nalloc(net, &net->d1, n1 * 32));
  A(nalloc(net, &net->u0, n0 * 32));
  A(nalloc(net, &net->d0, n0 * 16));
  A(nalloc(net, &net->out, n0 * kOutC));
  A(nalloc(net, &net->gout, n0 * kOutC));
  A(nalloc(net, &net->g0a, n0 * 16));
  A(nalloc(net, &net->g0b, n0 * 16));
  A(nalloc(net, &net->g0c, n0 * 32));
  A(nalloc(net, &net->g1a, n1 * 32));
  A(nalloc(net, &net->g1b, n1 * 32));
  A(nalloc(net, &net->g1c, n1 * 48));
  A(nalloc(net, &net->g2a, n2 * 48));
  A(nalloc(net, &net->g2b, n2 * 48));
  A(nalloc(net, &net->g2c, n2 * 64));
  A(nalloc(net, &net->g3, n3 * 64));
  A(nalloc(net, &net->dz, n0 * 32));
  A(nalloc(net, &net->Vst, n0 * 8));
  A(nalloc(net, &net->Dst, n0));
  if (e == cudaSuccess) {
    cudaMemsetAsync(net->P, 0, sizeof(float) * net->np, net->stream);
    cudaMemsetAsync(net->M, 0, sizeof(float) * net->np, net->stream);
    cudaMemsetAsync(net->V, 0, sizeof(float) * net->np, net->stream);
    cudaMemsetAsync(net->G, 0, sizeof(float) * net->np, net->stream);
    e = cudaStreamSynchronize(net->stream);
  }
  if (e != cudaSuccess) {
    sld_net_destroy(net);
    return ncuda(e, "network allocation");
  }
  *out = net;
  return SLD_OK;
}

sld_status sld_net_set_params(sld_net net, const float* params) {
  if (!net || !params) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(net->P, params, sizeof(float) * net->np, cudaMemcpyDefault, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "set params");
}

sld_status sld_net_get_params(sld_net net, float* params) {
  if (!net || !params) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(params, net->P, sizeof(float) * net->np, cudaMemcpyDefault, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "get params");
}

sld_status sld_net_get_grads(sld_net net, float* grads) {
  if (!net || !grads) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(grads, net->G, sizeof(float) * net->np, cudaMemcpyDefault, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "get grads");
}

sld_status sld_net_forward(sld_net net, const double* K, float* out) {
  if (!net || !K) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  const Dims& d = net->d[0];
  cudaStream_t s = net->stream;
  cudaError_t e = cudaMemcpyAsync(net->K, K, sizeof(double) * d.n, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return ncuda(e, "copy K");
  cudaMemsetAsync(net->stats, 0, sizeof(double) * 4, s);
  k_logk_stats<<<std::min<unsigned>(blocks(d.n, 256), 1024), 256, 0, s>>>(d.n, net->K, net->stats);
  k_features<<<blocks(d.n, 256), 256, 0, s>>>(d, net->K, net->stats, net->f);
  e = forward(net);
  if (e == cudaSuccess && out)
    e = cudaMemcpyAsync(out, net->out, sizeof(float) * d.n * kOutC, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "network forward");
}

sld_status sld_net_backward(sld_net net, const float* dout) {
  if (!net || !dout) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  const Dims& d = net->d[0];
  cudaError_t e = cudaMemcpyAsync(net->gout, dout, sizeof(float) * d.n * kOutC, cudaMemcpyDefault, net->stream);
  if (e == cudaSuccess) e = backward(net);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "network backward");
}

sld_status sld_net_loss_backward(sld_net net, const float* V, int m, const double* D, double* loss) {
  if (!net || !V || !D) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  if (m < 1 || m > 8) return nfail(SLD_ERR_INVALID_ARG, "m must be in [1, 8]");
  const Dims& d = net->d[0];
  cudaStream_t s = net->stream;
  const float* Vd = V;
  const double* Dd = D;
  cudaError_t e = cudaSuccess;
  if (!on_dev(V)) {
    e = cudaMemcpyAsync(net->Vst, V, sizeof(float) * d.n * m, cudaMemcpyHostToDevice, s);
    Vd = net->Vst;
  }
  if (e == cudaSuccess && !on_dev(D)) {
    e = cudaMemcpyAsync(net->Dst, D, sizeof(double) * d.n, cudaMemcpyHostToDevice, s);
    Dd = net->Dst;
  }
  if (e != cudaSuccess) return ncuda(e, "copy targets");
  const int nsum = 64 + 8 * m + 1;
  cudaMemsetAsync(net->S, 0, sizeof(double) * nsum, s);
  k_loss_sums<<<std::min<unsigned>(blocks(d.n, 128), 2048), 160, 0, s>>>(d.n, m, net->out, Vd, Dd, net->S);
  double S[64 + 64 + 1];
  e = cudaMemcpyAsync(S, net->S, sizeof(double) * nsum, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ncuda(e, "loss sums");
  // G (8x8) = Y^T D Y (+ a relative ridge for a rank-deficient Y), C (8 x m)
  double G[64], C[64], Lc[64];
  double tr = 0.0;
  for (int a = 0; a < 8; ++a) tr += S[a * 8 + a];
  for (int k = 0; k < 64; ++k) G[k] = 0.5 * (S[k] + S[(k % 8) * 8 + k / 8]);
  for (int a = 0; a < 8; ++a) G[a * 8 + a] += 1e-10 * tr / 8.0 + 1e-300;
  for (int k = 0; k < 8 * m; ++k) C[k] = S[64 + k];
  const double vv = S[64 + 8 * m];
  if (!(vv > 0.0)) return nfail(SLD_ERR_INVALID_ARG, "targets have zero D-norm");
  // Cholesky G = L L^T, then X = G^{-1} C by two triangular solves
  for (int j = 0; j < 8; ++j) {
    double s2 = G[j * 8 + j];
    for (int k = 0; k < j; ++k) s2 -= Lc[j * 8 + k] * Lc[j * 8 + k];
    if (!(s2 > 0.0)) return nfail(SLD_ERR_BREAKDOWN, "network output has a degenerate Gram matrix");
    Lc[j * 8 + j] = std::sqrt(s2);
    for (int i = j + 1; i < 8; ++i) {
      double t = G[i * 8 + j];
      for (int k = 0; k < j; ++k) t -= Lc[i * 8 + k] * Lc[j * 8 + k];
      Lc[i * 8 + j] = t / Lc[j * 8 + j];
    }
  }
  double X[64];
  for (int b = 0; b < m; ++b) {
    double y[8];
    for (int i = 0; i < 8; ++i) {
      double t = C[i * m + b];
      for (int k = 0; k < i; ++k) t -= Lc[i * 8 + k] * y[k];
      y[i] = t / Lc[i * 8 + i];
    }
    for (int i = 7; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < 8; ++k) t -= Lc[k * 8 + i] * X[k * m + b];
      X[i * m + b] = t / Lc[i * 8 + i];
    }
  }
  double proj = 0.0;
  for (int k = 0; k < 8 * m; ++k) proj += C[k] * X[k];
  if (loss) *loss = (vv - proj) / vv;
  Small sm{};
  sm.m = m;
  for (int k = 0; k < 8 * m; ++k) sm.M1[k] = (float)X[k];
  sm.scale = (float)(-2.0 / vv);
  k_loss_grad<<<blocks(d.n, 256), 256, 0, s>>>(d.n, sm, net->out, Vd, Dd, net->gout);
  e = backward(net);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SLD_OK : ncuda(e, "loss backward");
}

sld_status sld_net_adam(sld_net net, float lr, float beta1, float beta2, float eps, int step) {
  if (!net || step < 1) return nfail(SLD_ERR_INVALID_ARG, "bad network or step");
  const float c1 = 1.f - std::pow(beta1, (float)step), c2 = 1.f - std::pow(beta2, (float)step);
  k_adam<<<blocks(net->np, 256), 256, 0, net->stream>>>(net->np, net->P, net->G, net->M, net->V, lr, beta1, beta2,
                                                        eps, c1, c2);
  cudaError_t e = cudaStreamSynchronize(net->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? SLD_OK : ncuda(e, "adam");
}

void sld_default_train_options(sld_train_options* o) {
  if (!o) return;
  o->epochs = 12;
  o->lr = 2e-3f;
  o->lr_decay = 0.5f;
  o->decay_every = 0;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->seed = 0;
}

sld_status sld_learned_train(sld_net net, int nfields, const double* const* K, const float* const* V, int m,
                             const double* const* D, const sld_train_options* opt, double* epoch_loss) {
  sld::set_last_error("");
  if (!net || !K || !V || !D) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  if (nfields < 1) return nfail(SLD_ERR_INVALID_ARG, "nfields must be >= 1");
  if (m < 1 || m > 8) return nfail(SLD_ERR_INVALID_ARG, "m must be in [1, 8]");
  sld_train_options o;
  sld_default_train_options(&o);
  if (opt) o = *opt;
  if (o.epochs < 1 || !(o.lr > 0.f) || !(o.lr_decay > 0.f) || o.decay_every < 0 || !(o.beta1 >= 0.f) ||
      !(o.beta1 < 1.f) || !(o.beta2 >= 0.f) || !(o.beta2 < 1.f) || !(o.eps > 0.f))
    return nfail(SLD_ERR_INVALID_ARG, "training options out of range");
  for (int i = 0; i < nfields; ++i)
    if (!K[i] || !V[i] || !D[i]) return nfail(SLD_ERR_INVALID_ARG, "NULL field pointer");
  const int every = o.decay_every > 0 ? o.decay_every : std::max(1, o.epochs / 3);
  std::vector<int> order(nfields);
  int step = 0;
  for (int ep = 0; ep < o.epochs; ++ep) {
    // Fisher-Yates with SplitMix64 (Steele, Lea and Flood 2014) seeded by seed + epoch
    uint64_t st = o.seed + (uint64_t)ep;
    auto next = [&st]() {
      uint64_t z = (st += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    for (int i = 0; i < nfields; ++i) order[i] = i;
    for (int i = nfields - 1; i > 0; --i) std::swap(order[i], order[(int)(next() % (uint64_t)(i + 1))]);
    const float lr = o.lr * std::pow(o.lr_decay, (float)(ep / every));
    double sum = 0.0;
    for (int i : order) {
      sld_status r = sld_net_forward(net, K[i], nullptr);
      double loss = 0.0;
      if (r == SLD_OK) r = sld_net_loss_backward(net, V[i], m, D[i], &loss);
      if (r == SLD_OK) r = sld_net_adam(net, lr, o.beta1, o.beta2, o.eps, ++step);
      if (r != SLD_OK) return r;
      sum += loss;
    }
    if (epoch_loss) epoch_loss[ep] = sum / nfields;
  }
  return SLD_OK;
}

sld_status sld_learned_infer(sld_net net, sld_system s, float* Zextra_out) {
  sld::set_last_error("");
  if (!net || !s) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  const Dims& d = net->d[0];
  if (d.nx != s->g.nx || d.ny != s->g.ny || d.nz != s->g.nz)
    return nfail(SLD_ERR_INVALID_ARG, "the network's grid is not the system's");
  if (!s->label || s->have_labels_d < 1) return nfail(SLD_ERR_STATE, "make the system's labels first");
  sld_status r = sld_net_forward(net, s->K, nullptr);  // the handle's own K (device)
  if (r != SLD_OK) return r;
  if (Zextra_out) {
    cudaError_t e = cudaMemcpyAsync(Zextra_out, net->out, sizeof(float) * d.n * kOutC, cudaMemcpyDefault, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return ncuda(e, "copy the learned vectors");
  }
  return sld_build_deflation(s, nullptr, s->have_labels_d, net->out, kOutC, SLD_ZEXTRA_F32);
}

void sld_net_destroy(sld_net net) {
  if (!net) return;
  cudaStreamSynchronize(net->stream);
  for (void* p : net->allocs) cudaFree(p);
  delete net;
}

}  // extern "C"
