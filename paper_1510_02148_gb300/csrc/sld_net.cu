// sld_net.cu -- the deflation-vector network: 3x3x3 convolutions as implicit
// GEMMs on BF16 tensor cores (FP32 accumulation), their data and weight
// gradients, pooling/upsampling, the subspace loss and Adam.
//
// Activations are channels-last BF16 [cell][C]; gradients of activations are
// FP32.  A forward convolution is, per 3x3x3 tap, a GEMM of the shifted input
// (cells x Cin) with the tap's weights (Cin x Cout), accumulated over the 27
// taps: on the 5th-generation tensor cores (tcgen05.mma, accumulator in
// tensor memory), one CTA per 128 cells and all Cout columns.  The data
// gradient is the same kernel on the flipped, transposed weights; the weight
// gradient is a GEMM over cells (Cout x cells times cells x Cin per tap),
// also on tcgen05.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sld_net.h"
#include "sld_device.cuh"
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

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}



// ---------------------------------------------------------------------------
// Convolution: Y[r][co] = epi(sum_t sum_ci W[t][co][ci] X[r + off_t][ci])
// with epi = + bias, + skip, relu as requested.
// The same convolution on the 5th-generation tensor cores (tcgen05): one CTA
// of 128 threads owns 128 consecutive cells (the M = 128 rows of the GEMM)
// and all NP output channels (N, Cout padded to a multiple of 16); the FP32
// accumulator lives in tensor memory (TMEM, NP of its columns).  For each of
// the 27 taps every thread gathers its cell's neighbour row (Cin BF16,
// zero-padded to CINP) into shared memory and the CTA loads the tap's
// weights; one thread issues the CINP/16 MMAs (K = 16 each) of the tap and
// commits them to the stage's mbarrier.  Two stages: the gather of tap t+1
// overlaps the MMAs of tap t.  Operands use the canonical K-major layout
// without swizzle: 8 x 8 BF16 core matrices of 128 contiguous bytes, the
// ones adjacent in K 128 B apart (LBO), the 8-row groups CINP / 8 * 128 B
// apart (SBO).  Every wait is bounded; a wait that runs out sets *err,
// lets the MMAs in flight finish (bounded), frees the TMEM and leaves.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(const void* p, unsigned lbo, unsigned sbo) {
  const uint64_t a = sld::smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(unsigned* dst, unsigned ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sld::smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   sld::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <int CINP, int NP>
struct ConvTc {
  static constexpr int KC = CINP / 8;                           // core matrices along K
  static constexpr unsigned A_BYTES = 128u * CINP * 2u;         // one stage of A (128 rows)
  static constexpr unsigned B_BYTES = (unsigned)NP * CINP * 2u;  // one stage of B (NP rows)
  static constexpr unsigned SMEM = 2u * (A_BYTES + B_BYTES);
  static constexpr unsigned NCOLS = NP <= 32 ? 32u : 64u;        // TMEM columns (a power of 2, >= 32)
  static_assert(CINP % 16 == 0 && NP % 16 == 0 && NP <= 64 && CINP <= 64, "tile sizes");
};

template <int CINP, int NP>
__global__ void __launch_bounds__(128) k_conv_tc(Dims d, int Cin, int Cout, const bf16* __restrict__ X,
                                                 const bf16* __restrict__ W, const float* __restrict__ bias,
                                                 const bf16* __restrict__ skip, int relu, bf16* __restrict__ Y16,
                                                 float* __restrict__ Y32, int* __restrict__ err) {
  using C = ConvTc<CINP, NP>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ unsigned tmem_base;
  __shared__ int s_fail;
  unsigned char* const As[2] = {smem, smem + C::A_BYTES};
  unsigned char* const Bs[2] = {smem + 2 * C::A_BYTES, smem + 2 * C::A_BYTES + C::B_BYTES};
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned long long timeout = 2000000000ull;  // 2 s per wait
  if (warp == 0) tmem_alloc(&tmem_base, C::NCOLS);
  if (tid == 0) {
    sld::mbar_init(&mbar[0], 1);
    sld::mbar_init(&mbar[1], 1);
    sld::fence_mbar_init();
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tm = tmem_base;
  const int64_t r = (int64_t)blockIdx.x * 128 + tid;  // this thread's cell (row)
  int x = 0, y = 0, z = 0;
  if (r < d.n) {
    x = (int)(r % d.nx);
    y = (int)((r / d.nx) % d.ny);
    z = (int)(r / d.nxy);
  }
  constexpr uint32_t idesc = umma_idesc_bf16(128, NP);
  int issued = 0;  // taps whose MMAs were issued (thread 0's view, shared below)
  for (int tap = 0; tap < 27; ++tap) {
    const int s = tap & 1;
    if (tap >= 2 && !sld::mbar_wait_bounded(&mbar[s], (unsigned)(((tap - 2) >> 1) & 1), timeout)) s_fail = 1;
    __syncthreads();  // stage s is free (or a wait failed: every thread sees s_fail)
    if (s_fail) break;
    // gather: this thread's neighbour row for the tap, Cin BF16 zero-padded to CINP
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int xx = x + dx, yy = y + dy, zz = z + dz;
    const bool in = r < d.n && xx >= 0 && xx < d.nx && yy >= 0 && yy < d.ny && zz >= 0 && zz < d.nz;
    const bf16* src = X + (in ? (r + (int64_t)dz * d.nxy + (int64_t)dy * d.nx + dx) * Cin : 0);
    unsigned char* arow = As[s] + (tid >> 3) * (C::KC * 128) + (tid & 7) * 16;
#pragma unroll
    for (int j = 0; j < C::KC; ++j) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (in && 8 * j < Cin) v = *reinterpret_cast<const uint4*>(src + 8 * j);
      *reinterpret_cast<uint4*>(arow + j * 128) = v;
    }
    // the tap's weights W[tap][co][ci] (K-major rows), zero-padded to NP x CINP
    for (int i = tid; i < NP * C::KC; i += 128) {
      const int co = i / C::KC, j = i % C::KC;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (co < Cout && 8 * j < Cin) v = *reinterpret_cast<const uint4*>(W + ((int64_t)tap * Cout + co) * Cin + 8 * j);
      *reinterpret_cast<uint4*>(Bs[s] + (co >> 3) * (C::KC * 128) + j * 128 + (co & 7) * 16) = v;
    }
    sld::fence_proxy_async_smem();  // the generic stores above, before the tensor core reads them
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < CINP / 16; ++kk) {
        const uint64_t ad = umma_desc(As[s] + kk * 256, 128, C::KC * 128);
        const uint64_t bd = umma_desc(Bs[s] + kk * 256, 128, C::KC * 128);
        umma_bf16(tm, ad, bd, idesc, (tap > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&mbar[s]);
    }
    issued = tap + 1;
  }
  // wait for the last commit of each stage used (it covers every earlier MMA
  // of the issuing thread): the last tap of stage s is the largest t < issued
  // with t & 1 == s, its commit is use number t >> 1 of that stage
  bool ok = !s_fail;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int t = (issued - 1) - (((issued - 1) & 1) ^ s);
    if (t >= 0 && !sld::mbar_wait_bounded(&mbar[s], (unsigned)((t >> 1) & 1), timeout)) ok = false;
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc_fence_after();
  if (ok) {
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float v[16];
      tmem_ld16(tm + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
      if (r < d.n) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int co = c0 + j;
          if (co >= Cout) break;
          float v0 = v[j], v1 = v[j + 1];
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
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, C::NCOLS);
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: for one tap and one chunk of cells,
// dW[tap][co][ci] += sum_r G[r][co] X[r + off][ci], a GEMM with M = Cout
// (padded to 128: the accumulator's TMEM lane is the output channel), N =
// CINP = Cin and K = the chunk's cells, 64 per stage (four K = 16 MMAs).
// Staging transposes both operands into K-major core matrices (8 rows x 8
// cells): threads 0..63 scatter the G row of one cell, threads 64..127 the
// shifted X row.  Rows co >= Cout of A stay zero.  Two stages, bounded waits
// and the error path as in k_conv_tc; the chunk's result is added to dW with
// FP32 atomics (chunks run in any order).
// ---------------------------------------------------------------------------
template <int CINP>
struct WgradTc {
  static constexpr int KB = 64;                                  // cells per stage
  static constexpr unsigned A_BYTES = 128u * KB * 2u;            // 128 rows (co) x KB cells
  static constexpr unsigned B_BYTES = (unsigned)CINP * KB * 2u;  // CINP rows (ci) x KB cells
  static constexpr unsigned SMEM = 2u * (A_BYTES + B_BYTES);
  static constexpr unsigned NCOLS = CINP <= 32 ? 32u : 64u;
  static constexpr unsigned SBO = KB / 8 * 128;                  // next 8-row group
};

template <int CINP>
__global__ void __launch_bounds__(128) k_wgrad_tc(Dims d, int Cout, const bf16* __restrict__ G,
                                                  const bf16* __restrict__ X, float* __restrict__ dW, int64_t chunk,
                                                  int* __restrict__ err) {
  using C = WgradTc<CINP>;
  constexpr int Cin = CINP;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ unsigned tmem_base;
  __shared__ int s_fail;
  unsigned char* const As[2] = {smem, smem + C::A_BYTES};
  unsigned char* const Bs[2] = {smem + 2 * C::A_BYTES, smem + 2 * C::A_BYTES + C::B_BYTES};
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const unsigned long long timeout = 2000000000ull;
  if (warp == 0) tmem_alloc(&tmem_base, C::NCOLS);
  // rows co >= Cout of both A stages stay zero
  for (unsigned i = tid * 16; i < 2 * C::A_BYTES; i += 128 * 16) *reinterpret_cast<uint4*>(smem + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    sld::mbar_init(&mbar[0], 1);
    sld::mbar_init(&mbar[1], 1);
    sld::fence_mbar_init();
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tm = tmem_base;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(rb + chunk, d.n);
  const int nst = (int)((re - rb + C::KB - 1) / C::KB);
  constexpr uint32_t idesc = umma_idesc_bf16(128, CINP);
  int issued = 0;
  for (int st = 0; st < nst; ++st) {
    const int s = st & 1;
    if (st >= 2 && !sld::mbar_wait_bounded(&mbar[s], (unsigned)(((st - 2) >> 1) & 1), timeout)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    const int c = tid & 63;  // the cell of this thread within the stage
    const int64_t r = rb + (int64_t)st * C::KB + c;
    const unsigned cell_off = (unsigned)(c >> 3) * 128u + (unsigned)(c & 7) * 2u;
    if (tid < 64) {  // A[co][c] = G[r][co]
      for (int co0 = 0; co0 < Cout; co0 += 8) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < re) v = *reinterpret_cast<const uint4*>(G + r * Cout + co0);
        const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          *reinterpret_cast<bf16*>(As[s] + (unsigned)(co0 >> 3) * C::SBO + (unsigned)k * 16u + cell_off) = e[k];
      }
    } else {  // B[ci][c] = X[r + off][ci]
      int64_t q = -1;
      if (r < re) {
        const int x = (int)(r % d.nx), y = (int)((r / d.nx) % d.ny), z = (int)(r / d.nxy);
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        if (xx >= 0 && xx < d.nx && yy >= 0 && yy < d.ny && zz >= 0 && zz < d.nz)
          q = r + (int64_t)dz * d.nxy + (int64_t)dy * d.nx + dx;
      }
#pragma unroll
      for (int ci0 = 0; ci0 < Cin; ci0 += 8) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (q >= 0) v = *reinterpret_cast<const uint4*>(X + q * Cin + ci0);
        const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          *reinterpret_cast<bf16*>(Bs[s] + (unsigned)(ci0 >> 3) * C::SBO + (unsigned)k * 16u + cell_off) = e[k];
      }
    }
    sld::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < C::KB / 16; ++kk) {
        const uint64_t ad = umma_desc(As[s] + kk * 256, 128, C::SBO);
        const uint64_t bd = umma_desc(Bs[s] + kk * 256, 128, C::SBO);
        umma_bf16(tm, ad, bd, idesc, (st > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&mbar[s]);
    }
    issued = st + 1;
  }
  bool ok = !s_fail && issued > 0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int t = (issued - 1) - (((issued - 1) & 1) ^ s);
    if (t >= 0 && !sld::mbar_wait_bounded(&mbar[s], (unsigned)((t >> 1) & 1), timeout)) ok = false;
  }
  if (!ok && issued > 0 && tid == 0) atomicExch(err, 1);
  tc_fence_after();
  if (ok) {
    const int co = tid;  // TMEM lane = output channel
    float* base = dW + ((int64_t)tap * Cout + co) * Cin;
#pragma unroll
    for (int c0 = 0; c0 < CINP; c0 += 16) {
      float v[16];
      tmem_ld16(tm + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
      if (co < Cout) {
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(base + c0 + j, v[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, C::NCOLS);
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
  int* err = nullptr;     // set by a tensor-core kernel whose bounded wait ran out
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

// After a synchronised call: a tensor-core kernel whose bounded wait ran out
// left *err set (and its results unwritten); report it and clear the flag.
sld_status nchecked(sld_net net, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return ncuda(e, what);
  int h = 0;
  e = cudaMemcpy(&h, net->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ncuda(e, what);
  if (h) {
    cudaMemset(net->err, 0, sizeof(int));
    return nfail(SLD_ERR_TIMEOUT, std::string(what) + ": a tensor-core wait timed out");
  }
  return SLD_OK;
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

// A convolution on the tensor cores: k_conv_tc with Cin and Cout padded to
// multiples of 16 (the forward and data-gradient channel pairs of the net).
cudaError_t conv(sld_net net, int level, int l, const bf16* X, const bf16* W, const float* bias, const bf16* skip,
                 int relu, bf16* Y16, float* Y32, int Cin, int Cout) {
  const Dims& d = net->d[level];
  const unsigned grid = blocks(d.n, 128);
  const int cinp = (Cin + 15) / 16 * 16, np = (Cout + 15) / 16 * 16;
  bool done = false;
#define CONV_TC(CI, NN)                                                                                        \
  if (!done && cinp == CI && np == NN) {                                                                       \
    k_conv_tc<CI, NN><<<grid, 128, ConvTc<CI, NN>::SMEM, net->stream>>>(d, Cin, Cout, X, W, bias, skip, relu,  \
                                                                        Y16, Y32, net->err);                   \
    done = true;                                                                                               \
  }
  CONV_TC(16, 16)
  CONV_TC(16, 32)
  CONV_TC(32, 16)
  CONV_TC(32, 48)
  CONV_TC(48, 32)
  CONV_TC(48, 64)
  CONV_TC(64, 48)
#undef CONV_TC
  (void)l;
  if (!done) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t wgrad(sld_net net, int level, int l, const bf16* Gz, const bf16* X) {
  const Dims& d = net->d[level];
  const int Cin = kCin[l], Cout = kCout[l];
  const int64_t chunk = 4096;
  dim3 grid((unsigned)((d.n + chunk - 1) / chunk), 27, 1);
  float* dW = net->G + w_off(l);
  switch (Cin) {
#define WG_CASE(CI)                                                                                        \
  case CI: {                                                                                               \
    auto kern = k_wgrad_tc<CI>;                                                                            \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WgradTc<CI>::SMEM);       \
    kern<<<grid, 128, WgradTc<CI>::SMEM, net->stream>>>(d, Cout, Gz, X, dW, chunk, net->err);              \
    break;                                                                                                 \
  }
    WG_CASE(16)
    WG_CASE(32)
    WG_CASE(48)
    WG_CASE(64)
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
  A(nalloc(net, &net->err, 1));
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
    cudaMemsetAsync(net->err, 0, sizeof(int), net->stream);
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
  return nchecked(net, e, "network forward");
}

sld_status sld_net_backward(sld_net net, const float* dout) {
  if (!net || !dout) return nfail(SLD_ERR_INVALID_ARG, "NULL argument");
  const Dims& d = net->d[0];
  cudaError_t e = cudaMemcpyAsync(net->gout, dout, sizeof(float) * d.n * kOutC, cudaMemcpyDefault, net->stream);
  if (e == cudaSuccess) e = backward(net);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  return nchecked(net, e, "network backward");
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
  return nchecked(net, e, "loss backward");
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
