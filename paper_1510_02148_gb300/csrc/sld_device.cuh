// sld_device.cuh -- device helpers shared by the libsld kernels:
// bounded grid barrier, vector loads of four cells, warp reductions,
// cell geometry and Dirichlet tests.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sld_internal.h"

namespace sld {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Barrier of a team of CTAs in a cooperative launch (all CTAs co-resident).
// A monotone arrival counter: barrier number e completes when the counter
// reaches e * (team size).  Every wait is bounded by sy.timeout_ns; on expiry
// the CTA records SLD_ERR_TIMEOUT in *sy.status and the barrier returns
// false, as it does when another CTA has already recorded an error.  The
// caller then leaves the kernel.  No trap, no unbounded spin.
__device__ __forceinline__ bool grid_barrier(const SyncArgs& sy, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * (unsigned)sy.ncta;
    const bool skip = sy.skip_epoch > 0 && (int)blockIdx.x == sy.cta0 && epoch == (unsigned)sy.skip_epoch;
    // release: the CTA's writes (ordered before this thread by the CTA
    // barrier above) become visible before the arrival does
    if (!skip) red_release_add_u32(sy.count, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(sy.count) < target) {
      if (((++spins) & 63u) == 0) {
        if (ld_volatile_i32(sy.status) != 0) { ok = 0; break; }
        if (global_ns() - t0 > sy.timeout_ns) {
          atomicCAS(sy.status, 0, (int)SLD_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    // the acquire load that saw the count orders every later read of this
    // CTA (through the CTA barrier below).  An error recorded elsewhere is
    // seen by the bounded spin of a later barrier, which the failed CTA
    // never reaches.
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum of p[k * stride] over k = k0, k0 + step, ... < n, added in that order,
// the loads issued eight at a time: a long sum then waits for one memory
// round trip per eight terms instead of one per term (a loop whose trip
// count is known only at run time otherwise issues each load after the add
// before it).  Past n the batch reads nothing and adds +0, which leaves the
// sum unchanged.  For data written by the running kernel: plain loads.
__device__ __forceinline__ double ordered_sum(const double* p, int64_t stride, int k0, int n, int step) {
  double t = 0.0;
  for (int k = k0; k < n; k += 8 * step) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = k + u * step < n ? p[(int64_t)(k + u * step) * stride] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) t += v[u];
  }
  return t;
}

// ---------------------------------------------------------------------------
// Loads / stores of CX consecutive cells.  With CX == 4 and all four cells in
// range the access is one 16-byte vector (float) or two (double); otherwise
// element-wise with the missing cells read as 0.  `ro` selects the read-only
// (non-coherent) path and must only be used for data the kernel never writes.
// ---------------------------------------------------------------------------
template <typename T, int CX, bool RO>
__device__ __forceinline__ void ld_cells(const T* __restrict__ a, int64_t i, int nval, T (&v)[CX]) {
  if constexpr (CX == 4) {
    if (nval == 4) {
      if constexpr (sizeof(T) == 4) {
        float4 q = RO ? __ldg(reinterpret_cast<const float4*>(a + i)) : *reinterpret_cast<const float4*>(a + i);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
        double2 q0 = RO ? __ldg(reinterpret_cast<const double2*>(a + i)) : *reinterpret_cast<const double2*>(a + i);
        double2 q1 = RO ? __ldg(reinterpret_cast<const double2*>(a + i) + 1) : *(reinterpret_cast<const double2*>(a + i) + 1);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
      }
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < CX; ++c) v[c] = (c < nval) ? (RO ? __ldg(a + i + c) : a[i + c]) : T(0);
}

template <int CX>
__device__ __forceinline__ void ld_labels(const int32_t* __restrict__ a, int64_t i, int nval, int (&v)[CX]) {
  if constexpr (CX == 4) {
    if (nval == 4) {
      int4 q = __ldg(reinterpret_cast<const int4*>(a + i));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < CX; ++c) v[c] = (c < nval) ? __ldg(a + i + c) : -1;
}

template <typename T, int CX>
__device__ __forceinline__ void st_cells(T* __restrict__ a, int64_t i, int nval, const T (&v)[CX]) {
  if constexpr (CX == 4) {
    if (nval == 4) {
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(a + i) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        reinterpret_cast<double2*>(a + i)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(a + i)[1] = make_double2(v[2], v[3]);
      }
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < CX; ++c)
    if (c < nval) a[i + c] = v[c];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Rank of this CTA in its team, and the team size.
__device__ __forceinline__ int team_rank(const SyncArgs& sy) { return (int)blockIdx.x - sy.cta0; }

// Dirichlet-cell test along one axis: coordinate c on a Dirichlet face.
__device__ __forceinline__ bool dir_axis(int c, int n, unsigned lo, unsigned hi) {
  return (lo && c == 0) || (hi && c == n - 1);
}

}  // namespace sld

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) and mbarrier helpers.  Every wait is bounded.
// ---------------------------------------------------------------------------
namespace sld {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy accesses before later
// async-proxy (TMA) accesses, in global and shared memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Orders this thread's generic shared-memory accesses before later
// async-proxy (TMA) accesses of the CTA's shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait until phase `parity` of the barrier has completed, at most timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > timeout_ns) return false;
  }
}

// Fetch a tensor map (here a __grid_constant__ kernel parameter) into the
// TMA unit's descriptor cache ahead of its first use.
__device__ __forceinline__ void prefetch_tensormap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace sld
