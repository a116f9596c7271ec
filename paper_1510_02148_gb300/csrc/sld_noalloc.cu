// sld_noalloc.cu -- sld_restrict_noalloc: out = Z^T v (the segmented sum over
// labels) without allocating device memory.
//
// For callers that cannot call cudaMalloc: code running where the device
// memory is already handed out to another allocator (a framework's pool or
// arena, a hard memory cap), and loops that must not pay for cudaMalloc /
// cudaFree, which can block and (cudaFree) synchronise the whole device.
//
// The per-CTA partial sums live in a file-scope __device__ array of fixed
// size (kNoAllocCtas x kNoAllocMaxD doubles = 1 MiB).  Every GPU that loads
// this library holds that array until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is
// fetched with cudaGetSymbolAddress once per device, on the first call made
// with that device current, and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sld_internal.h"

namespace {

constexpr int kNoAllocCtas = 128;   // CTAs of the partial-sum pass (grid-stride over cells)
constexpr int kNoAllocMaxD = 1024;  // largest d this entry point takes
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device; each call overwrites the rows it reads,
// so nothing has to start at zero.  Calls whose kernels overlap on the GPU
// (two streams, or two host threads) race on it.
static __device__ __align__(256) double g_restrict_scratch[kNoAllocCtas * kNoAllocMaxD];

std::mutex g_mu;
double* g_scratch_addr[kNoAllocMaxDevices] = {};

sld_status na_fail(sld_status st, const std::string& m) {
  sld::set_last_error(m);  // read back with sld_last_error()
  return st;
}

// Pass 1: CTA b sums v over the cells it visits into shared memory and writes
// all d sums (zeros included) to row b of the scratch array.
__global__ void k_restrict_partials(int64_t n, int d, const int32_t* __restrict__ label,
                                    const double* __restrict__ v, double* __restrict__ scratch) {
  extern __shared__ double sacc[];
  for (int k = threadIdx.x; k < d; k += blockDim.x) sacc[k] = 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(&sacc[label[i]], v[i]);
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x) scratch[(int64_t)blockIdx.x * d + k] = sacc[k];
}

// Pass 2: out[k] = sum over the rows of the scratch array, in row order.
__global__ void k_restrict_finish(int d, int rows, const double* __restrict__ scratch, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d) return;
  double t = 0.0;
  for (int b = 0; b < rows; ++b) t += scratch[(int64_t)b * d + k];
  out[k] = t;
}

// True when the kernels of device `dev` may read p directly: device memory of
// that same GPU, or managed memory.  Device memory of another GPU is refused:
// this entry point copies nothing, and a direct read of a peer's memory
// without peer access enabled is an illegal address.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" {

sld_status sld_restrict_noalloc(sld_system s, const double* v, double* out) {
  sld::set_last_error("");
  if (!s || !v || !out) return na_fail(SLD_ERR_INVALID_ARG, "NULL argument");
  if (!s->label || s->d < 1) return na_fail(SLD_ERR_STATE, "no deflation built");
  if (s->d > kNoAllocMaxD)
    return na_fail(SLD_ERR_INVALID_ARG, "sld_restrict_noalloc takes d <= " + std::to_string(kNoAllocMaxD) +
                                            " (its scratch holds " + std::to_string(kNoAllocCtas) + " x " +
                                            std::to_string(kNoAllocMaxD) + " partial sums); d = " +
                                            std::to_string(s->d));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(SLD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != s->device || dev < 0 || dev >= kNoAllocMaxDevices)
    return na_fail(SLD_ERR_INVALID_ARG, "make the handle's device current before the call");
  if (!on_device(v, dev) || !on_device(out, dev))
    return na_fail(SLD_ERR_INVALID_ARG,
                   "v and out must be device memory of the handle's GPU (this entry point stages nothing)");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_restrict_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(SLD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  const int d = s->d;
  k_restrict_partials<<<kNoAllocCtas, 256, sizeof(double) * d, s->stream>>>(s->g.n, d, s->label, v, scratch);
  k_restrict_finish<<<(d + 127) / 128, 128, 0, s->stream>>>(d, kNoAllocCtas, scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(SLD_ERR_CUDA, std::string("restrict kernels: ") + cudaGetErrorString(e));
  return SLD_OK;
}

}  // extern "C"
