// sld_cc.cu -- automatic subdomain-levelset labels: every (subdomain,
// levelset class) region of the plain labels split into its face-connected
// components, one deflation vector per component (Section 3.2.2's
// subdomain-levelset vectors, built without manual input the way the
// physics-based vectors of Section 4 take one vector per layer).
// Canonical numbering: components ordered by (plain SLD label, smallest cell
// index of the component), numbered 0, 1, ...
//
//   k_cc_init     parent[i] = i
//   k_cc_hook     unite i with its +x, +y, +z neighbour when both carry the
//                 same plain label: lock-free union-find that always hooks
//                 the larger root under the smaller one (parent[i] <= i
//                 throughout), with path halving in the root search
//                 (Jaiganesh and Burtscher's ECL-CC scheme).  Every loop
//                 strictly decreases a cell index, so it ends.
//   k_cc_flatten  root[i] = the root of i = the smallest cell of its
//                 component, into a separate array: the path halving of
//                 other threads may still rewrite parent[] with non-root
//                 ancestors while this pass runs
//   k_cc_count    heads (root[i] == i) per block of cells
//   k_cc_scan     exclusive prefix of the block counts (one CTA)
//   k_cc_compact  the heads in cell order, and each head's rank
//   k_cc_number   one thread: counting sort of the heads by plain label
//                 (stable, so by smallest cell within a label)
//   k_cc_relabel  label[i] = number of the head of i's component
#include <cuda_runtime.h>

#include <climits>
#include <string>

#include "sld_internal.h"

namespace sld {
namespace {

constexpr int kCB = 1024;  // cells per block in the counting passes

__global__ void k_cc_init(int n, int* __restrict__ parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = i;
}

// Root of i with path halving; parent[x] <= x always, so the walk strictly
// decreases and ends.
__device__ __forceinline__ int cc_root(volatile int* parent, int i) {
  int cur = parent[i];
  if (cur != i) {
    int prev = i, next;
    while (cur > (next = parent[cur])) {
      parent[prev] = next;
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

__device__ __forceinline__ void cc_unite(int* parent, int a, int b) {
  volatile int* vp = parent;
  int ra = cc_root(vp, a), rb = cc_root(vp, b);
  while (ra != rb) {  // each failed CAS moves ra or rb to a strictly smaller cell
    if (ra < rb) {
      const int old = atomicCAS(parent + rb, rb, ra);
      if (old == rb) break;
      rb = old;
    } else {
      const int old = atomicCAS(parent + ra, ra, rb);
      if (old == ra) break;
      ra = old;
    }
  }
}

__global__ void k_cc_hook(Geo g, const int32_t* __restrict__ label, int* parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int)g.n) return;
  const int ix = i % g.nx, iy = (i / g.nx) % g.ny, iz = i / (int)g.nxy;
  const int32_t l = label[i];
  if (ix + 1 < g.nx && label[i + 1] == l) cc_unite(parent, i, i + 1);
  if (iy + 1 < g.ny && label[i + g.nx] == l) cc_unite(parent, i, i + g.nx);
  if (iz + 1 < g.nz && label[i + (int)g.nxy] == l) cc_unite(parent, i, i + (int)g.nxy);
}

__global__ void k_cc_flatten(int n, int* parent, int* __restrict__ root) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) root[i] = cc_root(parent, i);
}

__device__ __forceinline__ int block_excl(int flag, int* warp_tot, int* total) {
  // exclusive prefix of flag over the CTA in thread order; *total = CTA sum
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[warp] = __popc(bal);
  __syncthreads();
  int before = 0, tot = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    if (w < warp) before += warp_tot[w];
    tot += warp_tot[w];
  }
  *total = tot;
  return before + in_warp;
}

__global__ void k_cc_count(int n, const int* __restrict__ root, int* __restrict__ bcount) {
  __shared__ int wt[kCB / 32];
  const int i = blockIdx.x * kCB + threadIdx.x;
  int tot = 0;
  block_excl(i < n && root[i] == i, wt, &tot);
  if (threadIdx.x == 0) bcount[blockIdx.x] = tot;
}

// exclusive prefix of nb block counts in place; *total = their sum (one CTA of kCB threads)
__global__ void k_cc_scan(int nb, int* __restrict__ bcount, int* __restrict__ total) {
  __shared__ int part[kCB];
  const int per = (nb + kCB - 1) / kCB;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; ++b) s += bcount[b];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < kCB; ++t) {
      const int v = part[t];
      part[t] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int b = b0; b < b1; ++b) {
    const int v = bcount[b];
    bcount[b] = run;
    run += v;
  }
}

__global__ void k_cc_compact(int n, const int* __restrict__ root, const int* __restrict__ boff,
                             int* __restrict__ heads, int* __restrict__ hrank) {
  __shared__ int wt[kCB / 32];
  const int i = blockIdx.x * kCB + threadIdx.x;
  const bool h = i < n && root[i] == i;
  int tot = 0;
  const int r = boff[blockIdx.x] + block_excl(h, wt, &tot);
  if (h) {
    heads[r] = i;
    hrank[i] = r;
  }
}

// number[r] for the H heads (in cell order): counting sort by plain label,
// stable.  cnt: d0 + 1 ints of scratch.
__global__ void k_cc_number(int H, int d0, const int* __restrict__ heads, const int32_t* __restrict__ base,
                            int* __restrict__ cnt, int* __restrict__ number) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int k = 0; k <= d0; ++k) cnt[k] = 0;
  for (int r = 0; r < H; ++r) ++cnt[base[heads[r]]];
  int run = 0;
  for (int k = 0; k < d0; ++k) {
    const int v = cnt[k];
    cnt[k] = run;
    run += v;
  }
  for (int r = 0; r < H; ++r) number[r] = cnt[base[heads[r]]]++;
}

__global__ void k_cc_relabel(int n, const int* __restrict__ root, const int* __restrict__ hrank,
                             const int* __restrict__ number, int32_t* __restrict__ label) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) label[i] = number[hrank[root[i]]];
}

unsigned nb_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int run_cc_labels(sld_system s, int d0, int maxd, int* d_out, std::string* msg) {
  const int64_t n64 = s->g.n;
  if (n64 > INT_MAX) {
    *msg = "automatic labels need fewer than 2^31 cells";
    return SLD_ERR_INVALID_ARG;
  }
  const int n = (int)n64;
  cudaStream_t st = s->stream;
  const int nb = (int)nb_of(n, kCB);
  int *parent = nullptr, *root = nullptr, *hrank = nullptr, *bcount = nullptr, *small = nullptr;
  auto release = [&]() {
    cudaFree(parent);
    cudaFree(root);
    cudaFree(hrank);
    cudaFree(bcount);
    cudaFree(small);
  };
  cudaError_t e = cudaMalloc(&parent, sizeof(int) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&root, sizeof(int) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&hrank, sizeof(int) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&bcount, sizeof(int) * ((size_t)nb + 1));
  if (e != cudaSuccess) {
    release();
    *msg = std::string("automatic labels: ") + cudaGetErrorString(e);
    return SLD_ERR_OOM;
  }
  k_cc_init<<<nb_of(n, 256), 256, 0, st>>>(n, parent);
  k_cc_hook<<<nb_of(n, 256), 256, 0, st>>>(s->g, s->label, parent);
  k_cc_flatten<<<nb_of(n, 256), 256, 0, st>>>(n, parent, root);
  k_cc_count<<<nb, kCB, 0, st>>>(n, root, bcount);
  k_cc_scan<<<1, kCB, 0, st>>>(nb, bcount, bcount + nb);
  int H = 0;
  if ((e = cudaMemcpyAsync(&H, bcount + nb, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    release();
    *msg = std::string("automatic labels: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  *d_out = H;
  if (H > maxd) {
    release();
    *msg = "automatic labels: " + std::to_string(H) + " components exceed the limit of " + std::to_string(maxd) +
           " (use fewer thresholds or larger subdomains)";
    return SLD_ERR_INVALID_ARG;
  }
  // small: heads (H), number (H), counting-sort scratch (d0 + 1)
  if ((e = cudaMalloc(&small, sizeof(int) * ((size_t)2 * H + d0 + 1))) != cudaSuccess) {
    release();
    *msg = std::string("automatic labels: ") + cudaGetErrorString(e);
    return SLD_ERR_OOM;
  }
  int *heads = small, *number = small + H, *cnt = small + 2 * H;
  k_cc_compact<<<nb, kCB, 0, st>>>(n, root, bcount, heads, hrank);
  k_cc_number<<<1, 32, 0, st>>>(H, d0, heads, s->label, cnt, number);
  k_cc_relabel<<<nb_of(n, 256), 256, 0, st>>>(n, root, hrank, number, s->label);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  release();
  if (e != cudaSuccess) {
    *msg = std::string("automatic labels: ") + cudaGetErrorString(e);
    return SLD_ERR_CUDA;
  }
  return SLD_OK;
}

}  // namespace sld
