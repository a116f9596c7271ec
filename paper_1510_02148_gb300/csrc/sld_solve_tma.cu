// sld_solve_tma.cu -- instantiations of the TMA-pipelined persistent solve
// for label deflation alone (extra dense columns: sld_solve_tma_learned.cu).
#include <algorithm>
#include <cstring>
#include <memory>

#include "sld_solve_tma.cuh"

namespace sld {

// Row strides must be multiples of 16 bytes for every streamed array (the
// 16-bit labels are the narrowest): the FP32 and BF16 forms keep their inner
// arrays and labels at rows padded to 8 cells, so any grid qualifies; the
// FP64 form streams the unpadded FP64 operator: nx % 8 == 0.
bool tma_eligible(const Geo& g, bool fp64) { return (!fp64 || g.nx % 8 == 0) && encode_fn() != nullptr; }

// CTAs per SM of the 64 x 8-tile kernel for this coarse size.
template <typename F, bool WACC>
int tma_ctas_per_sm_8(const SolveArgs& a) {
  const size_t smem = tma_smem_bytes<float, F, 8, 3, WACC>(a.d, a.dk);
  auto kern = k_solve_tma<float, F, 8, 3, WACC, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 16 * 8, smem) != cudaSuccess) return 0;
  return per;
}

int launch_solve_tma(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg) {
  if (a.kL > 0) return launch_solve_tma_learned(s, a, o, ms, msg);
  const bool wacc = a.d <= kWarpAccMaxD;
  if (a.fp64)
    return wacc ? launch_tma<double, double, 8, 3, true, false>(s, a, o, ms, msg)
                : launch_tma<double, double, 8, 3, false, false>(s, a, o, ms, msg);
  // FP32 inner and BF16 faces: 64 x 8 tiles, 3-deep ring, four CTAs per SM
  // (on the 256 x 256 x 128 workload 1.5 % faster than 64 x 16 tiles at two
  // CTAs per SM, 10 % faster than 64 x 8 tiles with 4-deep rings or at three
  // CTAs per SM, 30 % faster than one CTA per SM).  When the coarse arrays in
  // shared memory (large d) leave room for fewer than four 64 x 8 CTAs, 64 x 16
  // tiles at two CTAs per SM (7 % faster at d = 1536 than three 64 x 8 CTAs).
  const int per8 = a.bf16 ? (wacc ? tma_ctas_per_sm_8<__nv_bfloat16, true>(a) : tma_ctas_per_sm_8<__nv_bfloat16, false>(a))
                          : (wacc ? tma_ctas_per_sm_8<float, true>(a) : tma_ctas_per_sm_8<float, false>(a));
  const bool small = per8 >= 4;
  if (a.bf16) {
    if (small)
      return wacc ? launch_tma<float, __nv_bfloat16, 8, 3, true, false>(s, a, o, ms, msg)
                  : launch_tma<float, __nv_bfloat16, 8, 3, false, false>(s, a, o, ms, msg);
    return wacc ? launch_tma<float, __nv_bfloat16, 16, 3, true, false>(s, a, o, ms, msg)
                : launch_tma<float, __nv_bfloat16, 16, 3, false, false>(s, a, o, ms, msg);
  }
  if (small)
    return wacc ? launch_tma<float, float, 8, 3, true, false>(s, a, o, ms, msg)
                : launch_tma<float, float, 8, 3, false, false>(s, a, o, ms, msg);
  return wacc ? launch_tma<float, float, 16, 3, true, false>(s, a, o, ms, msg)
              : launch_tma<float, float, 16, 3, false, false>(s, a, o, ms, msg);
}

// ---------------------------------------------------------------------------
// Batched FP32-inner solve on the TMA sweeps (64 x 8 tiles, 3-deep ring,
// four CTAs per SM, as the single solve).
// ---------------------------------------------------------------------------
constexpr int kBTY = 8;  // tile rows of the batched kernel

unsigned tma_batch_args_off(int dmax, bool wacc) {
  const size_t b = wacc ? tma_smem_bytes<float, float, kBTY, 3, true>(dmax, dmax)
                        : tma_smem_bytes<float, float, kBTY, 3, false>(dmax, dmax);
  return (unsigned)((b + 15) / 16 * 16);
}

size_t tma_batch_smem(int dmax, bool wacc) { return tma_batch_args_off(dmax, wacc) + sizeof(SolveArgs); }

int tma_batch_occupancy(bool wacc, size_t smem) {
  // both kernels (arguments in shared memory / in the parameter space) must fit
  const void* kerns[2] = {wacc ? (const void*)k_solve_tma_batch<float, float, kBTY, 3, true>
                               : (const void*)k_solve_tma_batch<float, float, kBTY, 3, false>,
                          wacc ? (const void*)k_solve_tma_batch_p<float, float, kBTY, 3, true>
                               : (const void*)k_solve_tma_batch_p<float, float, kBTY, 3, false>};
  int best = 1 << 30;
  for (const void* kern : kerns) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 16 * kBTY, smem);
    best = std::min(best, per);
  }
  return best;
}

int tma_batch_param_max() { return kBatchParamMax; }

void tma_batch_tiles(SolveArgs* a) {
  a->ntx = (a->g.nx + kTX - 1) / kTX;
  a->nty = (a->g.ny + kBTY - 1) / kBTY;
  a->ntiles = (int64_t)a->ntx * a->nty * a->g.nz;
}

size_t tma_maps_bytes() { return sizeof(Maps); }

bool tma_batch_maps(const SolveArgs& a, void* out) { return build_maps<float, float, kBTY>(a, static_cast<Maps*>(out)); }

cudaError_t tma_batch_launch(int G, size_t smem, unsigned args_off, bool wacc, const SolveArgs* d_args,
                             const SolveArgs* h_args, int count, const void* d_maps, const int* d_cta,
                             cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(16 * kBTY);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const Maps* mp = static_cast<const Maps*>(d_maps);
  if (h_args && count <= kBatchParamMax) {
    // host staging of the parameter: the launch (or the graph capture) copies it
    auto P = std::make_unique<BatchParam>();
    std::memset(P.get(), 0, sizeof(BatchParam));
    std::memcpy(P->a, h_args, sizeof(SolveArgs) * count);
    if (wacc) return cudaLaunchKernelEx(&cfg, k_solve_tma_batch_p<float, float, kBTY, 3, true>, *P, mp, d_cta);
    return cudaLaunchKernelEx(&cfg, k_solve_tma_batch_p<float, float, kBTY, 3, false>, *P, mp, d_cta);
  }
  if (wacc) return cudaLaunchKernelEx(&cfg, k_solve_tma_batch<float, float, kBTY, 3, true>, d_args, mp, d_cta, args_off);
  return cudaLaunchKernelEx(&cfg, k_solve_tma_batch<float, float, kBTY, 3, false>, d_args, mp, d_cta, args_off);
}

}  // namespace sld
