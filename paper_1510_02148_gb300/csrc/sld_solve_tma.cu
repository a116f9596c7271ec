// sld_solve_tma.cu -- instantiations of the TMA-pipelined persistent solve
// for label deflation alone (extra dense columns: sld_solve_tma_learned.cu).
#include "sld_solve_tma.cuh"

namespace sld {

// Row strides must be multiples of 16 bytes for every streamed array (the
// 16-bit labels are the narrowest): nx % 8 == 0.
bool tma_eligible(const Geo& g) { return g.nx % 8 == 0 && encode_fn() != nullptr; }

int launch_solve_tma(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg) {
  if (a.kL > 0) return launch_solve_tma_learned(s, a, o, ms, msg);
  const bool wacc = a.d <= kWarpAccMaxD;
  if (a.fp64)
    return wacc ? launch_tma<double, double, 8, 3, true, false>(s, a, o, ms, msg)
                : launch_tma<double, double, 8, 3, false, false>(s, a, o, ms, msg);
  if (a.bf16)
    return wacc ? launch_tma<float, __nv_bfloat16, 16, 3, true, false>(s, a, o, ms, msg)
                : launch_tma<float, __nv_bfloat16, 16, 3, false, false>(s, a, o, ms, msg);
  // FP32 inner: 64 x 16 tiles, 3-deep ring (measured faster than 64 x 8
  // tiles with 4- or 5-deep rings on the 256 x 256 x 128 workload)
  return wacc ? launch_tma<float, float, 16, 3, true, false>(s, a, o, ms, msg)
              : launch_tma<float, float, 16, 3, false, false>(s, a, o, ms, msg);
}

}  // namespace sld
