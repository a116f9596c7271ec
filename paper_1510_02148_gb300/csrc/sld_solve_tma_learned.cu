// sld_solve_tma_learned.cu -- instantiations of the TMA-pipelined persistent
// solve with extra dense deflation columns (Z = [Z_lab, Z_L]): FP64 and the
// FP32 inner iteration.
#include "sld_solve_tma.cuh"

namespace sld {

int launch_solve_tma_learned(sld_system s, SolveArgs& a, const sld_options& o, float* ms, std::string* msg) {
  const bool wacc = a.d <= kWarpAccMaxD;
  if (a.bf16) {
    *msg = "extra dense deflation columns are not supported with BF16 coefficients";
    return SLD_ERR_INVALID_ARG;
  }
  if (a.fp64)
    return wacc ? launch_tma<double, double, 8, 3, true, true>(s, a, o, ms, msg)
                : launch_tma<double, double, 8, 3, false, true>(s, a, o, ms, msg);
  return wacc ? launch_tma<float, float, 16, 3, true, true>(s, a, o, ms, msg)
              : launch_tma<float, float, 16, 3, false, true>(s, a, o, ms, msg);
}

}  // namespace sld
