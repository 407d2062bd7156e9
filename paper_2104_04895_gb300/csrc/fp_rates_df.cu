// FP64-accurate instantiations whose vertex contraction runs in double-float on the FP32 pipes
// (FP_PREC_DOUBLE_FLOAT), for 1, 2 and 4 atoms per cell.
#include "fp_rates_kernel.cuh"

namespace fp {
const void* rates_kernel_df(int nb, int maxt) {
  switch (nb * 100 + maxt) {
    case 301: return reinterpret_cast<const void*>(rates_kernel<double, 3, 1, false, true>);
    case 308: return reinterpret_cast<const void*>(rates_kernel<double, 3, kMaxT, false, true>);
    case 601: return reinterpret_cast<const void*>(rates_kernel<double, 6, 1, false, true>);
    case 608: return reinterpret_cast<const void*>(rates_kernel<double, 6, kMaxT, false, true>);
    case 1201: return reinterpret_cast<const void*>(rates_kernel<double, 12, 1, false, true>);
    case 1208: return reinterpret_cast<const void*>(rates_kernel<double, 12, kMaxT, false, true>);
    default: return nullptr;
  }
}
}  // namespace fp
