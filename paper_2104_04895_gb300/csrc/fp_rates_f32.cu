// Mixed-precision (FP32 vertex) instantiations of the rate kernel for 1, 2 and 4 atoms per cell.
#include "fp_rates_kernel.cuh"

namespace fp {
const void* rates_kernel_f32(int nb, int maxt) {
  switch (nb * 100 + maxt) {
    case 301: return reinterpret_cast<const void*>(rates_kernel<float, 3, 1>);
    case 308: return reinterpret_cast<const void*>(rates_kernel<float, 3, kMaxT>);
    case 601: return reinterpret_cast<const void*>(rates_kernel<float, 6, 1>);
    case 608: return reinterpret_cast<const void*>(rates_kernel<float, 6, kMaxT>);
    case 1201: return reinterpret_cast<const void*>(rates_kernel<float, 12, 1>);
    case 1208: return reinterpret_cast<const void*>(rates_kernel<float, 12, kMaxT>);
    default: return nullptr;
  }
}
// the tensor-core T contraction (nb = 6 only)
const void* rates_kernel_f32_tc(int nb, int maxt) {
  if (nb != 6) return nullptr;
  return maxt == 1 ? reinterpret_cast<const void*>(rates_kernel<float, 6, 1, true>)
                   : reinterpret_cast<const void*>(rates_kernel<float, 6, kMaxT, true>);
}
}  // namespace fp
