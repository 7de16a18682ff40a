// ops_su3_full.cu -- SU(3) in full storage (18 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su3_full(int precision) {
  if (precision == 32) return ops_instance<float, 3, kFull>();
  if (precision == 64) return ops_instance<double, 3, kFull>();
  return nullptr;
}
}  // namespace sun
