// ops_su3.cu -- SU(3): two-row storage (12 reals, third row rebuilt) and full storage (18 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su3(int storage, int precision) {
  if (precision == 32) {
    if (storage == 12) return ops_instance<float, 3, kTwoRow>();
    if (storage == 18) return ops_instance<float, 3, kFull>();
  } else if (precision == 64) {
    if (storage == 12) return ops_instance<double, 3, kTwoRow>();
    if (storage == 18) return ops_instance<double, 3, kFull>();
  }
  return nullptr;
}
}  // namespace sun
