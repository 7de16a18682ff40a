// ops_su2.cu -- SU(2): quaternion storage (4 reals, Eq. 6) and full 2x2 storage (8 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su2(int storage, int precision) {
  if (precision == 32) {
    if (storage == 4) return ops_instance<float, 2, kQuat>();
    if (storage == 8) return ops_instance<float, 2, kFull>();
  } else if (precision == 64) {
    if (storage == 4) return ops_instance<double, 2, kQuat>();
    if (storage == 8) return ops_instance<double, 2, kFull>();
  }
  return nullptr;
}
}  // namespace sun
