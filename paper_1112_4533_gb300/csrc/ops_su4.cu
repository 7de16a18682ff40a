// ops_su4.cu -- SU(4), generic path: full storage (32 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su4(int storage, int precision) {
  if (storage != 32) return nullptr;
  if (precision == 32) return ops_instance<float, 4, kFull>();
  if (precision == 64) return ops_instance<double, 4, kFull>();
  return nullptr;
}
}  // namespace sun
