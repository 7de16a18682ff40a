// ops_su6.cu -- SU(6), generic path: full storage (72 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su6(int storage, int precision) {
  if (storage != 72) return nullptr;
  if (precision == 32) return ops_instance<float, 6, kFull>();
  if (precision == 64) return ops_instance<double, 6, kFull>();
  return nullptr;
}
}  // namespace sun
