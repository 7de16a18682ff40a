// ops_su5.cu -- SU(5), generic path: full storage (50 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su5(int storage, int precision) {
  if (storage != 50) return nullptr;
  if (precision == 32) return ops_instance<float, 5, kFull>();
  if (precision == 64) return ops_instance<double, 5, kFull>();
  return nullptr;
}
}  // namespace sun
