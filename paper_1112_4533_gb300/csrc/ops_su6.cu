// ops_su6.cu -- SU(6), generic path: full storage (72 reals), FP32 and FP64 units.
#include "sun_runtime.h"

namespace sun {
const Ops* ops_su6(int storage, int precision) {
  if (storage != 72) return nullptr;
  if (precision == 32) return ops_su6_f32();
  if (precision == 64) return ops_su6_f64();
  return nullptr;
}
}  // namespace sun
