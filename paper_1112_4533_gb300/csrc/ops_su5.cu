// ops_su5.cu -- SU(5), generic path: full storage (50 reals), FP32 and FP64 units.
#include "sun_runtime.h"

namespace sun {
const Ops* ops_su5(int storage, int precision) {
  if (storage != 50) return nullptr;
  if (precision == 32) return ops_su5_f32();
  if (precision == 64) return ops_su5_f64();
  return nullptr;
}
}  // namespace sun
