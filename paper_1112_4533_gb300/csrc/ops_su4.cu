// ops_su4.cu -- SU(4), generic path: full storage (32 reals), FP32 and FP64 units.
#include "sun_runtime.h"

namespace sun {
const Ops* ops_su4(int storage, int precision) {
  if (storage != 32) return nullptr;
  if (precision == 32) return ops_su4_f32();
  if (precision == 64) return ops_su4_f64();
  return nullptr;
}
}  // namespace sun
