// ops_su6_f32.cu -- SU(6), generic path, FP32: full storage (72 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su6_f32() { return ops_instance<float, 6, kFull>(); }
}  // namespace sun
