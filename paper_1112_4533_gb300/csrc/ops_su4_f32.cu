// ops_su4_f32.cu -- SU(4), generic path, FP32: full storage (32 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su4_f32() { return ops_instance<float, 4, kFull>(); }
}  // namespace sun
