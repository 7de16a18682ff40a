// ops_su5_f32.cu -- SU(5), generic path, FP32: full storage (50 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su5_f32() { return ops_instance<float, 5, kFull>(); }
}  // namespace sun
