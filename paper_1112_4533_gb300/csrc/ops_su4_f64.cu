// ops_su4_f64.cu -- SU(4), generic path, FP64: full storage (32 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su4_f64() { return ops_instance<double, 4, kFull>(); }
}  // namespace sun
