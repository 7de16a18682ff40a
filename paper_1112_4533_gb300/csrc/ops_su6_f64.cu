// ops_su6_f64.cu -- SU(6), generic path, FP64: full storage (72 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su6_f64() { return ops_instance<double, 6, kFull>(); }
}  // namespace sun
