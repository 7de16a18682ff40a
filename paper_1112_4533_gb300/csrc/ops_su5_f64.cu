// ops_su5_f64.cu -- SU(5), generic path, FP64: full storage (50 reals).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su5_f64() { return ops_instance<double, 5, kFull>(); }
}  // namespace sun
