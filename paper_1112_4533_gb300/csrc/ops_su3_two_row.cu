// ops_su3_two_row.cu -- SU(3) in two-row storage: rows 0 and 1 stored (12 reals, Sec. 3),
// the third row rebuilt as conj(row0 x row1).
#include "sun_kernels.cuh"

namespace sun {
const Ops* ops_su3_two_row(int precision) {
  if (precision == 32) return ops_instance<float, 3, kTwoRow>();
  if (precision == 64) return ops_instance<double, 3, kTwoRow>();
  return nullptr;
}
}  // namespace sun
