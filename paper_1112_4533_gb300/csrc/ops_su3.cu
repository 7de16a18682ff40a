// ops_su3.cu -- SU(3): two-row storage (12 reals, third row rebuilt) and full storage (18 reals),
// instantiated in ops_su3_two_row.cu and ops_su3_full.cu.
#include "sun_runtime.h"

namespace sun {
const Ops* ops_su3(int storage, int precision) {
  if (storage == 12) return ops_su3_two_row(precision);
  if (storage == 18) return ops_su3_full(precision);
  return nullptr;
}
}  // namespace sun
