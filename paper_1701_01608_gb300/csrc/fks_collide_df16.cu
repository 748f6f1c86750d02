// fks_collide_df16.cu -- the collision kernel in double-float arithmetic over an FP32 state at n = 16
// (the last escalation tier; one translation unit per n, so that the large kernels compile in parallel).
#include "fks_internal.h"

namespace fks {

bool find_collide_variant_dfloat_16(CollideVariant* out) { return collide_variant<dfloat, 16, 2, float>(out); }

}  // namespace fks
