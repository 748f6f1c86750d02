// fks_collide_df8.cu -- the collision kernel in double-float arithmetic over an FP32 state at n = 8
// (the last escalation tier; one translation unit per n, so that the large kernels compile in parallel).
#include "fks_internal.h"

namespace fks {

bool find_collide_variant_dfloat_8(CollideVariant* out) { return collide_variant<dfloat, 8, 1, float>(out); }

}  // namespace fks
