// fks_collide_df32.cu -- the collision kernel in double-float arithmetic over an FP32 state at n = 32
// (the last escalation tier; one translation unit per n, so that the large kernels compile in parallel).
#include "fks_internal.h"

namespace fks {

bool find_collide_variant_dfloat_32(CollideVariant* out) { return collide_variant<dfloat, 32, 8, float>(out); }

}  // namespace fks
