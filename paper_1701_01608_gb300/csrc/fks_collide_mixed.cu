// fks_collide_mixed.cu -- the collision kernel with FP64-accurate arithmetic over an FP32 state:
// the last tier of the precision escalation of FP32 and split-BF16 contexts (cells near
// equilibrium, where the gain and the loss cancel to a few digits and FP32 transforms cannot
// reach the tolerance).  Two arithmetics: FP64, and double-float pairs on the FP32 pipes (about
// 48 bits; GB300's FP64 pipe runs at 1/64 of its FP32 rate).
#include "fks_internal.h"

namespace fks {

// one cluster size per n: the FP64 default.  The double-float instantiations sit in translation
// units of their own (fks_collide_df*.cu), compiled in parallel: each is a large kernel.
bool find_collide_variant_mixed(int N, int C, CollideVariant* out) {
    switch (N * 16 + C) {
        case 8 * 16 + 1: return collide_variant<double, 8, 1, float>(out);
        case 16 * 16 + 2: return collide_variant<double, 16, 2, float>(out);
        case 24 * 16 + 4: return collide_variant<double, 24, 4, float>(out);
        case 32 * 16 + 8: return collide_variant<double, 32, 8, float>(out);
        default: return false;
    }
}

bool find_collide_variant_dfloat(int N, int C, CollideVariant* out) {
    switch (N * 16 + C) {
        case 8 * 16 + 1: return find_collide_variant_dfloat_8(out);
        case 16 * 16 + 2: return find_collide_variant_dfloat_16(out);
        case 24 * 16 + 4: return find_collide_variant_dfloat_24(out);
        case 32 * 16 + 8: return find_collide_variant_dfloat_32(out);
        default: return false;
    }
}

}  // namespace fks
