// fks_collide_f32_radix.cu -- FP32 instantiations of the collision kernel with alternative radix
// schedules of the length-n transforms (the autotuner's second dimension beside the cluster size).
#include "fks_internal.h"

namespace fks {

// top radix R0 of an n-point transform (default schedules: 32 = 4 x 8, 24 = 3 x 8, 16 = 4 x 4), at the
// default cluster size of each n
bool find_collide_variant_f32_radix(int N, int C, int R0, CollideVariant* out) {
    switch ((N * 16 + C) * 16 + R0) {
        case (32 * 16 + 8) * 16 + 2: return collide_variant<float, 32, 8, float, 2>(out);
        case (32 * 16 + 8) * 16 + 8: return collide_variant<float, 32, 8, float, 8>(out);
        case (24 * 16 + 2) * 16 + 2: return collide_variant<float, 24, 2, float, 2>(out);
        case (24 * 16 + 2) * 16 + 4: return collide_variant<float, 24, 2, float, 4>(out);
        case (24 * 16 + 2) * 16 + 8: return collide_variant<float, 24, 2, float, 8>(out);
        case (16 * 16 + 1) * 16 + 2: return collide_variant<float, 16, 1, float, 2>(out);
        case (16 * 16 + 1) * 16 + 8: return collide_variant<float, 16, 1, float, 8>(out);
        default: return false;
    }
}

}  // namespace fks
