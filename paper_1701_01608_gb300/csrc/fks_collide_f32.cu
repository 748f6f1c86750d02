// fks_collide_f32.cu -- FP32 instantiations of the per-cell collision kernel.
#include "fks_internal.h"

namespace fks {

template <int N, int C>
static bool variant(CollideVariant* out) {
    using Cfg = CollideCfg<float, N, C>;
    out->func = reinterpret_cast<const void*>(&collide_kernel<float, N, C, false>);
    out->func_batch = reinterpret_cast<const void*>(&collide_kernel<float, N, C, true>);
    out->N = N;
    out->C = C;
    out->NT = Cfg::NT;
    out->smem = Cfg::SMEM_BYTES;
    out->fp64 = false;
    return true;
}

bool find_collide_variant_f32(int N, int C, CollideVariant* out) {
    switch (N * 16 + C) {
        case 8 * 16 + 1: return variant<8, 1>(out);
        case 8 * 16 + 2: return variant<8, 2>(out);
        case 16 * 16 + 1: return variant<16, 1>(out);
        case 16 * 16 + 2: return variant<16, 2>(out);
        case 24 * 16 + 2: return variant<24, 2>(out);
        case 24 * 16 + 4: return variant<24, 4>(out);
        case 32 * 16 + 4: return variant<32, 4>(out);
        case 32 * 16 + 8: return variant<32, 8>(out);
        case 32 * 16 + 16: return variant<32, 16>(out);
        default: return false;
    }
}

}  // namespace fks
