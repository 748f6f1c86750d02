// fks_collide_mixed.cu -- the collision kernel with FP64 arithmetic over an FP32 state: the last
// tier of the precision escalation of FP32 and split-BF16 contexts (cells near equilibrium, where
// the gain and the loss cancel to a few digits and FP32 transforms cannot reach the tolerance).
#include "fks_internal.h"

namespace fks {

template <int N, int C>
static bool variant(CollideVariant* out) {
    using Cfg = CollideCfg<double, N, C>;
    out->func = reinterpret_cast<const void*>(&collide_kernel<double, N, C, false, float>);
    out->func_batch = reinterpret_cast<const void*>(&collide_kernel<double, N, C, true, float>);
    out->N = N;
    out->C = C;
    out->NT = Cfg::NT;
    out->smem = Cfg::SMEM_BYTES;
    out->fp64 = true;
    return true;
}

// one cluster size per n: the FP64 default
bool find_collide_variant_mixed(int N, int C, CollideVariant* out) {
    switch (N * 16 + C) {
        case 8 * 16 + 1: return variant<8, 1>(out);
        case 16 * 16 + 2: return variant<16, 2>(out);
        case 24 * 16 + 4: return variant<24, 4>(out);
        case 32 * 16 + 8: return variant<32, 8>(out);
        default: return false;
    }
}

}  // namespace fks
