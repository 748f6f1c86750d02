// fks_collide_mixed.cu -- the collision kernel with FP64-accurate arithmetic over an FP32 state:
// the last tier of the precision escalation of FP32 and split-BF16 contexts (cells near
// equilibrium, where the gain and the loss cancel to a few digits and FP32 transforms cannot
// reach the tolerance).  Two arithmetics: FP64, and double-float pairs on the FP32 pipes (about
// 48 bits; GB300's FP64 pipe runs at 1/64 of its FP32 rate).
#include "fks_internal.h"

namespace fks {

template <typename T, int N, int C>
static bool variant(CollideVariant* out) {
    using Cfg = CollideCfg<T, N, C>;
    out->func = reinterpret_cast<const void*>(&collide_kernel<T, N, C, false, float>);
    out->func_batch = reinterpret_cast<const void*>(&collide_kernel<T, N, C, true, float>);
    out->N = N;
    out->C = C;
    out->NT = Cfg::NT;
    out->smem = Cfg::SMEM_BYTES;
    out->fp64 = true;
    return true;
}

// one cluster size per n: the FP64 default
template <typename T>
static bool find(int N, int C, CollideVariant* out) {
    switch (N * 16 + C) {
        case 8 * 16 + 1: return variant<T, 8, 1>(out);
        case 16 * 16 + 2: return variant<T, 16, 2>(out);
        case 24 * 16 + 4: return variant<T, 24, 4>(out);
        case 32 * 16 + 8: return variant<T, 32, 8>(out);
        default: return false;
    }
}

bool find_collide_variant_mixed(int N, int C, CollideVariant* out) { return find<double>(N, C, out); }
bool find_collide_variant_dfloat(int N, int C, CollideVariant* out) { return find<dfloat>(N, C, out); }

}  // namespace fks
