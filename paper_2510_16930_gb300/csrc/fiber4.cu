// Instances of the fiber-factored pass for order-4 tensors (two prefix modes,
// PP = K_a * K_b; the split of PP is a launch argument).
#include "fiber.cuh"

namespace hoqri {

// k_fib<3, PP, KL> for the prefix rank product PP and the last other mode's rank KL, and
// its shared memory per warp (4-byte words) with zs prefix floats per piece; false if none
bool fib_kernel4(int PP, int KL, int zs, const void **fn, int *warp_floats) {
#define HQ_FIB4(P, L)                                                  \
    if (PP == P && KL == L) {                                         \
        *fn = reinterpret_cast<const void *>(&k_fib<3, P, L>);     \
        *warp_floats = fib_warp_floats<P, L>(zs);                     \
        return true;                                                  \
    }
    HQ_FIB4(16, 4)
    HQ_FIB4(16, 8)
    HQ_FIB4(16, 16)
    HQ_FIB4(16, 32)
    HQ_FIB4(32, 4)
    HQ_FIB4(32, 8)
    HQ_FIB4(32, 16)
    HQ_FIB4(32, 32)
    HQ_FIB4(64, 4)
    HQ_FIB4(64, 8)
    HQ_FIB4(64, 16)
    HQ_FIB4(128, 4)
    HQ_FIB4(128, 8)
    HQ_FIB4(256, 4)
#undef HQ_FIB4
    return false;
}

}  // namespace hoqri
