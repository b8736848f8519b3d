// Instances of the fiber-factored pass for order-3 tensors (one prefix mode).
#include "fiber.cuh"

namespace hoqri {

// k_fib<2, PP, KL> for the prefix rank PP and the last other mode's rank KL, and its
// shared memory per warp (4-byte words) with zs prefix floats per piece; false if none
bool fib_kernel3(int PP, int KL, int zs, const void **fn, int *warp_floats) {
#define HQ_FIB3(P, L)                                                  \
    if (PP == P && KL == L) {                                         \
        *fn = reinterpret_cast<const void *>(&k_fib<2, P, L>);     \
        *warp_floats = fib_warp_floats<P, L>(zs);                     \
        return true;                                                  \
    }
    HQ_FIB3(4, 8)
    HQ_FIB3(4, 16)
    HQ_FIB3(4, 32)
    HQ_FIB3(8, 4)
    HQ_FIB3(8, 8)
    HQ_FIB3(8, 16)
    HQ_FIB3(8, 32)
    HQ_FIB3(16, 4)
    HQ_FIB3(16, 8)
    HQ_FIB3(16, 16)
    HQ_FIB3(16, 32)
    HQ_FIB3(32, 4)
    HQ_FIB3(32, 8)
    HQ_FIB3(32, 16)
    HQ_FIB3(32, 32)
#undef HQ_FIB3
    return false;
}

}  // namespace hoqri
