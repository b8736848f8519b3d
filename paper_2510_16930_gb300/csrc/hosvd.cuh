// HOSVD initialisation of the factors (hosvd.cu).
#pragma once

#include "internal.cuh"

namespace hoqri {

// factors <- orthonormal bases of the leading left singular subspaces of the
// unfoldings, power_iters steps of orthogonal iteration from the seeded start
hoqri_status init_hosvd(hoqri_ctx *c, int power_iters);

}  // namespace hoqri
