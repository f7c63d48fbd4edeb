// Tensor-core (tcgen05) exact Gram with BF16 hi/lo split channel entries.
#include "common.cuh"

namespace xl {

int launch_gram_tc(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st) {
    (void)g; (void)users; (void)K; (void)B; (void)gram; (void)st;
    set_error("XLMIMO_BF16X3 is not available in this build");
    return XLMIMO_EUNSUPPORTED;
}

}  // namespace xl
