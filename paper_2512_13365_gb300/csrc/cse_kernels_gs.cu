// The step engine (cse_engine.cuh) instantiated with shared Greedy-
// Intersections coins (CSE_FLAG_GI_SHARED_COINS).  A separate translation
// unit, compiled in parallel with cse_kernels.cu, so that the option costs
// neither build time nor registers in the default engine.

#include "cse_engine.cuh"

namespace cse {

cudaError_t launch_round_gs(int W, bool gm, const DevMat* mats, int n_mats, const DevSearch* searches,
                            int total_units, int* work, const WarpLayout& L, int ppc, cudaStream_t stream,
                            bool prepare_only) {
    return launch_round_variant<true>(W, gm, mats, n_mats, searches, total_units, work, L, ppc, stream,
                                      prepare_only);
}

}  // namespace cse
