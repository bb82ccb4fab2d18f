// Tensor-core delayed flush (placeholder until the tcgen05 kernel lands).
#include "internal.h"

namespace lru {

bool launch_flush_tc(int mode, bool pf, const DevLayout& L, double* G, const float* Ph, const float* Pl,
                     const float* Qh, const float* Ql, const int* tau, const uint8_t* force_mask, int* err,
                     cudaStream_t st) {
    (void)mode; (void)pf; (void)L; (void)G; (void)Ph; (void)Pl; (void)Qh; (void)Ql; (void)tau;
    (void)force_mask; (void)err; (void)st;
    return false;
}

}  // namespace lru
