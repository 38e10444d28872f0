// tcgen05 (5th-generation tensor core) TF32 Gram kernel.
#include "internal.h"

namespace ttgb {

bool gram_rows_tc_tf32(Ctx& c, int n, long K, const float* X, long ldx, float* G) {
    (void)c; (void)n; (void)K; (void)X; (void)ldx; (void)G;
    return false;
}

}  // namespace ttgb
