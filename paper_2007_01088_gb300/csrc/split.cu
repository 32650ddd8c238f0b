// Split-precision path (placeholder until the tcgen05 kernels land).
#include "split.h"

namespace cc3 {
int split_omega(cc3_ctx *, cudaStream_t) { return CC3_ERR_UNSUPPORTED; }
void split_invalidate(cc3_ctx *) {}
void split_destroy(cc3_ctx *) {}
}  // namespace cc3
