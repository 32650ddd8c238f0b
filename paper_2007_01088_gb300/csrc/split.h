// Split-precision (BF16 slice) path of libcc3.
#pragma once
#include "cc3_internal.h"

namespace cc3 {
int split_omega(cc3_ctx *c, cudaStream_t s);
void split_invalidate(cc3_ctx *c);
void split_destroy(cc3_ctx *c);
size_t split_footprint(int no, int nv, int slices, int ntri);
}  // namespace cc3
