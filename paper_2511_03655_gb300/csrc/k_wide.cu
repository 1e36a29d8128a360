// k_wide.cu -- instantiations and launcher of the wide (ragged-batch) kernel.
#include <cuda_runtime.h>

#include "irkgl.h"
#include "irkgl_wide.cuh"

namespace irkgl {


template <int TEAM, int BLOCK, int SLOTS, int MIX, int CVS>
void wide_launch(dim3 g, dim3 b, size_t smem, cudaStream_t st, const WideArgs& a, const Coef& c) {
  irkgl_wide_kernel<TEAM, BLOCK, SLOTS, MIX, CVS><<<g, b, smem, st>>>(a, c);
}

#define IRKGL_WIDE_SHAPE(TEAM, BLOCK, SLOTS, MIX, CVS)                                                \
  WideShape {                                                                                       \
    TEAM, BLOCK, SLOTS, MIX, CVS, (const void*)irkgl_wide_kernel<TEAM, BLOCK, SLOTS, MIX, CVS>,     \
        wide_launch<TEAM, BLOCK, SLOTS, MIX, CVS>                                                   \
  }
#define IRKGL_WIDE_MIX(TEAM, BLOCK, SLOTS, MIX) IRKGL_WIDE_SHAPE(TEAM, BLOCK, SLOTS, MIX, 1)
#define IRKGL_WIDE(TEAM, BLOCK, SLOTS) IRKGL_WIDE_MIX(TEAM, BLOCK, SLOTS, 0)

static const WideShape kWide[] = {
    IRKGL_WIDE(32, 128, 2),    // d <= 64, 4 instances per block
    IRKGL_WIDE(32, 64, 2),     // d <= 64, 2 instances per block
    IRKGL_WIDE(64, 64, 4),     // d <= 256
    IRKGL_WIDE(128, 128, 4),   // d <= 512
    IRKGL_WIDE(256, 256, 2),   // d <= 512
    IRKGL_WIDE(256, 256, 4),   // d <= 1024
    IRKGL_WIDE_SHAPE(256, 256, 6, 0, 0),  // d <= 1536, c_i v recomputed (shared memory)
    // fixed-point stage mixing (IRKGL_OPT_MIX = 1)
    IRKGL_WIDE_MIX(32, 128, 2, 1),
    IRKGL_WIDE_MIX(64, 64, 4, 1),
    IRKGL_WIDE_MIX(128, 128, 4, 1),
    IRKGL_WIDE_MIX(256, 256, 2, 1),
    IRKGL_WIDE_MIX(256, 256, 4, 1),
    IRKGL_WIDE_SHAPE(256, 256, 6, 1, 0),
};

int wide_shapes(const WideShape** out) {
  *out = kWide;
  return static_cast<int>(sizeof(kWide) / sizeof(kWide[0]));
}

}  // namespace irkgl
