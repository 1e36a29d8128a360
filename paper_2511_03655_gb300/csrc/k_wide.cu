// k_wide.cu -- instantiations and launcher of the wide (ragged-batch) kernel.
#include <cuda_runtime.h>

#include "irkgl.h"
#include "irkgl_wide.cuh"

namespace irkgl {

// Team shapes: one warp per instance (small d), or the whole block.
struct WideShape {
  int team, block, slots;
  const void* fn;
  void (*launch)(dim3, dim3, size_t, cudaStream_t, const WideArgs&, const Coef&);
};
int wide_shapes(const WideShape** out);

template <int TEAM, int BLOCK, int SLOTS>
void wide_launch(dim3 g, dim3 b, size_t smem, cudaStream_t st, const WideArgs& a, const Coef& c) {
  irkgl_wide_kernel<TEAM, BLOCK, SLOTS><<<g, b, smem, st>>>(a, c);
}

#define IRKGL_WIDE(TEAM, BLOCK, SLOTS) \
  WideShape { TEAM, BLOCK, SLOTS, (const void*)irkgl_wide_kernel<TEAM, BLOCK, SLOTS>, wide_launch<TEAM, BLOCK, SLOTS> }

static const WideShape kWide[] = {
    IRKGL_WIDE(32, 128, 2),    // d <= 64, 4 instances per block
    IRKGL_WIDE(32, 64, 2),     // d <= 64, 2 instances per block
    IRKGL_WIDE(64, 64, 4),     // d <= 256
    IRKGL_WIDE(128, 128, 4),   // d <= 512
    IRKGL_WIDE(256, 256, 2),   // d <= 512
    IRKGL_WIDE(256, 256, 4),   // d <= 1024
};

int wide_shapes(const WideShape** out) {
  *out = kWide;
  return static_cast<int>(sizeof(kWide) / sizeof(kWide[0]));
}

}  // namespace irkgl
