// k_wide_repro.cu -- instantiations of the reproducible wide kernel
// (IRKGL_OPT_MIX = 2 on the ragged calls): the team shapes of the wide
// kernel, so every team size a caller or the autotuner picks is compiled.
#include <cuda_runtime.h>

#include "irkgl.h"
#include "irkgl_wide_repro.cuh"

namespace irkgl {

template <int TEAM, int BLOCK, int SLOTS>
void wide_repro_launch(dim3 g, dim3 b, size_t smem, cudaStream_t st, const WideArgs& a, const CoefRepro& c) {
  irkgl_wide_repro_kernel<TEAM, BLOCK, SLOTS><<<g, b, smem, st>>>(a, c);
}

#define IRKGL_WIDE_REPRO(TEAM, BLOCK, SLOTS)                                                        \
  WideReproShape {                                                                                \
    TEAM, BLOCK, SLOTS, (const void*)irkgl_wide_repro_kernel<TEAM, BLOCK, SLOTS>,                  \
        wide_repro_launch<TEAM, BLOCK, SLOTS>                                                     \
  }

static const WideReproShape kWideRepro[] = {
    IRKGL_WIDE_REPRO(32, 128, 2),   // d <= 64, 4 instances per block
    IRKGL_WIDE_REPRO(32, 64, 2),    // d <= 64, 2 instances per block
    IRKGL_WIDE_REPRO(64, 64, 4),    // d <= 256
    IRKGL_WIDE_REPRO(128, 128, 4),  // d <= 512
    IRKGL_WIDE_REPRO(256, 256, 2),  // d <= 512
    IRKGL_WIDE_REPRO(256, 256, 4),  // d <= 1024
    IRKGL_WIDE_REPRO(256, 256, 6),  // d <= 1536
};

int wide_repro_shapes(const WideReproShape** out) {
  *out = kWideRepro;
  return static_cast<int>(sizeof(kWideRepro) / sizeof(kWideRepro[0]));
}

}  // namespace irkgl
