// k_split.cu -- compiled instantiations of the explicit splitting baselines.
#include "irkgl.h"
#include "irkgl_split.cuh"

namespace {

const ::irkgl::SplitEntry kEntries[] = {
    IRKGL_SPLIT_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<1>, 1),
    IRKGL_SPLIT_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<5>, 5),
    IRKGL_SPLIT_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<1>, 1),
    IRKGL_SPLIT_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<5>, 5),
    IRKGL_SPLIT_NBODY_ENTRY(6, 1),
    IRKGL_SPLIT_NBODY_ENTRY(6, 5),
};
}  // namespace

namespace irkgl {
SplitTable kernels_split() {
  return SplitTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))};
}
}  // namespace irkgl
