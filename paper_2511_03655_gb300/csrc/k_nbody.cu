// k_nbody.cu -- compiled instantiations of the batched IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl_kernels.h"

namespace {
using NB3 = ::irkgl::NBody<1, 3>;
using NB4 = ::irkgl::NBody<1, 4>;
using NB5 = ::irkgl::NBody<1, 5>;
using NB6 = ::irkgl::NBody<1, 6>;

const ::irkgl::KernelEntry kEntries[] = {
    IRKGL_ENTRY(IRKGL_RHS_NBODY, 9, NB3, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_NBODY, 12, NB4, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_NBODY, 15, NB5, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_NBODY, 18, NB6, 8, 128),
    // fixed-point stage mixing, one stage row per lane
    IRKGL_ENTRY_MIX(IRKGL_RHS_NBODY, 9, NB3, 8, 128, 1),
    IRKGL_ENTRY_MIX(IRKGL_RHS_NBODY, 12, NB4, 8, 128, 1),
    IRKGL_ENTRY_MIX(IRKGL_RHS_NBODY, 15, NB5, 8, 128, 1),
    IRKGL_ENTRY_MIX(IRKGL_RHS_NBODY, 18, NB6, 8, 128, 1),
};
}  // namespace

namespace irkgl {
KernelTable kernels_nbody() { return KernelTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))}; }
}  // namespace irkgl
