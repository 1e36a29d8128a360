// k_henon_heiles.cu -- compiled instantiations of the batched IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl_kernels.h"

namespace {

const ::irkgl::KernelEntry kEntries[] = {
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<8>, 1, 128),
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<4>, 2, 128),
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<2>, 4, 128),
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<1>, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES_FORCED, 2, ::irkgl::HenonHeilesForced<8>, 1, 128),
    IRKGL_ENTRY(IRKGL_RHS_HENON_HEILES_FORCED, 2, ::irkgl::HenonHeilesForced<4>, 2, 128),
    IRKGL_ENTRY_CS(IRKGL_RHS_HENON_HEILES, ::irkgl::HenonHeiles<4>, 128, 0, 1),
    IRKGL_ENTRY_MIX(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeiles<8>, 1, 128, 1),
    IRKGL_ENTRY_CS(IRKGL_RHS_HENON_HEILES, ::irkgl::HenonHeiles<4>, 128, 1, 1),
};
}  // namespace

namespace irkgl {
KernelTable kernels_henon_heiles() { return KernelTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))}; }
}  // namespace irkgl
