// k_kepler.cu -- compiled instantiations of the batched IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl_kernels.h"

namespace {

// The two tiles the 65,536-orbit ensemble runs on carry a minimum-blocks
// hint for the register allocator, chosen by timing on GB300: LPT = 2 with
// FP64 mixing at 3 blocks per SM (+8 % over no hint), LPT = 1 with
// fixed-point mixing with a hint of 2 (+10 %); other hints were slower.
const ::irkgl::KernelEntry kEntries[] = {
    IRKGL_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<8>, 1, 128),
    IRKGL_ENTRY_TUNED(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<8>, 1, 128, 1, 2),
    IRKGL_ENTRY_MIX(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<8>, 1, 64, 1),
    IRKGL_ENTRY_TUNED(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<4>, 2, 128, 0, 3),
    IRKGL_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<4>, 2, 64),
    IRKGL_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<4>, 2, 256),
    IRKGL_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<2>, 4, 128),
    IRKGL_ENTRY(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<1>, 8, 128),
    IRKGL_ENTRY_CS(IRKGL_RHS_KEPLER, ::irkgl::Kepler<4>, 128, 0, 1),
    IRKGL_ENTRY_CS(IRKGL_RHS_KEPLER, ::irkgl::Kepler<4>, 128, 1, 1),
    // fixed-point mixing with the stage rows spread over 2 and 8 lanes (the
    // N-body tiles' form; here for bitwise checks against the one-lane tile)
    IRKGL_ENTRY_MIX(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<4>, 2, 128, 1),
    IRKGL_ENTRY_MIX(IRKGL_RHS_KEPLER, 2, ::irkgl::Kepler<1>, 8, 128, 1),
};
}  // namespace

namespace irkgl {
KernelTable kernels_kepler() { return KernelTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))}; }
}  // namespace irkgl
