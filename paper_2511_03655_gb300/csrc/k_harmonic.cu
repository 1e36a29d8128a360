// k_harmonic.cu -- compiled instantiations of the batched IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl_kernels.h"

namespace {
using Ha8x1 = ::irkgl::Harmonic<8, 1>;
using Ha1x1 = ::irkgl::Harmonic<1, 1>;
using Ha4x2 = ::irkgl::Harmonic<4, 2>;
using Ha1x2 = ::irkgl::Harmonic<1, 2>;
using Ha4x3 = ::irkgl::Harmonic<4, 3>;
using Ha1x3 = ::irkgl::Harmonic<1, 3>;

const ::irkgl::KernelEntry kEntries[] = {
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 1, Ha8x1, 1, 128),
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 1, Ha1x1, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 2, Ha4x2, 2, 128),
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 2, Ha1x2, 8, 128),
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 3, Ha4x3, 2, 128),
    IRKGL_ENTRY(IRKGL_RHS_HARMONIC, 3, Ha1x3, 8, 128),
};
}  // namespace

namespace irkgl {
KernelTable kernels_harmonic() { return KernelTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))}; }
}  // namespace irkgl
