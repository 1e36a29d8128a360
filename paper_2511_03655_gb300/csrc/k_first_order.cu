// k_first_order.cu -- compiled instantiations of the first-order IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl_first_order.cuh"

namespace {

const ::irkgl::KernelEntry1 kEntries[] = {
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<8>, 1, 128),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<4>, 2, 128),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<2>, 4, 128),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<8>, 1, 128),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<4>, 2, 128),
};
}  // namespace

namespace irkgl {
KernelTable1 kernels_first_order() {
  return KernelTable1{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))};
}
}  // namespace irkgl
