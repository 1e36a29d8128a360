// k_first_order.cu -- compiled instantiations of the first-order IRKGL16 kernel.
#include "irkgl.h"
#include "irkgl1_cs.cuh"
#include "irkgl_first_order.cuh"

namespace {

// The fixed-point component-split tile takes the FP64 sincos (its mixing
// already fills the integer pipes); every other Schwarzschild tile the
// fixed-point one.
using SchwarzschildFp64Trig = ::irkgl::Schwarzschild<2, false>;

// Functor template argument = stages per lane (NST / LPT).
const ::irkgl::KernelEntry1 kEntries[] = {
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<8>, 1, 128, 8),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<4>, 2, 128, 8),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<2>, 4, 128, 8),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<8>, 1, 128, 8),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<4>, 2, 128, 8),
    // s-stage IRKGL schemes, s = 2, 4, 6 (Sec. 5.2 comparison)
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<2>, 1, 128, 2),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<1>, 2, 128, 2),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<4>, 1, 128, 4),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<2>, 2, 128, 4),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<6>, 1, 128, 6),
    IRKGL_ENTRY1(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<3>, 2, 128, 6),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<2>, 1, 128, 2),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<4>, 1, 128, 4),
    IRKGL_ENTRY1(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<6>, 1, 128, 6),
    // component split (one component of all eight stages per lane)
    IRKGL_ENTRY1_CS(IRKGL_RHS_SCHWARZSCHILD, 4, ::irkgl::Schwarzschild<2>, 128, 0),
    IRKGL_ENTRY1_CS(IRKGL_RHS_SCHWARZSCHILD, 4, SchwarzschildFp64Trig, 128, 1),
    IRKGL_ENTRY1_CS(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<4>, 128, 0),
    IRKGL_ENTRY1_CS(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1<4>, 128, 1),
};
}  // namespace

namespace irkgl {
KernelTable1 kernels_first_order() {
  return KernelTable1{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))};
}
}  // namespace irkgl
