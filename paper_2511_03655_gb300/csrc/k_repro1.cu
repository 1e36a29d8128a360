// k_repro1.cu -- compiled instantiations of the first-order reproducible
// kernel (IRKGL_OPT_MIX = 2): the right-hand sides whose operations are all
// correctly rounded, for the s = 2, 4, 6, 8 schemes.
#include "irkgl.h"
#include "irkgl_repro1.cuh"

namespace {
const ::irkgl::KernelEntry1 kEntries[] = {
    IRKGL_ENTRY1_REPRO(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1Seq, 8),
    IRKGL_ENTRY1_REPRO(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1Seq, 6),
    IRKGL_ENTRY1_REPRO(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1Seq, 4),
    IRKGL_ENTRY1_REPRO(IRKGL_RHS_HARMONIC1, 2, ::irkgl::Harmonic1Seq, 2),
};
}  // namespace

namespace irkgl {
KernelTable1 kernels_first_order_repro() {
  return KernelTable1{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))};
}
}  // namespace irkgl
