// k_repro.cu -- compiled instantiations of the reproducible kernel
// (IRKGL_OPT_MIX = 2) for the right-hand sides and dimensions the register
// tiles serve.
#include "irkgl.h"
#include "irkgl_kernels.h"

namespace {
const ::irkgl::ReproEntry kEntries[] = {
    IRKGL_ENTRY_REPRO(IRKGL_RHS_KEPLER, 2, ::irkgl::KeplerSeq, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_HENON_HEILES, 2, ::irkgl::HenonHeilesSeq, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_HARMONIC, 1, ::irkgl::HarmonicSeq<1>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_HARMONIC, 2, ::irkgl::HarmonicSeq<2>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_HARMONIC, 3, ::irkgl::HarmonicSeq<3>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_NBODY, 9, ::irkgl::NBodySeq<3>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_NBODY, 12, ::irkgl::NBodySeq<4>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_NBODY, 15, ::irkgl::NBodySeq<5>, 128, 1),
    IRKGL_ENTRY_REPRO(IRKGL_RHS_NBODY, 18, ::irkgl::NBodySeq<6>, 128, 1),
};
}  // namespace

namespace irkgl {
ReproTable kernels_repro() { return ReproTable{kEntries, static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0]))}; }
}  // namespace irkgl
