// irkgl_kernels.h -- internal: the table of compiled kernel instantiations.
//
// Each right-hand side's instantiations live in their own translation unit
// (k_*.cu) so that they compile in parallel; irkgl_api.cu looks kernels up
// by (kind, dimension, lanes per trajectory, block size).
#pragma once

#include <cuda_runtime.h>

#include "irkgl_cs.cuh"
#include "irkgl_device.cuh"
#include "irkgl_repro.cuh"

namespace irkgl {

struct KernelEntry {
  int kind;
  int dim;
  int lpt;
  int block;
  int mix;     // 0: FP64 FMA mixing, 1: fixed-point mixing on the integer pipes
  int layout;  // 0: stage split (irkgl_kernel), 1: component split (irkgl_kernel_cs, lpt = 2)
  const void* fn;
  void (*launch)(dim3, dim3, cudaStream_t, const KArgs&, const Coef&);
};

template <class Rhs, int LPT, int BLOCK, int MIX, int MINB>
void launch_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs& a, const Coef& c) {
  irkgl_kernel<Rhs, LPT, BLOCK, MIX, MINB><<<grid, block, 0, st>>>(a, c);
}

template <class Rhs, int BLOCK, int MIX, int MINB>
void launch_cs_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs& a, const Coef& c) {
  irkgl_kernel_cs<Rhs, BLOCK, MIX, MINB><<<grid, block, 0, st>>>(a, c);
}

struct KernelTable {
  const KernelEntry* entries;
  int count;
};

// the reproducible form (IRKGL_OPT_MIX = 2): one thread per trajectory
struct ReproEntry {
  int kind;
  int dim;
  const void* fn;
  void (*launch)(dim3, dim3, cudaStream_t, const KArgs&, const CoefRepro&);
};

template <class Rhs, int BLOCK, int MINB>
void launch_repro_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs& a, const CoefRepro& c) {
  irkgl_kernel_repro<Rhs, BLOCK, MINB><<<grid, block, 0, st>>>(a, c);
}

struct ReproTable {
  const ReproEntry* entries;
  int count;
};
ReproTable kernels_repro();

KernelTable kernels_kepler();
KernelTable kernels_henon_heiles();
KernelTable kernels_harmonic();
KernelTable kernels_nbody();

}  // namespace irkgl

#define IRKGL_ENTRY_TUNED(KIND, DIM, RHS, LPT, BLOCK, MIX, MINB)                                    \
  ::irkgl::KernelEntry {                                                                            \
    KIND, DIM, LPT, BLOCK, MIX, 0, (const void*)::irkgl::irkgl_kernel<RHS, LPT, BLOCK, MIX, MINB>,  \
        ::irkgl::launch_impl<RHS, LPT, BLOCK, MIX, MINB>                                            \
  }
// component-split tile (two lanes per trajectory, one component each)
#define IRKGL_ENTRY_CS(KIND, RHS, BLOCK, MIX, MINB)                                               \
  ::irkgl::KernelEntry {                                                                         \
    KIND, 2, 2, BLOCK, MIX, 1, (const void*)::irkgl::irkgl_kernel_cs<RHS, BLOCK, MIX, MINB>,     \
        ::irkgl::launch_cs_impl<RHS, BLOCK, MIX, MINB>                                           \
  }
#define IRKGL_ENTRY_MIX(KIND, DIM, RHS, LPT, BLOCK, MIX) IRKGL_ENTRY_TUNED(KIND, DIM, RHS, LPT, BLOCK, MIX, 1)
#define IRKGL_ENTRY(KIND, DIM, RHS, LPT, BLOCK) IRKGL_ENTRY_MIX(KIND, DIM, RHS, LPT, BLOCK, 0)
#define IRKGL_ENTRY_REPRO(KIND, DIM, RHS, BLOCK, MINB)                                          \
  ::irkgl::ReproEntry {                                                                          \
    KIND, DIM, (const void*)::irkgl::irkgl_kernel_repro<RHS, BLOCK, MINB>,                       \
        ::irkgl::launch_repro_impl<RHS, BLOCK, MINB>                                             \
  }
