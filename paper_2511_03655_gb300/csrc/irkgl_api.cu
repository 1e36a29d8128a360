// irkgl_api.cu -- host side of libirkgl.so: the C-ABI declared in include/irkgl.h.
//
// The context owns: the FP64 tables (Sec. 2.4 of arXiv 2511.03655, plus the
// fused initial-guess matrix W), a device copy of the right-hand-side
// parameters, a work counter for the persistent launch, and host-API staging
// buffers.  Kernels are instantiated per (right-hand side, dimension, lanes
// per trajectory) and dispatched from a table.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "irkgl.h"
#include "irkgl_first_order.cuh"
#include "irkgl_kernels.h"
#include "irkgl_repro1.cuh"
#include "irkgl_split.cuh"
#include "irkgl_wide.cuh"
#include "irkgl_wide_repro.cuh"
#include "irkgl_tables.h"

using irkgl::Coef;
using irkgl::Coef1;
using irkgl::KArgs;
using irkgl::KArgs1;

namespace {

thread_local char g_cuda_err[256] = "no error";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", cudaGetErrorString(e));
  return IRKGL_ERR_CUDA;
}

#define IRKGL_CUDA(call)                         \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

using irkgl::KernelEntry;

const KernelEntry* find_kernel(int kind, int dim, int lpt, int block, int mix = 0, int layout = 0) {
  const irkgl::KernelTable tables[] = {irkgl::kernels_kepler(), irkgl::kernels_henon_heiles(),
                                       irkgl::kernels_harmonic(), irkgl::kernels_nbody()};
  for (const irkgl::KernelTable& t : tables)
    for (int i = 0; i < t.count; i++) {
      const KernelEntry& e = t.entries[i];
      if (e.kind == kind && e.dim == dim && e.lpt == lpt && e.block == block && e.mix == mix &&
          e.layout == layout)
        return &e;
    }
  return nullptr;
}

const irkgl::ReproEntry* find_repro(int kind, int dim) {
  const irkgl::ReproTable t = irkgl::kernels_repro();
  for (int i = 0; i < t.count; i++)
    if (t.entries[i].kind == kind && t.entries[i].dim == dim) return &t.entries[i];
  return nullptr;
}

// Built-in default tile per (kind, dim): the smallest LPT that is compiled,
// preferring 2 for d = 2 (both components' compensated updates in one pass).
const irkgl::KernelEntry1* find_kernel1(int kind, int dim, int lpt, int block, int nst = 8, int mix = 0,
                                        int layout = 0) {
  const irkgl::KernelTable1 t = irkgl::kernels_first_order();
  for (int i = 0; i < t.count; i++) {
    const irkgl::KernelEntry1& e = t.entries[i];
    if (e.kind == kind && e.dim == dim && e.lpt == lpt && e.block == block && e.nst == nst && e.mix == mix &&
        e.layout == layout)
      return &e;
  }
  return nullptr;
}

const irkgl::KernelEntry1* find_repro1(int kind, int dim, int nst) {
  const irkgl::KernelTable1 t = irkgl::kernels_first_order_repro();
  for (int i = 0; i < t.count; i++)
    if (t.entries[i].kind == kind && t.entries[i].dim == dim && t.entries[i].nst == nst) return &t.entries[i];
  return nullptr;
}

// Tables of the s-stage first-order form (s = 2, 4, 6 generated; s = 8 is
// the context's own IRKGL16 table).
bool small_stage_tables(int s, Coef1* out) {
  const double *b = nullptr, *mu = nullptr, *nu = nullptr;
  switch (s) {
    case 2: b = IRKGL_TAB2_B; mu = IRKGL_TAB2_MU; nu = IRKGL_TAB2_NU; break;
    case 4: b = IRKGL_TAB4_B; mu = IRKGL_TAB4_MU; nu = IRKGL_TAB4_NU; break;
    case 6: b = IRKGL_TAB6_B; mu = IRKGL_TAB6_MU; nu = IRKGL_TAB6_NU; break;
    default: return false;
  }
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < s; i++) out->b[i] = b[i];
  for (int x = 0; x < s * s; x++) {
    out->mu[x] = mu[x];
    out->nu[x] = nu[x];
  }
  return true;
}

// Right-hand sides of first-order systems y' = f(y) (the mu form).
bool first_order_kind(int kind) {
  return kind == IRKGL_RHS_SCHWARZSCHILD || kind == IRKGL_RHS_HARMONIC1;
}

int default_lpt(int kind, int dim, int nst = 8, int mix = 0) {
  // measured preferences: two lanes for the second-order kinds (Kepler
  // ensemble); four for the first-order ones (Schwarzschild: 128 registers,
  // no spills, 10 % faster than two lanes); with the fixed-point mixing the
  // one-lane tile (compile-time coefficient rows) where it is compiled, else
  // one stage row per lane (N-body)
  const int prefs2[] = {2, 1, 8, 4};
  const int prefs2_mix[] = {1, 8, 4, 2};
  const int prefs1[] = {4, 2, 1, 8};
  for (int i = 0; i < 4; i++) {
    const int p = first_order_kind(kind) ? prefs1[i] : (mix ? prefs2_mix[i] : prefs2[i]);
    if (first_order_kind(kind) ? find_kernel1(kind, dim, p, 128, nst) != nullptr
                               : find_kernel(kind, dim, p, 128, mix) != nullptr)
      return p;
  }
  return 0;
}

bool is_default_table(const irkgl_coeffs* c) {
  irkgl_coeffs d;
  irkgl_default_coeffs(&d);
  return std::memcmp(&d, c, sizeof(d)) == 0;
}

// FP64 FMA throughput probe: 8 independent dependency chains per thread, a
// full grid; the issued FMA count is returned to the caller, who times the
// launch on its stream.  Used to measure the FP64 roof the kernels run against.
constexpr int kProbeIters = 4096;
__global__ void __launch_bounds__(256) fp64_fma_probe(double* out, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
#pragma unroll 4
  for (int i = 0; i < kProbeIters; i++) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[0] = s;  // never true; keeps the chains alive
}

}  // namespace

struct irkgl_ctx {
  int kind;
  int dim;
  double h;
  int device;
  int sm_count;
  Coef coef;
  Coef1 coef1;  // first-order kinds: b, mu, nu
  irkgl::CoefRepro coefr;  // the caller's tables for the reproducible form (mix = 2)
  double* d_params;
  int nparams;
  unsigned* d_counter;
  int lpt;       // 0 = default
  int kmax;
  int monitor;
  int block;
  int grid_blocks;
  int wide_team;
  int monitor_local;
  int mix;             // IRKGL_OPT_MIX
  int stages;          // IRKGL_OPT_STAGES (first-order kinds: 2, 4, 6 or 8)
  int layout;          // IRKGL_OPT_TILE_LAYOUT: 0 auto, 1 stage split, 2 component split
  int default_tables;  // the context uses irkgl_default_coeffs (needed by mix = 1)
  // staging for irkgl_integrate_host
  void* d_stage;
  size_t stage_bytes;
};

extern "C" {

int irkgl_default_coeffs(irkgl_coeffs* out) {
  if (!out) return IRKGL_ERR_INVALID;
  for (int i = 0; i < 8; i++) {
    out->c[i] = IRKGL_TAB_C[i];
    out->b[i] = IRKGL_TAB_B[i];
  }
  for (int x = 0; x < 64; x++) {
    out->mu[x] = IRKGL_TAB_MU[x];
    out->eta[x] = IRKGL_TAB_ETA[x];
    out->nu[x] = IRKGL_TAB_NU[x];
  }
  return IRKGL_OK;
}

const char* irkgl_strerror(int code) {
  switch (code) {
    case IRKGL_OK: return "ok";
    case IRKGL_ERR_INVALID: return "invalid argument";
    case IRKGL_ERR_NOMEM: return "out of memory";
    case IRKGL_ERR_CUDA: return "CUDA runtime error";
    case IRKGL_ERR_UNSUPPORTED: return "no compiled kernel for this right-hand side, dimension and tile";
    case IRKGL_STATUS_MAXITER: return "status: fixed-point sweep cap reached";
    case IRKGL_STATUS_NONFINITE: return "status: non-finite stage value";
    case IRKGL_STATUS_BAD_INSTANCE: return "status: invalid instance descriptor";
    default: return "unknown code";
  }
}

const char* irkgl_last_cuda_error(void) { return g_cuda_err; }

int irkgl_probe_fp64_fma(double* scratch, long long* fma_count, void* stream) {
  if (!scratch || !fma_count) return IRKGL_ERR_INVALID;
  int dev = 0, sms = 0;
  IRKGL_CUDA(cudaGetDevice(&dev));
  IRKGL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  fp64_fma_probe<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(scratch, 0.999999, 1e-7);
  IRKGL_CUDA(cudaGetLastError());
  *fma_count = static_cast<long long>(blocks) * threads * kProbeIters * 8;
  return IRKGL_OK;
}

static int check_rhs(const irkgl_rhs& f, int dim) {
  if (dim < 1 || dim > 4096) return IRKGL_ERR_INVALID;
  if (f.nparams < 1 || !f.params) return IRKGL_ERR_INVALID;
  for (int i = 0; i < f.nparams; i++)
    if (!std::isfinite(f.params[i])) return IRKGL_ERR_INVALID;
  switch (f.kind) {
    case IRKGL_RHS_KEPLER:
    case IRKGL_RHS_HENON_HEILES:
      return dim == 2 ? IRKGL_OK : IRKGL_ERR_INVALID;
    case IRKGL_RHS_HENON_HEILES_FORCED:
      return (dim == 2 && f.nparams == 2) ? IRKGL_OK : IRKGL_ERR_INVALID;
    case IRKGL_RHS_SCHWARZSCHILD:
      return (dim == 4 && f.nparams == 3) ? IRKGL_OK : IRKGL_ERR_INVALID;
    case IRKGL_RHS_HARMONIC1:
      return (dim == 2 && f.nparams == 1) ? IRKGL_OK : IRKGL_ERR_INVALID;
    case IRKGL_RHS_HARMONIC:
    case IRKGL_RHS_FPUT:
      return IRKGL_OK;
    case IRKGL_RHS_NBODY:
      return (dim % 3 == 0 && f.nparams == 1 + dim / 3) ? IRKGL_OK : IRKGL_ERR_INVALID;
    default:
      return IRKGL_ERR_INVALID;
  }
}

int irkgl_create(irkgl_ctx** out, irkgl_rhs f, int dim, double h, const irkgl_coeffs* coeffs) {
  if (!out) return IRKGL_ERR_INVALID;
  *out = nullptr;
  if (!std::isfinite(h) || h == 0.0) return IRKGL_ERR_INVALID;
  int rc = check_rhs(f, dim);
  if (rc != IRKGL_OK) return rc;
  irkgl_coeffs tab;
  if (coeffs) {
    tab = *coeffs;
    const double* all = reinterpret_cast<const double*>(&tab);
    for (size_t i = 0; i < sizeof(tab) / sizeof(double); i++)
      if (!std::isfinite(all[i])) return IRKGL_ERR_INVALID;
  } else {
    irkgl_default_coeffs(&tab);
  }
  irkgl_ctx* c = static_cast<irkgl_ctx*>(std::calloc(1, sizeof(irkgl_ctx)));
  if (!c) return IRKGL_ERR_NOMEM;
  c->kind = f.kind;
  c->dim = dim;
  c->h = h;
  c->kmax = 100;
  c->monitor = 1;
  c->block = 128;
  c->lpt = 0;
  c->grid_blocks = 0;
  c->stages = 8;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    std::free(c);
    return cuda_fail(e);
  }
  for (int i = 0; i < 8; i++) {
    c->coef.c[i] = tab.c[i];
    c->coef.b[i] = tab.b[i];
  }
  for (int x = 0; x < 64; x++) c->coef.eta[x] = tab.eta[x];
  for (int i = 0; i < 8; i++) c->coef1.b[i] = tab.b[i];
  for (int i = 0; i < 8; i++) {
    c->coefr.c[i] = tab.c[i];
    c->coefr.b[i] = tab.b[i];
  }
  for (int x = 0; x < 64; x++) {
    c->coefr.mu[x] = tab.mu[x];
    c->coefr.nu[x] = tab.nu[x];
    c->coefr.eta[x] = tab.eta[x];
  }
  for (int x = 0; x < 64; x++) {
    c->coef1.mu[x] = tab.mu[x];
    c->coef1.nu[x] = tab.nu[x];
  }
  c->default_tables = is_default_table(&tab) ? 1 : 0;
  if (c->default_tables) {
    for (int x = 0; x < 64; x++) c->coef.W[x] = IRKGL_TAB_W[x];
  } else {
    // W = mu diag(b) nu in FP64, fixed summation order (host code is built
    // without floating-point contraction, so this is the same on every host)
    for (int i = 0; i < 8; i++)
      for (int k = 0; k < 8; k++) {
        double acc = 0.0;
        for (int j = 0; j < 8; j++) acc += (tab.mu[i * 8 + j] * tab.b[j]) * tab.nu[j * 8 + k];
        c->coef.W[i * 8 + k] = acc;
      }
  }
  c->nparams = f.nparams;
  e = cudaMalloc(&c->d_params, sizeof(double) * f.nparams);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_params, f.params, sizeof(double) * f.nparams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, 2 * sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaFree(c->d_params);
    std::free(c);
    return e == cudaErrorMemoryAllocation ? IRKGL_ERR_NOMEM : cuda_fail(e);
  }
  *out = c;
  return IRKGL_OK;
}

void irkgl_destroy(irkgl_ctx* c) {
  if (!c) return;
  cudaFree(c->d_params);
  cudaFree(c->d_counter);
  cudaFree(c->d_stage);
  std::free(c);
}

int irkgl_set_option(irkgl_ctx* c, int option, long long value) {
  if (!c) return IRKGL_ERR_INVALID;
  switch (option) {
    case IRKGL_OPT_LANES_PER_TRAJ:
      if (!(value == 0 || value == 1 || value == 2 || value == 4 || value == 8)) return IRKGL_ERR_INVALID;
      c->lpt = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_KMAX:
      if (value < 1 || value > 1000) return IRKGL_ERR_INVALID;
      c->kmax = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_MONITOR_EVERY:
      if (value < 0 || value > (1LL << 30)) return IRKGL_ERR_INVALID;
      c->monitor = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_BLOCK_THREADS:
      if (!(value == 64 || value == 128 || value == 256)) return IRKGL_ERR_INVALID;
      c->block = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_GRID_BLOCKS:
      if (value < 0 || value > (1 << 20)) return IRKGL_ERR_INVALID;
      c->grid_blocks = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_MIX:
      if (value < 0 || value > 2) return IRKGL_ERR_INVALID;
      c->mix = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_TILE_LAYOUT:
      if (value < 0 || value > 2) return IRKGL_ERR_INVALID;
      c->layout = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_STAGES:
      if (!(value == 2 || value == 4 || value == 6 || value == 8)) return IRKGL_ERR_INVALID;
      c->stages = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_MONITOR_LOCAL:
      if (value != 0 && value != 1) return IRKGL_ERR_INVALID;
      c->monitor_local = static_cast<int>(value);
      return IRKGL_OK;
    case IRKGL_OPT_WIDE_TEAM:
      if (!(value == 0 || value == 32 || value == 64 || value == 128 || value == 256))
        return IRKGL_ERR_INVALID;
      c->wide_team = static_cast<int>(value);
      return IRKGL_OK;
    default:
      return IRKGL_ERR_INVALID;
  }
}

static void resolve_tile(const irkgl_ctx* c, int* lpt, int* layout);

// First-order tiles: the component split (D lanes) when requested, or by
// default with the fixed-point mixing; otherwise the stage split with the
// requested or default lanes.
static void resolve_tile1(const irkgl_ctx* c, int* lpt, int* layout) {
  const bool cs_ok = find_kernel1(c->kind, c->dim, c->dim, c->block, c->stages, c->mix, 1) != nullptr;
  if (c->layout == 2 || (c->layout == 0 && c->mix && cs_ok)) {
    *lpt = c->dim;
    *layout = 1;
  } else {
    *lpt = c->lpt ? c->lpt : default_lpt(c->kind, c->dim, c->stages);
    *layout = 0;
  }
}

int irkgl_get_layout(irkgl_ctx* c) {
  if (!c) return IRKGL_ERR_INVALID;
  int lpt = 0, layout = 0;
  if (c->mix == 2) return 3;  // the reproducible form: one thread per trajectory
  if (first_order_kind(c->kind)) resolve_tile1(c, &lpt, &layout);
  else resolve_tile(c, &lpt, &layout);
  return layout ? 2 : 1;
}

int irkgl_get_tile(irkgl_ctx* c) {
  if (!c) return IRKGL_ERR_INVALID;
  if (first_order_kind(c->kind)) {
    if (c->mix == 2) return find_repro1(c->kind, c->dim, c->stages) ? 1 : 0;
    int lpt = 0, layout = 0;
    resolve_tile1(c, &lpt, &layout);
    return find_kernel1(c->kind, c->dim, lpt, c->block, c->stages, c->mix, layout) ? lpt : 0;
  }
  int lpt = 0, layout = 0;
  if (c->mix == 2) return find_repro(c->kind, c->dim) ? 1 : 0;
  if (!first_order_kind(c->kind)) {
    resolve_tile(c, &lpt, &layout);
    return find_kernel(c->kind, c->dim, lpt, c->block, c->mix, layout) ? lpt : 0;
  }
  return c->lpt ? c->lpt : default_lpt(c->kind, c->dim);
}

// Right-hand sides that read t: no energy monitor (H(t) is not conserved).
static bool time_dependent_kind(int kind) { return kind == IRKGL_RHS_HENON_HEILES_FORCED; }

// The tile a second-order call runs: the component-split tile (two lanes)
// when requested, or by default with the fixed-point mixing where it is
// compiled (the fastest form measured on GB300: 1.31x the one-lane tile);
// else the requested or default lanes per trajectory of the stage-split
// tiles (with the fixed-point mixing: one lane where compiled, else one
// stage row per lane).
static void resolve_tile(const irkgl_ctx* c, int* lpt, int* layout) {
  const bool cs_ok = find_kernel(c->kind, c->dim, 2, c->block, c->mix, 1) != nullptr;
  if (c->layout == 2 || (c->layout == 0 && c->mix && cs_ok)) {
    *lpt = 2;
    *layout = 1;
  } else {
    *lpt = c->lpt ? c->lpt : default_lpt(c->kind, c->dim, 8, c->mix);
    *layout = 0;
  }
}

// The reproducible form: one thread per trajectory, a persistent grid of the
// occupancy's full wave (or the requested size), capped at the batch.
static int run_repro(irkgl_ctx* c, KArgs& a, cudaStream_t st) {
  const irkgl::ReproEntry* ke = find_repro(c->kind, c->dim);
  if (!ke) return IRKGL_ERR_UNSUPPORTED;
  constexpr int kBlock = 128;
  a.counter = c->d_counter;
  if (!a.params) a.params = c->d_params;
  a.kmax = c->kmax;
  a.monitor = c->monitor;
  a.monitor_local = c->monitor_local;
  const long long need = (static_cast<long long>(a.batch) + kBlock - 1) / kBlock;
  int grid = c->grid_blocks;
  if (grid <= 0) {
    int per_sm = 0;
    IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ke->fn, kBlock, 0));
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * c->sm_count;
  }
  if (grid > need) grid = static_cast<int>(need);
  if (grid < 1) grid = 1;
  IRKGL_CUDA(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), st));
  ke->launch(dim3(grid), dim3(kBlock), st, a, c->coefr);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

static int run(irkgl_ctx* c, KArgs& a, cudaStream_t st) {
  if (first_order_kind(c->kind)) return IRKGL_ERR_INVALID;  // use the irkgl_*1 calls
  if (c->stages != 8) return IRKGL_ERR_UNSUPPORTED;        // s-stage variants: first-order form only
  if (c->mix == 2) return run_repro(c, a, st);
  if (c->mix && !c->default_tables) return IRKGL_ERR_UNSUPPORTED;
  int lpt = 0, layout = 0;
  resolve_tile(c, &lpt, &layout);
  const KernelEntry* ke = lpt ? find_kernel(c->kind, c->dim, lpt, c->block, c->mix, layout) : nullptr;
  if (!ke) return IRKGL_ERR_UNSUPPORTED;
  a.counter = c->d_counter;
  if (!a.params) a.params = c->d_params;  // else per-trajectory (irkgl_advance_multi)
  a.kmax = c->kmax;
  a.monitor = time_dependent_kind(c->kind) ? 0 : c->monitor;
  a.monitor_local = c->monitor_local;
  const int traj_per_block = c->block / lpt;
  long long need = (static_cast<long long>(a.batch) + traj_per_block - 1) / traj_per_block;
  int grid = c->grid_blocks;
  if (grid <= 0) {
    int per_sm = 0;
    IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ke->fn, c->block, 0));
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * c->sm_count;
  }
  if (grid > need) grid = static_cast<int>(need);
  if (grid < 1) grid = 1;
  IRKGL_CUDA(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), st));
  ke->launch(dim3(grid), dim3(c->block), st, a, c->coef);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

int irkgl_step(irkgl_ctx* c, double* q, double* v, double* q_lo, double* v_lo, double* r_prev,
               const double* h, int batch, int nsteps, int* iters, int* status, void* stream) {
  if (!c || batch < 0 || nsteps < 0) return IRKGL_ERR_INVALID;
  if (batch == 0 || nsteps == 0) return IRKGL_OK;
  if (!q || !v) return IRKGL_ERR_INVALID;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.hist_len = nsteps;
  a.q_in = q;
  a.v_in = v;
  a.qlo_in = q_lo;
  a.vlo_in = v_lo;
  a.rp_in = r_prev;
  a.q_out = q;
  a.v_out = v;
  a.qlo_out = q_lo;
  a.vlo_out = v_lo;
  a.rp_out = r_prev;
  a.nsteps = nullptr;
  a.nsteps_all = nsteps;
  a.h = h;
  a.h_all = c->h;
  a.order = nullptr;
  a.iters_hist = iters;
  a.status = status;
  int saved_monitor = c->monitor;
  c->monitor = 0;  // no energy monitoring in the step-by-step form
  int rc = run(c, a, static_cast<cudaStream_t>(stream));
  c->monitor = saved_monitor;
  return rc;
}

int irkgl_advance(irkgl_ctx* c, double* q, double* v, double* q_lo, double* v_lo, double* r_prev,
                  const double* h, const long long* nsteps, double* H0, int h0_init,
                  double* dH_max, long long* iters, int* status, int batch, void* stream) {
  if (!c || batch < 0) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q || !v || !q_lo || !v_lo || !r_prev || !nsteps) return IRKGL_ERR_INVALID;
  if (dH_max && !H0) return IRKGL_ERR_INVALID;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.q_in = q;
  a.v_in = v;
  a.qlo_in = q_lo;
  a.vlo_in = v_lo;
  a.rp_in = r_prev;
  a.q_out = q;
  a.v_out = v;
  a.qlo_out = q_lo;
  a.vlo_out = v_lo;
  a.rp_out = r_prev;
  a.nsteps = nsteps;
  a.h = h;
  a.h_all = c->h;
  a.iters_total = iters;
  a.dH_max = dH_max;
  a.status = status;
  a.H0_io = H0;
  a.h0_init = h0_init ? 1 : 0;
  a.accumulate = 1;
  const int saved_monitor = c->monitor;
  if (!dH_max) c->monitor = 0;
  const int rc = run(c, a, static_cast<cudaStream_t>(stream));
  c->monitor = saved_monitor;
  return rc;
}

int irkgl_advance_multi(irkgl_ctx* c, double* q, double* v, double* q_lo, double* v_lo,
                        double* r_prev, const double* h, const long long* nsteps,
                        const double* params, int param_stride, const int* order, double* H0,
                        double* dH_max, long long* iters, int* status, int batch, void* stream) {
  if (!c || batch < 0 || param_stride < 0) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q || !v || !q_lo || !v_lo || !r_prev || !nsteps) return IRKGL_ERR_INVALID;
  if (dH_max && !H0) return IRKGL_ERR_INVALID;
  if (params ? param_stride < c->nparams : param_stride != 0) return IRKGL_ERR_INVALID;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.q_in = q;
  a.v_in = v;
  a.qlo_in = q_lo;
  a.vlo_in = v_lo;
  a.rp_in = r_prev;
  a.q_out = q;
  a.v_out = v;
  a.qlo_out = q_lo;
  a.vlo_out = v_lo;
  a.rp_out = r_prev;
  a.nsteps = nsteps;
  a.h = h;
  a.h_all = c->h;
  a.order = order;
  a.iters_total = iters;
  a.dH_max = dH_max;
  a.status = status;
  a.H0_io = H0;
  a.h0_init = 0;  // per trajectory: a NaN entry of H0 is computed at its first step
  a.accumulate = 1;
  a.params = params;
  a.param_stride = params ? param_stride : 0;
  a.sticky_status = 1;
  const int saved_monitor = c->monitor;
  if (!dH_max) c->monitor = 0;
  const int rc = run(c, a, static_cast<cudaStream_t>(stream));
  c->monitor = saved_monitor;
  return rc;
}

int irkgl_advance_t(irkgl_ctx* c, double* q, double* v, double* q_lo, double* v_lo, double* r_prev,
                    double* t, double* t_lo, const double* h, const long long* nsteps,
                    long long* iters, int* status, int batch, void* stream) {
  if (!c || batch < 0) return IRKGL_ERR_INVALID;
  if (!time_dependent_kind(c->kind)) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q || !v || !q_lo || !v_lo || !r_prev || !t || !nsteps) return IRKGL_ERR_INVALID;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.q_in = q;
  a.v_in = v;
  a.qlo_in = q_lo;
  a.vlo_in = v_lo;
  a.rp_in = r_prev;
  a.q_out = q;
  a.v_out = v;
  a.qlo_out = q_lo;
  a.vlo_out = v_lo;
  a.rp_out = r_prev;
  a.t_in = t;
  a.tlo_in = t_lo;
  a.t_out = t;
  a.tlo_out = t_lo;
  a.nsteps = nsteps;
  a.h = h;
  a.h_all = c->h;
  a.iters_total = iters;
  a.status = status;
  a.accumulate = 1;
  return run(c, a, static_cast<cudaStream_t>(stream));
}

static int run1(irkgl_ctx* c, KArgs1& a, cudaStream_t st) {
  if (!first_order_kind(c->kind)) return IRKGL_ERR_INVALID;
  if (c->mix == 1 && !c->default_tables) return IRKGL_ERR_UNSUPPORTED;  // fixed point: built-in tables
  int lpt = 0, layout = 0;
  int block = c->block;
  const irkgl::KernelEntry1* ke = nullptr;
  if (c->mix == 2) {  // the reproducible form: one thread per trajectory
    ke = find_repro1(c->kind, c->dim, c->stages);
    lpt = 1;
    if (ke) block = ke->block;  // its one compiled block size
  } else {
    resolve_tile1(c, &lpt, &layout);
    ke = lpt ? find_kernel1(c->kind, c->dim, lpt, c->block, c->stages, c->mix, layout) : nullptr;
  }
  if (!ke) return IRKGL_ERR_UNSUPPORTED;
  Coef1 small;
  if (c->stages != 8 && !small_stage_tables(c->stages, &small)) return IRKGL_ERR_UNSUPPORTED;
  a.counter = c->d_counter;
  a.params = c->d_params;
  a.kmax = c->kmax;
  a.monitor = c->monitor;
  a.monitor_local = c->monitor_local;
  const int traj_per_block = block / lpt;
  const long long need = (static_cast<long long>(a.batch) + traj_per_block - 1) / traj_per_block;
  int grid = c->grid_blocks;
  if (grid <= 0) {
    int per_sm = 0;
    IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ke->fn, block, 0));
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * c->sm_count;
  }
  if (grid > need) grid = static_cast<int>(need);
  if (grid < 1) grid = 1;
  IRKGL_CUDA(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), st));
  ke->launch(dim3(grid), dim3(block), st, a, c->stages == 8 ? c->coef1 : small);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

int irkgl_integrate1(irkgl_ctx* c, const double* y0, int batch, const long long* nsteps,
                     long long nsteps_all, const double* h, const int* order,
                     const irkgl_outputs1* out, void* stream) {
  if (!c || batch < 0 || !out) return IRKGL_ERR_INVALID;
  if (!first_order_kind(c->kind)) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!y0 || !out->y) return IRKGL_ERR_INVALID;
  if (!nsteps && nsteps_all < 0) return IRKGL_ERR_INVALID;
  KArgs1 a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.y_in = y0;
  a.y_out = out->y;
  a.ylo_out = out->y_lo;
  a.lp_out = out->l_prev;
  a.nsteps = nsteps;
  a.nsteps_all = nsteps_all;
  a.h = h;
  a.h_all = c->h;
  a.order = order;
  a.iters_total = out->iters;
  a.dH_max = out->dH_max;
  a.status = out->status;
  a.steps_done = out->steps;
  return run1(c, a, static_cast<cudaStream_t>(stream));
}

int irkgl_advance1(irkgl_ctx* c, double* y, double* y_lo, double* l_prev, const double* h,
                   const long long* nsteps, double* H0, int h0_init, double* dH_max,
                   long long* iters, int* status, int batch, void* stream) {
  if (!c || batch < 0) return IRKGL_ERR_INVALID;
  if (!first_order_kind(c->kind)) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!y || !y_lo || !l_prev || !nsteps) return IRKGL_ERR_INVALID;
  if (dH_max && !H0) return IRKGL_ERR_INVALID;
  KArgs1 a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.y_in = y;
  a.ylo_in = y_lo;
  a.lp_in = l_prev;
  a.y_out = y;
  a.ylo_out = y_lo;
  a.lp_out = l_prev;
  a.nsteps = nsteps;
  a.h = h;
  a.h_all = c->h;
  a.iters_total = iters;
  a.dH_max = dH_max;
  a.status = status;
  a.H0_io = H0;
  a.h0_init = h0_init ? 1 : 0;
  a.accumulate = 1;
  const int saved_monitor = c->monitor;
  if (!dH_max) c->monitor = 0;
  const int rc = run1(c, a, static_cast<cudaStream_t>(stream));
  c->monitor = saved_monitor;
  return rc;
}

int irkgl_split_integrate(irkgl_ctx* c, int scheme, const double* q0, const double* v0, int batch,
                          const long long* nsteps, long long nsteps_all, const double* h,
                          const irkgl_outputs* out, void* stream) {
  if (!c || batch < 0 || !out) return IRKGL_ERR_INVALID;
  if (first_order_kind(c->kind)) return IRKGL_ERR_INVALID;
  if (scheme != IRKGL_SPLIT_STRANG && scheme != IRKGL_SPLIT_SUZ90) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q0 || !v0 || !out->q || !out->v) return IRKGL_ERR_INVALID;
  if (!nsteps && nsteps_all < 0) return IRKGL_ERR_INVALID;
  const int nk = scheme == IRKGL_SPLIT_STRANG ? 1 : 5;
  const irkgl::SplitTable tab = irkgl::kernels_split();
  const irkgl::SplitEntry* se = nullptr;
  for (int i = 0; i < tab.count && !se; i++)
    if (tab.entries[i].kind == c->kind && tab.entries[i].dim == c->dim && tab.entries[i].nk == nk)
      se = &tab.entries[i];
  if (!se) return IRKGL_ERR_UNSUPPORTED;
  irkgl::SplitCoef sc;
  std::memset(&sc, 0, sizeof(sc));
  const double* A = nk == 1 ? IRKGL_SPLIT_STRANG_A : IRKGL_SPLIT_SUZ90_A;
  const double* B = nk == 1 ? IRKGL_SPLIT_STRANG_B : IRKGL_SPLIT_SUZ90_B;
  for (int j = 0; j <= nk; j++) sc.a[j] = A[j];
  for (int j = 0; j < nk; j++) sc.b[j] = B[j];
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.monitor = time_dependent_kind(c->kind) ? 0 : c->monitor;
  a.monitor_local = c->monitor_local;
  a.q_in = q0;
  a.v_in = v0;
  a.q_out = out->q;
  a.v_out = out->v;
  a.qlo_out = out->q_lo;
  a.vlo_out = out->v_lo;
  a.nsteps = nsteps;
  a.nsteps_all = nsteps_all;
  a.h = h;
  a.h_all = c->h;
  a.iters_total = out->iters;
  a.dH_max = out->dH_max;
  a.status = out->status;
  a.steps_done = out->steps;
  a.params = c->d_params;
  const long long threads = static_cast<long long>(batch) * se->lanes;
  const int grid = static_cast<int>((threads + 127) / 128);
  se->launch(dim3(grid), dim3(128), static_cast<cudaStream_t>(stream), a, sc);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

int irkgl_integrate(irkgl_ctx* c, const double* q0, const double* v0, int batch,
                    const long long* nsteps, long long nsteps_all, const double* h,
                    const int* order, const irkgl_outputs* out, void* stream) {
  if (!c || batch < 0 || !out) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q0 || !v0 || !out->q || !out->v) return IRKGL_ERR_INVALID;
  if (!nsteps && nsteps_all < 0) return IRKGL_ERR_INVALID;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.q_in = q0;
  a.v_in = v0;
  a.q_out = out->q;
  a.v_out = out->v;
  a.qlo_out = out->q_lo;
  a.vlo_out = out->v_lo;
  a.rp_out = out->r_prev;
  a.nsteps = nsteps;
  a.nsteps_all = nsteps_all;
  a.h = h;
  a.h_all = c->h;
  a.order = order;
  a.iters_total = out->iters;
  a.dH_max = out->dH_max;
  a.status = out->status;
  a.steps_done = out->steps;
  return run(c, a, static_cast<cudaStream_t>(stream));
}

// The reproducible wide kernel: the same team-shape rule as run_wide.
static int run_wide_repro(irkgl_ctx* c, irkgl::WideArgs& a, int ninst, int dmax, cudaStream_t st) {
  const irkgl::WideReproShape* shapes = nullptr;
  const int ns = irkgl::wide_repro_shapes(&shapes);
  const irkgl::WideReproShape* ws = nullptr;
  const int want_team = c->wide_team ? c->wide_team : 256;
  size_t smem = 0;
  for (int i = 0; i < ns && !ws; i++) {
    const irkgl::WideReproShape& x = shapes[i];
    if (x.team * x.slots < dmax || x.team != want_team) continue;
    const size_t need_smem = irkgl::wide_repro_smem_bytes(x.block / x.team, dmax);
    if (need_smem > 227 * 1024) continue;
    ws = &x;
    smem = need_smem;
  }
  if (!ws) return IRKGL_ERR_UNSUPPORTED;
  const int teams = ws->block / ws->team;
  IRKGL_CUDA(cudaFuncSetAttribute(ws->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
  int per_sm = 0;
  IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ws->fn, ws->block, smem));
  if (per_sm < 1) return IRKGL_ERR_UNSUPPORTED;
  int grid = c->grid_blocks > 0 ? c->grid_blocks : per_sm * c->sm_count;
  const int need = (ninst + teams - 1) / teams;
  if (grid > need) grid = need;
  a.ninst = ninst;
  a.kmax = c->kmax;
  a.dmax = dmax;
  a.counter = c->d_counter;
  a.monitor_local = c->monitor_local;
  IRKGL_CUDA(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), st));
  ws->launch(dim3(grid), dim3(ws->block), smem, st, a, c->coefr);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

static int run_wide(irkgl_ctx* c, irkgl::WideArgs& a, int ninst, int dmax, cudaStream_t st) {
  static_assert(sizeof(irkgl_instance) == sizeof(irkgl::WideInstance), "instance layout");
  if (dmax < 1) return IRKGL_ERR_INVALID;
  if (dmax > 1536) return IRKGL_ERR_UNSUPPORTED;
  if (c->mix == 2) return run_wide_repro(c, a, ninst, dmax, st);
  if (c->mix && !c->default_tables) return IRKGL_ERR_UNSUPPORTED;  // fixed point: built-in tables
  // team shape: the requested team size, else 256-thread teams (the
  // right-hand side runs team-parallel over (stage, body or particle), and
  // the autotuner measured the 256-thread team within a few per cent of the
  // best for every size bucket on GB300); the first shape of that team size
  // whose threads x slots cover dmax and whose shared memory fits
  const irkgl::WideShape* shapes = nullptr;
  const int ns = irkgl::wide_shapes(&shapes);
  const irkgl::WideShape* ws = nullptr;
  const int want_team = c->wide_team ? c->wide_team : 256;
  size_t smem = 0;
  for (int i = 0; i < ns && !ws; i++) {
    const irkgl::WideShape& x = shapes[i];
    if (x.team * x.slots < dmax) continue;
    if (x.team != want_team || x.mix != c->mix) continue;
    const size_t need_smem = irkgl::wide_smem_bytes(x.block / x.team, dmax, x.cvs);
    if (need_smem > 227 * 1024) continue;
    ws = &x;
    smem = need_smem;
  }
  if (!ws) return IRKGL_ERR_UNSUPPORTED;
  const int teams = ws->block / ws->team;
  IRKGL_CUDA(cudaFuncSetAttribute(ws->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
  int per_sm = 0;
  IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ws->fn, ws->block, smem));
  if (per_sm < 1) return IRKGL_ERR_UNSUPPORTED;
  int grid = c->grid_blocks > 0 ? c->grid_blocks : per_sm * c->sm_count;
  const int need = (ninst + teams - 1) / teams;
  if (grid > need) grid = need;
  a.ninst = ninst;
  a.kmax = c->kmax;
  a.dmax = dmax;
  a.counter = c->d_counter;
  a.monitor_local = c->monitor_local;
  IRKGL_CUDA(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), st));
  ws->launch(dim3(grid), dim3(ws->block), smem, st, a, c->coef);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}

int irkgl_integrate_ragged(irkgl_ctx* c, const irkgl_instance* inst, int ninst, int dmax,
                           const double* params, const double* q0, const double* v0,
                           const int* order, const irkgl_outputs* out, void* stream) {
  if (!c || ninst < 0 || !out) return IRKGL_ERR_INVALID;
  if (ninst == 0) return IRKGL_OK;
  if (!inst || !params || !q0 || !v0 || !out->q || !out->v) return IRKGL_ERR_INVALID;
  irkgl::WideArgs a;
  std::memset(&a, 0, sizeof(a));
  a.monitor = c->monitor;
  a.inst = reinterpret_cast<const irkgl::WideInstance*>(inst);
  a.params = params;
  a.q_in = q0;
  a.v_in = v0;
  a.q_out = out->q;
  a.v_out = out->v;
  a.qlo_out = out->q_lo;
  a.vlo_out = out->v_lo;
  a.rp_out = out->r_prev;
  a.dH_max = out->dH_max;
  a.iters_total = out->iters;
  a.steps_done = out->steps;
  a.status = out->status;
  a.order = order;
  return run_wide(c, a, ninst, dmax, static_cast<cudaStream_t>(stream));
}

int irkgl_advance_ragged(irkgl_ctx* c, const irkgl_instance* inst, int ninst, int dmax,
                         const double* params, double* q, double* v, double* q_lo, double* v_lo,
                         double* r_prev, const long long* nsteps, double* H0, int h0_init,
                         double* dH_max, long long* iters, int* status, const int* order,
                         void* stream) {
  if (!c || ninst < 0) return IRKGL_ERR_INVALID;
  if (ninst == 0) return IRKGL_OK;
  if (!inst || !params || !q || !v || !q_lo || !v_lo || !r_prev || !nsteps) return IRKGL_ERR_INVALID;
  if (dH_max && !H0) return IRKGL_ERR_INVALID;
  irkgl::WideArgs a;
  std::memset(&a, 0, sizeof(a));
  a.monitor = dH_max ? c->monitor : 0;
  a.inst = reinterpret_cast<const irkgl::WideInstance*>(inst);
  a.params = params;
  a.q_in = q;
  a.v_in = v;
  a.q_out = q;
  a.v_out = v;
  a.qlo_in = q_lo;
  a.vlo_in = v_lo;
  a.qlo_out = q_lo;
  a.vlo_out = v_lo;
  a.rp_in = r_prev;
  a.rp_out = r_prev;
  a.nsteps_call = nsteps;
  a.H0_io = H0;
  a.h0_init = h0_init ? 1 : 0;
  a.accumulate = 1;
  a.dH_max = dH_max;
  a.iters_total = iters;
  a.status = status;
  a.sticky_status = 1;
  a.order = order;
  return run_wide(c, a, ninst, dmax, static_cast<cudaStream_t>(stream));
}

int irkgl_integrate_host(irkgl_ctx* c, const double* q0, const double* v0, int batch,
                         const long long* nsteps, long long nsteps_all, const double* h,
                         const int* order, const irkgl_outputs* out, void* stream) {
  if (!c || batch < 0 || !out) return IRKGL_ERR_INVALID;
  if (batch == 0) return IRKGL_OK;
  if (!q0 || !v0 || !out->q || !out->v) return IRKGL_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t B = static_cast<size_t>(batch), D = static_cast<size_t>(c->dim);
  // staging layout (8-byte aligned slices)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_q0 = take(B * D * 8), o_v0 = take(B * D * 8);
  const size_t o_ns = nsteps ? take(B * 8) : 0, o_h = h ? take(B * 8) : 0, o_ord = order ? take(B * 4) : 0;
  const size_t o_q = take(B * D * 8), o_v = take(B * D * 8);
  const size_t o_ql = out->q_lo ? take(B * D * 8) : 0, o_vl = out->v_lo ? take(B * D * 8) : 0;
  const size_t o_rp = out->r_prev ? take(B * 8 * D * 8) : 0;
  const size_t o_dh = out->dH_max ? take(B * 8) : 0, o_it = out->iters ? take(B * 8) : 0;
  const size_t o_sd = out->steps ? take(B * 8) : 0, o_st = out->status ? take(B * 4) : 0;
  if (off > c->stage_bytes) {
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_stage, off);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IRKGL_ERR_NOMEM : cuda_fail(e);
    c->stage_bytes = off;
  }
  char* base = static_cast<char*>(c->d_stage);
  auto dp = [&](size_t o) { return static_cast<void*>(base + o); };
  IRKGL_CUDA(cudaMemcpyAsync(dp(o_q0), q0, B * D * 8, cudaMemcpyHostToDevice, st));
  IRKGL_CUDA(cudaMemcpyAsync(dp(o_v0), v0, B * D * 8, cudaMemcpyHostToDevice, st));
  if (nsteps) IRKGL_CUDA(cudaMemcpyAsync(dp(o_ns), nsteps, B * 8, cudaMemcpyHostToDevice, st));
  if (h) IRKGL_CUDA(cudaMemcpyAsync(dp(o_h), h, B * 8, cudaMemcpyHostToDevice, st));
  if (order) IRKGL_CUDA(cudaMemcpyAsync(dp(o_ord), order, B * 4, cudaMemcpyHostToDevice, st));
  irkgl_outputs dout;
  std::memset(&dout, 0, sizeof(dout));
  dout.q = static_cast<double*>(dp(o_q));
  dout.v = static_cast<double*>(dp(o_v));
  if (out->q_lo) dout.q_lo = static_cast<double*>(dp(o_ql));
  if (out->v_lo) dout.v_lo = static_cast<double*>(dp(o_vl));
  if (out->r_prev) dout.r_prev = static_cast<double*>(dp(o_rp));
  if (out->dH_max) dout.dH_max = static_cast<double*>(dp(o_dh));
  if (out->iters) dout.iters = static_cast<long long*>(dp(o_it));
  if (out->steps) dout.steps = static_cast<long long*>(dp(o_sd));
  if (out->status) dout.status = static_cast<int*>(dp(o_st));
  int rc = irkgl_integrate(c, static_cast<double*>(dp(o_q0)), static_cast<double*>(dp(o_v0)), batch,
                           nsteps ? static_cast<long long*>(dp(o_ns)) : nullptr, nsteps_all,
                           h ? static_cast<double*>(dp(o_h)) : nullptr,
                           order ? static_cast<int*>(dp(o_ord)) : nullptr, &dout, stream);
  if (rc != IRKGL_OK) return rc;
  IRKGL_CUDA(cudaMemcpyAsync(out->q, dout.q, B * D * 8, cudaMemcpyDeviceToHost, st));
  IRKGL_CUDA(cudaMemcpyAsync(out->v, dout.v, B * D * 8, cudaMemcpyDeviceToHost, st));
  if (out->q_lo) IRKGL_CUDA(cudaMemcpyAsync(out->q_lo, dout.q_lo, B * D * 8, cudaMemcpyDeviceToHost, st));
  if (out->v_lo) IRKGL_CUDA(cudaMemcpyAsync(out->v_lo, dout.v_lo, B * D * 8, cudaMemcpyDeviceToHost, st));
  if (out->r_prev)
    IRKGL_CUDA(cudaMemcpyAsync(out->r_prev, dout.r_prev, B * 8 * D * 8, cudaMemcpyDeviceToHost, st));
  if (out->dH_max) IRKGL_CUDA(cudaMemcpyAsync(out->dH_max, dout.dH_max, B * 8, cudaMemcpyDeviceToHost, st));
  if (out->iters) IRKGL_CUDA(cudaMemcpyAsync(out->iters, dout.iters, B * 8, cudaMemcpyDeviceToHost, st));
  if (out->steps) IRKGL_CUDA(cudaMemcpyAsync(out->steps, dout.steps, B * 8, cudaMemcpyDeviceToHost, st));
  if (out->status) IRKGL_CUDA(cudaMemcpyAsync(out->status, dout.status, B * 4, cudaMemcpyDeviceToHost, st));
  IRKGL_CUDA(cudaStreamSynchronize(st));
  return IRKGL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Integration without any device allocation.
//
// Some callers cannot call cudaMalloc: hosts that reserve (nearly) all device
// memory for their own pool allocator up front, real-time or certified code
// that forbids allocation after start-up, and plug-ins that must not touch
// the device heap of the application that loads them.  For them,
// irkgl_integrate_noalloc runs the same batched kernel as irkgl_integrate
// with default options, but its scratch (the work counter that hands
// trajectories to the persistent grid, and the right-hand-side parameters)
// lives in the file-scope array below instead of in a context.
//
// The array is fixed at 64 doubles (512 bytes) and belongs to the library
// image: every GPU that loads the library holds it until the process exits.
// All calls share it and it keeps the last call's contents; each call resets
// the counter and rewrites the parameters before its launch, so calls that
// overlap on the GPU (different streams without ordering, or different host
// threads on one device) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoallocScratchDoubles = 64;  // word 0: work counter; words 1..63: parameters
static __device__ __align__(256) double g_irkgl_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (host code sees only a host-side stand-in for the symbol).  The
// cached address belongs to the device's current context: after
// cudaDeviceReset (or any other teardown of the primary context) the module
// is loaded again and the array may move, so a process that resets a device
// must not call irkgl_integrate_noalloc on it afterwards.
int noalloc_scratch(double** out) {
  int dev = 0;
  IRKGL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return IRKGL_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    IRKGL_CUDA(cudaGetSymbolAddress(&p, g_irkgl_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return IRKGL_OK;
}

}  // namespace

extern "C" int irkgl_integrate_noalloc(irkgl_rhs f, int dim, double h, const double* q0,
                                       const double* v0, int batch, const long long* nsteps,
                                       long long nsteps_all, const double* h_per_traj,
                                       const int* order, const irkgl_outputs* out,
                                       void* stream) {
  if (batch < 0 || !out) return IRKGL_ERR_INVALID;
  if (!std::isfinite(h) || h == 0.0) return IRKGL_ERR_INVALID;
  int rc = check_rhs(f, dim);
  if (rc != IRKGL_OK) return rc;
  if (first_order_kind(f.kind)) return IRKGL_ERR_INVALID;  // the second-order form only
  if (f.nparams > IRKGL_NOALLOC_MAX_PARAMS) return IRKGL_ERR_INVALID;  // beyond the scratch capacity
  if (batch == 0) return IRKGL_OK;
  if (!q0 || !v0 || !out->q || !out->v) return IRKGL_ERR_INVALID;
  if (!nsteps && nsteps_all < 0) return IRKGL_ERR_INVALID;
  const int lpt = default_lpt(f.kind, dim, /*nst=*/8, /*mix=*/0);
  const int block = 128;
  const KernelEntry* ke = lpt ? find_kernel(f.kind, dim, lpt, block) : nullptr;
  if (!ke) return IRKGL_ERR_UNSUPPORTED;

  double* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc != IRKGL_OK) return rc;
  int dev = 0, sms = 0, per_sm = 0;
  IRKGL_CUDA(cudaGetDevice(&dev));
  IRKGL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  IRKGL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ke->fn, block, 0));
  if (per_sm < 1) per_sm = 1;

  Coef coef;
  for (int i = 0; i < 8; i++) {
    coef.c[i] = IRKGL_TAB_C[i];
    coef.b[i] = IRKGL_TAB_B[i];
  }
  for (int x = 0; x < 64; x++) {
    coef.eta[x] = IRKGL_TAB_ETA[x];
    coef.W[x] = IRKGL_TAB_W[x];
  }
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.kmax = 100;
  a.monitor = time_dependent_kind(f.kind) ? 0 : 1;  // H(t) is not conserved
  a.q_in = q0;
  a.v_in = v0;
  a.q_out = out->q;
  a.v_out = out->v;
  a.qlo_out = out->q_lo;
  a.vlo_out = out->v_lo;
  a.rp_out = out->r_prev;
  a.nsteps = nsteps;
  a.nsteps_all = nsteps_all;
  a.h = h_per_traj;
  a.h_all = h;
  a.order = order;
  a.iters_total = out->iters;
  a.dH_max = out->dH_max;
  a.status = out->status;
  a.steps_done = out->steps;
  a.counter = reinterpret_cast<unsigned*>(scratch);  // word 0, cleared below
  a.params = scratch + 1;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IRKGL_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double), st));
  IRKGL_CUDA(cudaMemcpyAsync(scratch + 1, f.params, sizeof(double) * f.nparams,
                             cudaMemcpyHostToDevice, st));
  const int traj_per_block = block / lpt;
  const long long need = (static_cast<long long>(batch) + traj_per_block - 1) / traj_per_block;
  int grid = per_sm * sms;
  if (grid > need) grid = static_cast<int>(need);
  if (grid < 1) grid = 1;
  ke->launch(dim3(grid), dim3(block), st, a, coef);
  IRKGL_CUDA(cudaGetLastError());
  return IRKGL_OK;
}
