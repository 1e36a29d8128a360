// k_diag.cu -- diagnostic kernel for the fixed-point mixing (tests only).
#include <cuda_runtime.h>

#include "irkgl.h"
#include "irkgl_device.cuh"

namespace {
__global__ void fixed_mix_kernel(const double* R, double* out, int n) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  double Rc[irkgl::S];
#pragma unroll
  for (int j = 0; j < irkgl::S; j++) Rc[j] = R[x * irkgl::S + j];
  unsigned long long rb[irkgl::S];
  bool nf;
  const int emax = irkgl::fixed_column(Rc, rb, nf);
#pragma unroll
  for (int i = 0; i < irkgl::S; i++) {
    out[(x * irkgl::S + i) * 2] = nf ? __longlong_as_double(0x7ff8000000000000LL)
                                     : irkgl::fixed_row<false>(i, rb, emax);
    out[(x * irkgl::S + i) * 2 + 1] = nf ? __longlong_as_double(0x7ff8000000000000LL)
                                         : irkgl::fixed_row<true>(i, rb, emax);
  }
}
// The same sums by the runtime-row form of the stage-split tiles with the
// rows spread over lanes (fixed_row_rt: one accumulator, signs applied to
// the operands, row constants rbias).
__global__ void fixed_mix_rows_kernel(const double* R, double* out, int n) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  double Rc[irkgl::S];
#pragma unroll
  for (int j = 0; j < irkgl::S; j++) Rc[j] = R[x * irkgl::S + j];
  unsigned long long rb[irkgl::S];
  bool nf;
  const int emax = irkgl::fixed_column(Rc, rb, nf);
  const irkgl::FixedRowTables& t = irkgl::kFixedRows;
  for (int i = 0; i < irkgl::S; i++) {
    const double e = irkgl::fixed_row_rt<IRKGL_ETA_SHIFT>(&t.mag[0][i * irkgl::S], t.negbits[0][i],
                                                         &t.rbias[0][i * 4], rb, emax);
    const double w = irkgl::fixed_row_rt<IRKGL_W_SHIFT>(&t.mag[1][i * irkgl::S], t.negbits[1][i],
                                                       &t.rbias[1][i * 4], rb, emax);
    out[(x * irkgl::S + i) * 2] = nf ? __longlong_as_double(0x7ff8000000000000LL) : e;
    out[(x * irkgl::S + i) * 2 + 1] = nf ? __longlong_as_double(0x7ff8000000000000LL) : w;
  }
}
// The device reciprocal square roots the right-hand sides use.
__global__ void rinv_kernel(const double* x, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[3 * i] = irkgl::rinv3(x[i]);
  out[3 * i + 1] = irkgl::rinv1(x[i]);
  out[3 * i + 2] = irkgl::rcp_int(x[i]);
}
// The fixed-point sine and cosine of the Schwarzschild right-hand side.
__global__ void sincos_kernel(const double* x, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s, c;
  irkgl::sincos_fx(x[i], s, c);
  out[2 * i] = s;
  out[2 * i + 1] = c;
}
}  // namespace

extern "C" int irkgl_diag_sincos(const double* x, double* out, int n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return IRKGL_ERR_INVALID;
  if (n == 0) return IRKGL_OK;
  sincos_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? IRKGL_OK : IRKGL_ERR_CUDA;
}

extern "C" int irkgl_diag_rinv(const double* x, double* out, int n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return IRKGL_ERR_INVALID;
  if (n == 0) return IRKGL_OK;
  rinv_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? IRKGL_OK : IRKGL_ERR_CUDA;
}

extern "C" int irkgl_diag_fixed_mix_rows(const double* R, double* out, int n, void* stream) {
  if (n < 0 || (n > 0 && (!R || !out))) return IRKGL_ERR_INVALID;
  if (n == 0) return IRKGL_OK;
  fixed_mix_rows_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(R, out, n);
  return cudaGetLastError() == cudaSuccess ? IRKGL_OK : IRKGL_ERR_CUDA;
}

extern "C" int irkgl_diag_fixed_mix(const double* R, double* out, int n, void* stream) {
  if (n < 0 || (n > 0 && (!R || !out))) return IRKGL_ERR_INVALID;
  if (n == 0) return IRKGL_OK;
  fixed_mix_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(R, out, n);
  return cudaGetLastError() == cudaSuccess ? IRKGL_OK : IRKGL_ERR_CUDA;
}
