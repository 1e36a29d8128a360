// irkgl_repro1.cuh -- the reproducible form (IRKGL_OPT_MIX = 2) of the
// first-order kernel, y' = f(y), for the s-stage schemes (s = 2, 4, 6, 8).
//
// The plain sequence of Eqs. IRK_init / IRK_FP / Yi2 with every FP64
// operation rounded separately (irkgl_repro.cuh's conventions):
//   * Y_i = y + sum_j nu_ij Lprev_j, sums left to right from j = 1;
//   * each sweep: F_i = f(Y_i), L_i = h (b_i F_i),
//     Yn_i = y + sum_j mu_ij L_j; a non-finite Yn ends the step (status 2);
//   * Eqs. Delta_n and stopping on all D components, FP64 values;
//   * y = y (+) sum_i L_i with TwoSum + Fast2Sum; L becomes Lprev;
//   * dH = |(H_n - H_0) / H_0|, or the local form.
// One thread per trajectory.  Right-hand sides here are those whose every
// operation is correctly rounded in IEEE arithmetic (no sin or cos), so any
// binary64 program of the sequence returns the same bits.
#pragma once

#include "irkgl_first_order.cuh"
#include "irkgl_repro.cuh"

namespace irkgl {

// Harmonic oscillator in first-order form, y = (q, p), params {omega}:
// f = (p, -((omega omega) q)); H = (p p + ((omega omega) q) q) / 2.
struct Harmonic1Seq {
  static constexpr int D = 2;
  double w2;
  __device__ void load(const double* p) { w2 = seq::mul(p[0], p[0]); }
  __device__ __forceinline__ void f(const double (&y)[D], double (&out)[D]) const {
    out[0] = y[1];
    out[1] = -seq::mul(w2, y[0]);
  }
  __device__ double H(const double (&y)[D]) const {
    using namespace seq;
    return div(add(mul(y[1], y[1]), mul(mul(w2, y[0]), y[0])), 2.0);
  }
};

// One step of the NST-stage scheme; L holds Lprev on entry and the last
// sweep's L on return (valid when the step succeeded).
template <class Rhs, int NST>
__device__ __forceinline__ int repro_step1(const Rhs& rhs, const Coef1& cf, double h, int kmax,
                                           double (&y)[Rhs::D], double (&ylo)[Rhs::D],
                                           double (&L)[NST][Rhs::D], int* kout) {
  using namespace seq;
  constexpr int D = Rhs::D;
  double Y[NST][D], Yn[NST][D];
#pragma unroll
  for (int i = 0; i < NST; i++)
#pragma unroll
    for (int l = 0; l < D; l++) {
      double acc = mul(cf.nu[i * NST], L[0][l]);
#pragma unroll
      for (int j = 1; j < NST; j++) acc = add(acc, mul(cf.nu[i * NST + j], L[j][l]));
      Y[i][l] = add(y[l], acc);
    }
  const double inf = __longlong_as_double(static_cast<long long>(INF_BITS));
  double dmin[D], dprev[D];
#pragma unroll
  for (int l = 0; l < D; l++) {
    dmin[l] = inf;
    dprev[l] = inf;
  }
  int k = 0;
  for (;;) {
    k++;
#pragma unroll
    for (int i = 0; i < NST; i++) {
      double F[D];
      rhs.f(Y[i], F);
#pragma unroll
      for (int l = 0; l < D; l++) L[i][l] = mul(h, mul(cf.b[i], F[l]));
    }
    bool finite = true;
#pragma unroll
    for (int i = 0; i < NST; i++)
#pragma unroll
      for (int l = 0; l < D; l++) {
        double acc = mul(cf.mu[i * NST], L[0][l]);
#pragma unroll
        for (int j = 1; j < NST; j++) acc = add(acc, mul(cf.mu[i * NST + j], L[j][l]));
        const double x = add(y[l], acc);
        Yn[i][l] = x;
        finite = finite && (abs_bits(x) < INF_BITS);
      }
    if (!finite) {
      *kout = k;
      return ST_NONFINITE;
    }
    bool stop = true;
#pragma unroll
    for (int l = 0; l < D; l++) {
      double delta = 0.0;
#pragma unroll
      for (int i = 0; i < NST; i++) {
        const double d = fabs(sub(Yn[i][l], Y[i][l]));
        if (d > delta) delta = d;
      }
      const double m = dprev[l] <= delta ? dprev[l] : delta;
      const bool cond = (delta == 0.0) || (dmin[l] <= m);
      stop = stop && cond;
      dmin[l] = dmin[l] <= dprev[l] ? dmin[l] : dprev[l];
      dprev[l] = delta;
    }
#pragma unroll
    for (int i = 0; i < NST; i++)
#pragma unroll
      for (int l = 0; l < D; l++) Y[i][l] = Yn[i][l];
    if (stop) break;
    if (k >= kmax) {
      *kout = k;
      return ST_MAXITER;
    }
  }
  *kout = k;
#pragma unroll
  for (int l = 0; l < D; l++) {
    double sL = L[0][l];
#pragma unroll
    for (int i = 1; i < NST; i++) sL = add(sL, L[i][l]);
    repro_two_sum_add(y[l], ylo[l], sL);
  }
  return ST_OK;
}

// Persistent grid, one trajectory per thread at a time (KArgs1 semantics of
// the first-order tiles: per-trajectory nsteps and h, H0_io with NaN entries
// computed at the first step, accumulate, per-step sweep history).
// l_prev is [batch][NST][D].
template <class Rhs, int NST, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    irkgl_kernel1_repro(const __grid_constant__ KArgs1 a, const __grid_constant__ Coef1 cf) {
  constexpr int D = Rhs::D;
  for (;;) {
    const unsigned idx = atomicAdd(a.counter, 1u);
    if (idx >= static_cast<unsigned>(a.batch)) break;
    const int t = a.order ? a.order[idx] : static_cast<int>(idx);
    if (t < 0 || t >= a.batch) continue;
    Rhs rhs;
    rhs.load(a.params);
    const long long N = a.nsteps ? a.nsteps[t] : a.nsteps_all;
    const double h = a.h ? a.h[t] : a.h_all;
    double dHmax = 0.0;
    long long itot = 0;
    if (a.accumulate) {
      if (a.dH_max) dHmax = a.dH_max[t];
      if (a.iters_total) itot = a.iters_total[t];
    }
    double y[D], ylo[D], L[NST][D];
    const size_t off = static_cast<size_t>(t) * D;
#pragma unroll
    for (int l = 0; l < D; l++) {
      y[l] = a.y_in[off + l];
      ylo[l] = a.ylo_in ? a.ylo_in[off + l] : 0.0;
    }
    const size_t loff = static_cast<size_t>(t) * NST * D;
#pragma unroll
    for (int i = 0; i < NST; i++)
#pragma unroll
      for (int l = 0; l < D; l++) L[i][l] = a.lp_in ? a.lp_in[loff + i * D + l] : 0.0;

    double H0 = 0.0, Hprev = 0.0;
    if (a.monitor > 0) {
      if (a.H0_io && !a.h0_init) H0 = a.H0_io[t];
      if (!a.H0_io || a.h0_init || (H0 != H0 && N > 0)) {
        H0 = rhs.H(y);
        if (a.H0_io) a.H0_io[t] = H0;
      }
      Hprev = H0;
    }
    int st = ST_OK;
    long long n = 0;
    while (n < N) {
      int k = 0;
      st = repro_step1<Rhs, NST>(rhs, cf, h, a.kmax, y, ylo, L, &k);
      if (a.iters_hist && n < a.hist_len) a.iters_hist[static_cast<size_t>(t) * a.hist_len + n] = k;
      itot += k;
      if (st != ST_OK) break;
      n++;
      if (a.monitor > 0 && (n % a.monitor) == 0) {
        const double Hn = rhs.H(y);
        double dH;
        if (a.monitor_local) {
          dH = fabs(seq::div(seq::sub(Hn, Hprev), Hprev));
          Hprev = Hn;
        } else {
          dH = fabs(seq::div(seq::sub(Hn, H0), H0));
        }
        if (dH > dHmax) dHmax = dH;
      }
    }
#pragma unroll
    for (int l = 0; l < D; l++) {
      a.y_out[off + l] = y[l];
      if (a.ylo_out) a.ylo_out[off + l] = ylo[l];
    }
    if (a.lp_out && st == ST_OK) {
#pragma unroll
      for (int i = 0; i < NST; i++)
#pragma unroll
        for (int l = 0; l < D; l++) a.lp_out[loff + i * D + l] = L[i][l];
    }
    if (a.dH_max) a.dH_max[t] = dHmax;
    if (a.iters_total) a.iters_total[t] = itot;
    if (a.status) a.status[t] = st;
    if (a.steps_done) a.steps_done[t] = n;
  }
}

template <class Rhs, int NST, int BLOCK>
void launch1_repro_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs1& a, const Coef1& c) {
  irkgl_kernel1_repro<Rhs, NST, BLOCK><<<grid, block, 0, st>>>(a, c);
}

// The first-order reproducible instantiations (k_repro1.cu): mix 2,
// layout 2, one lane per trajectory.
KernelTable1 kernels_first_order_repro();

}  // namespace irkgl

#define IRKGL_ENTRY1_REPRO(KIND, DIM, RHS, NST)                                                      \
  ::irkgl::KernelEntry1 {                                                                            \
    KIND, DIM, 1, 128, NST, 2, 2, (const void*)::irkgl::irkgl_kernel1_repro<RHS, NST, 128>,          \
        ::irkgl::launch1_repro_impl<RHS, NST, 128>                                                   \
  }
