// irkgl_split.cuh -- explicit symplectic splitting baselines for q'' = g(q).
//
// arXiv 2511.03655, Sec. 4: with the drift phi^A_t(q, v) = (q + t v, v) and
// the kick phi^B_t(q, v) = (q, v + t g(q)) (Eq. flowAB), a symmetric
// composition of NK Strang steps is the drift-kick sequence of
// Eq. high_order_splitting,
//   A_{a_1 h}, B_{b_1 h}, A_{a_2 h}, ..., B_{b_NK h}, A_{a_{NK+1} h},
// with NK evaluations of g per step.  Strang: NK = 1; Suzuki's
// fourth-order composition: NK = 5.  q and v are compensated (hi, lo)
// pairs updated by the same TwoSum + Fast2Sum rule as the IRKGL kernels.
//
// One thread per trajectory: the stages of an explicit method are
// sequential, so there is no stage parallelism to spread over lanes.  The
// right-hand-side functors of the IRKGL kernels are reused with one stage
// slot per kick: set_step(b_j h) makes stage_R(j, q, R) return (b_j h) g(q).
#pragma once

#include "irkgl_device.cuh"

namespace irkgl {

struct SplitCoef {
  double a[S + 1];  // drift weights a_1 .. a_{NK+1}
  double b[S];      // kick weights b_1 .. b_NK
};

template <class Rhs, int NK, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    irkgl_split_kernel(const __grid_constant__ KArgs a, const __grid_constant__ SplitCoef sc) {
  constexpr int D = Rhs::D;
  const long long idx = static_cast<long long>(blockIdx.x) * BLOCK + threadIdx.x;
  if (idx >= a.batch) return;
  const int t = a.order ? a.order[idx] : static_cast<int>(idx);
  if (t < 0 || t >= a.batch) return;

  Rhs rhs;
  rhs.load_params(a.params);
  const double h = a.h ? a.h[t] : a.h_all;
  const long long N = a.nsteps ? a.nsteps[t] : a.nsteps_all;
  double kick[NK];
#pragma unroll
  for (int j = 0; j < NK; j++) kick[j] = sc.b[j] * h;
  rhs.set_step(kick);
  double drift[NK + 1];
#pragma unroll
  for (int j = 0; j <= NK; j++) drift[j] = sc.a[j] * h;

  const size_t off = static_cast<size_t>(t) * D;
  double qh[D], ql[D], vh[D], vl[D];
#pragma unroll
  for (int l = 0; l < D; l++) {
    qh[l] = a.q_in[off + l];
    vh[l] = a.v_in[off + l];
    ql[l] = a.qlo_in ? a.qlo_in[off + l] : 0.0;
    vl[l] = a.vlo_in ? a.vlo_in[off + l] : 0.0;
  }
  double H0 = 0.0, Hprev = 0.0, dHmax = 0.0;
  if (a.monitor > 0) {
    H0 = rhs.H(qh, vh);
    Hprev = H0;
  }
  int st = ST_OK;
  long long n = 0;
  for (; n < N; n++) {
#pragma unroll
    for (int j = 0; j < NK; j++) {
#pragma unroll
      for (int l = 0; l < D; l++) two_sum_add(qh[l], ql[l], drift[j] * vh[l]);
      double R[D];
      rhs.stage_R(j, qh, R);
#pragma unroll
      for (int l = 0; l < D; l++) two_sum_add(vh[l], vl[l], R[l]);
    }
    bool bad = false;
#pragma unroll
    for (int l = 0; l < D; l++) {
      two_sum_add(qh[l], ql[l], drift[NK] * vh[l]);
      bad = bad || (abs_bits(qh[l]) >= INF_BITS) || (abs_bits(vh[l]) >= INF_BITS);
    }
    if (bad) {
      st = ST_NONFINITE;
      break;
    }
    if (a.monitor > 0 && ((n + 1) % a.monitor) == 0) {
      const double Hn = rhs.H(qh, vh);
      const double ref = a.monitor_local ? Hprev : H0;
      const double dH = fabs((Hn - ref) / ref);
      if (dH > dHmax) dHmax = dH;
      Hprev = Hn;
    }
  }
#pragma unroll
  for (int l = 0; l < D; l++) {
    a.q_out[off + l] = qh[l];
    a.v_out[off + l] = vh[l];
    if (a.qlo_out) a.qlo_out[off + l] = ql[l];
    if (a.vlo_out) a.vlo_out[off + l] = vl[l];
  }
  if (a.dH_max) a.dH_max[t] = dHmax;
  if (a.iters_total) a.iters_total[t] = n * NK;  // evaluations of g
  if (a.status) a.status[t] = st;
  if (a.steps_done) a.steps_done[t] = n;
}

// N-body (Eq. Ham2) splitting with one lane per body: a group of 8 lanes
// holds one system of NB <= 8 bodies; lane a owns body a's compensated q, v
// and forms its own acceleration G sum_{b != a} m_b (q_b - q_a)/|q_b - q_a|^3
// from the positions gathered by shuffles (every pair is evaluated from both
// ends: twice the pair count of the symmetric form, spread over NB lanes).
template <int NB, int NK, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    irkgl_split_nbody_kernel(const __grid_constant__ KArgs a, const __grid_constant__ SplitCoef sc) {
  constexpr int GL = 8;
  static_assert(NB >= 2 && NB <= GL, "one lane per body, at most 8 bodies");
  const int lane = threadIdx.x & 31;
  const int r = lane % GL;
  const int gbase = lane - r;
  const unsigned gmask = 0xffu << gbase;
  const long long sys = (static_cast<long long>(blockIdx.x) * BLOCK + threadIdx.x) / GL;
  if (sys >= a.batch) return;  // the whole group leaves together
  const int t = a.order ? a.order[sys] : static_cast<int>(sys);
  if (t < 0 || t >= a.batch) return;
  const bool body = r < NB;

  const double G = a.params[0];
  double m[NB];
#pragma unroll
  for (int b = 0; b < NB; b++) m[b] = a.params[1 + b];
  const double mr = body ? a.params[1 + r] : 0.0;
  const double h = a.h ? a.h[t] : a.h_all;
  const long long N = a.nsteps ? a.nsteps[t] : a.nsteps_all;
  double drift[NK + 1], kick[NK];
#pragma unroll
  for (int j = 0; j <= NK; j++) drift[j] = sc.a[j] * h;
#pragma unroll
  for (int j = 0; j < NK; j++) kick[j] = (sc.b[j] * h) * G;

  const size_t off = static_cast<size_t>(t) * 3 * NB + 3 * r;
  double qh[3], ql[3], vh[3], vl[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    qh[c] = body ? a.q_in[off + c] : 0.0;
    vh[c] = body ? a.v_in[off + c] : 0.0;
    ql[c] = (body && a.qlo_in) ? a.qlo_in[off + c] : 0.0;
    vl[c] = (body && a.vlo_in) ? a.vlo_in[off + c] : 0.0;
  }

  // H = sum_a m_a |v_a|^2 / 2 - G sum_{a<b} m_a m_b / |q_b - q_a|, lane a
  // taking its kinetic term and its pairs (a, b > a), summed over the group
  auto energy = [&]() {
    double pot = 0.0;
#pragma unroll
    for (int b = 0; b < NB; b++) {
      const double xb = __shfl_sync(gmask, qh[0], gbase + b);
      const double yb = __shfl_sync(gmask, qh[1], gbase + b);
      const double zb = __shfl_sync(gmask, qh[2], gbase + b);
      if (body && b > r) {
        const double dx = xb - qh[0], dy = yb - qh[1], dz = zb - qh[2];
        pot = fma(m[b], rinv1(fma(dx, dx, fma(dy, dy, dz * dz))), pot);
      }
    }
    double e = body ? fma(0.5 * mr, fma(vh[0], vh[0], fma(vh[1], vh[1], vh[2] * vh[2])), -G * mr * pot) : 0.0;
#pragma unroll
    for (int o = 1; o < GL; o <<= 1) e += __shfl_xor_sync(gmask, e, o);
    return e;
  };

  double H0 = 0.0, Hprev = 0.0, dHmax = 0.0;
  if (a.monitor > 0) {
    H0 = energy();
    Hprev = H0;
  }
  int st = ST_OK;
  long long n = 0;
  for (; n < N; n++) {
#pragma unroll
    for (int j = 0; j < NK; j++) {
#pragma unroll
      for (int c = 0; c < 3; c++) two_sum_add(qh[c], ql[c], drift[j] * vh[c]);
      double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int b = 0; b < NB; b++) {
        const double xb = __shfl_sync(gmask, qh[0], gbase + b);
        const double yb = __shfl_sync(gmask, qh[1], gbase + b);
        const double zb = __shfl_sync(gmask, qh[2], gbase + b);
        if (body && b != r) {
          const double dx = xb - qh[0], dy = yb - qh[1], dz = zb - qh[2];
          const double w = m[b] * rinv3(fma(dx, dx, fma(dy, dy, dz * dz)));
          acc[0] = fma(w, dx, acc[0]);
          acc[1] = fma(w, dy, acc[1]);
          acc[2] = fma(w, dz, acc[2]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; c++) two_sum_add(vh[c], vl[c], kick[j] * acc[c]);
    }
    int bad = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      two_sum_add(qh[c], ql[c], drift[NK] * vh[c]);
      bad |= (abs_bits(qh[c]) >= INF_BITS || abs_bits(vh[c]) >= INF_BITS) ? 1 : 0;
    }
#pragma unroll
    for (int o = 1; o < GL; o <<= 1) bad |= __shfl_xor_sync(gmask, bad, o);
    if (bad) {
      st = ST_NONFINITE;
      break;
    }
    if (a.monitor > 0 && ((n + 1) % a.monitor) == 0) {
      const double Hn = energy();
      const double ref = a.monitor_local ? Hprev : H0;
      const double dH = fabs((Hn - ref) / ref);
      if (dH > dHmax) dHmax = dH;
      Hprev = Hn;
    }
  }
  if (body) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a.q_out[off + c] = qh[c];
      a.v_out[off + c] = vh[c];
      if (a.qlo_out) a.qlo_out[off + c] = ql[c];
      if (a.vlo_out) a.vlo_out[off + c] = vl[c];
    }
  }
  if (r == 0) {
    if (a.dH_max) a.dH_max[t] = dHmax;
    if (a.iters_total) a.iters_total[t] = n * NK;
    if (a.status) a.status[t] = st;
    if (a.steps_done) a.steps_done[t] = n;
  }
}

struct SplitEntry {
  int kind;
  int dim;
  int nk;
  int lanes;  // threads per trajectory (1, or 8 for the lane-per-body N-body kernel)
  const void* fn;
  void (*launch)(dim3, dim3, cudaStream_t, const KArgs&, const SplitCoef&);
};

template <class Rhs, int NK>
void split_launch(dim3 g, dim3 b, cudaStream_t st, const KArgs& a, const SplitCoef& c) {
  irkgl_split_kernel<Rhs, NK, 128><<<g, b, 0, st>>>(a, c);
}

template <int NB, int NK>
void split_nbody_launch(dim3 g, dim3 b, cudaStream_t st, const KArgs& a, const SplitCoef& c) {
  irkgl_split_nbody_kernel<NB, NK, 128><<<g, b, 0, st>>>(a, c);
}

struct SplitTable {
  const SplitEntry* entries;
  int count;
};

SplitTable kernels_split();

}  // namespace irkgl

#define IRKGL_SPLIT_ENTRY(KIND, DIM, RHS, NK) \
  ::irkgl::SplitEntry { KIND, DIM, NK, 1, (const void*)::irkgl::irkgl_split_kernel<RHS, NK, 128>, ::irkgl::split_launch<RHS, NK> }
#define IRKGL_SPLIT_NBODY_ENTRY(NB, NK)                                                              \
  ::irkgl::SplitEntry {                                                                              \
    IRKGL_RHS_NBODY, 3 * (NB), NK, 8, (const void*)::irkgl::irkgl_split_nbody_kernel<NB, NK, 128>,  \
        ::irkgl::split_nbody_launch<NB, NK>                                                          \
  }
