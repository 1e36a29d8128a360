// irkgl_repro.cuh -- the reproducible form of the batched IRKGL16 kernel
// (IRKGL_OPT_MIX = 2).
//
// The fast tiles round differently from a plain FP64 program: they fuse
// multiply-adds, fuse the two-stage initial guess into one matrix W, form
// x^(-3/2) from an integer correction, and (with fixed-point mixing) round
// each stage sum once.  Each is at least as accurate as the plain sequence,
// but a last-bit difference can change where the stopping rule (Eqs.
// Delta_n, stopping) ends a step, so sweep counts and final states are not
// those of a CPU program.  This kernel instead performs the operation
// sequence of the method's plain definition with every FP64 operation
// rounded separately (explicit round-to-nearest intrinsics, so no
// contraction whatever the compiler flags):
//   * initial guess, Eq. IRK_init2 unfused: V_i = v + sum_j nu_ij Rprev_j,
//     Lq_i = h (b_i V_i), Q_i = q + sum_j mu_ij Lq_j;
//   * each sweep (Eq. IRK_FP2): G_i = g(Q_i), R_i = h (b_i G_i),
//     Qn_i = q + h (c_i v + sum_j eta_ij R_j);
//   * a non-finite Qn ends the step with status 2 and the state of its start;
//   * Eqs. Delta_n and stopping per component, on FP64 values;
//   * update, Eq. qnvn2: sum_i R_i and sum_i c_i R_i, TwoSum + Fast2Sum of
//     v and then of q with dq = h v_hi + (h v_lo - h sum_i c_i R_i);
//   * dH = |(H_n - H_0) / H_0| (Eq. DHglobmax), or the local form.
// Every sum runs left to right from its first term (j = 1, 2, ..., 8), and
// g and H use IEEE division and square root in the order the right-hand
// sides below state.  Any IEEE-754 binary64 implementation of this sequence
// (round to nearest even, no contraction, no flush to zero) returns the same
// bits: states, R_prev, sweep counts, dH_max and status.
//
// One thread per trajectory: the stage arrays (3 x 8 x D doubles) live in
// registers for D = 2 and spill to (cached) local memory for the N-body
// sizes.  The price of the plain sequence on GB300, where FP64 issues at
// 1/64 of the integer rate, is measured by the benchmark's sub-line.
#pragma once

#include "irkgl_device.cuh"

namespace irkgl {

// The tables of the plain definition (the caller's, not the fused W).
struct CoefRepro {
  double c[S];
  double b[S];
  double mu[S * S];   // Eq. IRK_init2, second mixing
  double nu[S * S];   // Eq. IRK_init2, first mixing (Rprev -> V)
  double eta[S * S];  // Eq. Qi2
};

namespace seq {
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
}  // namespace seq

// ---------------------------------------------------------------------------
// Right-hand sides in their stated operation order.  p: the trajectory's
// parameters.  g(q) and H(q, v) as written in each comment, evaluated left
// to right with every operation rounded.
// ---------------------------------------------------------------------------

// Kepler (Sec. 5): r2 = q1 q1 + q2 q2, r3 = r2 sqrt(r2), g_l = -(mu q_l) / r3;
// H = (v1 v1 + v2 v2) / 2 - mu / sqrt(r2).
struct KeplerSeq {
  static constexpr int D = 2;
  double mu;
  __device__ void load(const double* p) { mu = p[0]; }
  __device__ __forceinline__ void g(const double (&q)[D], double (&out)[D]) const {
    using namespace seq;
    const double r2 = add(mul(q[0], q[0]), mul(q[1], q[1]));
    const double r3 = mul(r2, seq::sqrt(r2));
    out[0] = div(-mul(mu, q[0]), r3);
    out[1] = div(-mul(mu, q[1]), r3);
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    using namespace seq;
    const double r2 = add(mul(q[0], q[0]), mul(q[1], q[1]));
    return sub(div(add(mul(v[0], v[0]), mul(v[1], v[1])), 2.0), div(mu, seq::sqrt(r2)));
  }
};

// Henon-Heiles (Sec. 5.1): g1 = -q1 - ((2 lam) q1) q2,
// g2 = -q2 - lam (q1 q1 - q2 q2);
// H = (v1 v1 + v2 v2) / 2 + (q1 q1 + q2 q2) / 2 + lam ((q1 q1) q2 - ((q2 q2) q2) / 3).
struct HenonHeilesSeq {
  static constexpr int D = 2;
  double lam;
  __device__ void load(const double* p) { lam = p[0]; }
  __device__ __forceinline__ void g(const double (&q)[D], double (&out)[D]) const {
    using namespace seq;
    out[0] = sub(-q[0], mul(mul(mul(2.0, lam), q[0]), q[1]));
    out[1] = sub(-q[1], mul(lam, sub(mul(q[0], q[0]), mul(q[1], q[1]))));
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    using namespace seq;
    const double ke = div(add(mul(v[0], v[0]), mul(v[1], v[1])), 2.0);
    const double pe = div(add(mul(q[0], q[0]), mul(q[1], q[1])), 2.0);
    const double cub = sub(mul(mul(q[0], q[0]), q[1]), div(mul(mul(q[1], q[1]), q[1]), 3.0));
    return add(add(ke, pe), mul(lam, cub));
  }
};

// Harmonic oscillator, d components: w2 = omega omega, g_l = -(w2 q_l);
// H = sum_l (v_l v_l + (w2 q_l) q_l) / 2, summed from 0.
template <int DIM>
struct HarmonicSeq {
  static constexpr int D = DIM;
  double w2;
  __device__ void load(const double* p) { w2 = seq::mul(p[0], p[0]); }
  __device__ __forceinline__ void g(const double (&q)[D], double (&out)[D]) const {
#pragma unroll
    for (int l = 0; l < D; l++) out[l] = -seq::mul(w2, q[l]);
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    using namespace seq;
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < D; l++) acc = add(acc, div(add(mul(v[l], v[l]), mul(mul(w2, q[l]), q[l])), 2.0));
    return acc;
  }
};

// N bodies in 3D, p = {G, m_1 .. m_N}: for each body a, over b != a in
// index order, dx = q_b - q_a, r2 = (dx1 dx1 + dx2 dx2) + dx3 dx3,
// w = (G m_b) / (r2 sqrt(r2)), acc_k = acc_k + w dx_k from acc = 0;
// H = sum_a (m_a |v_a|^2) / 2 - sum_{a<b} ((G m_a) m_b) / |q_b - q_a|, each
// sum from 0 in index order (|v|^2 and |dx|^2 as for r2).
template <int NB>
struct NBodySeq {
  static constexpr int D = 3 * NB;
  double G, m[NB];
  __device__ void load(const double* p) {
    G = p[0];
#pragma unroll
    for (int b = 0; b < NB; b++) m[b] = p[1 + b];
  }
  __device__ __forceinline__ void g(const double (&q)[D], double (&out)[D]) const {
    using namespace seq;
#pragma unroll
    for (int a = 0; a < NB; a++) {
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
#pragma unroll
      for (int b = 0; b < NB; b++) {
        if (b == a) continue;
        const double dx0 = sub(q[3 * b], q[3 * a]);
        const double dx1 = sub(q[3 * b + 1], q[3 * a + 1]);
        const double dx2 = sub(q[3 * b + 2], q[3 * a + 2]);
        const double r2 = add(add(mul(dx0, dx0), mul(dx1, dx1)), mul(dx2, dx2));
        const double w = div(mul(G, m[b]), mul(r2, seq::sqrt(r2)));
        acc0 = add(acc0, mul(w, dx0));
        acc1 = add(acc1, mul(w, dx1));
        acc2 = add(acc2, mul(w, dx2));
      }
      out[3 * a] = acc0;
      out[3 * a + 1] = acc1;
      out[3 * a + 2] = acc2;
    }
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    using namespace seq;
    double kin = 0.0, pot = 0.0;
#pragma unroll
    for (int a = 0; a < NB; a++) {
      const double v2 = add(add(mul(v[3 * a], v[3 * a]), mul(v[3 * a + 1], v[3 * a + 1])),
                            mul(v[3 * a + 2], v[3 * a + 2]));
      kin = add(kin, div(mul(m[a], v2), 2.0));
    }
#pragma unroll
    for (int a = 0; a < NB; a++)
#pragma unroll
      for (int b = a + 1; b < NB; b++) {
        const double dx0 = sub(q[3 * b], q[3 * a]);
        const double dx1 = sub(q[3 * b + 1], q[3 * a + 1]);
        const double dx2 = sub(q[3 * b + 2], q[3 * a + 2]);
        const double r = seq::sqrt(add(add(mul(dx0, dx0), mul(dx1, dx1)), mul(dx2, dx2)));
        pot = add(pot, div(mul(mul(G, m[a]), m[b]), r));
      }
    return sub(kin, pot);
  }
};

// hi + lo += x: TwoSum of (hi, x), then Fast2Sum of the sum with lo + error
__device__ __forceinline__ void repro_two_sum_add(double& hi, double& lo, double x) {
  using namespace seq;
  const double s = add(hi, x);
  const double bb = sub(s, hi);
  const double err = add(sub(hi, sub(s, bb)), sub(x, bb));
  const double lo2 = add(lo, err);
  const double hi2 = add(s, lo2);
  lo = sub(lo2, sub(hi2, s));
  hi = hi2;
}

// One step of one trajectory in the plain sequence.  R holds Rprev on entry
// and the last sweep's R on return (valid for the next step only when the
// step succeeded).  Returns the status; *kout the sweeps taken.
template <class Rhs>
__device__ __forceinline__ int repro_step(const Rhs& rhs, const CoefRepro& cf, double h, int kmax,
                                          double (&q)[Rhs::D], double (&v)[Rhs::D],
                                          double (&ql)[Rhs::D], double (&vl)[Rhs::D],
                                          double (&R)[S][Rhs::D], int* kout) {
  using namespace seq;
  constexpr int D = Rhs::D;
  double Q[S][D], L[S][D];
  // Eq. IRK_init2: V_i = v + sum_j nu_ij Rprev_j; Lq_i = h (b_i V_i)
#pragma unroll
  for (int i = 0; i < S; i++)
#pragma unroll
    for (int l = 0; l < D; l++) {
      double acc = mul(cf.nu[i * S], R[0][l]);
#pragma unroll
      for (int j = 1; j < S; j++) acc = add(acc, mul(cf.nu[i * S + j], R[j][l]));
      L[i][l] = mul(h, mul(cf.b[i], add(v[l], acc)));
    }
  // Q_i = q + sum_j mu_ij Lq_j
#pragma unroll
  for (int i = 0; i < S; i++)
#pragma unroll
    for (int l = 0; l < D; l++) {
      double acc = mul(cf.mu[i * S], L[0][l]);
#pragma unroll
      for (int j = 1; j < S; j++) acc = add(acc, mul(cf.mu[i * S + j], L[j][l]));
      Q[i][l] = add(q[l], acc);
    }

  double dmin[D], dprev[D];
#pragma unroll
  for (int l = 0; l < D; l++) {
    dmin[l] = __longlong_as_double(static_cast<long long>(INF_BITS));
    dprev[l] = dmin[l];
  }
  int k = 0;
  for (;;) {
    k++;
    // R_i = h (b_i g(Q_i)) (Eq. Gi)
#pragma unroll
    for (int i = 0; i < S; i++) {
      double G[D];
      rhs.g(Q[i], G);
#pragma unroll
      for (int l = 0; l < D; l++) R[i][l] = mul(h, mul(cf.b[i], G[l]));
    }
    // Qn_i = q + h (c_i v + sum_j eta_ij R_j) (Eq. Qi2) into L (free now)
    bool finite = true;
#pragma unroll
    for (int i = 0; i < S; i++)
#pragma unroll
      for (int l = 0; l < D; l++) {
        double acc = mul(cf.c[i], v[l]);
#pragma unroll
        for (int j = 0; j < S; j++) acc = add(acc, mul(cf.eta[i * S + j], R[j][l]));
        const double x = add(q[l], mul(h, acc));
        L[i][l] = x;
        finite = finite && (abs_bits(x) < INF_BITS);
      }
    if (!finite) {
      *kout = k;
      return ST_NONFINITE;
    }
    // Eqs. Delta_n and stopping, per component; every component's history
    // is updated
    bool stop = true;
#pragma unroll
    for (int l = 0; l < D; l++) {
      double delta = 0.0;
#pragma unroll
      for (int i = 0; i < S; i++) {
        const double d = fabs(sub(L[i][l], Q[i][l]));
        if (d > delta) delta = d;
      }
      const double m = dprev[l] <= delta ? dprev[l] : delta;
      const bool cond = (delta == 0.0) || (dmin[l] <= m);
      stop = stop && cond;
      dmin[l] = dmin[l] <= dprev[l] ? dmin[l] : dprev[l];
      dprev[l] = delta;
    }
#pragma unroll
    for (int i = 0; i < S; i++)
#pragma unroll
      for (int l = 0; l < D; l++) Q[i][l] = L[i][l];
    if (stop) break;
    if (k >= kmax) {
      *kout = k;
      return ST_MAXITER;
    }
  }
  *kout = k;
  // Eq. qnvn2, compensated
#pragma unroll
  for (int l = 0; l < D; l++) {
    double sR = R[0][l];
#pragma unroll
    for (int i = 1; i < S; i++) sR = add(sR, R[i][l]);
    double scR = mul(cf.c[0], R[0][l]);
#pragma unroll
    for (int i = 1; i < S; i++) scR = add(scR, mul(cf.c[i], R[i][l]));
    repro_two_sum_add(v[l], vl[l], sR);
    const double dq = add(mul(h, v[l]), sub(mul(h, vl[l]), mul(h, scR)));
    repro_two_sum_add(q[l], ql[l], dq);
  }
  return ST_OK;
}

// Persistent grid, one trajectory per thread at a time, taken from a.counter
// (through a.order when given).  KArgs semantics as the other tiles:
// per-trajectory nsteps/h/params, sticky status, H0_io (NaN entries computed
// at the first step), accumulate, per-step sweep history.
template <class Rhs, int BLOCK, int MINB = 1>
__global__ void __launch_bounds__(BLOCK, MINB)
    irkgl_kernel_repro(const __grid_constant__ KArgs a, const __grid_constant__ CoefRepro cf) {
  constexpr int D = Rhs::D;
  for (;;) {
    const unsigned idx = atomicAdd(a.counter, 1u);
    if (idx >= static_cast<unsigned>(a.batch)) break;
    const int t = a.order ? a.order[idx] : static_cast<int>(idx);
    if (t < 0 || t >= a.batch) continue;
    Rhs rhs;
    rhs.load(a.param_stride ? a.params + static_cast<size_t>(t) * a.param_stride : a.params);
    const long long N0 = a.nsteps ? a.nsteps[t] : a.nsteps_all;
    long long N = N0;
    int st = ST_OK;
    if (a.sticky_status && a.status) {
      const int s0 = a.status[t];
      if (s0 != ST_OK) {  // a failure is final: keep the status, take no step
        st = s0;
        N = 0;
      }
    }
    const double h = a.h ? a.h[t] : a.h_all;
    double dHmax = 0.0;
    long long itot = 0;
    if (a.accumulate) {
      if (a.dH_max) dHmax = a.dH_max[t];
      if (a.iters_total) itot = a.iters_total[t];
    }
    double q[D], v[D], ql[D], vl[D], R[S][D];
    const size_t off = static_cast<size_t>(t) * D;
#pragma unroll
    for (int l = 0; l < D; l++) {
      q[l] = a.q_in[off + l];
      v[l] = a.v_in[off + l];
      ql[l] = a.qlo_in ? a.qlo_in[off + l] : 0.0;
      vl[l] = a.vlo_in ? a.vlo_in[off + l] : 0.0;
    }
    const size_t roff = static_cast<size_t>(t) * S * D;
#pragma unroll
    for (int i = 0; i < S; i++)
#pragma unroll
      for (int l = 0; l < D; l++) R[i][l] = a.rp_in ? a.rp_in[roff + i * D + l] : 0.0;

    double H0 = 0.0, Hprev = 0.0;
    if (a.monitor > 0) {
      if (a.H0_io && !a.h0_init) H0 = a.H0_io[t];
      if (!a.H0_io || a.h0_init || (H0 != H0 && N > 0)) {
        H0 = rhs.H(q, v);
        if (a.H0_io) a.H0_io[t] = H0;
      }
      Hprev = H0;
    }
    long long n = 0;
    while (n < N) {
      int k = 0;
      st = repro_step(rhs, cf, h, a.kmax, q, v, ql, vl, R, &k);
      if (a.iters_hist && n < a.hist_len) a.iters_hist[static_cast<size_t>(t) * a.hist_len + n] = k;
      itot += k;
      if (st != ST_OK) break;
      n++;
      if (a.monitor > 0 && (n % a.monitor) == 0) {
        const double Hn = rhs.H(q, v);
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
      a.q_out[off + l] = q[l];
      a.v_out[off + l] = v[l];
      if (a.qlo_out) a.qlo_out[off + l] = ql[l];
      if (a.vlo_out) a.vlo_out[off + l] = vl[l];
    }
    if (a.rp_out && st == ST_OK) {
#pragma unroll
      for (int i = 0; i < S; i++)
#pragma unroll
        for (int l = 0; l < D; l++) a.rp_out[roff + i * D + l] = R[i][l];
    }
    if (a.dH_max) a.dH_max[t] = dHmax;
    if (a.iters_total) a.iters_total[t] = itot;
    if (a.status) a.status[t] = st;
    if (a.steps_done) a.steps_done[t] = n;
  }
}

}  // namespace irkgl
