// irkgl_wide_repro.cuh -- the reproducible form (IRKGL_OPT_MIX = 2) of the
// wide kernel for ragged batches (N-body with up to 128 bodies, FPUT chains,
// harmonic oscillators, d <= 1536).
//
// The operation sequence is that of irkgl_repro.cuh (the method's plain
// definition, every FP64 operation rounded separately), spread over a team
// without changing the order of any sum:
//   * each owned component l: the two-matrix initial guess of Eq. IRK_init2,
//     the stage sums of Eq. Qi2 (j = 1..8 left to right), Delta, Eq.
//     stopping and the compensated update, all sequential in one thread;
//   * g: one thread per (stage, body) or (stage, particle), each force a
//     sequential sum over the other bodies in index order, then
//     R_i = h (b_i G_i);
//   * H: the terms are formed in parallel into shared memory, and one thread
//     adds them in index order (chunks of 8 dmax terms), so H does not
//     depend on the team size;
//   * the non-finite check, Eq. stopping's AND and the sweep cap as in the
//     wide kernel.
// So every team shape returns the same bits, and those of any IEEE-754
// binary64 program of the same sequence.
//
// Right-hand sides in their stated order (p: the instance's parameters):
//   N-body (p = G, m_1..m_N): as NBodySeq in irkgl_repro.cuh;
//   FPUT (p = alpha), fixed ends q_0 = q_{d+1} = 0, bonds r_j = q_{j+1} - q_j
//     (one subtraction, an end taken as the constant 0):
//     g_l = (r_l + (alpha r_l) r_l) - (r_{l-1} + (alpha r_{l-1}) r_{l-1});
//     H = sum_l (v_l v_l) / 2, then per bond j = 0..d
//     acc = (acc + (r_j r_j) / 2) + (((alpha r_j) r_j) r_j) / 3, from 0;
//   harmonic (p = omega): as HarmonicSeq.
#pragma once

#include "irkgl_repro.cuh"
#include "irkgl_wide.cuh"

namespace irkgl {

struct WideReproShape {
  int team, block, slots;
  const void* fn;
  void (*launch)(dim3, dim3, size_t, cudaStream_t, const WideArgs&, const CoefRepro&);
};
int wide_repro_shapes(const WideReproShape** out);

// per team: Q, R [8][dmax]; qs, vs [dmax]; red [32]
__host__ __device__ inline size_t wide_repro_smem_bytes(int teams, int dmax) {
  const size_t per_team = 2 * S * static_cast<size_t>(dmax) + 2 * static_cast<size_t>(dmax) + 32;
  return static_cast<size_t>(teams) * per_team * sizeof(double);
}

// R_i = h (b_i g(Q_i)) for every stage, team-parallel, plain sequence.
template <int TEAM>
__device__ __forceinline__ void team_rhs_repro(int kind, int d, const double* p, const CoefRepro& cf,
                                               double h, const double* Q, double* R, int tid) {
  using namespace seq;
  if (kind == IRKGL_RHS_NBODY) {
    const int nb = d / 3;
    const double G = p[0];
    for (int x = tid; x < S * nb; x += TEAM) {
      const int i = x / nb, a = x - i * nb;
      const double* Qi = Q + i * d;
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
      for (int b = 0; b < nb; b++) {
        if (b == a) continue;
        const double dx0 = sub(Qi[3 * b], Qi[3 * a]);
        const double dx1 = sub(Qi[3 * b + 1], Qi[3 * a + 1]);
        const double dx2 = sub(Qi[3 * b + 2], Qi[3 * a + 2]);
        const double r2 = add(add(mul(dx0, dx0), mul(dx1, dx1)), mul(dx2, dx2));
        const double w = div(mul(G, p[1 + b]), mul(r2, seq::sqrt(r2)));
        acc0 = add(acc0, mul(w, dx0));
        acc1 = add(acc1, mul(w, dx1));
        acc2 = add(acc2, mul(w, dx2));
      }
      R[i * d + 3 * a] = mul(h, mul(cf.b[i], acc0));
      R[i * d + 3 * a + 1] = mul(h, mul(cf.b[i], acc1));
      R[i * d + 3 * a + 2] = mul(h, mul(cf.b[i], acc2));
    }
  } else if (kind == IRKGL_RHS_FPUT) {
    const double al = p[0];
    for (int x = tid; x < S * d; x += TEAM) {
      const int i = x / d, l = x - i * d;
      const double* Qi = Q + i * d;
      const double rr = sub(l + 1 < d ? Qi[l + 1] : 0.0, Qi[l]);
      const double rl = sub(Qi[l], l > 0 ? Qi[l - 1] : 0.0);
      const double g = sub(add(rr, mul(mul(al, rr), rr)), add(rl, mul(mul(al, rl), rl)));
      R[x] = mul(h, mul(cf.b[i], g));
    }
  } else {  // IRKGL_RHS_HARMONIC
    const double w2 = mul(p[0], p[0]);
    for (int x = tid; x < S * d; x += TEAM) {
      const int i = x / d;
      R[x] = mul(h, mul(cf.b[i], -mul(w2, Q[x])));
    }
  }
}

// Number of H terms of an instance (N-body: nb kinetic terms, then the
// nb (nb - 1) / 2 pair terms in the order (a, b > a); FPUT: d kinetic terms,
// then two per bond j = 0..d; harmonic: d).
__device__ __forceinline__ int repro_energy_terms(int kind, int d) {
  if (kind == IRKGL_RHS_NBODY) {
    const int nb = d / 3;
    return nb + nb * (nb - 1) / 2;
  }
  if (kind == IRKGL_RHS_FPUT) return d + 2 * (d + 1);
  return d;
}

__device__ __forceinline__ double repro_energy_term(int kind, int d, const double* p, const double* qs,
                                                    const double* vs, int x) {
  using namespace seq;
  if (kind == IRKGL_RHS_NBODY) {
    const int nb = d / 3;
    if (x < nb) {
      const int a = x;
      const double v2 = add(add(mul(vs[3 * a], vs[3 * a]), mul(vs[3 * a + 1], vs[3 * a + 1])),
                            mul(vs[3 * a + 2], vs[3 * a + 2]));
      return div(mul(p[1 + a], v2), 2.0);
    }
    int a = 0, b = x - nb;  // pair index -> (a, b), b > a, lexicographic
    while (b >= nb - 1 - a) {
      b -= nb - 1 - a;
      a++;
    }
    b += a + 1;
    const double dx0 = sub(qs[3 * b], qs[3 * a]);
    const double dx1 = sub(qs[3 * b + 1], qs[3 * a + 1]);
    const double dx2 = sub(qs[3 * b + 2], qs[3 * a + 2]);
    const double r = seq::sqrt(add(add(mul(dx0, dx0), mul(dx1, dx1)), mul(dx2, dx2)));
    return div(mul(mul(p[0], p[1 + a]), p[1 + b]), r);
  }
  if (kind == IRKGL_RHS_FPUT) {
    if (x < d) return div(mul(vs[x], vs[x]), 2.0);
    const int j = (x - d) >> 1;  // bond j = 0..d
    const double r = sub(j < d ? qs[j] : 0.0, j > 0 ? qs[j - 1] : 0.0);
    if (((x - d) & 1) == 0) return div(mul(r, r), 2.0);
    return div(mul(mul(mul(p[0], r), r), r), 3.0);
  }
  const double w2 = mul(p[0], p[0]);
  return div(add(mul(vs[x], vs[x]), mul(mul(w2, qs[x]), qs[x])), 2.0);
}

// H of the staged state qs, vs: terms in parallel into scratch (C doubles),
// summed in index order by thread 0; every thread returns H.
template <int TEAM>
__device__ double team_energy_repro(int kind, int d, const double* p, const double* qs, const double* vs,
                                    double* scratch, int C, double* red, int tid) {
  using namespace seq;
  const int T = repro_energy_terms(kind, d);
  const int nkin = kind == IRKGL_RHS_NBODY ? d / 3 : T;  // N-body: kin - pot
  double kin = 0.0, pot = 0.0;
  for (int c0 = 0; c0 < T; c0 += C) {
    const int c1 = c0 + C < T ? c0 + C : T;
    for (int x = c0 + tid; x < c1; x += TEAM) scratch[x - c0] = repro_energy_term(kind, d, p, qs, vs, x);
    team_sync<TEAM>();
    if (tid == 0)
      for (int x = c0; x < c1; x++) {
        if (x < nkin) kin = add(kin, scratch[x - c0]);
        else pot = add(pot, scratch[x - c0]);
      }
    team_sync<TEAM>();
  }
  if (tid == 0) red[0] = kind == IRKGL_RHS_NBODY ? sub(kin, pot) : kin;
  team_sync<TEAM>();
  const double H = red[0];
  team_sync<TEAM>();
  return H;
}

template <int TEAM, int BLOCK, int SLOTS>
__global__ void __launch_bounds__(BLOCK)
    irkgl_wide_repro_kernel(const __grid_constant__ WideArgs a, const __grid_constant__ CoefRepro cf) {
  static_assert(TEAM == 32 || TEAM == BLOCK, "a team is one warp or the whole block");
  using namespace seq;
  constexpr int TEAMS = BLOCK / TEAM;
  extern __shared__ double smem[];
  const int team = threadIdx.x / TEAM;
  const int tid = threadIdx.x - team * TEAM;
  const int dmax = a.dmax;
  const size_t per_team = 2 * S * static_cast<size_t>(dmax) + 2 * static_cast<size_t>(dmax) + 32;
  double* Q = smem + team * per_team;
  double* R = Q + S * dmax;
  double* qs = R + S * dmax;
  double* vs = qs + dmax;
  double* red = vs + dmax;
  __shared__ unsigned s_idx[TEAMS];

  double qh[SLOTS], ql[SLOTS], vh[SLOTS], vl[SLOTS], dmin[SLOTS], dprev[SLOTS];
  const double inf = __longlong_as_double(static_cast<long long>(INF_BITS));

  for (;;) {
    if (tid == 0) s_idx[team] = atomicAdd(a.counter, 1u);
    team_sync<TEAM>();
    const unsigned idx = s_idx[team];
    team_sync<TEAM>();
    if (idx >= static_cast<unsigned>(a.ninst)) break;
    const int t = a.order ? a.order[idx] : static_cast<int>(idx);
    if (t < 0 || t >= a.ninst) continue;
    const WideInstance in = a.inst[t];
    const int d = in.dim;
    // descriptor checks (no memory of a rejected instance is touched)
    bool ok_desc = d >= 1 && d <= dmax && d <= TEAM * SLOTS && in.nsteps >= 0 && in.nparams >= 1;
    if (in.kind == IRKGL_RHS_NBODY)
      ok_desc = ok_desc && (d % 3 == 0) && d / 3 <= kWideMaxBodies && in.nparams >= 1 + d / 3;
    else ok_desc = ok_desc && (in.kind == IRKGL_RHS_FPUT || in.kind == IRKGL_RHS_HARMONIC);
    if (!ok_desc) {
      if (tid == 0) {
        if (a.status) a.status[t] = ST_BADDESC;
        if (a.steps_done) a.steps_done[t] = 0;
        if (a.iters_total) a.iters_total[t] = 0;
      }
      continue;
    }
    const double* p = a.params + in.param_offset;
    const double h = in.h;
    long long N = a.nsteps_call ? a.nsteps_call[t] : in.nsteps;
    int st = ST_OK;
    if (a.sticky_status && a.status) {
      const int s0 = a.status[t];
      if (s0 != ST_OK) {  // stopped in an earlier call: a failure is final
        st = s0;
        N = 0;
      }
    }
    const size_t off = static_cast<size_t>(in.offset);
#pragma unroll
    for (int s = 0; s < SLOTS; s++) {
      const int l = tid + s * TEAM;
      const bool own = l < d;
      qh[s] = own ? a.q_in[off + l] : 0.0;
      vh[s] = own ? a.v_in[off + l] : 0.0;
      ql[s] = (own && a.qlo_in) ? a.qlo_in[off + l] : 0.0;
      vl[s] = (own && a.vlo_in) ? a.vlo_in[off + l] : 0.0;
    }
    for (int x = tid; x < S * d; x += TEAM) R[x] = a.rp_in ? a.rp_in[off * S + x] : 0.0;
    double H0 = 0.0, dHmax = 0.0;
    long long itot = 0;
    if (a.accumulate) {
      if (a.dH_max) dHmax = a.dH_max[t];
      if (a.iters_total) itot = a.iters_total[t];
    }
    bool have_h0 = false;
    if (a.H0_io && !a.h0_init) {
      H0 = a.H0_io[t];
      have_h0 = (H0 == H0);  // NaN: an instance joining a running batch
    }
    if (!have_h0 && a.monitor > 0 && N > 0) {
#pragma unroll
      for (int s = 0; s < SLOTS; s++) {
        const int l = tid + s * TEAM;
        if (l < d) {
          qs[l] = qh[s];
          vs[l] = vh[s];
        }
      }
      team_sync<TEAM>();
      H0 = team_energy_repro<TEAM>(in.kind, d, p, qs, vs, Q, S * dmax, red, tid);
      if (a.H0_io && tid == 0) a.H0_io[t] = H0;
    }
    double Hprev = H0;
    team_sync<TEAM>();

    long long n = 0;
    while (n < N) {
      // Eq. IRK_init2 unfused, per owned component
#pragma unroll
      for (int s = 0; s < SLOTS; s++) {
        const int l = tid + s * TEAM;
        if (l < d) {
          double Rj[S], L[S];
#pragma unroll
          for (int j = 0; j < S; j++) Rj[j] = R[j * d + l];
#pragma unroll
          for (int i = 0; i < S; i++) {
            double acc = mul(cf.nu[i * S], Rj[0]);
#pragma unroll
            for (int j = 1; j < S; j++) acc = add(acc, mul(cf.nu[i * S + j], Rj[j]));
            L[i] = mul(h, mul(cf.b[i], add(vh[s], acc)));
          }
#pragma unroll
          for (int i = 0; i < S; i++) {
            double acc = mul(cf.mu[i * S], L[0]);
#pragma unroll
            for (int j = 1; j < S; j++) acc = add(acc, mul(cf.mu[i * S + j], L[j]));
            Q[i * d + l] = add(qh[s], acc);
          }
        }
        dmin[s] = inf;
        dprev[s] = inf;
      }
      team_sync<TEAM>();
      int k = 0;
      for (;;) {
        k++;
        team_rhs_repro<TEAM>(in.kind, d, p, cf, h, Q, R, tid);
        team_sync<TEAM>();
        bool cond = true, bad = false;
#pragma unroll
        for (int s = 0; s < SLOTS; s++) {
          const int l = tid + s * TEAM;
          if (l < d) {
            double Rj[S];
#pragma unroll
            for (int j = 0; j < S; j++) Rj[j] = R[j * d + l];
            double delta = 0.0;
#pragma unroll
            for (int i = 0; i < S; i++) {
              double acc = mul(cf.c[i], vh[s]);
#pragma unroll
              for (int j = 0; j < S; j++) acc = add(acc, mul(cf.eta[i * S + j], Rj[j]));
              const double x = add(qh[s], mul(h, acc));
              bad = bad || !(abs_bits(x) < INF_BITS);
              const double dd = fabs(sub(x, Q[i * d + l]));
              if (dd > delta) delta = dd;
              Q[i * d + l] = x;
            }
            const double m = dprev[s] <= delta ? dprev[s] : delta;
            cond = cond && ((delta == 0.0) || (dmin[s] <= m));
            dmin[s] = dmin[s] <= dprev[s] ? dmin[s] : dprev[s];
            dprev[s] = delta;
          }
        }
        team_sync<TEAM>();  // new Q visible to the whole team before the next g
        const bool any_bad = team_or<TEAM>(bad);
        const bool stop = team_and<TEAM>(cond);
        if (any_bad) {
          st = ST_NONFINITE;
          break;
        }
        if (stop) break;
        if (k >= a.kmax) {
          st = ST_MAXITER;
          break;
        }
      }
      itot += k;
      if (st != ST_OK) break;
      // Eq. qnvn2, compensated, per owned component
#pragma unroll
      for (int s = 0; s < SLOTS; s++) {
        const int l = tid + s * TEAM;
        if (l < d) {
          double sR = R[l], scR = mul(cf.c[0], R[l]);
#pragma unroll
          for (int i = 1; i < S; i++) {
            const double Ri = R[i * d + l];
            sR = add(sR, Ri);
            scR = add(scR, mul(cf.c[i], Ri));
          }
          repro_two_sum_add(vh[s], vl[s], sR);
          const double dq = add(mul(h, vh[s]), sub(mul(h, vl[s]), mul(h, scR)));
          repro_two_sum_add(qh[s], ql[s], dq);
        }
      }
      n++;
      if (a.monitor > 0 && (n % a.monitor) == 0) {
#pragma unroll
        for (int s = 0; s < SLOTS; s++) {
          const int l = tid + s * TEAM;
          if (l < d) {
            qs[l] = qh[s];
            vs[l] = vh[s];
          }
        }
        team_sync<TEAM>();  // (Q is free until the next step's guess: the terms' scratch)
        const double Hn = team_energy_repro<TEAM>(in.kind, d, p, qs, vs, Q, S * dmax, red, tid);
        double dH;
        if (a.monitor_local) {
          dH = fabs(div(sub(Hn, Hprev), Hprev));
          Hprev = Hn;
        } else {
          dH = fabs(div(sub(Hn, H0), H0));
        }
        if (dH > dHmax) dHmax = dH;
      }
      team_sync<TEAM>();
    }

#pragma unroll
    for (int s = 0; s < SLOTS; s++) {
      const int l = tid + s * TEAM;
      if (l < d) {
        a.q_out[off + l] = qh[s];
        a.v_out[off + l] = vh[s];
        if (a.qlo_out) a.qlo_out[off + l] = ql[s];
        if (a.vlo_out) a.vlo_out[off + l] = vl[s];
      }
    }
    if (a.rp_out && st == ST_OK)
      for (int x = tid; x < S * d; x += TEAM) a.rp_out[off * S + x] = R[x];
    if (tid == 0) {
      if (a.dH_max) a.dH_max[t] = dHmax;
      if (a.iters_total) a.iters_total[t] = itot;
      if (a.steps_done) a.steps_done[t] = n;
      if (a.status) a.status[t] = st;
    }
    team_sync<TEAM>();
  }
}

}  // namespace irkgl
