// irkgl_cs.cuh -- the "component split" tile of the batched IRKGL16 kernel
// for two-component right-hand sides (Kepler, Henon-Heiles).
//
// The stage-split tiles (irkgl_kernel with LPT lanes) give each lane a block
// of stages and every component; the stage mixing of Eq. Qi2 then needs the
// other lanes' R by shuffle and, with LPT > 1, the eta rows of its own
// stages from shared memory.  Here the two lanes of a trajectory split the
// COMPONENTS instead: lane r keeps component r of q, v (compensated), of all
// eight stage values Q_i, of all eight increments R_i and of c_i v.  So
//   * the mixing Qn_i = q + h (c_i v + sum_j eta_ij R_j) of a lane involves
//     only its own registers, with every eta_ij (or its fixed-point form) a
//     compile-time constant-bank operand, the same on both lanes;
//   * Delta, Eq. stopping, and the compensated update (Eq. qnvn2) are per
//     component and need no reduction across lanes;
//   * only g needs both components: lane r evaluates stages 4r..4r+3 from
//     its own component and the partner's (one shuffle per stage) and hands
//     the partner its component of the result (one shuffle per stage).
// A lane holds 3 x 8 stage values of one component instead of 3 x 4 x 2 or
// 3 x 8 x 2, so more warps fit on an SM.
//
// The operation sequence is that of an existing tile, so the results are
// bit-identical to it: with FP64 mixing (MIX = 0) to the stage-split tile
// with two lanes (the update sums each half of the stages, then adds the
// halves, as that tile's butterfly does); with fixed-point mixing (MIX = 1)
// to the one-lane tile (sequential update sums).
#pragma once

#include "irkgl_device.cuh"

namespace irkgl {

template <class Rhs, int BLOCK, int MIX = 0, int MINB = 1>
__global__ void __launch_bounds__(BLOCK, MINB)
    irkgl_kernel_cs(const __grid_constant__ KArgs a, const __grid_constant__ Coef cf) {
  static_assert(Rhs::D == 2, "component split: two components, one per lane");
  static_assert(!time_dependent<Rhs>::value, "time-dependent right-hand sides use the stage-split tiles");
  constexpr int SPL = 4;  // g stages evaluated per lane
  const int lane = threadIdx.x & 31;
  const int r = lane & 1;  // the component this lane owns
  const int gbase = lane - r;
  const int i0 = 4 * r;
  const bool leader = (r == 0);

  Rhs rhs;
  rhs.load_params(a.params);
  double qh = 0.0, ql = 0.0, vh = 0.0, vl = 0.0;  // own component, compensated pairs
  unsigned long long dmin = INF_BITS, dprev = INF_BITS;
  double Rc[S], Qc[S], cvc[S];  // own component of all eight stages
  double h = 0.0, H0 = 0.0, invH0 = 0.0, dHmax = 0.0;
  double Hprev = 0.0, invHprev = 0.0;
  long long n = 0, N = 0, itot = 0;
  int traj = -1, st = ST_OK;
  bool active = false, exhausted = false;
  constexpr unsigned leaders_all = 0x55555555u;

  // H(q, v) of the pair's trajectory (both lanes get it)
  auto energy = [&](unsigned mask) {
    const double qo = __shfl_xor_sync(mask, qh, 1);
    const double vo = __shfl_xor_sync(mask, vh, 1);
    double qf[2], vf[2];
    qf[0] = r ? qo : qh;
    qf[1] = r ? qh : qo;
    vf[0] = r ? vo : vh;
    vf[1] = r ? vh : vo;
    return rhs.H(qf, vf);
  };

  for (;;) {
    // ---------------- refill: pairs without a trajectory grab the next one
    const bool need = !active && !exhausted;
    const unsigned needmask = __ballot_sync(FULL, need) & leaders_all;
    if (needmask) {
      const int first = __ffs(needmask) - 1;
      unsigned base = 0;
      if (lane == first) base = atomicAdd(a.counter, static_cast<unsigned>(__popc(needmask)));
      base = __shfl_sync(FULL, base, first);
      if (need) {
        const unsigned idx = base + __popc(needmask & ((1u << gbase) - 1u));
        if (idx >= static_cast<unsigned>(a.batch)) {
          exhausted = true;
        } else {
          int t = a.order ? a.order[idx] : static_cast<int>(idx);
          if (t < 0 || t >= a.batch) t = -1;
          traj = t;
          if (t >= 0) {
            active = true;
            st = ST_OK;
            n = 0;
            itot = 0;
            dHmax = 0.0;
            N = a.nsteps ? a.nsteps[t] : a.nsteps_all;
            if (a.sticky_status && a.status) {
              const int s0 = a.status[t];
              if (s0 != ST_OK) {  // a failure is final: keep the status, take no step
                st = s0;
                N = 0;
              }
            }
            h = a.h ? a.h[t] : a.h_all;
            if (a.accumulate) {
              if (a.dH_max) dHmax = a.dH_max[t];
              if (a.iters_total) itot = a.iters_total[t];
            }
            if (a.H0_io && !a.h0_init) {
              H0 = a.H0_io[t];
              invH0 = 1.0 / H0;
              Hprev = H0;
              invHprev = invH0;
            }
            if (a.param_stride) rhs.load_params(a.params + static_cast<size_t>(t) * a.param_stride);
            const size_t off = static_cast<size_t>(t) * 2 + r;
            qh = a.q_in[off];
            vh = a.v_in[off];
            ql = a.qlo_in ? a.qlo_in[off] : 0.0;
            vl = a.vlo_in ? a.vlo_in[off] : 0.0;
            const size_t roff = static_cast<size_t>(t) * S * 2 + r;
#pragma unroll
            for (int i = 0; i < S; i++) Rc[i] = a.rp_in ? a.rp_in[roff + 2 * i] : 0.0;
            double hb[SPL];
#pragma unroll
            for (int tt = 0; tt < SPL; tt++) hb[tt] = h * cf.b[i0 + tt];
            rhs.set_step(hb);
          }
        }
      }
    }
    if (__all_sync(FULL, exhausted && !active)) break;

    // ---------------- H_0 before the first step (exact ballot of the lanes)
    {
      const bool want = active && n == 0 && a.monitor > 0 && (!a.H0_io || a.h0_init || (H0 != H0 && N > 0));
      const unsigned h0mask = __ballot_sync(FULL, want);
      if (want) {
        H0 = energy(h0mask);
        invH0 = 1.0 / H0;
        Hprev = H0;
        invHprev = invH0;
        if (a.H0_io && leader) a.H0_io[traj] = H0;
      }
    }

    // ---------------- one step for every pair that still has steps to take
    const bool stepping = active && (n < N);
    const unsigned stepmask = __ballot_sync(FULL, stepping);
    if (stepping) {
      // init (Eq. IRK_init2, fused): Q_i = q + h (c_i v + sum_k W_ik Rprev_k)
      if constexpr (MIX == 1) {
        unsigned long long rb[S];
        bool nf;
        const int emax = fixed_column(Rc, rb, nf);
#pragma unroll
        for (int i = 0; i < S; i++) {
          // c_i v + T in one rounding (fixed-point tiles: no c_i v array)
          double T = fixed_row<true>(i, rb, emax);
          if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
          Qc[i] = fma(h, fma(cf.c[i], vh, T), qh);
        }
      } else {
#pragma unroll
        for (int i = 0; i < S; i++) {
          cvc[i] = cf.c[i] * vh;
          double acc = cvc[i];
#pragma unroll
          for (int j = 0; j < S; j++) acc = fma(cf.W[i * S + j], Rc[j], acc);
          Qc[i] = fma(h, acc, qh);
        }
      }
      dmin = INF_BITS;
      dprev = INF_BITS;
      int k = 0;
      bool conv = false;
      for (;;) {
        const unsigned sweepmask = __ballot_sync(stepmask, !conv);
        if (sweepmask == 0) break;
        if (!conv) {
          k++;
          // R_i = h b_i g(Q_i) (Eq. Gi): this lane's four stages, then swap
          // the components with the partner
#pragma unroll
          for (int t = 0; t < SPL; t++) {
            const double own = r ? Qc[4 + t] : Qc[t];   // my component, my stage i0 + t
            const double send = r ? Qc[t] : Qc[4 + t];  // my component, the partner's stage
            const double oth = __shfl_xor_sync(sweepmask, send, 1);
            double x[2], R2[2];
            x[0] = r ? oth : own;
            x[1] = r ? own : oth;
            rhs.stage_R(t, x, R2);
            const double mine = r ? R2[1] : R2[0];
            const double give = r ? R2[0] : R2[1];
            const double got = __shfl_xor_sync(sweepmask, give, 1);  // my component, partner's stage
            Rc[t] = r ? got : mine;
            Rc[4 + t] = r ? mine : got;
          }
          // Qn_i = q + h (c_i v + sum_j eta_ij R_j) (Eq. Qi2), own component
          unsigned long long dl = 0;
          if constexpr (MIX == 1) {
            unsigned long long rb[S];
            bool nf;
            const int emax = fixed_column(Rc, rb, nf);
#pragma unroll
            for (int i = 0; i < S; i++) {
              double T = fixed_row<false>(i, rb, emax);
              if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
              const double qn = fma(h, fma(cf.c[i], vh, T), qh);
              dl = umax64(dl, abs_bits(qn - Qc[i]));
              Qc[i] = qn;
            }
          } else {
#pragma unroll
            for (int i = 0; i < S; i++) {
              double acc = cvc[i];
#pragma unroll
              for (int j = 0; j < S; j++) acc = fma(cf.eta[i * S + j], Rc[j], acc);
              const double qn = fma(h, acc, qh);
              dl = umax64(dl, abs_bits(qn - Qc[i]));
              Qc[i] = qn;
            }
          }
          // Eq. stopping on the own component; the pair stops (or fails)
          // together: the shuffles run on both lanes, no short-circuit
          int bad_i = (dl >= INF_BITS) ? 1 : 0;
          const bool cond = (dl == 0) || (dmin <= umin64(dprev, dl));
          dmin = umin64(dmin, dprev);
          dprev = dl;
          int stop_i = cond ? 1 : 0;
          bad_i |= __shfl_xor_sync(sweepmask, bad_i, 1);
          stop_i &= __shfl_xor_sync(sweepmask, stop_i, 1);
          if (bad_i) {
            st = ST_NONFINITE;
            conv = true;
          } else if (stop_i) {
            conv = true;
          } else if (k >= a.kmax) {
            st = ST_MAXITER;
            conv = true;
          }
        }
      }

      if (a.iters_hist && leader && n < a.hist_len)
        a.iters_hist[static_cast<size_t>(traj) * a.hist_len + n] = k;
      itot += k;

      const unsigned okmask = __ballot_sync(stepmask, st == ST_OK);
      if (st == ST_OK) {
        // update (Eq. qnvn2), own component, compensated
        double x, y;
        if constexpr (MIX == 1) {
          // the one-lane tile's order: sequential over the stages
          x = Rc[0];
          y = cf.c[0] * Rc[0];
#pragma unroll
          for (int i = 1; i < S; i++) {
            x = x + Rc[i];
            y = fma(cf.c[i], Rc[i], y);
          }
        } else {
          // the two-lane stage-split tile's order: each half, then the halves
          double x0 = Rc[0], y0 = cf.c[0] * Rc[0], x1 = Rc[4], y1 = cf.c[4] * Rc[4];
#pragma unroll
          for (int i = 1; i < 4; i++) {
            x0 = x0 + Rc[i];
            y0 = fma(cf.c[i], Rc[i], y0);
            x1 = x1 + Rc[4 + i];
            y1 = fma(cf.c[4 + i], Rc[4 + i], y1);
          }
          x = x0 + x1;
          y = y0 + y1;
        }
        two_sum_add(vh, vl, x);
        const double dq = fma(h, vh, fma(h, vl, -(h * y)));
        two_sum_add(qh, ql, dq);
        n++;
        if (a.monitor > 0) {
          const bool mon = (n % a.monitor) == 0;
          const unsigned monmask = __ballot_sync(okmask, mon);
          if (mon) {
            const double Hn = energy(monmask);
            double dH;
            if (a.monitor_local) {
              dH = fabs((Hn - Hprev) * invHprev);
              Hprev = Hn;
              invHprev = 1.0 / Hn;
            } else {
              dH = fabs((Hn - H0) * invH0);
            }
            if (dH > dHmax) dHmax = dH;
          }
        }
      }
    }

    // ---------------- finish
    const bool fin = active && (n >= N || st != ST_OK);
    if (fin) {
      const size_t off = static_cast<size_t>(traj) * 2 + r;
      a.q_out[off] = qh;
      a.v_out[off] = vh;
      if (a.qlo_out) a.qlo_out[off] = ql;
      if (a.vlo_out) a.vlo_out[off] = vl;
      if (a.rp_out && st == ST_OK) {
        const size_t roff = static_cast<size_t>(traj) * S * 2 + r;
#pragma unroll
        for (int i = 0; i < S; i++) a.rp_out[roff + 2 * i] = Rc[i];
      }
      if (leader) {
        if (a.dH_max) a.dH_max[traj] = dHmax;
        if (a.iters_total) a.iters_total[traj] = itot;
        if (a.status) a.status[traj] = st;
        if (a.steps_done) a.steps_done[traj] = n;
      }
      active = false;
    }
  }
}

}  // namespace irkgl
