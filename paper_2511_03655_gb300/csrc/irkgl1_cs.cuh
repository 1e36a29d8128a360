// irkgl1_cs.cuh -- component-split tile of the first-order (mu form) kernel.
//
// The first-order counterpart of irkgl_cs.cuh (Eqs. Yi2, IRK_init, IRK_FP,
// stopping on all D components, Eq. yn2): a trajectory of D components
// (D = 2 or 4) runs on D lanes, lane r keeping component r of y
// (compensated), of the eight stage values Y_i and of the eight increments
// L_i.  The mixings Y_i = y + sum_j mu_ij L_j (sweeps) and
// Y_i = y + sum_j nu_ij Lprev_j (guess) then use only a lane's own registers
// with compile-time coefficients, as FP64 FMA chains (MIX = 0) or as exact
// fixed-point sums on the integer pipes rounded once (MIX = 1: mu is on the
// 2^-62 grid, nu is rounded to 2^-47 because it only seeds the guess).
// f needs all components of a stage: lane r evaluates stages r*SPL .. r*SPL
// + SPL - 1 (SPL = 8/D); the components come and go by D - 1 rotation
// shuffles per stage each way.  Stage and component indices that depend on
// the lane are resolved with unrolled selects, so nothing is indexed
// dynamically (no local memory).
//
// With MIX = 0 the results equal the stage-split first-order kernel's to
// roundoff (the sums over stages are associated differently); with MIX = 1
// the mixing is the correctly rounded exact sum.
#pragma once

#include "irkgl_first_order.cuh"

namespace irkgl {

// sum_j coef_ij L_j for row i (compile-time after unrolling) from the offset
// fixed-point column rb with shared exponent emax: coef = mu (IS_NU false,
// exact) or nu (rounded).
template <bool IS_NU>
__device__ __forceinline__ double fixed_row1(int i, const unsigned long long (&rb)[S], int emax) {
  // one accumulator: a negative coefficient takes the two's complement of
  // the operand, and the row constant rbias absorbs the n_ij 2^64 that adds
  U128 P{0u, 0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < S; j++) {
    const int k = i * S + j;
    const unsigned long long m = IS_NU ? irkgl_nu_mag(k) : irkgl_mu_mag(k);
    const bool neg = IS_NU ? irkgl_nu_neg(k) : irkgl_mu_neg(k);
    mac64(P, m, neg ? (0ull - rb[j]) : rb[j]);
  }
  if (IS_NU) sub128(P, irkgl_nu_rbias(i, 0), irkgl_nu_rbias(i, 1), irkgl_nu_rbias(i, 2), irkgl_nu_rbias(i, 3));
  else sub128(P, irkgl_mu_rbias(i, 0), irkgl_mu_rbias(i, 1), irkgl_mu_rbias(i, 2), irkgl_mu_rbias(i, 3));
  constexpr int shift = IS_NU ? IRKGL_NU_SHIFT : IRKGL_MU_SHIFT;
  return s128_to_double(P, emax - 1083 - shift);
}

// arr[idx] for a runtime idx < N without dynamic register indexing
template <int N>
__device__ __forceinline__ double pick(const double (&arr)[N], int idx) {
  double x = arr[0];
#pragma unroll
  for (int k = 1; k < N; k++) x = (idx == k) ? arr[k] : x;
  return x;
}
template <int N>
__device__ __forceinline__ void place(double (&arr)[N], int idx, double v) {
#pragma unroll
  for (int k = 0; k < N; k++) arr[k] = (idx == k) ? v : arr[k];
}

template <class Rhs, int BLOCK, int MIX = 0>
__global__ void __launch_bounds__(BLOCK)
    irkgl1_kernel_cs(const __grid_constant__ KArgs1 a, const __grid_constant__ Coef1 cf) {
  constexpr int D = Rhs::D;
  static_assert(D == 2 || D == 4, "component split: 2 or 4 components, one per lane");
  constexpr int SPL = S / D;  // f stages evaluated per lane
  const int lane = threadIdx.x & 31;
  const int r = lane % D;  // the component this lane owns
  const int gbase = lane - r;
  const bool leader = (r == 0);

  Rhs rhs;
  rhs.load_params(a.params);
  double yh = 0.0, yl = 0.0;
  unsigned long long dmin = INF_BITS, dprev = INF_BITS;
  double Lc[S], Yc[S];  // own component of all eight stages
  double h = 0.0, H0 = 0.0, invH0 = 0.0, dHmax = 0.0;
  double Hprev = 0.0, invHprev = 0.0;
  long long n = 0, N = 0, itot = 0;
  int traj = -1, st = ST_OK;
  bool active = false, exhausted = false;
  unsigned leaders_all = 0;
#pragma unroll
  for (int g = 0; g < 32; g += D) leaders_all |= 1u << g;

  auto energy = [&](unsigned mask) {
    double yf[D];
#pragma unroll
    for (int c = 0; c < D; c++) yf[c] = __shfl_sync(mask, yh, gbase + c);
    return rhs.H(yf);
  };

  for (;;) {
    // ---------------- refill
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
            const size_t off = static_cast<size_t>(t) * D + r;
            yh = a.y_in[off];
            yl = a.ylo_in ? a.ylo_in[off] : 0.0;
            const size_t loff = static_cast<size_t>(t) * S * D + r;
#pragma unroll
            for (int i = 0; i < S; i++) Lc[i] = a.lp_in ? a.lp_in[loff + i * D] : 0.0;
            double hb[SPL];
#pragma unroll
            for (int tt = 0; tt < SPL; tt++) hb[tt] = h * cf.b[r * SPL + tt];
            rhs.set_step(hb);
          }
        }
      }
    }
    if (__all_sync(FULL, exhausted && !active)) break;

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

    const bool stepping = active && (n < N);
    const unsigned stepmask = __ballot_sync(FULL, stepping);
    if (stepping) {
      // init, Eq. IRK_init: Y_i = y + sum_j nu_ij Lprev_j (own component)
      if constexpr (MIX == 1) {
        unsigned long long rb[S];
        bool nf;
        const int emax = fixed_column(Lc, rb, nf);
#pragma unroll
        for (int i = 0; i < S; i++) {
          double T = fixed_row1<true>(i, rb, emax);
          if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
          Yc[i] = yh + T;
        }
      } else {
#pragma unroll
        for (int i = 0; i < S; i++) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < S; j++) acc = fma(cf.nu[i * S + j], Lc[j], acc);
          Yc[i] = yh + acc;
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
          // L_i = h b_i f(Y_i): this lane's stages, components by rotation
#pragma unroll
          for (int t = 0; t < SPL; t++) {
            const int myst = r * SPL + t;
            double x[D];
#pragma unroll
            for (int c = 0; c < D; c++) x[c] = 0.0;
            place<D>(x, r, pick<S>(Yc, myst));
#pragma unroll
            for (int kk = 1; kk < D; kk++) {
              // pull from src = r + kk: it sends its component at the stage of
              // the lane kk below it
              const int src = (r + kk) % D;
              const int req = (r - kk + D) % D;  // the lane this lane serves
              const double send = pick<S>(Yc, req * SPL + t);
              const double got = __shfl_sync(sweepmask, send, gbase + src);
              place<D>(x, src, got);
            }
            double L2[D];
            rhs.stage_L(t, x, L2);
            place<S>(Lc, myst, L2[r]);
#pragma unroll
            for (int kk = 1; kk < D; kk++) {
              // pull from src = r - kk its result for this lane's component
              const int src = (r - kk + D) % D;
              const int dst = (r + kk) % D;  // the lane pulling from this lane
              const double send = pick<D>(L2, dst);
              const double got = __shfl_sync(sweepmask, send, gbase + src);
              place<S>(Lc, src * SPL + t, got);
            }
          }
          // Yn_i = y + sum_j mu_ij L_j (Eq. Yi2), own component
          unsigned long long dl = 0;
          if constexpr (MIX == 1) {
            unsigned long long rb[S];
            bool nf;
            const int emax = fixed_column(Lc, rb, nf);
#pragma unroll
            for (int i = 0; i < S; i++) {
              double T = fixed_row1<false>(i, rb, emax);
              if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
              const double yn = yh + T;
              dl = umax64(dl, abs_bits(yn - Yc[i]));
              Yc[i] = yn;
            }
          } else {
#pragma unroll
            for (int i = 0; i < S; i++) {
              double acc = 0.0;
#pragma unroll
              for (int j = 0; j < S; j++) acc = fma(cf.mu[i * S + j], Lc[j], acc);
              const double yn = yh + acc;
              dl = umax64(dl, abs_bits(yn - Yc[i]));
              Yc[i] = yn;
            }
          }
          int bad_i = (dl >= INF_BITS) ? 1 : 0;
          const bool cond = (dl == 0) || (dmin <= umin64(dprev, dl));
          dmin = umin64(dmin, dprev);
          dprev = dl;
          int stop_i = cond ? 1 : 0;
#pragma unroll
          for (int off = 1; off < D; off <<= 1) {
            bad_i |= __shfl_xor_sync(sweepmask, bad_i, off);
            stop_i &= __shfl_xor_sync(sweepmask, stop_i, off);
          }
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
        // update, Eq. yn2, own component, compensated
        double x = Lc[0];
#pragma unroll
        for (int i = 1; i < S; i++) x = x + Lc[i];
        two_sum_add(yh, yl, x);
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

    const bool fin = active && (n >= N || st != ST_OK);
    if (fin) {
      const size_t off = static_cast<size_t>(traj) * D + r;
      a.y_out[off] = yh;
      if (a.ylo_out) a.ylo_out[off] = yl;
      if (a.lp_out && st == ST_OK) {
        const size_t loff = static_cast<size_t>(traj) * S * D + r;
#pragma unroll
        for (int i = 0; i < S; i++) a.lp_out[loff + i * D] = Lc[i];
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

template <class Rhs, int BLOCK, int MIX>
void launch1_cs_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs1& a, const Coef1& c) {
  irkgl1_kernel_cs<Rhs, BLOCK, MIX><<<grid, block, 0, st>>>(a, c);
}

}  // namespace irkgl
