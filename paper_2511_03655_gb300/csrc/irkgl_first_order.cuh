// irkgl_first_order.cuh -- first-order IRKGL16 (the mu form) for y' = f(y).
//
// The exactly-symplectic floating-point form of arXiv 2511.03655, Sec. 2.4
// (Eq. Yi2), iterated as in Eqs. IRK_init / IRK_FP, per step:
//
//   init   Y_i = y + sum_j nu_ij Lprev_j                    Eq. IRK_init (Eq. Pol0)
//   sweep  L_i = h b_i f(Y_i)                                Eq. IRK_FP
//          Yn_i = y + sum_j mu_ij L_j                        Eq. Yi2
//          Delta_l = max_i |Yn_il - Y_il| on all D components, Eq. stopping
//   update y += sum_i L_i, compensated (TwoSum + Fast2Sum)  Eq. yn2, Sec. 5
//
// Same layout as the second-order kernel: LPT lanes per trajectory, SPL =
// 8/LPT stages per lane, component l of the compensated state and its
// stopping history on lane l % LPT; stage values of other lanes are gathered
// with shuffles; |x|, max and the vote run on integer bit patterns.
#pragma once

#include "irkgl_device.cuh"

namespace irkgl {

struct Coef1 {
  double b[S];
  double mu[S * S];  // Eq. Yi2, row-major [i*s+j] for an s-stage kernel
  double nu[S * S];  // Eq. IRK_init, scaled by 1/b_j, same layout
};

struct KArgs1 {
  int batch;
  int kmax;
  int monitor;
  int hist_len;
  const double* y_in;
  const double* ylo_in;  // may be null (zeros)
  const double* lp_in;   // [batch][s][D] L of the previous step, may be null (zeros)
  double* y_out;
  double* ylo_out;       // may be null
  double* lp_out;        // may be null
  const long long* nsteps;
  long long nsteps_all;
  const double* h;
  double h_all;
  const int* order;
  int* iters_hist;
  long long* iters_total;
  double* dH_max;
  int* status;
  long long* steps_done;
  unsigned int* counter;
  const double* params;
  double* H0_io;  // read, or written when h0_init or when the entry is NaN (computed at
                  // the trajectory's first step of the call)
  int h0_init;
  int accumulate;
  int monitor_local;  // 1: dH_max = max_n |(H_n - H_{n-1}) / H_{n-1}| (Eq. DHlocmax)
};

// ------------------------------------------------------------------------
// first-order right-hand sides: stage_L(t, y, L) sets L = (h b_i) f(y) for
// the lane's stage t; H(y) is the conserved Hamiltonian
// ------------------------------------------------------------------------

// Charged particle near a Schwarzschild black hole in a magnetic field,
// Eq. Ham_SBH, y = (r, theta, p_r, p_theta), params {E, L, beta}.  With
// u = 1 - 2/r and s = sin^2 theta (derivatives of Eq. Ham_SBH):
//   r' = u p_r,  theta' = p_theta / r^2,
//   p_r' = -(p_r^2/r^2 + E^2/(r^2 u^2) - p_theta^2/r^3 - L^2/(r^3 s) + beta^2 r s/4),
//   p_theta' = (L^2/(r^2 s^2) - beta^2 r^2/4) sin theta cos theta.
template <int SPL, bool FX_TRIG = true>
struct Schwarzschild {
  static constexpr int D = 4;
  // sin and cos of theta: fixed point on the integer pipes (FX_TRIG), or the
  // FP64 sincos.  Tiles whose mixing already fills the integer pipes (the
  // fixed-point component split) run faster with the FP64 form, tiles with
  // FP64 mixing with the fixed-point one (measured on GB300: 1.72e8 against
  // 1.49e8, and 1.66e8 against 1.41e8, trajectory-steps/s).
  __device__ static __forceinline__ void trig(double x, double& sn, double& cs) {
    if constexpr (FX_TRIG) sincos_fx(x, sn, cs);
    else sincos(x, &sn, &cs);
  }
  double E2, L2, Lc, bh, b2q;  // E^2, L^2, L, beta/2, beta^2/4
  double hb[SPL];
  __device__ void load_params(const double* p) {
    E2 = p[0] * p[0];
    Lc = p[1];
    L2 = p[1] * p[1];
    bh = 0.5 * p[2];
    b2q = 0.25 * (p[2] * p[2]);
  }
  __device__ void set_step(const double (&x)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) hb[t] = x[t];
  }
  __device__ __forceinline__ void stage_L(int t, const double (&y)[D], double (&L)[D]) const {
    const double r = y[0], pr = y[2], pth = y[3];
    double sn, cs;
    trig(y[1], sn, cs);
    const double s = sn * sn;
    const double ri = rcp_int(r);
    const double u = fma(-2.0, ri, 1.0);
    const double ui = rcp_int(u);
    const double si = rcp_int(s);
    const double r2i = ri * ri;
    const double r3i = r2i * ri;
    // dH/dr
    double dr = pr * pr * r2i;
    dr = fma(E2 * r2i, ui * ui, dr);
    dr = fma(-(pth * pth), r3i, dr);
    dr = fma(-L2 * r3i, si, dr);
    dr = fma(b2q * r, s, dr);
    // dH/dtheta
    const double dth = fma(-L2 * r2i, si * si, b2q * (r * r)) * (sn * cs);
    L[0] = hb[t] * (u * pr);
    L[1] = hb[t] * (pth * r2i);
    L[2] = -(hb[t] * dr);
    L[3] = -(hb[t] * dth);
  }
  __device__ double H(const double (&y)[D]) const {
    const double r = y[0], pr = y[2], pth = y[3];
    double sn, cs;
    trig(y[1], sn, cs);
    const double s = sn * sn;
    const double u = 1.0 - 2.0 / r;
    const double a = fma(-bh * (r * r), s, Lc);
    const double r2 = r * r;
    return 0.5 * u * (pr * pr) - 0.5 * E2 / u + 0.5 * (pth * pth) / r2 + 0.5 * (a * a) / (r2 * s);
  }
};

// q' = p, p' = -omega^2 q (D = 2), params {omega}.
template <int SPL>
struct Harmonic1 {
  static constexpr int D = 2;
  double w2;
  double hb[SPL];
  __device__ void load_params(const double* p) { w2 = p[0] * p[0]; }
  __device__ void set_step(const double (&x)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) hb[t] = x[t];
  }
  __device__ __forceinline__ void stage_L(int t, const double (&y)[D], double (&L)[D]) const {
    L[0] = hb[t] * y[1];
    L[1] = -(hb[t] * (w2 * y[0]));
  }
  __device__ double H(const double (&y)[D]) const { return 0.5 * fma(y[1], y[1], w2 * (y[0] * y[0])); }
};

template <class Rhs, int LPT, int NS>
__device__ __forceinline__ double group_energy1(const Rhs& rhs, const double (&yh)[NS], unsigned mask,
                                                int gbase) {
  constexpr int D = Rhs::D;
  double yf[D];
#pragma unroll
  for (int l = 0; l < D; l++) yf[l] = owned_get<LPT, NS>(yh, l, mask, gbase);
  return rhs.H(yf);
}

template <class Rhs, int LPT, int BLOCK, int NST = S>
__global__ void __launch_bounds__(BLOCK)
    irkgl1_kernel(const __grid_constant__ KArgs1 a, const __grid_constant__ Coef1 cf) {
  // NST stages (the s of an s-stage IRKGL scheme; 8 for IRKGL16); the
  // tables hold the NST x NST matrices row-major with stride NST
  static_assert(NST >= 1 && NST <= S && NST % LPT == 0, "stages must split evenly over the lanes");
  constexpr int D = Rhs::D;
  constexpr int SPL = NST / LPT;
  constexpr int NS = (D + LPT - 1) / LPT;
  constexpr int PAD = NST + 1;

  __shared__ double s_mu[(LPT > 1) ? NST * PAD : 1];
  __shared__ double s_nu[(LPT > 1) ? NST * PAD : 1];
  if constexpr (LPT > 1) {
    for (int x = threadIdx.x; x < NST * NST; x += BLOCK) {
      s_mu[(x / NST) * PAD + (x % NST)] = cf.mu[x];
      s_nu[(x / NST) * PAD + (x % NST)] = cf.nu[x];
    }
    __syncthreads();
  }

  const int lane = threadIdx.x & 31;
  const int r = lane % LPT;
  const int gbase = lane - r;
  const int i0 = r * SPL;
  const bool leader = (r == 0);
#define IRKGL1_MU(t, j) ((LPT == 1) ? cf.mu[(t) * NST + (j)] : s_mu[(i0 + (t)) * PAD + (j)])
#define IRKGL1_NU(t, j) ((LPT == 1) ? cf.nu[(t) * NST + (j)] : s_nu[(i0 + (t)) * PAD + (j)])

  Rhs rhs;
  rhs.load_params(a.params);
  double yh[NS], yl[NS];
  unsigned long long dmin[NS], dprev[NS];
  double L[SPL][D];  // own stages' L (Lprev between steps)
  double Y[SPL][D];  // own stages' values
  double h = 0.0, H0 = 0.0, invH0 = 0.0, dHmax = 0.0;
  double Hprev = 0.0, invHprev = 0.0;  // local-error monitor
  long long n = 0, N = 0, itot = 0;
  int traj = -1, st = ST_OK;
  bool active = false, exhausted = false;

  unsigned leaders_all = 0;
#pragma unroll
  for (int g = 0; g < 32; g += LPT) leaders_all |= 1u << g;

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
            const size_t off = static_cast<size_t>(t) * D;
#pragma unroll
            for (int s = 0; s < NS; s++) {
              const int l = s * LPT + r;
              const bool in = l < D;
              yh[s] = in ? a.y_in[off + l] : 0.0;
              yl[s] = (a.ylo_in && in) ? a.ylo_in[off + l] : 0.0;
            }
            const size_t loff = static_cast<size_t>(t) * NST * D;
#pragma unroll
            for (int tt = 0; tt < SPL; tt++)
#pragma unroll
              for (int l = 0; l < D; l++) L[tt][l] = a.lp_in ? a.lp_in[loff + (i0 + tt) * D + l] : 0.0;
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
        H0 = group_energy1<Rhs, LPT, NS>(rhs, yh, h0mask, gbase);
        invH0 = 1.0 / H0;
        Hprev = H0;
        invHprev = invH0;
        if (a.H0_io && leader) a.H0_io[traj] = H0;
      }
    }

    // ---------------- one step
    const bool stepping = active && (n < N);
    const unsigned stepmask = __ballot_sync(FULL, stepping);
    if (stepping) {
      // init, Eq. IRK_init: Y_i = y + sum_j nu_ij Lprev_j
#pragma unroll
      for (int l = 0; l < D; l++) {
        const double ylv = owned_get<LPT, NS>(yh, l, stepmask, gbase);
        double acc[SPL];
#pragma unroll
        for (int t = 0; t < SPL; t++) acc[t] = 0.0;
#pragma unroll
        for (int j = 0; j < NST; j++) {
          double Lj;
          if constexpr (LPT == 1) Lj = L[j][l];
          else Lj = __shfl_sync(stepmask, L[j % SPL][l], gbase + j / SPL);
#pragma unroll
          for (int t = 0; t < SPL; t++) acc[t] = fma(IRKGL1_NU(t, j), Lj, acc[t]);
        }
#pragma unroll
        for (int t = 0; t < SPL; t++) Y[t][l] = ylv + acc[t];
      }
#pragma unroll
      for (int s = 0; s < NS; s++) {
        dmin[s] = INF_BITS;
        dprev[s] = INF_BITS;
      }
      int k = 0;
      bool conv = false;
      for (;;) {
        const unsigned sweepmask = __ballot_sync(stepmask, !conv);
        if (sweepmask == 0) break;
        if (!conv) {
          k++;
#pragma unroll
          for (int t = 0; t < SPL; t++) rhs.stage_L(t, Y[t], L[t]);
          bool cond_own = true, bad = false;
#pragma unroll
          for (int l = 0; l < D; l++) {
            const double ylv = owned_get<LPT, NS>(yh, l, sweepmask, gbase);
            double acc[SPL];
#pragma unroll
            for (int t = 0; t < SPL; t++) acc[t] = 0.0;
#pragma unroll
            for (int j = 0; j < NST; j++) {
              double Lj;
              if constexpr (LPT == 1) Lj = L[j][l];
              else Lj = __shfl_sync(sweepmask, L[j % SPL][l], gbase + j / SPL);
#pragma unroll
              for (int t = 0; t < SPL; t++) acc[t] = fma(IRKGL1_MU(t, j), Lj, acc[t]);
            }
            unsigned long long dl = 0;
#pragma unroll
            for (int t = 0; t < SPL; t++) {
              const double yn = ylv + acc[t];
              dl = umax64(dl, abs_bits(yn - Y[t][l]));
              Y[t][l] = yn;
            }
#pragma unroll
            for (int off = 1; off < LPT; off <<= 1) dl = umax64(dl, __shfl_xor_sync(sweepmask, dl, off));
            bad = bad || (dl >= INF_BITS);
#pragma unroll
            for (int s = 0; s < NS; s++) {
              if (s * LPT + r == l) {
                const bool cond = (dl == 0) || (dmin[s] <= umin64(dprev[s], dl));
                cond_own = cond_own && cond;
                dmin[s] = umin64(dmin[s], dprev[s]);
                dprev[s] = dl;
              }
            }
          }
          int stop_i = cond_own ? 1 : 0;
#pragma unroll
          for (int off = 1; off < LPT; off <<= 1) stop_i &= __shfl_xor_sync(sweepmask, stop_i, off);
          if (bad) {
            st = ST_NONFINITE;
            conv = true;
          } else if (stop_i != 0) {
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
        // update, Eq. yn2: y += sum_i L_i, compensated
        double sL[D];
#pragma unroll
        for (int l = 0; l < D; l++) {
          double x = L[0][l];
#pragma unroll
          for (int t = 1; t < SPL; t++) x = x + L[t][l];
#pragma unroll
          for (int off = 1; off < LPT; off <<= 1) x = x + __shfl_xor_sync(okmask, x, off);
          sL[l] = x;
        }
#pragma unroll
        for (int s = 0; s < NS; s++)
          if (s * LPT + r < D) two_sum_add(yh[s], yl[s], select_own<LPT, D>(sL, s, r));
        n++;
        if (a.monitor > 0) {
          const bool mon = (n % a.monitor) == 0;
          const unsigned monmask = __ballot_sync(okmask, mon);
          if (mon) {
            const double Hn = group_energy1<Rhs, LPT, NS>(rhs, yh, monmask, gbase);
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
      const size_t off = static_cast<size_t>(traj) * D;
#pragma unroll
      for (int s = 0; s < NS; s++) {
        const int l = s * LPT + r;
        if (l < D) {
          a.y_out[off + l] = yh[s];
          if (a.ylo_out) a.ylo_out[off + l] = yl[s];
        }
      }
      if (a.lp_out && st == ST_OK) {
        const size_t loff = static_cast<size_t>(traj) * NST * D;
#pragma unroll
        for (int tt = 0; tt < SPL; tt++)
#pragma unroll
          for (int l = 0; l < D; l++) a.lp_out[loff + (i0 + tt) * D + l] = L[tt][l];
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
#undef IRKGL1_MU
#undef IRKGL1_NU
}

struct KernelEntry1 {
  int kind;
  int dim;
  int lpt;
  int block;
  int nst;     // stages
  int mix;     // 0: FP64 FMA mixing, 1: fixed-point mixing (component split only)
  int layout;  // 0: stage split (irkgl1_kernel), 1: component split (irkgl1_kernel_cs, lpt = dim)
  const void* fn;
  void (*launch)(dim3, dim3, cudaStream_t, const KArgs1&, const Coef1&);
};

template <class Rhs, int LPT, int BLOCK, int NST>
void launch1_impl(dim3 grid, dim3 block, cudaStream_t st, const KArgs1& a, const Coef1& c) {
  irkgl1_kernel<Rhs, LPT, BLOCK, NST><<<grid, block, 0, st>>>(a, c);
}

struct KernelTable1 {
  const KernelEntry1* entries;
  int count;
};

KernelTable1 kernels_first_order();

}  // namespace irkgl

#define IRKGL_ENTRY1(KIND, DIM, RHS, LPT, BLOCK, NST)                                              \
  ::irkgl::KernelEntry1 {                                                                            \
    KIND, DIM, LPT, BLOCK, NST, 0, 0, (const void*)::irkgl::irkgl1_kernel<RHS, LPT, BLOCK, NST>,    \
        ::irkgl::launch1_impl<RHS, LPT, BLOCK, NST>                                                  \
  }
// component-split tile (irkgl1_cs.cuh): DIM lanes per trajectory, 8 stages
#define IRKGL_ENTRY1_CS(KIND, DIM, RHS, BLOCK, MIX)                                                  \
  ::irkgl::KernelEntry1 {                                                                            \
    KIND, DIM, DIM, BLOCK, 8, MIX, 1, (const void*)::irkgl::irkgl1_kernel_cs<RHS, BLOCK, MIX>,      \
        ::irkgl::launch1_cs_impl<RHS, BLOCK, MIX>                                                    \
  }
