// irkgl_wide.cuh -- the "wide" IRKGL16 kernel for instances of large and uneven
// dimension (N-body with many bodies, FPUT chains), heterogeneous in one launch.
//
// A team of TEAM threads (one warp, or the whole block) owns one instance at a
// time; persistent teams take instances from a work counter.  Per instance the
// 8 stage values Q, the increments R and c_i v live in shared memory
// ([8][d] each); thread `tid` owns components l = tid, tid + TEAM, ... and
// keeps their compensated q, v pairs and Eq. stopping history in registers.
// One step (arXiv 2511.03655):
//   init   Q_i = q + h (c_i v + sum_k W_ik Rprev_k)          Eq. IRK_init2 (fused)
//   sweep  R_i = h b_i g(Q_i)                                 Eq. Gi   (team-parallel
//          over (stage, body) or (stage, particle))
//          Qn_i = q + h (c_i v + sum_j eta_ij R_j)            Eq. Qi2  (thread per component,
//          all 8 stages: eta are compile-time constant-bank operands)
//          Delta, Eq. stopping per owned component, team-wide AND
//   update v += sum R_i, q += h v - h sum c_i R_i, compensated Eq. qnvn2, Sec. 5
#pragma once

#include "irkgl.h"
#include "irkgl_device.cuh"

namespace irkgl {

// Largest N-body instance the wide kernel takes (its per-stage body weights
// are staged in shared memory); a larger one gets IRKGL_STATUS_BAD_INSTANCE.
constexpr int kWideMaxBodies = 128;
__host__ __device__ constexpr int wide_nbmax(int dmax) {
  return (dmax / 3 < kWideMaxBodies ? dmax / 3 : kWideMaxBodies) + 1;
}

// One instance of a ragged batch (mirrors irkgl_instance in irkgl.h).
struct WideInstance {
  int kind;
  int dim;
  long long offset;  // first element in the packed [.][d] state arrays
  int param_offset;  // first parameter in the packed parameter array
  int nparams;
  double h;
  long long nsteps;
};

struct WideArgs {
  int ninst;
  int kmax;
  int monitor;
  int dmax;  // largest dimension in the batch (shared-memory layout)
  const WideInstance* inst;
  const double* params;
  const double* q_in;
  const double* v_in;
  double* q_out;
  double* v_out;
  double* qlo_out;  // may be null
  double* vlo_out;
  double* rp_out;   // [.][8][d] packed with offset * 8, may be null
  double* dH_max;   // [ninst] or null
  long long* iters_total;
  long long* steps_done;
  int* status;
  const int* order;
  unsigned int* counter;
  // continuation (irkgl_advance_ragged); all may be null
  const double* qlo_in;
  const double* vlo_in;
  const double* rp_in;
  const long long* nsteps_call;  // [ninst] steps for this call, overrides inst.nsteps
  double* H0_io;  // an entry that is NaN is computed at this call's first step
  int h0_init;
  int accumulate;
  int monitor_local;  // dH_max = max_n |(H_n - H_{n-1}) / H_{n-1}|
  int sticky_status;  // status in/out: an instance with a nonzero entry is not advanced
};

// Compiled team shapes (k_wide.cu): one warp per instance (small d) or the
// whole block, SLOTS components per thread, FP64 or fixed-point mixing,
// c_i v kept in shared memory or formed again where it is used.
struct WideShape {
  int team, block, slots;
  int mix;  // 0: FP64 FMA mixing, 1: fixed-point mixing
  int cvs;  // 1: c_i v in shared memory; 0: recomputed (same bits, less shared memory)
  const void* fn;
  void (*launch)(dim3, dim3, size_t, cudaStream_t, const WideArgs&, const Coef&);
};
int wide_shapes(const WideShape** out);

// team barrier and team-wide AND / OR
template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM == 32) __syncwarp();
  else __syncthreads();
}
template <int TEAM>
__device__ __forceinline__ bool team_and(bool x) {
  if constexpr (TEAM == 32) return __all_sync(FULL, x);
  else return __syncthreads_and(x) != 0;
}
template <int TEAM>
__device__ __forceinline__ bool team_or(bool x) {
  if constexpr (TEAM == 32) return __any_sync(FULL, x);
  else return __syncthreads_or(x) != 0;
}
template <int TEAM>
__device__ __forceinline__ double team_sum(double x, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
  if constexpr (TEAM == 32) {
    return x;
  } else {
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < TEAM / 32; i++) s += red[i];  // same order on every thread
    return s;
  }
}

// x^(-3/2) of the wide kernel's pair forces.  kWideRinv3Fp64 selects the
// FP64 form (six dependent FP64 operations after the FP32 seed) over the
// integer one (about forty dependent integer operations).  The integer form
// is the faster one on GB300 here too (ragged batch: 1.66e6 against 1.42e6
// trajectory-steps/s with the FP64 form), although its chain is longer.
//
// The pair force is evaluated from both ends (each body sums over all
// others).  Evaluating each pair once per stage, with tiles of 8 or 16
// bodies whose pairs a round-robin schedule visits (a travelling
// accumulator carrying the partner's sum through the lanes), cut the FP64
// instructions of the 33-64-body bucket by only 8 % (partly filled tiles
// and masked lanes cost full warp instructions) and ran 1.39x slower
// (2,285 against 1,644 ms for 1,090 systems x 1,000 steps), so it is not
// used.
constexpr bool kWideRinv3Fp64 = false;
__device__ __forceinline__ double wide_rinv3(double x) {
  if (!positive_normal(x)) return rinv3_special(x);
  return kWideRinv3Fp64 ? rinv3_fp64(x) : rinv3_int(x);
}

// R_i = (h b_i) g(Q_i) for every stage, team-parallel.  w8 holds (h b_i) per stage
// and, for N-body, (h b_i) G m_b at w8[8 + i * nb + b].
template <int TEAM>
__device__ __forceinline__ void team_rhs(int kind, int d, const double* p, const double* w8,
                                         const double* Q, double* R, int tid) {
  if (kind == IRKGL_RHS_NBODY) {
    const int nb = d / 3;
    // each (stage, body) thread sums over all other bodies, so every pair is
    // evaluated from both ends: nearly every lane is busy, which on GB300
    // beats evaluating each pair once (see the note at wide_rinv3)
    for (int x = tid; x < S * nb; x += TEAM) {
      const int i = x / nb, a = x - i * nb;
      const double* Qi = Q + i * d;
      const double xa = Qi[3 * a], ya = Qi[3 * a + 1], za = Qi[3 * a + 2];
      const double* wi = w8 + S + i * nb;
      double gx = 0.0, gy = 0.0, gz = 0.0;
      for (int b = 0; b < nb; b++) {
        if (b == a) continue;
        const double dx = Qi[3 * b] - xa, dy = Qi[3 * b + 1] - ya, dz = Qi[3 * b + 2] - za;
        const double wz = wi[b] * wide_rinv3(fma(dx, dx, fma(dy, dy, dz * dz)));
        gx = fma(wz, dx, gx);
        gy = fma(wz, dy, gy);
        gz = fma(wz, dz, gz);
      }
      R[i * d + 3 * a] = gx;
      R[i * d + 3 * a + 1] = gy;
      R[i * d + 3 * a + 2] = gz;
    }
  } else if (kind == IRKGL_RHS_FPUT) {
    const double al = p[0];
    for (int x = tid; x < S * d; x += TEAM) {
      const int i = x / d, l = x - i * d;
      const double* Qi = Q + i * d;
      const double ql = Qi[l];
      const double rr = (l + 1 < d ? Qi[l + 1] : 0.0) - ql;   // q_{l+1} - q_l
      const double rl = ql - (l > 0 ? Qi[l - 1] : 0.0);       // q_l - q_{l-1}
      const double g = fma(al * rr, rr, rr) - fma(al * rl, rl, rl);
      R[x] = w8[i] * g;
    }
  } else {  // IRKGL_RHS_HARMONIC
    const double mw2 = -(p[0] * p[0]);
    for (int x = tid; x < S * d; x += TEAM) {
      const int i = x / d;
      R[x] = (w8[i] * mw2) * Q[x];
    }
  }
}

// Energy share of thread tid (components / bonds / pairs it owns), with the
// positions and velocities staged in shared memory qs, vs.
template <int TEAM>
__device__ __forceinline__ double team_energy_part(int kind, int d, const double* p,
                                                   const double* qs, const double* vs, int tid) {
  double acc = 0.0;
  if (kind == IRKGL_RHS_NBODY) {
    const int nb = d / 3;
    const double G = p[0];
    for (int a = tid; a < nb; a += TEAM)
      acc = fma(0.5 * p[1 + a], fma(vs[3 * a], vs[3 * a], fma(vs[3 * a + 1], vs[3 * a + 1], vs[3 * a + 2] * vs[3 * a + 2])), acc);
    const int np = nb * (nb - 1) / 2;
    double pot = 0.0;
    for (int x = tid; x < np; x += TEAM) {
      int a = 0, b = x;
      while (b >= nb - 1 - a) {
        b -= nb - 1 - a;
        a++;
      }
      b += a + 1;
      const double dx = qs[3 * b] - qs[3 * a], dy = qs[3 * b + 1] - qs[3 * a + 1],
                   dz = qs[3 * b + 2] - qs[3 * a + 2];
      pot = fma(p[1 + a] * p[1 + b], rinv1(fma(dx, dx, fma(dy, dy, dz * dz))), pot);
    }
    acc = fma(-G, pot, acc);
  } else if (kind == IRKGL_RHS_FPUT) {
    const double al3 = p[0] * (1.0 / 3.0);
    for (int l = tid; l < d; l += TEAM) acc = fma(0.5 * vs[l], vs[l], acc);
    for (int j = tid; j <= d; j += TEAM) {  // bonds j = 0..d
      const double r = (j < d ? qs[j] : 0.0) - (j > 0 ? qs[j - 1] : 0.0);
      acc = fma(r * r, fma(al3, r, 0.5), acc);
    }
  } else {
    const double w2 = p[0] * p[0];
    for (int l = tid; l < d; l += TEAM) acc = fma(0.5 * vs[l], vs[l], fma(0.5 * w2 * qs[l], qs[l], acc));
  }
  return acc;
}

// SLOTS: owned components per thread (d <= TEAM * SLOTS).
// MIX = 1: the stage mixing of Eq. Qi2 and the initial guess as exact
// fixed-point sums on the integer pipes, rounded once (the register kernel's
// fixed-point form, per owned component).
// CVS = 1: c_i v of the owned components is stored once per step in shared
// memory; CVS = 0 forms the same product again at each use (one FP64
// multiply, identical bits), which frees 8 d doubles of shared memory per
// team so that chains up to d = 1536 fit one block.
template <int TEAM, int BLOCK, int SLOTS, int MIX = 0, int CVS = 1>
__global__ void __launch_bounds__(BLOCK)
    irkgl_wide_kernel(const __grid_constant__ WideArgs a, const __grid_constant__ Coef cf) {
  static_assert(TEAM == 32 || TEAM == BLOCK, "a team is one warp or the whole block");
  constexpr int TEAMS = BLOCK / TEAM;
  extern __shared__ double smem[];
  const int team = threadIdx.x / TEAM;
  const int tid = threadIdx.x - team * TEAM;
  const int dmax = a.dmax;
  // per team: Q, R [, cv] [8][dmax]; w8 [8 + 8 * nb]; qs, vs [dmax]; red [32]
  const int nbmax = wide_nbmax(dmax);
  const int per_team = (CVS ? 3 : 2) * S * dmax + (S + S * nbmax) + 2 * dmax + 32;
  double* Q = smem + team * per_team;
  double* R = Q + S * dmax;
  double* CV = R + S * dmax;  // used only when CVS
  double* w8 = CV + (CVS ? S * dmax : 0);
  double* qs = w8 + S + S * nbmax;
  double* vs = qs + dmax;
  double* red = vs + dmax;
  __shared__ unsigned s_idx[TEAMS];

  double qh[SLOTS], ql[SLOTS], vh[SLOTS], vl[SLOTS];
  unsigned long long dmin[SLOTS], dprev[SLOTS];

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

    // load owned components, Rprev (zero for a fresh run), per-stage weights
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
    if (tid < S) w8[tid] = h * cf.b[tid];
    if (in.kind == IRKGL_RHS_NBODY) {
      const int nb = d / 3;
      for (int x = tid; x < S * nb; x += TEAM) {
        const int i = x / nb, b = x - i * nb;
        w8[S + x] = ((h * cf.b[i]) * p[0]) * p[1 + b];
      }
    }
    double H0 = 0.0, invH0 = 0.0, dHmax = 0.0;
    long long itot = 0;
    if (a.accumulate) {
      if (a.dH_max) dHmax = a.dH_max[t];
      if (a.iters_total) itot = a.iters_total[t];
    }
    bool have_h0 = false;
    if (a.H0_io && !a.h0_init) {
      H0 = a.H0_io[t];
      invH0 = 1.0 / H0;
      have_h0 = (H0 == H0);  // NaN: a trajectory joining a running batch
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
      H0 = team_sum<TEAM>(team_energy_part<TEAM>(in.kind, d, p, qs, vs, tid), red);
      invH0 = 1.0 / H0;
      if (a.H0_io && tid == 0) a.H0_io[t] = H0;
    }
    double Hprev = H0, invHprev = invH0;
    team_sync<TEAM>();

    long long n = 0;
    while (n < N) {
      // init (fused Eq. IRK_init2): owner threads, all 8 stages of their components
#pragma unroll
      for (int s = 0; s < SLOTS; s++) {
        const int l = tid + s * TEAM;
        if (l < d) {
          double Rj[S];
#pragma unroll
          for (int j = 0; j < S; j++) Rj[j] = R[j * d + l];
          if constexpr (MIX == 1) {
            unsigned long long rb[S];
            bool nf;
            const int emax = fixed_column(Rj, rb, nf);
#pragma unroll
            for (int i = 0; i < S; i++) {
              // c_i v and c_i v + T rounded separately on every shape: the
              // intrinsics keep the compiler from fusing them into one FMA
              // in some shapes and not in others (team shapes stay bitwise equal)
              const double cvil = __dmul_rn(cf.c[i], vh[s]);
              if constexpr (CVS) CV[i * d + l] = cvil;
              double T = fixed_row<true>(i, rb, emax);
              if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
              Q[i * d + l] = fma(h, __dadd_rn(cvil, T), qh[s]);
            }
          } else {
#pragma unroll
            for (int i = 0; i < S; i++) {
              const double cvil = __dmul_rn(cf.c[i], vh[s]);
              if constexpr (CVS) CV[i * d + l] = cvil;
              double acc = cvil;
#pragma unroll
              for (int j = 0; j < S; j++) acc = fma(cf.W[i * S + j], Rj[j], acc);
              Q[i * d + l] = fma(h, acc, qh[s]);
            }
          }
        }
        dmin[s] = INF_BITS;
        dprev[s] = INF_BITS;
      }
      team_sync<TEAM>();
      int k = 0;
      for (;;) {
        k++;
        team_rhs<TEAM>(in.kind, d, p, w8, Q, R, tid);
        team_sync<TEAM>();
        bool cond = true, bad = false;
#pragma unroll
        for (int s = 0; s < SLOTS; s++) {
          const int l = tid + s * TEAM;
          if (l < d) {
            double Rj[S];
#pragma unroll
            for (int j = 0; j < S; j++) Rj[j] = R[j * d + l];
            unsigned long long dl = 0;
            if constexpr (MIX == 1) {
              unsigned long long rb[S];
              bool nf;
              const int emax = fixed_column(Rj, rb, nf);
#pragma unroll
              for (int i = 0; i < S; i++) {
                double T = fixed_row<false>(i, rb, emax);
                if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
                const double cvil = CVS ? CV[i * d + l] : __dmul_rn(cf.c[i], vh[s]);
                const double qn = fma(h, __dadd_rn(cvil, T), qh[s]);
                dl = umax64(dl, abs_bits(qn - Q[i * d + l]));
                Q[i * d + l] = qn;
              }
            } else {
#pragma unroll
              for (int i = 0; i < S; i++) {
                double acc = CVS ? CV[i * d + l] : __dmul_rn(cf.c[i], vh[s]);
#pragma unroll
                for (int j = 0; j < S; j++) acc = fma(cf.eta[i * S + j], Rj[j], acc);
                const double qn = fma(h, acc, qh[s]);
                dl = umax64(dl, abs_bits(qn - Q[i * d + l]));
                Q[i * d + l] = qn;
              }
            }
            bad = bad || (dl >= INF_BITS);
            cond = cond && ((dl == 0) || (dmin[s] <= umin64(dprev[s], dl)));
            dmin[s] = umin64(dmin[s], dprev[s]);
            dprev[s] = dl;
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
      // compensated update (Eq. qnvn2) of the owned components
#pragma unroll
      for (int s = 0; s < SLOTS; s++) {
        const int l = tid + s * TEAM;
        if (l < d) {
          double sR = R[l], scR = cf.c[0] * R[l];
#pragma unroll
          for (int i = 1; i < S; i++) {
            const double Ri = R[i * d + l];
            sR = sR + Ri;
            scR = fma(cf.c[i], Ri, scR);
          }
          two_sum_add(vh[s], vl[s], sR);
          const double dq = fma(h, vh[s], fma(h, vl[s], -(h * scR)));
          two_sum_add(qh[s], ql[s], dq);
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
        team_sync<TEAM>();
        const double Hn = team_sum<TEAM>(team_energy_part<TEAM>(in.kind, d, p, qs, vs, tid), red);
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
      team_sync<TEAM>();
    }

    // outputs
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

// shared memory bytes per block for a given dmax
__host__ __device__ inline size_t wide_smem_bytes(int teams, int dmax, int cvs = 1) {
  const int nbmax = wide_nbmax(dmax);
  const size_t per_team = (cvs ? 3 : 2) * S * dmax + (S + S * nbmax) + 2 * dmax + 32;
  return static_cast<size_t>(teams) * per_team * sizeof(double);
}

}  // namespace irkgl
