/*
 * IRKGL16 second-order step in plain C: TEST INFRASTRUCTURE ONLY.
 *
 * The same algorithm as oracle/irkgl.py (arXiv 2511.03655, Eqs. IRK_init2,
 * IRK_FP2, Delta_n, stopping, qnvn2, compensated update of Sec. 5), with the
 * identical operation sequence: sequential sums j = 1..8, every operation
 * rounded separately.  Build with -O2 -ffp-contract=off (no fast-math, no
 * FMA contraction) so that its results are bit-identical to the Python form;
 * tests/test_oracle_step.py::test_c_equals_python_bitwise checks that.  Used
 * by the tests for large cases and by bench.py as the timed CPU baseline;
 * never by the CUDA product path.
 *
 * Readings where the paper is silent are those stated in oracle/irkgl.py:
 * Rprev = 0 on the first step, kmax = 100 (status 1), a non-finite stage
 * value stops the trajectory (status 2) and leaves the state of the start of
 * that step, the update uses the R of the last sweep, and the compensated
 * pair update is TwoSum + Fast2Sum with dq = h v_hi + (h v_lo - h sum c_i R_i).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define S 8

typedef struct {
  double c[S], b[S], mu[S * S], eta[S * S], nu[S * S]; /* row-major [i*8+j] */
} orc_tab;

enum {
  ORC_KEPLER = 1,
  ORC_NBODY = 2,
  ORC_FPUT = 3,
  ORC_HENON_HEILES = 4,
  ORC_HARMONIC = 5,
  ORC_HH_FORCED = 6 /* the non-autonomous example of Sec. 3: lam + xi sin t */
};

static int time_dependent(int kind) { return kind == ORC_HH_FORCED; }
enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_NONFINITE = 2 };

/* ---------------- right-hand sides g(q) and Hamiltonians ---------------- */

/* FPUT bond r_j = q_{j+1} - q_j (1-based particles, fixed ends q_0 = q_{n+1} = 0). */
static double bond(const double* q, int d, int j) {
  double left = j >= 1 ? q[j - 1] : 0.0;
  double right = j <= d - 1 ? q[j] : 0.0;
  return right - left;
}

/* g(t, q); only ORC_HH_FORCED reads t. */
static void rhs_g(int kind, const double* p, int d, const double* q, double* g, double t) {
  switch (kind) {
    case ORC_KEPLER: {
      double mu = p[0];
      double r2 = q[0] * q[0] + q[1] * q[1];
      double r3 = r2 * sqrt(r2);
      g[0] = -(mu * q[0]) / r3;
      g[1] = -(mu * q[1]) / r3;
      break;
    }
    case ORC_HENON_HEILES: {
      double lam = p[0];
      g[0] = -q[0] - 2.0 * lam * q[0] * q[1];
      g[1] = -q[1] - lam * (q[0] * q[0] - q[1] * q[1]);
      break;
    }
    case ORC_HH_FORCED: {
      double aux = p[0] + p[1] * sin(t);
      g[0] = -q[0] - 2.0 * aux * q[0] * q[1];
      g[1] = -q[1] - aux * (q[0] * q[0] - q[1] * q[1]);
      break;
    }
    case ORC_HARMONIC: {
      double w2 = p[0] * p[0];
      for (int l = 0; l < d; l++) g[l] = -(w2 * q[l]);
      break;
    }
    case ORC_NBODY: {
      /* p[0] = G, p[1..N] = masses */
      int n = d / 3;
      double G = p[0];
      for (int a = 0; a < n; a++) {
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
        for (int b = 0; b < n; b++) {
          if (b == a) continue;
          double dx0 = q[3 * b] - q[3 * a];
          double dx1 = q[3 * b + 1] - q[3 * a + 1];
          double dx2 = q[3 * b + 2] - q[3 * a + 2];
          double r2 = dx0 * dx0 + dx1 * dx1 + dx2 * dx2;
          double w = (G * p[1 + b]) / (r2 * sqrt(r2));
          acc0 = acc0 + w * dx0;
          acc1 = acc1 + w * dx1;
          acc2 = acc2 + w * dx2;
        }
        g[3 * a] = acc0;
        g[3 * a + 1] = acc1;
        g[3 * a + 2] = acc2;
      }
      break;
    }
    case ORC_FPUT: {
      double al = p[0];
      for (int j = 1; j <= d; j++) {
        double rr = bond(q, d, j);     /* q_{j+1} - q_j */
        double rl = bond(q, d, j - 1); /* q_j - q_{j-1} */
        g[j - 1] = (rr + al * rr * rr) - (rl + al * rl * rl);
      }
      break;
    }
    default:
      for (int l = 0; l < d; l++) g[l] = NAN;
  }
}

static double rhs_H(int kind, const double* p, int d, const double* q, const double* v) {
  switch (kind) {
    case ORC_KEPLER: {
      double r2 = q[0] * q[0] + q[1] * q[1];
      return (v[0] * v[0] + v[1] * v[1]) / 2.0 - p[0] / sqrt(r2);
    }
    case ORC_HENON_HEILES: {
      double lam = p[0];
      return (v[0] * v[0] + v[1] * v[1]) / 2.0 + (q[0] * q[0] + q[1] * q[1]) / 2.0 +
             lam * (q[0] * q[0] * q[1] - q[1] * q[1] * q[1] / 3.0);
    }
    case ORC_HARMONIC: {
      double w2 = p[0] * p[0];
      double acc = 0.0;
      for (int l = 0; l < d; l++) acc = acc + (v[l] * v[l] + w2 * q[l] * q[l]) / 2.0;
      return acc;
    }
    case ORC_NBODY: {
      int n = d / 3;
      double G = p[0];
      double kin = 0.0, pot = 0.0;
      for (int a = 0; a < n; a++)
        kin = kin + p[1 + a] * (v[3 * a] * v[3 * a] + v[3 * a + 1] * v[3 * a + 1] +
                                v[3 * a + 2] * v[3 * a + 2]) / 2.0;
      for (int a = 0; a < n; a++)
        for (int b = a + 1; b < n; b++) {
          double dx0 = q[3 * b] - q[3 * a];
          double dx1 = q[3 * b + 1] - q[3 * a + 1];
          double dx2 = q[3 * b + 2] - q[3 * a + 2];
          double r = sqrt(dx0 * dx0 + dx1 * dx1 + dx2 * dx2);
          pot = pot + (G * p[1 + a] * p[1 + b]) / r;
        }
      return kin - pot;
    }
    case ORC_FPUT: {
      double al = p[0];
      double acc = 0.0;
      for (int j = 0; j < d; j++) acc = acc + v[j] * v[j] / 2.0;
      for (int j = 0; j <= d; j++) {
        double r = bond(q, d, j);
        acc = acc + r * r / 2.0 + al * r * r * r / 3.0;
      }
      return acc;
    }
    default:
      return NAN;
  }
}

/* ------------------------------ the step ------------------------------ */

static void two_sum_add(double* hi, double* lo, double x) {
  double s = *hi + x;
  double bb = s - *hi;
  double err = (*hi - (s - bb)) + (x - bb);
  double lo2 = *lo + err;
  double hi2 = s + lo2;
  *lo = lo2 - (hi2 - s);
  *hi = hi2;
}

/* One step for one trajectory; work arrays sized 5*S*d + 3*d doubles.
 * (*th, *tl) is the time t_n as a compensated pair; a time-dependent g is
 * evaluated at the stage times *th + h c_i.  Returns the status; *k
 * receives the number of sweeps. */
static int one_step(const orc_tab* t, int kind, const double* p, int d, double h, int kmax,
                    double* q, double* v, double* qlo, double* vlo, double* rp, double* th,
                    double* tl, int* kout, double* work) {
  double tau[S];
  for (int i = 0; i < S; i++) tau[i] = *th + h * t->c[i];
  double* V = work;             /* S*d, reused as Lq */
  double* Q = V + S * d;        /* S*d */
  double* Qn = Q + S * d;       /* S*d */
  double* G = Qn + S * d;       /* S*d */
  double* R = G + S * d;        /* S*d */
  double* dmin = R + S * d;     /* d */
  double* dprev = dmin + d;     /* d */

  /* init, Eq. IRK_init2 */
  for (int i = 0; i < S; i++)
    for (int l = 0; l < d; l++) {
      double acc = t->nu[i * S] * rp[l];
      for (int j = 1; j < S; j++) acc = acc + t->nu[i * S + j] * rp[j * d + l];
      V[i * d + l] = v[l] + acc;
    }
  for (int i = 0; i < S; i++)
    for (int l = 0; l < d; l++) V[i * d + l] = h * (t->b[i] * V[i * d + l]); /* Lq */
  for (int i = 0; i < S; i++)
    for (int l = 0; l < d; l++) {
      double acc = t->mu[i * S] * V[l];
      for (int j = 1; j < S; j++) acc = acc + t->mu[i * S + j] * V[j * d + l];
      Q[i * d + l] = q[l] + acc;
    }

  /* sweeps, Eq. IRK_FP2, stopping rule Eqs. Delta_n / stopping */
  for (int l = 0; l < d; l++) {
    dmin[l] = INFINITY;
    dprev[l] = INFINITY;
  }
  int k = 0;
  for (;;) {
    k++;
    for (int i = 0; i < S; i++) rhs_g(kind, p, d, Q + i * d, G + i * d, tau[i]);
    for (int i = 0; i < S; i++)
      for (int l = 0; l < d; l++) R[i * d + l] = h * (t->b[i] * G[i * d + l]);
    int finite = 1;
    for (int i = 0; i < S; i++)
      for (int l = 0; l < d; l++) {
        double acc = t->c[i] * v[l];
        for (int j = 0; j < S; j++) acc = acc + t->eta[i * S + j] * R[j * d + l];
        double x = q[l] + h * acc;
        Qn[i * d + l] = x;
        if (!isfinite(x)) finite = 0;
      }
    if (!finite) {
      *kout = k;
      return ORC_NONFINITE;
    }
    int stop = 1;
    for (int l = 0; l < d; l++) {
      double delta = 0.0;
      for (int i = 0; i < S; i++) {
        double a = fabs(Qn[i * d + l] - Q[i * d + l]);
        if (a > delta) delta = a;
      }
      double m = dprev[l] <= delta ? dprev[l] : delta;
      int cond = (delta == 0.0) || (dmin[l] <= m);
      stop = stop && cond;
      dmin[l] = dmin[l] <= dprev[l] ? dmin[l] : dprev[l];
      dprev[l] = delta;
    }
    memcpy(Q, Qn, sizeof(double) * S * d);
    if (stop) break;
    if (k >= kmax) {
      *kout = k;
      return ORC_MAXITER;
    }
  }
  *kout = k;

  /* update, Eq. qnvn2, compensated */
  for (int l = 0; l < d; l++) {
    double sR = R[l];
    for (int i = 1; i < S; i++) sR = sR + R[i * d + l];
    double scR = t->c[0] * R[l];
    for (int i = 1; i < S; i++) scR = scR + t->c[i] * R[i * d + l];
    double vh = v[l], vl = vlo[l];
    two_sum_add(&vh, &vl, sR);
    double dq = h * vh + (h * vl - h * scR);
    double qh = q[l], ql = qlo[l];
    two_sum_add(&qh, &ql, dq);
    q[l] = qh;
    qlo[l] = ql;
    v[l] = vh;
    vlo[l] = vl;
  }
  memcpy(rp, R, sizeof(double) * S * d);
  two_sum_add(th, tl, h); /* t_{n+1} = t_n + h */
  return ORC_OK;
}

typedef struct {
  const orc_tab* tab;
  int kind;
  const double* params;
  int pstride, d, batch;
  double *q, *v, *qlo, *vlo, *rp;
  double *t_hi, *t_lo; /* may be NULL: time starts at 0 and is not returned */
  const double* h;
  const long long* nsteps;
  int kmax;
  int* iters;
  int iters_stride;
  long long* iters_total;
  double* dH_max;
  int* status;
  long long* steps_done;
  int t0, t1;
  int err;
} job_t;

static void* run_range(void* arg) {
  job_t* J = (job_t*)arg;
  int d = J->d;
  double* work = (double*)malloc(sizeof(double) * (5 * S * d + 3 * d));
  if (!work) {
    J->err = -1;
    return NULL;
  }
  for (int t = J->t0; t < J->t1; t++) {
    const double* p = J->params + (size_t)t * J->pstride;
    double* q = J->q + (size_t)t * d;
    double* v = J->v + (size_t)t * d;
    double* ql = J->qlo + (size_t)t * d;
    double* vl = J->vlo + (size_t)t * d;
    double* rp = J->rp + (size_t)t * S * d;
    double th0 = 0.0, tl0 = 0.0;
    double* th = J->t_hi ? J->t_hi + t : &th0;
    double* tl = J->t_lo ? J->t_lo + t : &tl0;
    const int timed = time_dependent(J->kind);
    double H0 = timed ? 0.0 : rhs_H(J->kind, p, d, q, v);
    double dmax = 0.0;
    long long tot = 0, n = 0;
    int st = ORC_OK;
    for (n = 0; n < J->nsteps[t]; n++) {
      int k = 0;
      st = one_step(J->tab, J->kind, p, d, J->h[t], J->kmax, q, v, ql, vl, rp, th, tl, &k, work);
      if (J->iters && n < J->iters_stride) J->iters[(size_t)t * J->iters_stride + n] = k;
      tot += k;
      if (st != ORC_OK) break;
      if (timed) continue; /* H(t) is not conserved: no monitor */
      double Hn = rhs_H(J->kind, p, d, q, v);
      double dH = fabs((Hn - H0) / H0);
      if (dH > dmax) dmax = dH;
    }
    if (J->iters_total) J->iters_total[t] = tot;
    if (J->dH_max) J->dH_max[t] = dmax;
    if (J->status) J->status[t] = st;
    if (J->steps_done) J->steps_done[t] = n;
  }
  free(work);
  return NULL;
}

/*
 * Advance `batch` independent trajectories of dimension d (positions) by
 * nsteps[t] steps of size h[t].  t_hi, t_lo [batch] (may be NULL) hold each
 * trajectory's time t_n as a compensated pair, read and updated in place.  State arrays are trajectory-major and are
 * updated in place: q, v, q_lo, v_lo [batch*d], r_prev [batch*8*d].
 * params points at the right-hand-side parameters of trajectory 0;
 * trajectory t uses params + t*pstride (pstride 0: shared).
 * Optional outputs (may be NULL): iters [batch*iters_stride] (sweeps of the
 * first iters_stride steps), iters_total, dH_max (max_n |(H_n-H_0)/H_0| with
 * H_0 at entry), status, steps_done.  nthreads >= 1 splits the batch into
 * contiguous ranges.  Returns 0, or -1 on allocation failure.
 */
int orc_run_t(const orc_tab* tab, int kind, const double* params, int pstride, int d, int batch,
              double* q, double* v, double* q_lo, double* v_lo, double* r_prev, double* t_hi,
              double* t_lo, const double* h, const long long* nsteps, int kmax, int* iters,
              int iters_stride, long long* iters_total, double* dH_max, int* status,
              long long* steps_done, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > batch) nthreads = batch > 0 ? batch : 1;
  job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int w = 0; w < nthreads; w++) {
    job_t* J = &jobs[w];
    J->tab = tab;
    J->kind = kind;
    J->params = params;
    J->pstride = pstride;
    J->d = d;
    J->batch = batch;
    J->q = q;
    J->v = v;
    J->qlo = q_lo;
    J->vlo = v_lo;
    J->rp = r_prev;
    J->t_hi = t_hi;
    J->t_lo = t_lo;
    J->h = h;
    J->nsteps = nsteps;
    J->kmax = kmax;
    J->iters = iters;
    J->iters_stride = iters_stride;
    J->iters_total = iters_total;
    J->dH_max = dH_max;
    J->status = status;
    J->steps_done = steps_done;
    J->t0 = (int)((long long)batch * w / nthreads);
    J->t1 = (int)((long long)batch * (w + 1) / nthreads);
  }
  int err = 0;
  if (nthreads == 1) {
    run_range(&jobs[0]);
  } else {
    int started = 0;
    for (int w = 0; w < nthreads; w++) {
      if (pthread_create(&th[w], NULL, run_range, &jobs[w]) != 0) {
        run_range(&jobs[w]);
        th[w] = 0;
      } else {
        started |= 1;
      }
    }
    for (int w = 0; w < nthreads; w++)
      if (th[w]) pthread_join(th[w], NULL);
    (void)started;
  }
  for (int w = 0; w < nthreads; w++)
    if (jobs[w].err) err = -1;
  free(jobs);
  free(th);
  return err;
}

/* orc_run_t without time arrays: every trajectory starts at t = 0. */
int orc_run(const orc_tab* tab, int kind, const double* params, int pstride, int d, int batch,
            double* q, double* v, double* q_lo, double* v_lo, double* r_prev, const double* h,
            const long long* nsteps, int kmax, int* iters, int iters_stride,
            long long* iters_total, double* dH_max, int* status, long long* steps_done,
            int nthreads) {
  return orc_run_t(tab, kind, params, pstride, d, batch, q, v, q_lo, v_lo, r_prev, NULL, NULL, h,
                   nsteps, kmax, iters, iters_stride, iters_total, dH_max, status, steps_done,
                   nthreads);
}

/* H of one state (for tests). */
double orc_hamiltonian(int kind, const double* params, int d, const double* q, const double* v) {
  return rhs_H(kind, params, d, q, v);
}

/* ======================================================================
 * First-order form (Eq. Yi2 with Eqs. IRK_init / IRK_FP, stopping rule on
 * all D components, compensated update Eq. yn2): the same operation
 * sequence as oracle/first_order.py.
 * ====================================================================== */
enum {
  ORC1_SCHWARZSCHILD = 7, /* Eq. Ham_SBH, y = (r, theta, p_r, p_theta), params {E, L, beta} */
  ORC1_HARMONIC = 8       /* q' = p, p' = -omega^2 q, params {omega} */
};

static void rhs_f1(int kind, const double* p, const double* y, double* f) {
  if (kind == ORC1_SCHWARZSCHILD) {
    double r = y[0], th = y[1], pr = y[2], pth = y[3];
    double sn = sin(th), cs = cos(th);
    double s = sn * sn;
    double u = 1.0 - 2.0 / r;
    double r2 = r * r;
    double r3 = r2 * r;
    double E2 = p[0] * p[0], L2 = p[1] * p[1], b2 = p[2] * p[2];
    double dr = pr * pr / r2 + E2 / (r2 * (u * u)) - pth * pth / r3 - L2 / (r3 * s) + b2 * r * s / 4.0;
    double dth = (-L2 / (r2 * (s * s)) + b2 * r2 / 4.0) * (sn * cs);
    f[0] = u * pr;
    f[1] = pth / r2;
    f[2] = -dr;
    f[3] = -dth;
  } else { /* ORC1_HARMONIC */
    f[0] = y[1];
    f[1] = -(p[0] * p[0] * y[0]);
  }
}

static double rhs_H1(int kind, const double* p, const double* y) {
  if (kind == ORC1_SCHWARZSCHILD) {
    double r = y[0], th = y[1], pr = y[2], pth = y[3];
    double sn = sin(th);
    double s = sn * sn;
    double u = 1.0 - 2.0 / r;
    double a = p[1] - p[2] / 2.0 * (r * r) * s;
    return u * (pr * pr) / 2.0 - p[0] * p[0] / (2.0 * u) + pth * pth / (2.0 * (r * r)) +
           a * a / (2.0 * (r * r) * s);
  }
  return (y[1] * y[1] + p[0] * p[0] * y[0] * y[0]) / 2.0;
}

static int dim1(int kind) { return kind == ORC1_SCHWARZSCHILD ? 4 : 2; }

/* One first-order step of the ns-stage scheme (tables packed row-major with
 * stride ns); work sized 4*ns*D + 2*D doubles. */
static int one_step1(const orc_tab* t, int ns, int kind, const double* p, int D, double h, int kmax,
                     double* y, double* ylo, double* lp, int* kout, double* work) {
  double* Y = work;          /* ns*D */
  double* Yn = Y + ns * D;   /* ns*D */
  double* F = Yn + ns * D;   /* ns*D */
  double* L = F + ns * D;    /* ns*D */
  double* dmin = L + ns * D;  /* D */
  double* dprev = dmin + D;  /* D */
  /* init, Eq. IRK_init */
  for (int i = 0; i < ns; i++)
    for (int l = 0; l < D; l++) {
      double acc = t->nu[i * ns] * lp[l];
      for (int j = 1; j < ns; j++) acc = acc + t->nu[i * ns + j] * lp[j * D + l];
      Y[i * D + l] = y[l] + acc;
    }
  for (int l = 0; l < D; l++) {
    dmin[l] = INFINITY;
    dprev[l] = INFINITY;
  }
  int k = 0;
  for (;;) {
    k++;
    for (int i = 0; i < ns; i++) rhs_f1(kind, p, Y + i * D, F + i * D);
    for (int i = 0; i < ns; i++)
      for (int l = 0; l < D; l++) L[i * D + l] = h * (t->b[i] * F[i * D + l]);
    int finite = 1;
    for (int i = 0; i < ns; i++)
      for (int l = 0; l < D; l++) {
        double acc = t->mu[i * ns] * L[l];
        for (int j = 1; j < ns; j++) acc = acc + t->mu[i * ns + j] * L[j * D + l];
        double x = y[l] + acc;
        Yn[i * D + l] = x;
        if (!isfinite(x)) finite = 0;
      }
    if (!finite) {
      *kout = k;
      return ORC_NONFINITE;
    }
    int stop = 1;
    for (int l = 0; l < D; l++) {
      double delta = 0.0;
      for (int i = 0; i < ns; i++) {
        double a = fabs(Yn[i * D + l] - Y[i * D + l]);
        if (a > delta) delta = a;
      }
      double m = dprev[l] <= delta ? dprev[l] : delta;
      int cond = (delta == 0.0) || (dmin[l] <= m);
      stop = stop && cond;
      dmin[l] = dmin[l] <= dprev[l] ? dmin[l] : dprev[l];
      dprev[l] = delta;
    }
    memcpy(Y, Yn, sizeof(double) * ns * D);
    if (stop) break;
    if (k >= kmax) {
      *kout = k;
      return ORC_MAXITER;
    }
  }
  *kout = k;
  for (int l = 0; l < D; l++) {
    double sL = L[l];
    for (int i = 1; i < ns; i++) sL = sL + L[i * D + l];
    two_sum_add(&y[l], &ylo[l], sL);
  }
  memcpy(lp, L, sizeof(double) * ns * D);
  return ORC_OK;
}

/*
 * Advance `batch` first-order trajectories (D = 4 for ORC1_SCHWARZSCHILD,
 * 2 for ORC1_HARMONIC) of the ns-stage scheme (ns <= 8; tab holds b, mu,
 * nu packed with stride ns) by nsteps[t] steps of size h[t], in place: y,
 * y_lo [batch*D], l_prev [batch*ns*D].  Optional outputs as for orc_run
 * (dH_max relative to H at entry).  Single-threaded.  Returns 0, -1 on
 * allocation failure, -2 for an unknown kind.
 */
int orc_run1(const orc_tab* tab, int ns, int kind, const double* params, int pstride, int batch,
             double* y, double* y_lo, double* l_prev, const double* h, const long long* nsteps,
             int kmax, int* iters, int iters_stride, long long* iters_total, double* dH_max,
             int* status, long long* steps_done) {
  if (kind != ORC1_SCHWARZSCHILD && kind != ORC1_HARMONIC) return -2;
  if (ns < 1 || ns > S) return -2;
  const int D = dim1(kind);
  double* work = (double*)malloc(sizeof(double) * (4 * ns * D + 2 * D));
  if (!work) return -1;
  for (int t = 0; t < batch; t++) {
    const double* p = params + (size_t)t * pstride;
    double* yy = y + (size_t)t * D;
    double* yl = y_lo + (size_t)t * D;
    double* lp = l_prev + (size_t)t * ns * D;
    double H0 = rhs_H1(kind, p, yy);
    double dmax = 0.0;
    long long tot = 0, n = 0;
    int st = ORC_OK;
    for (n = 0; n < nsteps[t]; n++) {
      int k = 0;
      st = one_step1(tab, ns, kind, p, D, h[t], kmax, yy, yl, lp, &k, work);
      if (iters && n < iters_stride) iters[(size_t)t * iters_stride + n] = k;
      tot += k;
      if (st != ORC_OK) break;
      double dH = fabs((rhs_H1(kind, p, yy) - H0) / H0);
      if (dH > dmax) dmax = dH;
    }
    if (iters_total) iters_total[t] = tot;
    if (dH_max) dH_max[t] = dmax;
    if (status) status[t] = st;
    if (steps_done) steps_done[t] = n;
  }
  free(work);
  return 0;
}

double orc_hamiltonian1(int kind, const double* params, const double* y) {
  return rhs_H1(kind, params, y);
}

/* ======================================================================
 * Explicit splitting baselines (Sec. 4, Eqs. flowAB, high_order_splitting):
 * the same operation sequence as oracle/splitting.py.  a[0..s], b[0..s-1].
 * ====================================================================== */
int orc_split(const double* a, const double* b, int s, int kind, const double* params, int pstride,
              int d, int batch, double* q, double* v, double* q_lo, double* v_lo, const double* h,
              const long long* nsteps, int local, double* dH_max, int* status,
              long long* steps_done) {
  double* G = (double*)malloc(sizeof(double) * (size_t)d);
  if (!G) return -1;
  for (int t = 0; t < batch; t++) {
    const double* p = params + (size_t)t * pstride;
    double* qq = q + (size_t)t * d;
    double* vv = v + (size_t)t * d;
    double* ql = q_lo + (size_t)t * d;
    double* vl = v_lo + (size_t)t * d;
    double H0 = rhs_H(kind, p, d, qq, vv), Hp = H0, dmax = 0.0;
    long long n = 0;
    int st = ORC_OK;
    for (n = 0; n < nsteps[t]; n++) {
      const double hh = h[t];
      for (int j = 0; j < s; j++) {
        const double ah = a[j] * hh;
        for (int l = 0; l < d; l++) two_sum_add(&qq[l], &ql[l], ah * vv[l]);
        rhs_g(kind, p, d, qq, G, 0.0);
        const double bh = b[j] * hh;
        for (int l = 0; l < d; l++) two_sum_add(&vv[l], &vl[l], bh * G[l]);
      }
      const double ah = a[s] * hh;
      for (int l = 0; l < d; l++) two_sum_add(&qq[l], &ql[l], ah * vv[l]);
      int finite = 1;
      for (int l = 0; l < d; l++)
        if (!isfinite(qq[l]) || !isfinite(vv[l])) finite = 0;
      if (!finite) {
        st = ORC_NONFINITE;
        break;
      }
      const double Hn = rhs_H(kind, p, d, qq, vv);
      const double ref = local ? Hp : H0;
      const double dH = fabs((Hn - ref) / ref);
      if (dH > dmax) dmax = dH;
      Hp = Hn;
    }
    if (dH_max) dH_max[t] = dmax;
    if (status) status[t] = st;
    if (steps_done) steps_done[t] = n;
  }
  free(G);
  return 0;
}
