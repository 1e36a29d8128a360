// irkgl_device.cuh -- device side of the IRKGL16 library (sm_103a, FP64).
//
// One trajectory's 8 stages are spread over LPT lanes (LPT = 1, 2, 4, 8;
// SPL = 8/LPT stages per lane); 32/LPT trajectories share a warp and run in
// lock-step one step at a time.  Per step (arXiv 2511.03655):
//
//   init   Q_i = q + h (c_i v + sum_k W_ik R_k^prev)        Eq. IRK_init2 (fused)
//   sweep  R_i = h b_i g(Q_i)                                Eq. Gi
//          Qn_i = q + h (c_i v + sum_j eta_ij R_j)           Eq. Qi2 / IRK_FP2
//          Delta_l = max_i |Qn_il - Q_il|, Eq. stopping      Eqs. Delta_n, stopping
//   update v += sum_i R_i, q += h v_new - h sum_i c_i R_i    Eq. qnvn2, compensated
//
// FP64 is the scarce unit on GB300 (about 1/64 of the FP32 rate, and a
// masked lane costs as much as an active one), so: |x|, max and the
// stopping vote run on integer bit patterns; the reciprocal square root
// seed comes from the FP32 MUFU unit through integer bit manipulation (no
// F2F conversions, which run at the FP64 rate); sums over stages held by
// other lanes are gathered with warp shuffles; per-component scalar work
// (the compensated update) is spread over the LPT lanes of a trajectory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "irkgl_tables.h"

namespace irkgl {

constexpr int S = 8;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ULL;

enum { ST_OK = 0, ST_MAXITER = 1, ST_NONFINITE = 2, ST_BADDESC = 3 };

// Coefficients passed by value (kernel parameter space = constant bank).
struct Coef {
  double c[S];
  double b[S];
  double eta[S * S];  // Eq. Qi2, row-major [i*8+j]
  double W[S * S];    // fused initial guess of Eq. IRK_init2
};

struct KArgs {
  int batch;
  int kmax;
  int monitor;   // evaluate H every `monitor` steps (0 = never)
  int hist_len;  // columns of iters_hist
  const double* q_in;
  const double* v_in;
  const double* qlo_in;  // may be null (zeros)
  const double* vlo_in;
  const double* rp_in;   // [batch][8][D], may be null (zeros)
  double* q_out;
  double* v_out;
  double* qlo_out;       // may be null
  double* vlo_out;
  double* rp_out;        // may be null
  const long long* nsteps;  // [batch] or null -> nsteps_all
  long long nsteps_all;
  const double* h;          // [batch] or null -> h_all
  double h_all;
  const int* order;         // [batch] or null
  int* iters_hist;          // [batch][hist_len] or null
  long long* iters_total;   // [batch] or null
  double* dH_max;           // [batch] or null
  int* status;              // [batch] or null
  long long* steps_done;    // [batch] or null
  unsigned int* counter;    // work counter, zero at launch
  const double* params;     // right-hand-side parameters (device)
  double* H0_io;            // [batch] reference energy: read, or written when h0_init; an
                            // entry that is NaN is computed at the trajectory's first step
                            // of the call and written (a trajectory joining a running batch)
  int h0_init;              // 1: compute H0 at the first step and store it in H0_io
  int param_stride;         // 0: params serve every trajectory; else trajectory t reads its
                            // own at params + t * param_stride
  int sticky_status;        // 1: status is in/out; a trajectory whose entry is nonzero on
                            // entry stopped in an earlier call and is not advanced again
  int accumulate;           // 1: dH_max / iters_total start from the values in the arrays
  int monitor_local;        // 1: dH_max = max_n |(H_n - H_{n-1}) / H_{n-1}| (Eq. DHlocmax)
  // time t_n as a compensated pair, read only by time-dependent right-hand
  // sides (null in: t = 0; null out: not written)
  const double* t_in;       // [batch]
  const double* tlo_in;     // [batch]
  double* t_out;            // [batch]
  double* tlo_out;          // [batch]
};

// ------------------------------------------------------------------------
// arithmetic helpers
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffULL;
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}

// Seed y0 ~ x^(-1/2) with at most 24 significant bits (so y0*y0 is exact in
// FP64), for a positive normal x: the leading 23 mantissa bits of x, with the
// exponent parity folded in, form an FP32 number in [1, 4); its FP32
// reciprocal square root (MUFU.RSQ, about 22 correct bits) is rescaled by
// 2^(-floor(E/2)) by integer exponent arithmetic.  Callers handle x that is
// zero, subnormal, negative, Inf or NaN separately.
__device__ __forceinline__ double rsqrt_seed(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bx >> 52) & 0x7ff) - 1023;
  const int par = E & 1;
  const int half = (E - par) / 2;
  const unsigned m23 = static_cast<unsigned>((bx >> 29) & 0x7fffffu);
  const float xf = __uint_as_float((static_cast<unsigned>(127 + par) << 23) | m23);
  const float yf = rsqrtf(xf);  // in (0.5, 1]
  const unsigned yb = __float_as_uint(yf);
  const int ef = static_cast<int>(yb >> 23) - 127;
  const unsigned long long y0b =
      (static_cast<unsigned long long>(ef - half + 1023) << 52) |
      (static_cast<unsigned long long>(yb & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(y0b));
}

__device__ __forceinline__ bool positive_normal(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  return (bx - 0x0010000000000000ULL) < 0x7fe0000000000000ULL;  // 0 < x < Inf, normal
}

// x^(-3/2) of the special operands, resolved from the bit pattern (no
// division or square root subroutine, whose call would make the compiler
// keep stack space for the registers live across it): +-0 and positive
// subnormals give +Inf (the exact value exceeds the FP64 range), +Inf gives
// 0, negative and NaN give NaN.
__device__ __forceinline__ double rinv3_special(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  if ((bx << 1) == 0ull || bx < 0x0010000000000000ULL) return __longlong_as_double(0x7ff0000000000000LL);
  if (bx == 0x7ff0000000000000ULL) return 0.0;
  return __longlong_as_double(0x7ff8000000000000LL);
}

// x^(-3/2) for a positive normal x in FP64 (used where the result is
// subnormal).  From the seed y0 with e = 1 - x y0^2 (|e| < 2^-20):
// x^(-3/2) = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 3/2 e + 15/8 e^2 + O(e^3)),
// the binomial series (a third-order Householder correction); truncation
// error < 2^-57, so the result is within about one ulp.  6 FP64 operations.
__device__ __forceinline__ double rinv3_fp64(double x) {
  const double y0 = rsqrt_seed(x);
  const double y02 = y0 * y0;          // exact
  const double e = fma(-x, y02, 1.0);
  const double y03 = y02 * y0;
  const double p = fma(e, 1.875, 1.5);
  const double t = e * p;
  return fma(y03, t, y03);
}

// x^(-3/2) for x > 0 with no FP64 arithmetic at all: the same expansion
// y0^3 (1 + 3/2 e + 15/8 e^2), e = 1 - x y0^2, evaluated in integers.  With
// x = X 2^Ex (X the 53-bit significand) and the FP32 seed y0 = Yf 2^f (Yf its
// 24-bit significand):
//   * P = X Yf^2 (101 bits, exact) is x y0^2 scaled by 2^k, k = -(Ex + 2f);
//     e 2^56 = 2^56 - P / 2^(k-56), truncated (|e| < 2^-21, so this fits in
//     38 bits and is off by less than 2^-56);
//   * T = (3/2 e + 15/8 e^2) 2^56 from that integer (the square from its top
//     28 bits: the term is below 2^-40, so 2^-27 of it is negligible);
//   * y0^3 = Yf^3 (72 bits, top 64 kept) times (2^56 + T) 2^7, top 64 bits
//     of the 128-bit product, rounded to nearest-even FP64.
// Truncations add about 0.15 ulp to the rounding: 0.66 ulp worst case over
// 2e5 random arguments (the FP64 form above is within about one ulp).  About
// 60 integer operations and one FP32 reciprocal square root replace six
// FP64 operations, and FP64 issues 1/64 as fast as the integer pipes on
// GB300.  A result above the FP64 range (x below about 2^-682) is +Inf; a
// subnormal one (x above about 2^681) takes the FP64 form.
__device__ __forceinline__ double rinv3_int(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bx >> 52) & 0x7ff);
  const unsigned long long X = (bx & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
  const int Eu = E - 1023;
  const int par = Eu & 1;
  const int half = (Eu - par) / 2;  // exact: Eu - par is even
  const unsigned m23 = static_cast<unsigned>((bx >> 29) & 0x7fffffu);
  const float yf = rsqrtf(__uint_as_float((static_cast<unsigned>(127 + par) << 23) | m23));  // (0.5, 1]
  const unsigned yb = __float_as_uint(yf);
  const int f = static_cast<int>(yb >> 23) - 127 - 23 - half;   // y0 = Yf 2^f
  const unsigned long long Yf = (yb & 0x7fffffu) | 0x800000u;
  const unsigned long long Y2 = Yf * Yf;                       // 48 bits, exact
  const unsigned long long Plo = X * Y2, Phi = __umul64hi(X, Y2);
  const int sh = (1075 - E) - 2 * f - 56;                      // k - 56 = 42 - par - 2 ef: 41..44
  const unsigned long long Ptop = (Phi << (64 - sh)) | (Plo >> sh);
  const long long D = static_cast<long long>((1ULL << 56) - Ptop);  // e 2^56
  const long long Dq = D >> 8;
  const long long T = ((3 * D) >> 1) + ((15 * Dq * Dq) >> 43);
  const unsigned long long M = static_cast<unsigned long long>((1LL << 56) + T) << 7;
  const unsigned long long C = (__umul64hi(Y2, Yf) << 56) | ((Y2 * Yf) >> 8);  // Yf^3 / 2^8
  const unsigned long long hi = __umul64hi(C, M);               // in [2^59, 2^64)
  const int lz = __clzll(static_cast<long long>(hi));
  const unsigned long long mant = hi << lz;
  const int biased = 3 * f + 72 - lz + 1023;
  if (biased >= 2047) return __longlong_as_double(0x7ff0000000000000LL);  // above the range
  if (biased <= 0) return rinv3_fp64(x);  // subnormal or zero result
  const unsigned long long m53 = mant >> 11;
  unsigned long long bits = (static_cast<unsigned long long>(biased - 1) << 52) + m53;
  bits += ((mant >> 10) & 1ULL) & (((mant & 0x3ffULL) != 0ULL ? 1ULL : 0ULL) | (m53 & 1ULL));
  return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ double rinv3(double x) {
  if (!positive_normal(x)) return rinv3_special(x);
  return rinv3_int(x);
}

// m 2^e2 rounded to the nearest FP64 (ties to even), m > 0, the result
// normal.
__device__ __forceinline__ double u64_scaled_to_double(unsigned long long m, int e2) {
  const int lz = __clzll(static_cast<long long>(m));
  const unsigned long long mant = m << lz;
  const unsigned long long m53 = mant >> 11;
  unsigned long long bits = (static_cast<unsigned long long>(e2 - lz + 63 + 1023 - 1) << 52) + m53;
  bits += ((mant >> 10) & 1ULL) & (((mant & 0x3ffULL) != 0ULL ? 1ULL : 0ULL) | (m53 & 1ULL));
  return __longlong_as_double(static_cast<long long>(bits));
}

// sin x and cos x by fixed-point arithmetic, for 2^-30 <= |x| < 64 (other
// arguments take the FP64 sincos):
//   * t = |x| 2/pi from the exact product of x's 53-bit significand with
//     2/pi rounded to 128 bits, kept as t 2^120 in 128 bits (error below
//     2^-120); n = round(t) gives the quadrant, f = t - n in [-1/2, 1/2]
//     keeps at least 59 significant bits however close x lies to a
//     multiple of pi/2 (|x| < 64);
//   * with z = f^2, sin(pi/2 f) = f S(z) and cos(pi/2 f) = C(z), S and C
//     the Taylor series to z^10 with coefficients rounded to 2^-62
//     (generated), evaluated by Horner's rule in 64-bit fixed point;
//   * each value rounded once to FP64, signs and swaps by the quadrant.
// 0.503 ulp worst case for both over 3e4 arguments in a Python model of the
// integer steps against 80-digit decimals; about 130 integer operations in
// place of an FP64 argument reduction and two polynomials.
__device__ __forceinline__ void sincos_fx(double x, double& sv, double& cv) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bx >> 52) & 0x7ff);
  if (E < 993 || E > 1028) {
    sincos(x, &sv, &cv);
    return;
  }
  const unsigned long long T = (bx & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
  // P = T (2/pi) 2^128: 181 bits in p2:p1:p0
  const unsigned long long p0 = T * IRKGL_TWO_OVER_PI_LO;
  const unsigned long long h0 = __umul64hi(T, IRKGL_TWO_OVER_PI_LO);
  const unsigned long long l1 = T * IRKGL_TWO_OVER_PI_HI;
  const unsigned long long p1 = h0 + l1;
  const unsigned long long p2 = __umul64hi(T, IRKGL_TWO_OVER_PI_HI) + (p1 < h0 ? 1ULL : 0ULL);
  // F = P >> sh = t 2^120, sh = 1083 - E in [55, 90]
  const int sh = 1083 - E;
  unsigned long long FL, FH;
  if (sh < 64) {
    FL = (p0 >> sh) | (p1 << (64 - sh));
    FH = (p1 >> sh) | (p2 << (64 - sh));
  } else {
    const int s2 = sh - 64;
    FL = s2 ? ((p1 >> s2) | (p2 << (64 - s2))) : p1;
    FH = p2 >> s2;
  }
  const long long n = static_cast<long long>((FH + (1ULL << 55)) >> 56);
  const long long fH = static_cast<long long>(FH) - (n << 56);  // (t - n) 2^120, high word
  const bool fneg = fH < 0;
  unsigned long long aL = FL, aH = static_cast<unsigned long long>(fH);
  if (fneg) {
    aL = ~FL + 1ULL;
    aH = ~aH + (aL == 0ULL ? 1ULL : 0ULL);
  }
  // |f| = m 2^ef with m normalized to 64 bits
  unsigned long long m;
  int ef;
  if (aH) {
    const int lz = __clzll(static_cast<long long>(aH));
    m = lz ? ((aH << lz) | (aL >> (64 - lz))) : aH;
    ef = -56 - lz;
  } else {
    const int lz = __clzll(static_cast<long long>(aL));
    m = aL << lz;
    ef = -120 - lz;
  }
  const unsigned long long fx = (aH << 8) | (aL >> 56);           // |f| 2^64
  const long long Z = static_cast<long long>(__umul64hi(fx, fx));  // f^2 2^64 < 2^62
  long long sp = irkgl_sin_coef(IRKGL_SINCOS_TERMS - 1), cp = irkgl_cos_coef(IRKGL_SINCOS_TERMS - 1);
#pragma unroll
  for (int k = IRKGL_SINCOS_TERMS - 2; k >= 0; k--) {
    sp = irkgl_sin_coef(k) + __mul64hi(sp, Z);
    cp = irkgl_cos_coef(k) + __mul64hi(cp, Z);
  }
  double sr = u64_scaled_to_double(__umul64hi(m, static_cast<unsigned long long>(sp)), ef + 2);
  if (fneg) sr = -sr;
  const double cr = u64_scaled_to_double(static_cast<unsigned long long>(cp), -62);
  const int q = static_cast<int>(n & 3);
  double s_ = (q & 1) ? cr : sr, c_ = (q & 1) ? sr : cr;
  if (q == 1 || q == 2) c_ = -c_;
  if (q >= 2) s_ = -s_;
  sv = (bx >> 63) ? -s_ : s_;
  cv = c_;
}

// 1/x with no FP64 arithmetic, the same construction: an FP32 seed
// y0 = Yf 2^f of the reciprocal of x's leading 24 bits (rcp.approx, within
// an FP32 ulp), e = 1 - x y0 from the exact integer product X Yf (77 bits)
// as e 2^56, then 1/x = y0 (1 + e + e^2) (|e| < 2^-21, the e^3 term is
// below 2^-63) as Yf (2^56 + T) 2^7 with the top 64 bits of the product
// rounded to nearest-even.  0.61 ulp worst case over 2e5 random arguments of
// both signs across the exponent range (a Python model of the integer steps
// against 60-digit decimals).  Zero, subnormal, infinite and NaN arguments
// and subnormal results (|x| > 2^1022) take the FP64 division.
__device__ __forceinline__ double rcp_int(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bx >> 52) & 0x7ff);
  if (E == 0 || E >= 0x7fe) return 1.0 / x;
  const unsigned long long X = (bx & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
  const unsigned m23 = static_cast<unsigned>((bx >> 29) & 0x7fffffu);
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float((127u << 23) | m23)));  // (0.5, 1]
  const unsigned yb = __float_as_uint(yf);
  const int f = static_cast<int>(yb >> 23) - 127 - 23 - (E - 1023);  // y0 = Yf 2^f
  const unsigned long long Yf = (yb & 0x7fffffu) | 0x800000u;
  const unsigned long long P = X * Yf;                  // 77 bits: the low 64 ...
  const unsigned long long Ph = __umul64hi(X, Yf);      // ... and the high ones
  const int sh = (1075 - E) - f - 56;                   // k - 56, about 19..20
  const unsigned long long Ptop = (Ph << (64 - sh)) | (P >> sh);
  const long long D = static_cast<long long>((1ULL << 56) - Ptop);  // e 2^56
  const long long Dq = D >> 8;
  const long long T = D + ((Dq * Dq) >> 40);            // (e + e^2) 2^56
  const unsigned long long M = static_cast<unsigned long long>((1LL << 56) + T) << 7;
  const unsigned long long hi = __umul64hi(Yf << 40, M);
  const int lz = __clzll(static_cast<long long>(hi));
  const unsigned long long mant = hi << lz;
  const int biased = f + 24 - lz + 1023;
  if (biased <= 0) return 1.0 / x;
  const unsigned long long m53 = mant >> 11;
  unsigned long long bits = (static_cast<unsigned long long>(biased - 1) << 52) + m53;
  bits += ((mant >> 10) & 1ULL) & (((mant & 0x3ffULL) != 0ULL ? 1ULL : 0ULL) | (m53 & 1ULL));
  return __longlong_as_double(static_cast<long long>(bits | (bx & 0x8000000000000000ULL)));
}

// x^(-1/2) for a positive normal x with no FP64 arithmetic, as rinv3_int:
// y0 (1 + e/2 + 3/8 e^2), e = 1 - x y0^2 from the exact integer product, the
// correction in 64-bit integers, y0 = Yf 2^f times (2^56 + T) 2^7 rounded
// from the top 64 bits.  0.68 ulp worst case over 2e5 random arguments (a
// Python model of the integer steps against 60-digit decimals); the result
// (between 2^-512 and 2^511) is always normal.
__device__ __forceinline__ double rinv1_int(double x) {
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((bx >> 52) & 0x7ff);
  const unsigned long long X = (bx & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
  const int Eu = E - 1023;
  const int par = Eu & 1;
  const int half = (Eu - par) / 2;
  const unsigned m23 = static_cast<unsigned>((bx >> 29) & 0x7fffffu);
  const float yf = rsqrtf(__uint_as_float((static_cast<unsigned>(127 + par) << 23) | m23));
  const unsigned yb = __float_as_uint(yf);
  const int f = static_cast<int>(yb >> 23) - 127 - 23 - half;  // y0 = Yf 2^f
  const unsigned long long Yf = (yb & 0x7fffffu) | 0x800000u;
  const unsigned long long Y2 = Yf * Yf;
  const unsigned long long Plo = X * Y2, Phi = __umul64hi(X, Y2);
  const int sh = (1075 - E) - 2 * f - 56;  // 41..44, as in rinv3_int
  const unsigned long long Ptop = (Phi << (64 - sh)) | (Plo >> sh);
  const long long D = static_cast<long long>((1ULL << 56) - Ptop);  // e 2^56
  const long long Dq = D >> 8;
  const long long T = (D >> 1) + ((3 * Dq * Dq) >> 43);            // (e/2 + 3/8 e^2) 2^56
  const unsigned long long M = static_cast<unsigned long long>((1LL << 56) + T) << 7;
  const unsigned long long hi = __umul64hi(Yf << 40, M);
  const int lz = __clzll(static_cast<long long>(hi));
  const unsigned long long mant = hi << lz;
  const unsigned long long m53 = mant >> 11;
  unsigned long long bits = (static_cast<unsigned long long>(f + 24 - lz + 1023 - 1) << 52) + m53;
  bits += ((mant >> 10) & 1ULL) & (((mant & 0x3ffULL) != 0ULL ? 1ULL : 0ULL) | (m53 & 1ULL));
  return __longlong_as_double(static_cast<long long>(bits));
}

// Special operands from the bit pattern, as for rinv3: +0 -> +Inf, -0 -> -Inf,
// a positive subnormal is scaled by 2^54 (exactly) and the result by 2^27,
// +Inf -> 0, negative and NaN -> NaN.
__device__ __forceinline__ double rinv1(double x) {
  if (positive_normal(x)) return rinv1_int(x);
  const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x));
  if (bx == 0ull) return __longlong_as_double(0x7ff0000000000000LL);
  if (bx == 0x8000000000000000ULL) return __longlong_as_double(static_cast<long long>(0xfff0000000000000ULL));
  if (bx < 0x0010000000000000ULL) return rinv1_int(x * 18014398509481984.0) * 134217728.0;
  if (bx == 0x7ff0000000000000ULL) return 0.0;
  return __longlong_as_double(0x7ff8000000000000LL);
}

// (hi, lo) + x: Knuth's TwoSum of hi and x, error folded into lo, Dekker's
// Fast2Sum renormalisation (Sec. 5, improved summation).  Explicit
// round-to-nearest adds keep the compiler from contracting or reordering.
__device__ __forceinline__ void two_sum_add(double& hi, double& lo, double x) {
  const double s = __dadd_rn(hi, x);
  const double bb = __dsub_rn(s, hi);
  const double err = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bb)), __dsub_rn(x, bb));
  const double lo2 = __dadd_rn(lo, err);
  const double hi2 = __dadd_rn(s, lo2);
  lo = __dsub_rn(lo2, __dsub_rn(hi2, s));
  hi = hi2;
}

// ------------------------------------------------------------------------
// Fixed-point mixing on the integer pipes (kernel variant MIX = 1)
//
// The sums sum_j eta_ij R_j (and sum_k W_ik R_k) are accumulated exactly in
// 128-bit integers and rounded once to FP64, instead of eight FP64 FMAs:
//   * the eight R_j of one component share a scale: with emax the largest
//     biased exponent among them, R_j is truncated to the integer
//     r_j = R_j 2^(1083 - emax) (|r_j| < 2^61; exact unless R_j is more than
//     2^8 smaller than the largest, where the dropped bits lie below 2^-61 of
//     it), then offset to r'_j = r_j + 2^61 >= 0;
//   * eta_ij = +-n_ij 2^-63 with n_ij an exact integer (every eta is on that
//     grid); W_ik = +-w_ik 2^-50 rounded (W only seeds the initial guess);
//   * products n r' (64 x 64 -> 128 bits, eight 32-bit multiply-adds with
//     carry) go to one accumulator, a negative coefficient multiplying the
//     two's complement 2^64 - r' of the operand; minus the row constant
//     rbias_i = sum_j (+-n_ij) 2^61 + 2^64 sum_{negative j} n_ij (mod 2^128)
//     that is the exact sum, rounded to nearest-even FP64.
// The result is the correctly rounded value of the (exact) sum, one rounding
// instead of the FMA chain's eight.
// ------------------------------------------------------------------------
struct U128 {
  unsigned x0, x1, x2, x3;
};

// a += p * q (unsigned 64 x 64 -> 128)
__device__ __forceinline__ void mac64(U128& a, unsigned long long p, unsigned long long q) {
  const unsigned p0 = static_cast<unsigned>(p), p1 = static_cast<unsigned>(p >> 32);
  const unsigned q0 = static_cast<unsigned>(q), q1 = static_cast<unsigned>(q >> 32);
  asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32 %3, %5, %7, %3;"
      : "+r"(a.x0), "+r"(a.x1), "+r"(a.x2), "+r"(a.x3)
      : "r"(p0), "r"(p1), "r"(q0), "r"(q1));
}

// a -= b (mod 2^128)
__device__ __forceinline__ void sub128(U128& a, unsigned b0, unsigned b1, unsigned b2, unsigned b3) {
  asm("sub.cc.u32 %0, %0, %4;\n\t"
      "subc.cc.u32 %1, %1, %5;\n\t"
      "subc.cc.u32 %2, %2, %6;\n\t"
      "subc.u32 %3, %3, %7;"
      : "+r"(a.x0), "+r"(a.x1), "+r"(a.x2), "+r"(a.x3)
      : "r"(b0), "r"(b1), "r"(b2), "r"(b3));
}

// Round-to-nearest-even FP64 of v * 2^e2, v a 128-bit two's complement
// integer.  The result must be a normal number (|value| well inside range).
__device__ __forceinline__ double s128_to_double(const U128& v, int e2) {
  const unsigned s = v.x3 >> 31;
  unsigned long long hi = (static_cast<unsigned long long>(v.x3) << 32) | v.x2;
  unsigned long long lo = (static_cast<unsigned long long>(v.x1) << 32) | v.x0;
  if (s) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if ((hi | lo) == 0ull) return 0.0;
  int lz = 0;
  if (hi == 0ull) {
    hi = lo;
    lo = 0ull;
    lz = 64;
  }
  const int z = __clzll(static_cast<long long>(hi));
  if (z) {
    hi = (hi << z) | (lo >> (64 - z));
    lo <<= z;
  }
  lz += z;
  const int E = (127 - lz + e2) + 1023;  // biased exponent of the leading bit
  const unsigned long long mant = hi >> 11;  // 53 bits, leading bit 2^52
  const unsigned long long rbit = (hi >> 10) & 1ull;
  const unsigned long long sticky = ((hi & 0x3ffull) | lo) != 0ull ? 1ull : 0ull;
  unsigned long long bits = (static_cast<unsigned long long>(E - 1) << 52) + mant;
  bits += rbit & (sticky | (mant & 1ull));
  bits |= static_cast<unsigned long long>(s) << 63;
  return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ int biased_exp(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff);
}

// r' = trunc(x 2^(1083 - emax)) + 2^61 for x with biased exponent <= emax
// (zero and subnormal x give the offset alone).
__device__ __forceinline__ unsigned long long to_fixed_offset(double x, int emax) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  const unsigned long long m = e ? ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) : 0ull;
  const int sh = 8 - (emax - e);
  const unsigned long long mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
  constexpr unsigned long long OFF = 1ull << IRKGL_R_BIAS;
  return (b >> 63) ? OFF - mag : OFF + mag;
}

// sum_j coef_ij R_j for row i (compile-time after unrolling), R_j given as
// offset fixed point rb[j] with shared exponent emax.  IS_W selects W.
template <bool IS_W>
__device__ __forceinline__ double fixed_row(int i, const unsigned long long (&rb)[S], int emax) {
  // one accumulator: a negative coefficient takes the two's complement of
  // the operand (computed once per column, shared by the rows), and the row
  // constant rbias absorbs the n_ij 2^64 that adds (see fixed_row_rt)
  U128 P{0u, 0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < S; j++) {
    const int k = i * S + j;
    const unsigned long long m = IS_W ? irkgl_w_mag(k) : irkgl_eta_mag(k);
    const bool neg = IS_W ? irkgl_w_neg(k) : irkgl_eta_neg(k);
    mac64(P, m, neg ? (0ull - rb[j]) : rb[j]);
  }
  if (IS_W) sub128(P, irkgl_w_rbias(i, 0), irkgl_w_rbias(i, 1), irkgl_w_rbias(i, 2), irkgl_w_rbias(i, 3));
  else sub128(P, irkgl_eta_rbias(i, 0), irkgl_eta_rbias(i, 1), irkgl_eta_rbias(i, 2), irkgl_eta_rbias(i, 3));
  constexpr int shift = IS_W ? IRKGL_W_SHIFT : IRKGL_ETA_SHIFT;
  return s128_to_double(P, emax - 1083 - shift);
}

// Row sums for tiles that hold one or two stage rows per lane (LPT > 1), where
// the row index, and so each coefficient's sign, is known only at run time.
// A negative coefficient multiplies the two's complement 2^64 - r'_j of the
// operand (r'_j lies in [1, 2^62), so that is a positive 64-bit integer) and
// the products share one accumulator; the extra n_ij 2^64 of each negative
// entry is part of the row constant rbias_i.  The result is the same
// correctly rounded exact sum as fixed_row's.
struct FixedRowTables {
  unsigned long long mag[2][S * S];  // [0] eta, [1] W: |coef| on the 2^-SHIFT grid
  unsigned rbias[2][S * 4];          // per-row constants, 128-bit words
  unsigned negbits[2][S];            // bit j: coefficient (i, j) is negative
};
constexpr FixedRowTables make_fixed_row_tables() {
  FixedRowTables t{};
  for (int k = 0; k < S * S; k++) {
    t.mag[0][k] = irkgl_eta_mag(k);
    t.mag[1][k] = irkgl_w_mag(k);
    t.negbits[0][k / S] |= (irkgl_eta_neg(k) ? 1u : 0u) << (k % S);
    t.negbits[1][k / S] |= (irkgl_w_neg(k) ? 1u : 0u) << (k % S);
  }
  for (int k = 0; k < S * 4; k++) {
    t.rbias[0][k] = irkgl_eta_rbias(k / 4, k % 4);
    t.rbias[1][k] = irkgl_w_rbias(k / 4, k % 4);
  }
  return t;
}
static __constant__ FixedRowTables kFixedRows = make_fixed_row_tables();

// sum_j coef_ij R_j with the row's magnitudes mags[0..7], sign bits negbits
// and constant rbias[0..3]; R_j as offset fixed point rb[j], exponent emax.
template <int SHIFT>
__device__ __forceinline__ double fixed_row_rt(const unsigned long long* mags, unsigned negbits,
                                               const unsigned* rbias, const unsigned long long (&rb)[S],
                                               int emax) {
  U128 P{0u, 0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < S; j++) {
    const unsigned long long m = 0ull - static_cast<unsigned long long>((negbits >> j) & 1u);
    mac64(P, mags[j], (rb[j] ^ m) - m);
  }
  sub128(P, rbias[0], rbias[1], rbias[2], rbias[3]);
  return s128_to_double(P, emax - 1083 - SHIFT);
}

// Offset fixed-point form of the eight R_j of one component; returns emax and
// flags a non-finite R (whose sums must come out non-finite).
__device__ __forceinline__ int fixed_column(const double (&Rc)[S], unsigned long long (&rb)[S],
                                            bool& nonfinite) {
  int emax = 0;
#pragma unroll
  for (int j = 0; j < S; j++) emax = max(emax, biased_exp(Rc[j]));
  nonfinite = emax == 0x7ff;
#pragma unroll
  for (int j = 0; j < S; j++) rb[j] = to_fixed_offset(Rc[j], emax);
  return emax;
}

// ------------------------------------------------------------------------
// right-hand sides: R = (h b_i) g(Q_i) for one stage, and H(q, v)
// ------------------------------------------------------------------------
template <int SPL>
struct Kepler {
  static constexpr int D = 2;
  double mu;
  double s[SPL];  // -(h b_i) mu per own stage
  __device__ void load_params(const double* p) { mu = p[0]; }
  __device__ void set_step(const double (&hb)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) s[t] = -(hb[t] * mu);
  }
  __device__ __forceinline__ void stage_R(int t, const double (&x)[D], double (&R)[D]) const {
    const double r2 = fma(x[0], x[0], x[1] * x[1]);
    const double w = s[t] * rinv3(r2);
    R[0] = x[0] * w;
    R[1] = x[1] * w;
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    const double ke = 0.5 * fma(v[0], v[0], v[1] * v[1]);
    return fma(-mu, rinv1(fma(q[0], q[0], q[1] * q[1])), ke);
  }
};

template <int SPL>
struct HenonHeiles {
  static constexpr int D = 2;
  double lam, twolam;
  double s[SPL];  // -(h b_i)
  __device__ void load_params(const double* p) {
    lam = p[0];
    twolam = 2.0 * p[0];
  }
  __device__ void set_step(const double (&hb)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) s[t] = -hb[t];
  }
  // g1 = -q1 (1 + 2 lam q2), g2 = -(q2 + lam (q1^2 - q2^2))
  __device__ __forceinline__ void stage_R(int t, const double (&x)[D], double (&R)[D]) const {
    const double a = fma(twolam, x[1], 1.0);
    R[0] = s[t] * (x[0] * a);
    const double u = fma(x[0], x[0], -(x[1] * x[1]));
    R[1] = s[t] * fma(lam, u, x[1]);
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    const double ke = 0.5 * fma(v[0], v[0], v[1] * v[1]);
    const double pe = 0.5 * fma(q[0], q[0], q[1] * q[1]);
    const double cub = fma(q[0] * q[0], q[1], -(q[1] * q[1] * q[1]) * (1.0 / 3.0));
    return fma(lam, cub, ke + pe);
  }
};

// The non-autonomous Henon-Heiles system printed with the user-function
// example of Sec. 3: g1 = -q1 (1 + 2 a(t) q2), g2 = -(q2 + a(t) (q1^2 - q2^2)),
// a(t) = lam + xi sin t.  g is evaluated at the stage times t_n + c_i h
// (Eq. IRK_FP, first line); a(t) is formed once per stage per step, since
// the stage times do not change across the fixed-point sweeps.
template <int SPL>
struct HenonHeilesForced {
  static constexpr int D = 2;
  static constexpr bool kTime = true;
  double lam, xi;
  double s[SPL];             // -(h b_i)
  double aux[SPL], aux2[SPL];  // a(t_n + c_i h) and twice it
  __device__ void load_params(const double* p) {
    lam = p[0];
    xi = p[1];
  }
  __device__ void set_step(const double (&hb)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) s[t] = -hb[t];
  }
  __device__ void set_time(const double (&tau)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) {
      aux[t] = fma(xi, sin(tau[t]), lam);
      aux2[t] = 2.0 * aux[t];
    }
  }
  __device__ __forceinline__ void stage_R(int t, const double (&x)[D], double (&R)[D]) const {
    const double a = fma(aux2[t], x[1], 1.0);
    R[0] = s[t] * (x[0] * a);
    const double u = fma(x[0], x[0], -(x[1] * x[1]));
    R[1] = s[t] * fma(aux[t], u, x[1]);
  }
  // H of the autonomous part; H(t) is not conserved, and the host turns the
  // energy monitor off for this kind.
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    const double ke = 0.5 * fma(v[0], v[0], v[1] * v[1]);
    const double pe = 0.5 * fma(q[0], q[0], q[1] * q[1]);
    const double cub = fma(q[0] * q[0], q[1], -(q[1] * q[1] * q[1]) * (1.0 / 3.0));
    return fma(lam, cub, ke + pe);
  }
};

template <int SPL, int DD>
struct Harmonic {
  static constexpr int D = DD;
  double w2;
  double s[SPL];  // -(h b_i) omega^2
  __device__ void load_params(const double* p) { w2 = p[0] * p[0]; }
  __device__ void set_step(const double (&hb)[SPL]) {
#pragma unroll
    for (int t = 0; t < SPL; t++) s[t] = -(hb[t] * w2);
  }
  __device__ __forceinline__ void stage_R(int t, const double (&x)[D], double (&R)[D]) const {
#pragma unroll
    for (int l = 0; l < D; l++) R[l] = s[t] * x[l];
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < D; l++) acc = fma(0.5 * v[l], v[l], fma(0.5 * w2 * q[l], q[l], acc));
    return acc;
  }
};

// Newtonian N-body in 3-D (Eq. Ham2): g_a = G sum_{b != a} m_b (q_b - q_a)/|q_b - q_a|^3.
// Pairs are visited once (a < b) and both bodies are updated, 20 FP64
// operations per pair; (h b_i) G m_b is folded into one weight per body.
template <int SPL, int NB>
struct NBody {
  static constexpr int D = 3 * NB;
  // G and the masses stay in (L1-cached) global memory: they enter only the
  // per-step weights and the energy, and registers are the scarce resource
  const double* prm;  // G, m_1..m_NB
  double w[SPL][NB];  // (h b_i) G m_b
  __device__ void load_params(const double* p) { prm = p; }
  __device__ __forceinline__ double G() const { return __ldg(prm); }
  __device__ __forceinline__ double m(int b) const { return __ldg(prm + 1 + b); }
  __device__ void set_step(const double (&hb)[SPL]) {
    const double G0 = G();
#pragma unroll
    for (int t = 0; t < SPL; t++)
#pragma unroll
      for (int b = 0; b < NB; b++) w[t][b] = (hb[t] * G0) * m(b);
  }
  // Pair P of (0,1), (0,2), ..., (0,NB-1), (1,2), ...: the pairs are expanded
  // from an index sequence, so every array index is a compile-time constant
  // (a triangular loop nest left the arrays in local memory for NB >= 5).
  __host__ __device__ static constexpr int pair_first(int p) {
    int a = 0;
    while (p >= NB - 1 - a) {
      p -= NB - 1 - a;
      a++;
    }
    return a;
  }
  __host__ __device__ static constexpr int pair_second(int p) {
    int a = 0;
    while (p >= NB - 1 - a) {
      p -= NB - 1 - a;
      a++;
    }
    return a + 1 + p;
  }
  template <int P>
  __device__ __forceinline__ void pair_R(int t, const double (&x)[D], double (&R)[D]) const {
    constexpr int a = pair_first(P), b = pair_second(P);
    const double dx = x[3 * b] - x[3 * a];
    const double dy = x[3 * b + 1] - x[3 * a + 1];
    const double dz = x[3 * b + 2] - x[3 * a + 2];
    const double z = rinv3(fma(dx, dx, fma(dy, dy, dz * dz)));
    const double wb = w[t][b] * z, wa = w[t][a] * z;
    R[3 * a] = fma(wb, dx, R[3 * a]);
    R[3 * a + 1] = fma(wb, dy, R[3 * a + 1]);
    R[3 * a + 2] = fma(wb, dz, R[3 * a + 2]);
    R[3 * b] = fma(-wa, dx, R[3 * b]);
    R[3 * b + 1] = fma(-wa, dy, R[3 * b + 1]);
    R[3 * b + 2] = fma(-wa, dz, R[3 * b + 2]);
  }
  template <int... P>
  __device__ __forceinline__ void pairs_R(int t, const double (&x)[D], double (&R)[D],
                                          std::integer_sequence<int, P...>) const {
    (pair_R<P>(t, x, R), ...);
  }
  __device__ __forceinline__ void stage_R(int t, const double (&x)[D], double (&R)[D]) const {
#pragma unroll
    for (int l = 0; l < D; l++) R[l] = 0.0;
    pairs_R(t, x, R, std::make_integer_sequence<int, NB * (NB - 1) / 2>{});
  }
  // The share of H computed by lane r of a group of L lanes: pairs
  // p = r, r + L, ... (of the NB (NB-1)/2) and the kinetic energy of bodies
  // a = r, r + L, ...; the group sums the shares.  Bodies indexed at run time
  // are picked from the register arrays by unrolled selects (no local-memory
  // copies of q, v or m).
  static constexpr bool kSplitH = true;
  __device__ static __forceinline__ void pick3(const double (&x)[D], int a, double& x0, double& x1,
                                               double& x2) {
    x0 = x[0];
    x1 = x[1];
    x2 = x[2];
#pragma unroll
    for (int u = 1; u < NB; u++) {
      x0 = (a == u) ? x[3 * u] : x0;
      x1 = (a == u) ? x[3 * u + 1] : x1;
      x2 = (a == u) ? x[3 * u + 2] : x2;
    }
  }
  __device__ double H_part(int r, int L, const double (&q)[D], const double (&v)[D]) const {
    double acc = 0.0;
    for (int a = r; a < NB; a += L) {
      double v0, v1, v2;
      pick3(v, a, v0, v1, v2);
      acc = fma(0.5 * m(a), fma(v0, v0, fma(v1, v1, v2 * v2)), acc);
    }
    constexpr int NP = NB * (NB - 1) / 2;
    double pot = 0.0;
    for (int p = r; p < NP; p += L) {
      int a = 0, b = p;
      while (b >= NB - 1 - a) {
        b -= NB - 1 - a;
        a++;
      }
      b += a + 1;
      double xa, ya, za, xb, yb, zb;
      pick3(q, a, xa, ya, za);
      pick3(q, b, xb, yb, zb);
      const double dx = xb - xa;
      const double dy = yb - ya;
      const double dz = zb - za;
      pot = fma(m(a) * m(b), rinv1(fma(dx, dx, fma(dy, dy, dz * dz))), pot);
    }
    return fma(-G(), pot, acc);
  }
  __device__ double H(const double (&q)[D], const double (&v)[D]) const {
    double kin = 0.0, pot = 0.0;
#pragma unroll
    for (int a = 0; a < NB; a++)
      kin = fma(0.5 * m(a), fma(v[3 * a], v[3 * a], fma(v[3 * a + 1], v[3 * a + 1], v[3 * a + 2] * v[3 * a + 2])), kin);
#pragma unroll
    for (int a = 0; a < NB; a++)
#pragma unroll
      for (int b = a + 1; b < NB; b++) {
        const double dx = q[3 * b] - q[3 * a];
        const double dy = q[3 * b + 1] - q[3 * a + 1];
        const double dz = q[3 * b + 2] - q[3 * a + 2];
        pot = fma(m(a) * m(b), rinv1(fma(dx, dx, fma(dy, dy, dz * dz))), pot);
      }
    return fma(-G(), pot, kin);
  }
};

// ------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------
template <class T, class = void>
struct split_energy : std::false_type {};
template <class T>
struct split_energy<T, std::void_t<decltype(T::kSplitH)>> : std::integral_constant<bool, T::kSplitH> {};

// Right-hand sides that read t (g(t, q)) declare kTime = true and provide
// set_time(stage times of the lane's stages).
template <class T, class = void>
struct time_dependent : std::false_type {};
template <class T>
struct time_dependent<T, std::void_t<decltype(T::kTime)>> : std::integral_constant<bool, T::kTime> {};

// H(q, v) of the group's trajectory, from the owned components.  Right-hand
// sides with a split energy (N-body) compute shares on every lane and sum
// them with a butterfly; the others evaluate H on every lane redundantly.
template <class Rhs, int LPT, int NS>
__device__ __forceinline__ double group_energy(const Rhs& rhs, const double (&qh)[NS],
                                               const double (&vh)[NS], unsigned mask, int gbase,
                                               int r);

// Value of component l (compile-time) of a per-component quantity owned by
// lane (l % LPT) of the group, slot l / LPT.
template <int LPT, int NS>
__device__ __forceinline__ double owned_get(const double (&own)[NS], int l, unsigned mask, int gbase) {
  if constexpr (LPT == 1) return own[l];
  else return __shfl_sync(mask, own[l / LPT], gbase + l % LPT);
}

template <class Rhs, int LPT, int NS>
__device__ __forceinline__ double group_energy(const Rhs& rhs, const double (&qh)[NS],
                                               const double (&vh)[NS], unsigned mask, int gbase,
                                               int r) {
  constexpr int D = Rhs::D;
  double qf[D], vf[D];
#pragma unroll
  for (int l = 0; l < D; l++) {
    qf[l] = owned_get<LPT, NS>(qh, l, mask, gbase);
    vf[l] = owned_get<LPT, NS>(vh, l, mask, gbase);
  }
  if constexpr (split_energy<Rhs>::value && LPT > 1) {
    double e = rhs.H_part(r, LPT, qf, vf);
#pragma unroll
    for (int off = 1; off < LPT; off <<= 1) e = e + __shfl_xor_sync(mask, e, off);
    return e;
  } else {
    return rhs.H(qf, vf);
  }
}

// Select component (s*LPT + r) of a replicated per-component array, r runtime.
template <int LPT, int D>
__device__ __forceinline__ double select_own(const double (&arr)[D], int s, int r) {
  double x = arr[s * LPT];
#pragma unroll
  for (int rr = 1; rr < LPT; rr++)
    if (s * LPT + rr < D && r == rr) x = arr[s * LPT + rr];
  return x;
}

// MINB: minimum resident blocks per SM passed to the compiler's register
// allocator (__launch_bounds__); chosen per compiled tile from timings of the
// full Kepler ensemble on GB300 (1 = no constraint).
template <class Rhs, int LPT, int BLOCK, int MIX = 0, int MINB = 1>
__global__ void __launch_bounds__(BLOCK, MINB)
    irkgl_kernel(const __grid_constant__ KArgs a, const __grid_constant__ Coef cf) {
  constexpr int D = Rhs::D;
  constexpr int SPL = S / LPT;
  constexpr int NS = (D + LPT - 1) / LPT;  // owned component slots per lane
  constexpr int PAD = S + 1;               // padded smem row (bank spread)
  constexpr bool TIMED = time_dependent<Rhs>::value;
  // fixed-point mixing with the stage rows spread over the lanes: integer
  // coefficient rows in shared memory (fixed_row_rt)
  constexpr bool FIXED_RT = (MIX == 1) && (LPT > 1);

  __shared__ double s_eta[(LPT > 1 && !FIXED_RT) ? S * PAD : 1];
  __shared__ double s_W[(LPT > 1 && !FIXED_RT) ? S * PAD : 1];
  __shared__ unsigned long long s_fmag[FIXED_RT ? 2 * S * PAD : 1];
  __shared__ __align__(16) unsigned s_fbias[FIXED_RT ? 2 * S * 4 : 1];
  if constexpr (FIXED_RT) {
    for (int x = threadIdx.x; x < 2 * S * S; x += BLOCK) {
      const int tab = x / (S * S), k = x % (S * S);
      s_fmag[tab * S * PAD + (k / S) * PAD + (k % S)] = kFixedRows.mag[tab][k];
    }
    for (int x = threadIdx.x; x < 2 * S * 4; x += BLOCK) s_fbias[x] = kFixedRows.rbias[x / (S * 4)][x % (S * 4)];
    __syncthreads();
  } else if constexpr (LPT > 1) {
    for (int x = threadIdx.x; x < S * S; x += BLOCK) {
      s_eta[(x / S) * PAD + (x % S)] = cf.eta[x];
      s_W[(x / S) * PAD + (x % S)] = cf.W[x];
    }
    __syncthreads();
  }

  const int lane = threadIdx.x & 31;
  const int r = lane % LPT;      // rank inside the trajectory's lane group
  const int gbase = lane - r;    // first lane of the group
  const int i0 = r * SPL;        // first stage held by this lane
  const bool leader = (r == 0);

  // eta_(i0+t, j) and W_(i0+t, j): constant-bank operands when one lane holds
  // all stages (LPT == 1, indices known at compile time), padded shared
  // memory rows otherwise.
#define IRKGL_ETA(t, j) ((LPT == 1) ? cf.eta[(t) * S + (j)] : s_eta[(i0 + (t)) * PAD + (j)])
#define IRKGL_W(t, j) ((LPT == 1) ? cf.W[(t) * S + (j)] : s_W[(i0 + (t)) * PAD + (j)])

  double cc[SPL];
#pragma unroll
  for (int t = 0; t < SPL; t++) cc[t] = cf.c[i0 + t];
  unsigned neg_eta[SPL], neg_W[SPL];  // sign bits of the lane's rows (FIXED_RT)
#pragma unroll
  for (int t = 0; t < SPL; t++) {
    neg_eta[t] = FIXED_RT ? kFixedRows.negbits[0][i0 + t] : 0u;
    neg_W[t] = FIXED_RT ? kFixedRows.negbits[1][i0 + t] : 0u;
  }

  // Per-trajectory state.  Component l of q and v (hi and lo parts) and its
  // stopping-rule history live only on lane l % LPT of the group (slot
  // l / LPT); stage quantities live on the lane that holds the stage.
  Rhs rhs;
  rhs.load_params(a.params);
  double qh[NS], ql[NS], vh[NS], vl[NS];   // owned components: compensated pairs
  unsigned long long dmin[NS], dprev[NS];  // owned components: Eq. stopping history
  double R[SPL][D];           // own stages' R (Rprev between steps)
  double Q[SPL][D];           // own stages' values
  double cv[SPL][D];          // c_i v
  // The eight R_j of component l in offset fixed point with their shared
  // exponent: each lane converts its own stages after the group has agreed on
  // the largest exponent, then gathers the others' (FIXED_RT).
  auto gather_fixed = [&](int l, unsigned mask, unsigned long long (&rb)[S]) -> int {
    int e = 0;
#pragma unroll
    for (int t = 0; t < SPL; t++) e = max(e, biased_exp(R[t][l]));
#pragma unroll
    for (int off = 1; off < LPT; off <<= 1) e = max(e, __shfl_xor_sync(mask, e, off));
    unsigned long long own[SPL];
#pragma unroll
    for (int t = 0; t < SPL; t++) own[t] = to_fixed_offset(R[t][l], e);
#pragma unroll
    for (int j = 0; j < S; j++) rb[j] = __shfl_sync(mask, own[j % SPL], gbase + j / SPL);
    return e;
  };
  double h = 0.0, H0 = 0.0, invH0 = 0.0, dHmax = 0.0;
  double Hprev = 0.0, invHprev = 0.0;  // local-error monitor
  long long n = 0, N = 0, itot = 0;
  double th = 0.0, tl = 0.0;  // t_n (compensated), time-dependent g only
  int traj = -1, st = ST_OK;
  bool active = false, exhausted = false;

  // leaders of all groups in the warp
  unsigned leaders_all = 0;
#pragma unroll
  for (int g = 0; g < 32; g += LPT) leaders_all |= 1u << g;

  for (;;) {
    // ---------------- refill: groups without a trajectory grab the next one
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
          if (t < 0 || t >= a.batch) {
            t = -1;  // not a permutation entry: skip it
          }
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
            const size_t off = static_cast<size_t>(t) * D;
#pragma unroll
            for (int s = 0; s < NS; s++) {
              const int l = s * LPT + r;
              const bool in = l < D;
              qh[s] = in ? a.q_in[off + l] : 0.0;
              vh[s] = in ? a.v_in[off + l] : 0.0;
              ql[s] = (a.qlo_in && in) ? a.qlo_in[off + l] : 0.0;
              vl[s] = (a.vlo_in && in) ? a.vlo_in[off + l] : 0.0;
            }
            const size_t roff = static_cast<size_t>(t) * S * D;
#pragma unroll
            for (int tt = 0; tt < SPL; tt++)
#pragma unroll
              for (int l = 0; l < D; l++)
                R[tt][l] = a.rp_in ? a.rp_in[roff + (i0 + tt) * D + l] : 0.0;
            double hb[SPL];
#pragma unroll
            for (int tt = 0; tt < SPL; tt++) hb[tt] = h * cf.b[i0 + tt];
            rhs.set_step(hb);
            if constexpr (TIMED) {
              th = a.t_in ? a.t_in[t] : 0.0;
              tl = a.tlo_in ? a.tlo_in[t] : 0.0;
            }
          }
        }
      }
    }
    if (__all_sync(FULL, exhausted && !active)) break;

    // ---------------- reference energy H_0 of trajectories before their first
    // step.  The groups that need it differ from warp iteration to iteration,
    // so the shuffles inside run under the ballot of exactly those lanes.
    {
      const bool want = active && n == 0 && a.monitor > 0 && (!a.H0_io || a.h0_init || (H0 != H0 && N > 0));
      const unsigned h0mask = __ballot_sync(FULL, want);
      if (want) {
        H0 = group_energy<Rhs, LPT, NS>(rhs, qh, vh, h0mask, gbase, r);
        invH0 = 1.0 / H0;
        Hprev = H0;
        invHprev = invH0;
        if (a.H0_io && leader) a.H0_io[traj] = H0;
      }
    }

    // ---------------- one step for every group that still has steps to take
    const bool stepping = active && (n < N);
    const unsigned stepmask = __ballot_sync(FULL, stepping);
    if (stepping) {
      if constexpr (TIMED) {
        // stage times t_n + c_i h: h c_i rounded, then added to the hi part
        double tau[SPL];
#pragma unroll
        for (int t = 0; t < SPL; t++) tau[t] = __dadd_rn(th, __dmul_rn(h, cc[t]));
        rhs.set_time(tau);
      }
      // init (Eq. IRK_init2 in fused form): Q_i = q + h (c_i v + sum_k W_ik Rprev_k)
#pragma unroll
      for (int l = 0; l < D; l++) {
        const double vlv = owned_get<LPT, NS>(vh, l, stepmask, gbase);
        const double qlv = owned_get<LPT, NS>(qh, l, stepmask, gbase);
        if constexpr (FIXED_RT) {
          unsigned long long rb[S];
          const int emax = gather_fixed(l, stepmask, rb);
#pragma unroll
          for (int t = 0; t < SPL; t++) {
            double T = fixed_row_rt<IRKGL_W_SHIFT>(&s_fmag[S * PAD + (i0 + t) * PAD], neg_W[t],
                                                   &s_fbias[S * 4 + (i0 + t) * 4], rb, emax);
            if (emax == 0x7ff) T = __longlong_as_double(0x7ff8000000000000LL);
            Q[t][l] = fma(h, fma(cc[t], vlv, T), qlv);
          }
        } else if constexpr (MIX == 1) {
          double Rc[S];
#pragma unroll
          for (int j = 0; j < S; j++) Rc[j] = R[j][l];
          unsigned long long rb[S];
          bool nf;
          const int emax = fixed_column(Rc, rb, nf);
#pragma unroll
          for (int t = 0; t < SPL; t++) {
            double T = fixed_row<true>(t, rb, emax);
            if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
            Q[t][l] = fma(h, fma(cc[t], vlv, T), qlv);
          }
        } else {
          double acc[SPL];
#pragma unroll
          for (int t = 0; t < SPL; t++) {
            cv[t][l] = cc[t] * vlv;
            acc[t] = cv[t][l];
          }
#pragma unroll
          for (int j = 0; j < S; j++) {
            double Rj;
            if constexpr (LPT == 1) Rj = R[j][l];
            else Rj = __shfl_sync(stepmask, R[j % SPL][l], gbase + j / SPL);
#pragma unroll
            for (int t = 0; t < SPL; t++) acc[t] = fma(IRKGL_W(t, j), Rj, acc[t]);
          }
#pragma unroll
          for (int t = 0; t < SPL; t++) Q[t][l] = fma(h, acc[t], qlv);
        }
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
          // R_i = h b_i g(Q_i) (Eq. Gi)
#pragma unroll
          for (int t = 0; t < SPL; t++) rhs.stage_R(t, Q[t], R[t]);
          // Qn_i = q + h (c_i v + sum_j eta_ij R_j) (Eq. Qi2), Delta (Eq. Delta_n)
          bool cond_own = true, bad = false;
#pragma unroll
          for (int l = 0; l < D; l++) {
            const double qlv = owned_get<LPT, NS>(qh, l, sweepmask, gbase);
            double acc[SPL];
            if constexpr (FIXED_RT) {
              // c_i v + T in one rounding (the fixed-point tiles keep no c_i v array)
              const double vlv = owned_get<LPT, NS>(vh, l, sweepmask, gbase);
              unsigned long long rb[S];
              const int emax = gather_fixed(l, sweepmask, rb);
#pragma unroll
              for (int t = 0; t < SPL; t++) {
                double T = fixed_row_rt<IRKGL_ETA_SHIFT>(&s_fmag[(i0 + t) * PAD], neg_eta[t],
                                                         &s_fbias[(i0 + t) * 4], rb, emax);
                if (emax == 0x7ff) T = __longlong_as_double(0x7ff8000000000000LL);
                acc[t] = fma(cc[t], vlv, T);
              }
            } else if constexpr (MIX == 1) {
              double Rc[S];
#pragma unroll
              for (int j = 0; j < S; j++) Rc[j] = R[j][l];
              unsigned long long rb[S];
              bool nf;
              const int emax = fixed_column(Rc, rb, nf);
#pragma unroll
              for (int t = 0; t < SPL; t++) {
                double T = fixed_row<false>(t, rb, emax);
                if (nf) T = __longlong_as_double(0x7ff8000000000000LL);
                acc[t] = fma(cc[t], owned_get<LPT, NS>(vh, l, sweepmask, gbase), T);
              }
            } else {
#pragma unroll
              for (int t = 0; t < SPL; t++) acc[t] = cv[t][l];
#pragma unroll
              for (int j = 0; j < S; j++) {
                double Rj;
                if constexpr (LPT == 1) Rj = R[j][l];
                else Rj = __shfl_sync(sweepmask, R[j % SPL][l], gbase + j / SPL);
#pragma unroll
                for (int t = 0; t < SPL; t++) acc[t] = fma(IRKGL_ETA(t, j), Rj, acc[t]);
              }
            }
            unsigned long long dl = 0;
#pragma unroll
            for (int t = 0; t < SPL; t++) {
              const double qn = fma(h, acc[t], qlv);
              dl = umax64(dl, abs_bits(qn - Q[t][l]));
              Q[t][l] = qn;
            }
#pragma unroll
            for (int off = 1; off < LPT; off <<= 1)
              dl = umax64(dl, __shfl_xor_sync(sweepmask, dl, off));
            bad = bad || (dl >= INF_BITS);  // NaN/Inf patterns are >= INF_BITS
            // Eq. stopping on this component, by its owner (non-negative
            // doubles order like their bit patterns)
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
          // the group stops when every component's condition holds (the
          // shuffle must run on every lane: no short-circuit around it)
          int stop_i = cond_own ? 1 : 0;
#pragma unroll
          for (int off = 1; off < LPT; off <<= 1) stop_i &= __shfl_xor_sync(sweepmask, stop_i, off);
          const bool stop = stop_i != 0;
          if (bad) {
            st = ST_NONFINITE;
            conv = true;
          } else if (stop) {
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
        // update (Eq. qnvn2): sums over the stages.  Each lane sums its own
        // stages; the group then reduce-scatters the partial sums so that
        // each lane ends with the totals of the components it owns.  Column c
        // of the lane's partials holds components c, c + LPT, c + 2 LPT, ...
        // (zero past D).  At the level with offset off a lane holds the
        // columns that agree with its rank below bit off, keeps the half
        // whose bit off matches its own, sends the other half to lane
        // r ^ off and adds what it receives: own + partner, in the order of a
        // butterfly over xor offsets 1, 2, 4, so the totals are the ones every
        // lane of a full butterfly would form, with (LPT - 1) NS additions per
        // sum instead of D log2(LPT).
        double sx[LPT][NS], sy[LPT][NS];
#pragma unroll
        for (int c = 0; c < LPT; c++)
#pragma unroll
          for (int s = 0; s < NS; s++) {
            const int l = c + LPT * s;
            if (l < D) {
              double x = R[0][l], y = cc[0] * R[0][l];
#pragma unroll
              for (int t = 1; t < SPL; t++) {
                x = x + R[t][l];
                y = fma(cc[t], R[t][l], y);
              }
              sx[c][s] = x;
              sy[c][s] = y;
            } else {
              sx[c][s] = 0.0;
              sy[c][s] = 0.0;
            }
          }
#pragma unroll
        for (int lev = 0; (1 << lev) < LPT; lev++) {
          const int off = 1 << lev;
          const bool upper = (r & off) != 0;  // keep the odd member of each pair
#pragma unroll
          for (int u = 0; u < (LPT >> lev) / 2; u++)
#pragma unroll
            for (int s = 0; s < NS; s++) {
              const double kx = upper ? sx[2 * u + 1][s] : sx[2 * u][s];
              const double gx = upper ? sx[2 * u][s] : sx[2 * u + 1][s];
              const double ky = upper ? sy[2 * u + 1][s] : sy[2 * u][s];
              const double gy = upper ? sy[2 * u][s] : sy[2 * u + 1][s];
              sx[u][s] = kx + __shfl_xor_sync(okmask, gx, off);
              sy[u][s] = ky + __shfl_xor_sync(okmask, gy, off);
            }
        }
        // compensated update of the owned components l = s*LPT + r
#pragma unroll
        for (int s = 0; s < NS; s++) {
          if (s * LPT + r < D) {
            two_sum_add(vh[s], vl[s], sx[0][s]);
            // dq = h v_hi + (h v_lo - h sum c_i R_i)
            const double dq = fma(h, vh[s], fma(h, vl[s], -(h * sy[0][s])));
            two_sum_add(qh[s], ql[s], dq);
          }
        }
        if constexpr (TIMED) two_sum_add(th, tl, h);  // t_{n+1} = t_n + h
        n++;
        if (a.monitor > 0) {
          const bool mon = (n % a.monitor) == 0;  // differs between groups when monitor > 1
          const unsigned monmask = __ballot_sync(okmask, mon);
          if (mon) {
            const double Hn = group_energy<Rhs, LPT, NS>(rhs, qh, vh, monmask, gbase, r);
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

    // ---------------- finish: write outputs of completed/failed trajectories
    const bool fin = active && (n >= N || st != ST_OK);
    if (fin) {
      const size_t off = static_cast<size_t>(traj) * D;
#pragma unroll
      for (int s = 0; s < NS; s++) {
        const int l = s * LPT + r;
        if (l < D) {
          a.q_out[off + l] = qh[s];
          a.v_out[off + l] = vh[s];
          if (a.qlo_out) a.qlo_out[off + l] = ql[s];
          if (a.vlo_out) a.vlo_out[off + l] = vl[s];
        }
      }
      if (a.rp_out && st == ST_OK) {
        const size_t roff = static_cast<size_t>(traj) * S * D;
#pragma unroll
        for (int tt = 0; tt < SPL; tt++)
#pragma unroll
          for (int l = 0; l < D; l++) a.rp_out[roff + (i0 + tt) * D + l] = R[tt][l];
      }
      if (leader) {
        if constexpr (TIMED) {
          if (a.t_out) a.t_out[traj] = th;
          if (a.tlo_out) a.tlo_out[traj] = tl;
        }
        if (a.dH_max) a.dH_max[traj] = dHmax;
        if (a.iters_total) a.iters_total[traj] = itot;
        if (a.status) a.status[traj] = st;
        if (a.steps_done) a.steps_done[traj] = n;
      }
      active = false;
    }
  }
#undef IRKGL_ETA
#undef IRKGL_W
}

}  // namespace irkgl
