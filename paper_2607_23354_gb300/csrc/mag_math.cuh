// FP64 exp(x) for x <= 0 by Tang's table-driven method (P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989), used wherever the solver
// needs Z_jk = exp(-t d_jk) in FP64.
//
//   x = (256 k + j) ln2/256 + r, |r| <= ln2/512 (N = 256k + j = round(256 x / ln 2),
//                                               r with the two-part ln2/256)
//   exp(x) = 2^k 2^(j/256) exp(r),  exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24
//   (Taylor, truncation below 4e-17 relative), 2^(j/256) = T_hi + T_lo.
//
// Ten FP64 operations; the range test and the final 2^k scaling are integer
// operations on the bit patterns (the FP64 pipe is the generator's limit).
// At most about one unit in the last place from the exact value (the tests
// compare it with the host libm exp).  Results below 2^-1021 (x below about
// -707.7) are returned as 0, NaN propagates.  The table (T_hi, T_lo pairs,
// then the FP32 pieces exp_neg_small uses) must be staged by the caller,
// usually in shared memory: EXPT_SMEM doubles filled by load_exp_table()
// (or the 2 * EXPT_SIZE doubles of load_exp_table_d() for exp_neg and
// exp_neg_small_d alone).
#pragma once

#include <cuda_runtime.h>

namespace mag {

#include "exp_table.inc"

// Doubles of the shared-memory table of load_exp_table.
constexpr int EXPT_SMEM = 4 * EXPT_SIZE;

__device__ __forceinline__ void load_exp_table_d(double* tab) {
  for (int i = threadIdx.x; i < 2 * EXPT_SIZE; i += blockDim.x) tab[i] = kExpTable[i];
}
__device__ __forceinline__ void load_exp_table(double* tab) {
  load_exp_table_d(tab);
  unsigned* x = reinterpret_cast<unsigned*>(tab + 2 * EXPT_SIZE);
  for (int i = threadIdx.x; i < 4 * EXPT_SIZE; i += blockDim.x) x[i] = kExpTableX[i];
}

__device__ __forceinline__ double exp_neg(double x, const double* tab) {
  // |x| >= 1024 (high word at least that of 1024.0), -inf and NaN leave on
  // the integer pipe: every such result is 0 (NaN propagates).  The test also
  // keeps N = round(256 x / ln 2) far inside the int32 low word read below,
  // which would wrap for x below about -5.8e6.
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40900000) return x != x ? x : 0.0;
  const double shift = 0x1.8p52;
  double kd = fma(x, EXPT_INV_L, shift);
  const int N = __double2loint(kd);        // round(x 256 / ln 2)
  if (N < -1021 * EXPT_SIZE) return 0.0;   // 2^k with k < -1021
  kd -= shift;
  double r = fma(-kd, EXPT_L1, x);
  r = fma(-kd, EXPT_L2, r);
  double a = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  a = fma(a, r, 0.5);
  a = fma(a, r, 1.0);
  const double p = a * r;
  static_assert(EXPT_SIZE == 256, "k = N >> 8 below");
  const int j = N & (EXPT_SIZE - 1), k = N >> 8;
  const double th = tab[2 * j], tl = tab[2 * j + 1];
  const double s = th + fma(th, p, tl);  // in [0.998, 2.003): 2^k s stays normal for k >= -1021
  return __hiloint2double(__double2hiint(s) + k * (1 << 20), __double2loint(s));
}

// exp(-a) for 0 <= a <= 64 (the caller bounds a): the reduction of exp_neg
// with N = round(256 a / ln 2) taken on the FP32 pipe from a's leading 24
// bits (truncation and the FP32 constant move a N below 23,700 by less than
// 0.005, so |r| <= 0.5042 ln2/256 and the first omitted series term stays
// below 4.1e-17 relative) and N widened to FP64 on the integer pipe: eight
// FP64 operations against exp_neg's ten, same accuracy.  Table of
// load_exp_table_d.
__device__ __forceinline__ double exp_neg_small_d(double a, const double* tab) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const float af = (b >> 52) < 1023 - 126 ? 0.0f : __uint_as_float((unsigned)(b >> 29) - ((1023u - 127u) << 23));
  // af 256/ln2 + 1.5 2^23, rounded once: the low bits hold N
  const float shifted = fmaf(af, 0x1.715476p+8f, 12582912.0f);
  const int N = __float_as_int(shifted) - 0x4B400000;
  const unsigned nb = __float_as_uint(shifted - 12582912.0f);  // N as an FP32, exact
  const double kd =
      nb == 0u ? 0.0
               : __longlong_as_double((long long)(((unsigned long long)((nb >> 23) + (1023u - 127u)) << 52) |
                                                  ((unsigned long long)(nb & 0x7fffffu) << 29)));
  // r = N ln2/256 - a with the two-part constant (kd EXPT_L1 is exact)
  double r = fma(kd, EXPT_L1, -a);
  r = fma(kd, EXPT_L2, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double p = q * r;
  // exp(-a) = 2^(-N/256) exp(r): -N = 256 k + j
  const int M = -N;
  const int j = M & (EXPT_SIZE - 1), k = M >> 8;
  const double th = tab[2 * j], tl = tab[2 * j + 1];
  const double s = th + fma(th, p, tl);
  return __hiloint2double(__double2hiint(s) + k * (1 << 20), __double2loint(s));
}

__device__ __forceinline__ double f32_to_f64_nonneg(float v);

// v (any FP32 value) to FP64 on the integer pipe; FP32 subnormals give 0.
__device__ __forceinline__ double f32_to_f64(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 255u) return (double)v;  // inf, NaN
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// exp(-a) for 0 <= a <= 64 in four FP64 operations (exp_neg_small), and
// exp(-t d) in four as well, the product t d included (exp_neg_td).
// N = round(256 a / ln 2) as in exp_neg_small_d and r = N ln2/256 - a =
// r1 + rc, r1 = N L1 - a rounded
// once (exact for exp_neg_small, whose a is a double; exp_neg_td forms N L1
// exactly on the integer pipe and r1 = fma(-t, d, N L1), so t d is never
// rounded), rc = N L2 in float-float.  exp(-a) = 2^(-N/256) exp(r) and
//   T exp(r) = T_hi + T_hi r1 + (T_hi (u + rc) + T_lo) + O(2^-100),
//   u = exp(r) - 1 - r = r^2/2 + r^3/6 + r^4/24 + r^5/120 + O(9e-21):
// the last bracket, below 1e-6 T_hi, needs only a relative accuracy of
// 2^-40 and is formed in float-float on the FP32 pipe from r split into
// FP32 parts (rh + rl, |rl| <= ulp(rh)) -- r^2 and r^3 from exact products
// (FMA), r^4 and r^5 in plain FP32 -- then widened to FP64 on the integer
// pipe.  The FP64 work after r1 is the sum of the two widened parts, one
// FMA and the final sum, whose rounding dominates: within about 0.51 units
// in the last place (compared with the host libm in the tests).
__device__ __forceinline__ double exp_neg_core(int N, float kf, double r1, const double* tab) {
  const float rch = kf * EXPT_L2H;
  const float rcl = fmaf(kf, EXPT_L2L, fmaf(kf, EXPT_L2H, -rch));
  // r1 = rh0 + rl0 on the integer pipe (leading 24 bits; the next 23 bits);
  // |r1| below 2^-103 counts as 0 here (it still enters through T_hi r1)
  const unsigned long long rb = (unsigned long long)__double_as_longlong(r1);
  const unsigned re = (unsigned)(rb >> 52) & 0x7ffu;
  const unsigned rs = (unsigned)(rb >> 32) & 0x80000000u;
  float rh0 = 0.0f, rl0 = 0.0f;
  if (re >= 920u) {
    rh0 = __uint_as_float(rs | ((re - (1023u - 127u)) << 23) | ((unsigned)(rb >> 29) & 0x7fffffu));
    const float f = __uint_as_float((((unsigned)rb & 0x1fffffffu) >> 6) | 0x3f800000u) - 1.0f;
    rl0 = __uint_as_float(__float_as_uint(f * __uint_as_float((re - 919u) << 23)) | rs);
  }
  // r = rh + rl: rc folded in, renormalized (|rl0 + rch| < |rh0| or rh0 = 0)
  const float t1 = rl0 + rch;
  const float rh = rh0 + t1;
  const float rl = (rh0 - rh) + t1;
  // u = uh + ul
  const float p = rh * rh;
  const float pe = fmaf(2.0f * rh, rl, fmaf(rh, rh, -p));  // r^2 = p + pe
  const float c = p * rh;
  const float ce = fmaf(pe, rh, fmaf(p, rl, fmaf(p, rh, -c)));  // r^3 = c + ce
  const float d = c * EXPT_S6H;
  const float de = fmaf(c, EXPT_S6L, fmaf(ce, EXPT_S6H, fmaf(c, EXPT_S6H, -d)));  // r^3/6 = d + de
  const float q = (p * p) * fmaf(rh, 1.0f / 120.0f, 1.0f / 24.0f);
  const float hp = 0.5f * p;  // |r^3/6| < |r^2/2|: the sum's error is exact below
  const float uh = hp + d;
  const float ul = (((hp - uh) + d) + 0.5f * pe) + (de + q);
  // g = u + rc (rc >= 0, either may be the larger)
  const float gh = uh + rch;
  const float bv = gh - uh;
  const float gl = ((uh - (gh - bv)) + (rch - bv)) + (ul + rcl);
  // exp(-a) = 2^(-N/256) exp(r): -N = 256 k + j
  const int M = -N;
  const int j = M & (EXPT_SIZE - 1), k = M >> 8;
  // one 16-byte entry: T_hi, TL = T_hi - TH (TH: T_hi's leading 24 bits), T_lo
  const uint4 T = reinterpret_cast<const uint4*>(tab + 2 * EXPT_SIZE)[j];
  const double th = __hiloint2double((int)T.y, (int)T.x);
  const float thh = __uint_as_float(((T.y << 3) | (T.x >> 29)) - ((1023u - 127u) << 23));
  const float thl = __uint_as_float(T.z), tlf = __uint_as_float(T.w);
  const float vh = thh * gh;  // >= 0
  const float vl = fmaf(thh, gl, fmaf(thl, gh, fmaf(thh, gh, -vh))) + tlf;
  const double w = f32_to_f64_nonneg(vh) + f32_to_f64(vl);
  const double s = th + fma(th, r1, w);
  return __hiloint2double(__double2hiint(s) + k * (1 << 20), __double2loint(s));
}

// N = round(256 af / ln 2) for 0 <= af < 64 (FP32) and N as an FP32.
__device__ __forceinline__ int exp_reduce_n(float af, float* kf) {
  const float shifted = fmaf(af, 0x1.715476p+8f, 12582912.0f);
  *kf = shifted - 12582912.0f;  // N as an FP32, exact
  return __float_as_int(shifted) - 0x4B400000;
}

__device__ __forceinline__ double exp_neg_small(double a, const double* tab) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const float af = (b >> 52) < 1023 - 126 ? 0.0f : __uint_as_float((unsigned)(b >> 29) - ((1023u - 127u) << 23));
  float kf;
  const int N = exp_reduce_n(af, &kf);
  const unsigned nb = __float_as_uint(kf);
  const double kd =
      nb == 0u ? 0.0
               : __longlong_as_double((long long)(((unsigned long long)((nb >> 23) + (1023u - 127u)) << 52) |
                                                  ((unsigned long long)(nb & 0x7fffffu) << 29)));
  return exp_neg_core(N, kf, fma(kd, EXPT_L1, -a), tab);
}

__device__ __forceinline__ float f64_to_f32_nonneg(double x);

// N L1 for 0 <= N < 2^15 exactly, on the integer pipe (L1 = L1M 2^L1E with
// a 32-bit L1M: the product has at most 47 bits).
__device__ __forceinline__ double nl1_exact(int N) {
  if (N <= 0) return 0.0;
  const unsigned long long pr = (unsigned long long)N * EXPT_L1M;
  const int top = 63 - __clzll((long long)pr);  // leading bit
  const unsigned long long mant = pr << (52 - top);
  return __longlong_as_double((long long)(((unsigned long long)(top + EXPT_L1E + 1022) << 52) + mant));
}

// exp(-t d) for t > 0, d >= 0 (NaN propagates): N from the FP32 product of
// t and d rounded on the integer pipe (within 2^-21 relative of t d, moving
// N by less than 0.006), then the reduction without rounding t d; for t d
// of about 63.5 or more the product is formed and exp_neg takes it.
__device__ __forceinline__ double exp_neg_td(double t, double d, const double* tab) {
  const float af = f64_to_f32_nonneg(t) * f64_to_f32_nonneg(d);
  if (!(af < 63.5f)) {
    const double a = t * d;
    return (unsigned long long)__double_as_longlong(a) < 0x4050000000000000ull ? exp_neg_small(a, tab)
                                                                               : exp_neg(-a, tab);
  }
  float kf;
  const int N = exp_reduce_n(af, &kf);
  return exp_neg_core(N, kf, fma(-t, d, nl1_exact(N)), tab);
}

// exp(x) - 1 for x <= 0 without the cancellation of exp(x) - 1 near 0: for
// x >= -1/4 the Taylor series x + x^2/2! + ... + x^14/14! in Horner form
// (the first omitted term is below 2^-63 |x|), else exp_neg(x) - 1, whose
// result lies in [-1, -0.22] so the subtraction costs at most two units in
// the last place.
__device__ __forceinline__ double expm1_neg(double x, const double* tab) {
  if (x < -0.25) return exp_neg(x, tab) - 1.0;
  double p = 1.0 / 87178291200.0;  // 1/14!
  p = fma(p, x, 1.0 / 6227020800.0);
  p = fma(p, x, 1.0 / 479001600.0);
  p = fma(p, x, 1.0 / 39916800.0);
  p = fma(p, x, 1.0 / 3628800.0);
  p = fma(p, x, 1.0 / 362880.0);
  p = fma(p, x, 1.0 / 40320.0);
  p = fma(p, x, 1.0 / 5040.0);
  p = fma(p, x, 1.0 / 720.0);
  p = fma(p, x, 1.0 / 120.0);
  p = fma(p, x, 1.0 / 24.0);
  p = fma(p, x, 1.0 / 6.0);
  p = fma(p, x, 0.5);
  return fma(p * x, x, x);
}

// Off-diagonal entry of the matrix a solve factors, from the FP64 distance
// dd (kind: MatKind of mag_internal.cuh): exp(-t d) (Eq. weighting);
// 1 - t d (the scale-zero system, t = 1/c); 1 + kc expm1(-t d) with
// kc = 1/(c t) (the deflated small-t system).  The diagonal is 1 for all.
__device__ __forceinline__ double mat_entry(int kind, double t, double kc, double dd, const double* tab) {
  if (kind == 1) return fma(-t, dd, 1.0);
  if (kind == 2) return fma(expm1_neg(-t * dd, tab), kc, 1.0);
  return exp_neg_td(t, dd, tab);
}

// exp(-a) for a > kTinyArg = 46 (mag_internal.cuh; results below
// e^-46 < 2^-66) in FP32, a = t d formed from FP32 roundings of t and d
// (exp_neg_tiny_td, no FP64 operation: GB300's FP64 pipe is the generator's
// limit): the CUDA expf of the argument, relative error below 2e-5
// (three roundings of 2^-24 in a <= 87, 1.6e-5, plus the expf error), and 0
// for a > 87 (below FP32's normal range).  In a row of Z that holds the unit
// diagonal these entries change the FP64 row sum by at most
// n (2e-5 e^-46 + 2^-126) < n 2^-81: for n <= 2^20 far below the 2^-53 of
// one FP64 rounding of that sum, so residuals and refinement see the same
// matrix as with FP64 exponentials everywhere.
__device__ __forceinline__ float exp_neg_tiny_f(float a) { return a > 87.0f ? 0.0f : expf(-a); }

// x in [0, 2^128) to FP32, round to nearest even, on the integer pipe; values
// below 2^-126 (FP32 subnormals) become 0.  Used for the FP32 copy of a Z
// entry, whose role is the factor's input.
__device__ __forceinline__ float f64_to_f32_nonneg(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if ((b >> 52) < 1023 - 126) return 0.0f;
  b += 0x0FFFFFFFull + ((b >> 29) & 1ull);  // round the 29 dropped bits, ties to even
  return __uint_as_float((unsigned)(b >> 29) - ((1023u - 127u) << 23));
}

// v >= 0 (an FP32 value, e.g. an FP32 entry of Z) to FP64 on the integer
// pipe: exponent rebiased, significand shifted; 0 and FP32 subnormals give 0.
__device__ __forceinline__ double f32_to_f64_nonneg(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned e = b >> 23;
  if (e == 0u) return 0.0;
  if (e == 255u) return (double)v;  // inf, NaN
  return __longlong_as_double(
      (long long)(((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// exp(-t d) below e^-46 (exp_neg_tiny_f) from FP64 d >= 0 and tf = t rounded
// to FP32: d rounded on the integer pipe, the product and the exponential on
// the FP32 pipe.  Returns the FP32 entry; its FP64 copy is
// f32_to_f64_nonneg of it.  d of 2^126 or more (or NaN) takes t d in FP64.
__device__ __forceinline__ float exp_neg_tiny_td(float tf, double t, double d);
// The same from d^2 (the square root on the FP32 pipe as well).
__device__ __forceinline__ float exp_neg_tiny_td2(float tf, double t, double d2);

// sqrt(v) for v >= 0 by Markstein's method (P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990): y ~ 1/sqrt(v) from the FP32 reciprocal square root of
// v's leading bits (|y sqrt(v) - 1| < 2^-20), s = v y, then two corrections
// s += (y/2)(v - s^2) whose residual is exact with an FMA; each multiplies
// the relative error by about that of y, leaving < 2^-60 before the final
// rounding (within one unit in the last place).  Five FP64 operations; the
// seed, its widening to FP64 and y/2 run on the FP32 and integer pipes.  Outside
// [2^-120, 2^120] (and for 0, inf, NaN) it defers to the library sqrt.
__device__ __forceinline__ double sqrt_pos(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned e = (unsigned)(b >> 52);
  if (e < 1023 - 120 || e > 1023 + 120) return sqrt(v);
  // v's top 24 significand bits as an FP32 (truncated: a seed needs no rounding)
  const float vf = __uint_as_float((unsigned)(b >> 29) - ((1023u - 127u) << 23));
  const float yf = rsqrtf(vf);
  const unsigned yb = __float_as_uint(yf);
  // FP32 -> FP64 of a normal positive float on the integer pipe
  const unsigned long long ywide =
      ((unsigned long long)((yb >> 23) + (1023u - 127u)) << 52) | ((unsigned long long)(yb & 0x7fffffu) << 29);
  const double y = __longlong_as_double((long long)ywide);
  const double h = __longlong_as_double((long long)(ywide - (1ull << 52)));  // y / 2 (y normal), integer pipe
  double s = v * y;
  double r = fma(-s, s, v);
  s = fma(h, r, s);
  r = fma(-s, s, v);
  return fma(h, r, s);
}

__device__ __forceinline__ float exp_neg_tiny_td(float tf, double t, double d) {
  if ((unsigned long long)__double_as_longlong(d) >= 0x47D0000000000000ull)  // 2^126, inf, NaN
    return d != d ? (float)d : exp_neg_tiny_f((float)fmin(t * d, 100.0));
  return exp_neg_tiny_f(tf * f64_to_f32_nonneg(d));
}
__device__ __forceinline__ float exp_neg_tiny_td2(float tf, double t, double d2) {
  if ((unsigned long long)__double_as_longlong(d2) >= 0x47D0000000000000ull)
    return d2 != d2 ? (float)d2 : exp_neg_tiny_f((float)fmin(t * sqrt(d2), 100.0));
  return exp_neg_tiny_f(tf * sqrtf(f64_to_f32_nonneg(d2)));
}

// Exact d^2 from quantized coordinates (quantize_points in the host
// code): every coordinate is an integer multiple of 2^-e relative to its
// dimension's minimum (x = lo_l + q 2^-e, |x - that| <= 2^-e), so a pair's
// d^2 = 2^-2e sum_l (q_il - q_jl)^2 is an exact integer sum, here in 128
// bits on the integer pipe: |D| < 2^(2L) in two L-bit limbs, three 64-bit
// sums (lo lo, hi lo, hi hi) of 32 x 32 -> 64-bit multiply-adds, combined
// and rounded to FP64 once.  The quantization moves d by at most
// 2 sqrt(m) 2^-e, no more than the FP64 differences' rounding (2^-52 d)
// once d >= sqrt(m) 2^(53-e); closer pairs (d^2 below tau2) take the FP64
// differences from the points instead.  Replaces 2m FP64 operations per
// pair; the square root stays FP64 (sqrt_pos).
struct QuantParams {
  int L;        // limb bits
  int e;        // coordinate scale exponent
  double tau2;  // d^2 below which a pair takes the FP64 differences
};

// 2^-2e (C 2^2L + Bx 2^(L+1) + A) rounded to nearest FP64 (A, Bx, C < 2^63)
__device__ __forceinline__ double q128_to_f64(unsigned long long A, unsigned long long Bx, unsigned long long C,
                                              int L, int e) {
  unsigned long long ql = A, qh = 0;
  const unsigned long long bl = Bx << (L + 1), bh = Bx >> (63 - L);
  ql += bl;
  qh += bh + (ql < bl ? 1ull : 0ull);
  const unsigned long long cl = C << (2 * L), ch = C >> (64 - 2 * L);
  ql += cl;
  qh += ch + (ql < cl ? 1ull : 0ull);
  if ((qh | ql) == 0ull) return 0.0;
  const int lz = qh ? __clzll((long long)qh) : 64 + __clzll((long long)ql);
  unsigned long long nh, nl;
  if (lz == 0) {
    nh = qh;
    nl = ql;
  } else if (lz < 64) {
    nh = (qh << lz) | (ql >> (64 - lz));
    nl = ql << lz;
  } else {
    nh = ql << (lz - 64);
    nl = 0ull;
  }
  // the top 53 of the 128 bits, rounded to nearest even on the other 75
  unsigned long long mant = nh >> 11;
  const unsigned long long rest = nh & 0x7ffull;
  const bool up = (rest >> 10) && ((rest & 0x3ffull) || nl || (mant & 1ull));
  mant += up ? 1ull : 0ull;
  // leading bit 127 - lz of the integer, times 2^-2e; mant carries the
  // implicit bit (a rounding carry to 2^53 moves the exponent by one)
  const long long ex = 127 - lz - 2 * e;
  return __longlong_as_double((long long)(((unsigned long long)(ex + 1022) << 52) + mant));
}

// d^2 of rows (x) and columns (y) given as quantized coordinates, m terms
__device__ __forceinline__ void q_accumulate(long long a, long long b, unsigned long long mask, int L,
                                             unsigned long long& A, unsigned long long& Bx,
                                             unsigned long long& C) {
  const long long dv = a - b;
  const unsigned long long ad = dv < 0 ? 0ull - (unsigned long long)dv : (unsigned long long)dv;
  const unsigned lo = (unsigned)(ad & mask), hi = (unsigned)(ad >> L);
  A += (unsigned long long)lo * lo;
  Bx += (unsigned long long)hi * lo;
  C += (unsigned long long)hi * hi;
}


}  // namespace mag
