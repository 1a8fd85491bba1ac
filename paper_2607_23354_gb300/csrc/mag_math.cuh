// FP64 exp(x) for x <= 0 by Tang's table-driven method (P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989), used wherever the solver
// needs Z_jk = exp(-t d_jk) in FP64.
//
//   x = (64 k + j) ln2/64 + r,  |r| <= ln2/128  (N = 64k + j = round(64 x / ln 2),
//                                                r with the two-part ln2/64)
//   exp(x) = 2^k 2^(j/64) exp(r),  exp(r) - 1 = r + r^2/2 + ... + r^5/120
//   (Taylor, truncation below 3.4e-17 relative), 2^(j/64) = T_hi + T_lo.
//
// About 12 FP64 operations; at most about one unit in the last place from the
// exact value (the tests compare it with the host libm exp).  Results below
// 2^-1021 (x < -708) are returned as 0, NaN propagates.  The 128-double table
// (T_hi, T_lo pairs) must be staged by the caller, usually in shared memory:
// load_exp_table().
#pragma once

#include <cuda_runtime.h>

namespace mag {

#include "exp_table.inc"

__device__ __forceinline__ void load_exp_table(double* tab) {
  for (int i = threadIdx.x; i < 128; i += blockDim.x) tab[i] = kExpTable[i];
}

__device__ __forceinline__ double exp_neg(double x, const double* tab) {
  if (!(x > -708.0)) return x != x ? x : 0.0;
  const double shift = 0x1.8p52;
  double kd = fma(x, EXPT_INV_L, shift);
  const int N = __double2loint(kd);
  kd -= shift;
  double r = fma(-kd, EXPT_L1, x);
  r = fma(-kd, EXPT_L2, r);
  double a = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  a = fma(a, r, 1.0 / 6.0);
  a = fma(a, r, 0.5);
  a = fma(a, r, 1.0);
  const double p = a * r;
  const int j = N & 63, k = N >> 6;
  const double th = tab[2 * j], tl = tab[2 * j + 1];
  const double s = th + fma(th, p, tl);
  return s * __hiloint2double((k + 1023) << 20, 0);
}

}  // namespace mag
