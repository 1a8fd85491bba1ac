// K4: FP64 residual r = b - Z w of iterative refinement, with Z regenerated
// on the fly from the points (matrix free: nothing of size n^2 is read), and
// the norms the stopping test needs: ||r||inf, ||Z||inf (max row sum, Z > 0),
// ||w||inf.  K5: the FP64 solution update.  K6: Mag = 1^T w (compensated),
// min_j w_j and the sign information.  K7: the fused gradient reductions.
//
// Accuracy: every pair is d^2 = sum_l (x_jl - x_kl)^2 in FP64, Z_jk =
// exp(-t sqrt(d^2)) in FP64, and each row sum is accumulated with Kahan
// compensation per thread and then combined across column chunks with
// Neumaier's rule, so the residual is good to a few units of FP64 rounding
// relative to ||Z||inf ||w||inf (the refinement target is 1e-14).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/magnitude.h"
#include "mag_internal.cuh"
#include "mag_math.cuh"

namespace mag {

namespace {

constexpr int RES_THREADS = 128;

__device__ inline void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// Row j = blockIdx.x*128 + threadIdx.x, columns of chunk blockIdx.y.  Row point
// in registers when m <= MR (MR > 0), else read through the read-only cache.
template <int MR>
__global__ void __launch_bounds__(RES_THREADS) k_resid_mf(const double* __restrict__ X, int64_t n,
                                                          int m, double t,
                                                          const double* __restrict__ w,
                                                          double* __restrict__ part, int chunks,
                                                          int64_t np, int ct, int kind, double kc) {
  extern __shared__ double sm[];
  double* xc = sm;            // [ct][m]
  double* wc = sm + ct * m;   // [ct]
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  load_exp_table(exptab);
  const int64_t j = (int64_t)blockIdx.x * RES_THREADS + threadIdx.x;
  const int64_t ntiles = (n + ct - 1) / ct;
  const int64_t per = (ntiles + chunks - 1) / chunks;
  const int64_t c0 = blockIdx.y * per * ct;
  const int64_t c1 = min(n, (blockIdx.y + 1) * per * ct);
  const bool live = j < n;
  double xr[MR > 0 ? MR : 1];
  if (MR > 0) {
#pragma unroll
    for (int l = 0; l < (MR > 0 ? MR : 1); ++l) xr[l] = (live && l < m) ? X[j * m + l] : 0.0;
  }
  double s = 0.0, c = 0.0, zs = 0.0;
  for (int64_t k0 = c0; k0 < c1; k0 += ct) {
    const int cnt = (int)min((int64_t)ct, c1 - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * m; e += RES_THREADS) xc[e] = X[k0 * m + e];
    for (int e = threadIdx.x; e < cnt; e += RES_THREADS) wc[e] = w[k0 + e];
    __syncthreads();
    if (!live) continue;
    for (int q = 0; q < cnt; ++q) {
      const double* xk = xc + q * m;
      double d2 = 0.0;
      if (MR > 0) {
#pragma unroll
        for (int l = 0; l < (MR > 0 ? MR : 1); ++l) {
          if (l < m) {
            const double diff = xr[l] - xk[l];
            d2 = fma(diff, diff, d2);
          }
        }
      } else {
        for (int l = 0; l < m; ++l) {
          const double diff = __ldg(X + j * m + l) - xk[l];
          d2 = fma(diff, diff, d2);
        }
      }
      const double dd = sqrt_pos(d2);
      const double z = mat_entry(kind, t, kc, dd, exptab);  // dd = 0 (k = j): the unit diagonal
      zs += z;
      // Kahan step for s += z * w_k
      const double y = fma(z, wc[q], -c);
      const double tt = s + y;
      c = (tt - s) - y;
      s = tt;
    }
  }
  if (live) {
    part[((int64_t)0 * chunks + blockIdx.y) * np + j] = s;
    part[((int64_t)1 * chunks + blockIdx.y) * np + j] = -c;
    part[((int64_t)2 * chunks + blockIdx.y) * np + j] = zs;
  }
}

// Stored-tile residual: Zw from the FP64 lower tiles (Z_IJ for I >= J; the
// diagonal tiles are stored in full).  CTA (t, J) works on column block J:
// t = 0 takes the diagonal tile; t >= 1 the strip of RS_STRIP tiles (I, J),
// I in [J+1+(t-1)S, J+1+tS).  For each tile it stores the row contributions
// Z_IJ w_J (rows of block I) as partial P[I][J][r]; over the strip it
// accumulates the transposed contributions Z_IJ^T w_I (rows of block J) in
// registers and stores their sum once as P[J][J+t][c], so the cross-lane
// reduction of the column sums is paid once per strip.  Every product is one
// FP64 FMA; within a row the 128 terms are a short tree, across tiles
// k_resid_stored_finish adds a row's partials with Neumaier compensation.
// Thread layout (256 threads): lane = 8 * rs + cg; column group cg owns the
// 16 columns 16k + 2cg, 16k + 2cg + 1 (k < 8); warp wp and row slot rs cover
// tile rows 16 wp + 4 i + rs (i < 4).  Each load instruction reads four
// 128-byte row segments.
constexpr int RS_STRIP = 8;

__global__ void __launch_bounds__(256) k_resid_stored(const double* __restrict__ Zd, int64_t n, int64_t N,
                                                      const double* __restrict__ w,
                                                      double* __restrict__ P) {
  __shared__ double colp[8][TILE];
  const int64_t J = blockIdx.y;
  const int64_t t = blockIdx.x;
  const int64_t nstrips = (N - 1 - J + RS_STRIP - 1) / RS_STRIP;
  if (t > nstrips) return;  // uniform
  const int tid = threadIdx.x, wp = tid >> 5, l = tid & 31, cg = l & 7, rs = l >> 3;
  double wc[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t col = J * TILE + 16 * k + 2 * cg;
    wc[2 * k] = col < n ? w[col] : 0.0;
    wc[2 * k + 1] = col + 1 < n ? w[col + 1] : 0.0;
  }
  const int64_t I0 = t == 0 ? J : J + 1 + (t - 1) * RS_STRIP;
  const int64_t I1 = t == 0 ? J + 1 : (I0 + RS_STRIP < N ? I0 + RS_STRIP : N);
  double cs[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) cs[k] = 0.0;
  for (int64_t I = I0; I < I1; ++I) {
    const double* tile = Zd + tri_index(I, J) * TILE_ELEMS;
#pragma unroll 2
    for (int i = 0; i < 4; ++i) {
      const int r = wp * 16 + 4 * i + rs;
      const int64_t row = I * TILE + r;
      const double wr = row < n ? w[row] : 0.0;
      const double* rp = tile + r * TILE + 2 * cg;
      double sr = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double2 z = *reinterpret_cast<const double2*>(rp + 16 * k);
        sr = fma(z.x, wc[2 * k], sr);
        sr = fma(z.y, wc[2 * k + 1], sr);
        cs[2 * k] = fma(z.x, wr, cs[2 * k]);
        cs[2 * k + 1] = fma(z.y, wr, cs[2 * k + 1]);
      }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1);
      sr += __shfl_xor_sync(0xffffffffu, sr, 2);
      sr += __shfl_xor_sync(0xffffffffu, sr, 4);
      if (cg == 0) P[(I * N + J) * TILE + r] = sr;
    }
  }
  if (t == 0) return;  // uniform: the diagonal tile's rows already cover both triangles
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    cs[k] += __shfl_xor_sync(0xffffffffu, cs[k], 8);
    cs[k] += __shfl_xor_sync(0xffffffffu, cs[k], 16);
  }
  if (rs == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      colp[wp][16 * k + 2 * cg] = cs[2 * k];
      colp[wp][16 * k + 2 * cg + 1] = cs[2 * k + 1];
    }
  }
  __syncthreads();
  if (tid < TILE) {
    double sc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sc += colp[k][tid];
    P[(J * N + J + t) * TILE + tid] = sc;
  }
}

// The same product Z w from the same FP64 tiles in float-float arithmetic on
// the FP32 pipe, for the inner iterations of GMRES-IR (GB300 runs FP64 at
// 1/64 of FP32, and k_resid_stored is bound by its FP64 FMAs).  Each entry
// z in [0, 1] (Z = exp(-t D)) is split on the integer pipe into z_h (its
// leading 24 bits) and z_l (the next 23 of the 29 remaining), w into
// w_h + w_l (k_split_ff); a product is z_h w_h exactly (FMA) plus
// z_h w_l + z_l w_h, and the sums are float-float (Knuth's TwoSum on the
// leading parts, the trailing parts added plainly).  Dropping z_l w_l, the
// last 6 bits of z and the rounding of the trailing parts leave a relative
// error of a few units of 2^-46 of sum_k |z_jk| |w_k| -- far below what a
// preconditioned inner iteration resolves, not the FP64 residual (the outer
// steps of GMRES-IR keep k_resid_stored).  Layout, partials and the finish
// (k_resid_stored_finish) as in k_resid_stored.
struct ffp {
  float h, l;
};

__device__ __forceinline__ void ff_split_unit(double z, float* zh, float* zl) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(z);
  const unsigned e = (unsigned)(b >> 52);  // z >= 0: the biased exponent
  const float h = __uint_as_float((unsigned)(b >> 29) - ((1023u - 127u) << 23));
  // the 29 bits below z_h: (m >> 6) 2^-23 exactly, times 2^(e - 1046)
  const unsigned m = (unsigned)b & 0x1FFFFFFFu;
  const float f = __uint_as_float((m >> 6) | 0x3F800000u) - 1.0f;
  const int se = (int)e - (1046 - 127);
  *zh = e >= 1023u - 126u ? h : 0.0f;  // below 2^-126: 0
  *zl = se > 0 ? f * __uint_as_float((unsigned)se << 23) : 0.0f;
}

// s += z w in float-float
__device__ __forceinline__ void ff_fma(ffp& s, float zh, float zl, float wh, float wl) {
  const float ph = zh * wh;
  float pl = fmaf(zh, wh, -ph);
  pl = fmaf(zh, wl, pl);
  pl = fmaf(zl, wh, pl);
  const float t = s.h + ph;
  const float bp = t - s.h;
  const float e = (s.h - (t - bp)) + (ph - bp);
  s.l += pl + e;
  s.h = t;
}

__device__ __forceinline__ void ff_add(ffp& s, const ffp& o) {
  const float t = s.h + o.h;
  const float bp = t - s.h;
  const float e = (s.h - (t - bp)) + (o.h - bp);
  s.l += o.l + e;
  s.h = t;
}

__device__ __forceinline__ ffp ff_shfl_xor(const ffp& v, int o) {
  return ffp{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}

__global__ void k_split_ff(const double* __restrict__ w, int64_t n, int64_t np, float2* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const double v = j < n ? w[j] : 0.0;
  const float h = __double2float_rn(v);
  out[j] = make_float2(h, __double2float_rn(v - (double)h));
}

__global__ void __launch_bounds__(256) k_resid_stored_ff(const double* __restrict__ Zd, int64_t n, int64_t N,
                                                         const float2* __restrict__ wf, double* __restrict__ P) {
  __shared__ ffp colp[8][TILE];
  const int64_t J = blockIdx.y;
  const int64_t t = blockIdx.x;
  const int64_t nstrips = (N - 1 - J + RS_STRIP - 1) / RS_STRIP;
  if (t > nstrips) return;  // uniform
  const int tid = threadIdx.x, wp = tid >> 5, l = tid & 31, cg = l & 7, rs = l >> 3;
  float2 wc[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t col = J * TILE + 16 * k + 2 * cg;
    wc[2 * k] = wf[col];  // wf is zero-padded to a whole tile row
    wc[2 * k + 1] = wf[col + 1];
  }
  const int64_t I0 = t == 0 ? J : J + 1 + (t - 1) * RS_STRIP;
  const int64_t I1 = t == 0 ? J + 1 : (I0 + RS_STRIP < N ? I0 + RS_STRIP : N);
  ffp cs[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) cs[k] = ffp{0.0f, 0.0f};
  for (int64_t I = I0; I < I1; ++I) {
    const double* tile = Zd + tri_index(I, J) * TILE_ELEMS;
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      const int r = wp * 16 + 4 * i + rs;
      const float2 wr = wf[I * TILE + r];
      const double* rp = tile + r * TILE + 2 * cg;
      ffp sr{0.0f, 0.0f};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double2 z = *reinterpret_cast<const double2*>(rp + 16 * k);
        float zh0, zl0, zh1, zl1;
        ff_split_unit(z.x, &zh0, &zl0);
        ff_split_unit(z.y, &zh1, &zl1);
        ff_fma(sr, zh0, zl0, wc[2 * k].x, wc[2 * k].y);
        ff_fma(sr, zh1, zl1, wc[2 * k + 1].x, wc[2 * k + 1].y);
        ff_fma(cs[2 * k], zh0, zl0, wr.x, wr.y);
        ff_fma(cs[2 * k + 1], zh1, zl1, wr.x, wr.y);
      }
      ff_add(sr, ff_shfl_xor(sr, 1));
      ff_add(sr, ff_shfl_xor(sr, 2));
      ff_add(sr, ff_shfl_xor(sr, 4));
      if (cg == 0) P[(I * N + J) * TILE + r] = (double)sr.h + (double)sr.l;
    }
  }
  if (t == 0) return;  // uniform: the diagonal tile's rows already cover both triangles
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    ff_add(cs[k], ff_shfl_xor(cs[k], 8));
    ff_add(cs[k], ff_shfl_xor(cs[k], 16));
  }
  if (rs == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      colp[wp][16 * k + 2 * cg] = cs[2 * k];
      colp[wp][16 * k + 2 * cg + 1] = cs[2 * k + 1];
    }
  }
  __syncthreads();
  if (tid < TILE) {
    ffp sc = colp[0][tid];
#pragma unroll
    for (int k = 1; k < 8; ++k) ff_add(sc, colp[k][tid]);
    P[(J * N + J + t) * TILE + tid] = (double)sc.h + (double)sc.l;
  }
}

// Matrix-free FP64 residual over the lower triangle of tiles only (Z is
// symmetric): one CTA per lower tile (I, J) computes its 128 x 128 entries
// Z_jk = exp(-t d_jk) once -- the FP64 differences, square root and
// exponential of the generator, entries below e^-46 in FP32 as the generator
// writes them for a solve -- and uses each twice: the row contributions
// Z_IJ w_J (rows of block I) go to partial P[I][J], and for I != J the
// column contributions Z_IJ^T w_I (rows of block J) to P[J][I], so every row
// block X has exactly N partials P[X][0..N-1] (J <= X: its tiles' rows;
// J > X: the tiles below it, transposed).  Within a tile each thread adds its
// 4 (row) or 8 (column) products with FMAs and the partial is a shuffle /
// shared-memory tree; across tiles k_resid_sym_finish adds the N partials of
// a row with Neumaier compensation (the accuracy class of the stored-tile
// residual).  Row sums of Z for ||Z||inf go to rowsum (FP32 within a tile,
// FP64 atomics across tiles: a norm).  Thread layout as in the generator:
// warp w has tile rows w + 16 i (i < 8), lane l columns l + 32 q (q < 4).
constexpr int SYM_THREADS = 512;
constexpr int SYM_MC = 32;

__global__ void __launch_bounds__(SYM_THREADS, 1)
    k_resid_sym(const double* __restrict__ X, int64_t n, int m, double t, const double* __restrict__ w,
                double* __restrict__ P, double* __restrict__ rowsum, int64_t N, int kind, double kc) {
  extern __shared__ double smem[];
  double* xr = smem;                   // [TILE][SYM_MC] row points
  double* xc = smem + TILE * SYM_MC;   // [SYM_MC][TILE] column points
  __shared__ double colpart[SYM_THREADS / 32][TILE];
  __shared__ float zcol[SYM_THREADS / 32][TILE];
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  load_exp_table(exptab);
  int64_t I, J;
  tri_coords((int64_t)blockIdx.x, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = I * TILE, col0 = J * TILE;
  double d2[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) d2[i][q] = 0.0;
  for (int l0 = 0; l0 < m; l0 += SYM_MC) {
    const int mc = min(SYM_MC, m - l0);
    for (int e = threadIdx.x; e < TILE * mc; e += SYM_THREADS) {
      const int r = e / mc, l = e - r * mc;
      const int64_t gr = row0 + r, gc = col0 + r;
      xr[r * SYM_MC + l] = gr < n ? X[gr * m + l0 + l] : 0.0;
      xc[l * TILE + r] = gc < n ? X[gc * m + l0 + l] : 0.0;
    }
    __syncthreads();
    for (int l = 0; l < mc; ++l) {
      double a[8], b[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = xr[(warp + 16 * i) * SYM_MC + l];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = xc[l * TILE + lane + 32 * q];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double diff = a[i] - b[q];
          d2[i][q] = fma(diff, diff, d2[i][q]);
        }
    }
    __syncthreads();
  }
  __shared__ double s_wr[TILE], s_wc[TILE];
  if (threadIdx.x < TILE) {
    const int64_t gr = row0 + threadIdx.x, gc = col0 + threadIdx.x;
    s_wr[threadIdx.x] = gr < n ? w[gr] : 0.0;
    s_wc[threadIdx.x] = gc < n ? w[gc] : 0.0;
  }
  __syncthreads();
  double cs[4] = {0.0, 0.0, 0.0, 0.0};
  float zc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  // d^2 above (kTinyArg / t)^2: t d > kTinyArg, the entry below e^-46
  const double dcut = kTinyArg / t;
  const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(dcut * dcut);
  const float tf = (float)t;
  // rows of block I: each row's 4 products per lane, then a lane tree -> P[I][J]
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = warp + 16 * i;
    const int64_t gr = row0 + r;
    const double wri = s_wr[r];
    double v = 0.0;
    float zv = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gc = col0 + lane + 32 * q;
      double z = 0.0;
      if (gr < n && gc < n) {
        if (gr == gc) {
          z = 1.0;
        } else if (kind == MAT_EXP) {
          // the solver's entries: FP32 below e^-46 (as the generator writes
          // them for a solve; decided on d^2, then sqrt and exp on the FP32
          // pipe), the FP32-reduced FP64 exponential above
          if ((unsigned long long)__double_as_longlong(d2[i][q]) > tiny_bits) {
            z = f32_to_f64_nonneg(exp_neg_tiny_td2(tf, t, d2[i][q]));
          } else {
            z = exp_neg_td(t, sqrt_pos(d2[i][q]), exptab);
          }
        } else {
          z = mat_entry(kind, t, kc, sqrt_pos(d2[i][q]), exptab);
        }
      }
      v = fma(z, s_wc[lane + 32 * q], v);
      cs[q] = fma(z, wri, cs[q]);
      const float zf = kind ? __double2float_rn(z) : f64_to_f32_nonneg(z);
      zv += zf;
      zc[q] += zf;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      zv += __shfl_xor_sync(0xffffffffu, zv, o);
    }
    if (lane == 0) {
      P[(I * N + J) * TILE + r] = v;
      if (gr < n) atomicAdd(rowsum + gr, (double)zv);
    }
  }
  if (I == J) return;  // uniform: a diagonal tile's rows cover both triangles
  // rows of block J (the transposed tile): P[J][I]
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    colpart[warp][lane + 32 * q] = cs[q];
    zcol[warp][lane + 32 * q] = zc[q];
  }
  __syncthreads();
  if (threadIdx.x < TILE) {
    double v = 0.0;
    float zv = 0.0f;
#pragma unroll
    for (int k = 0; k < SYM_THREADS / 32; ++k) {
      v += colpart[k][threadIdx.x];
      zv += zcol[k][threadIdx.x];
    }
    P[(J * N + I) * TILE + threadIdx.x] = v;
    if (col0 + threadIdx.x < n) atomicAdd(rowsum + col0 + threadIdx.x, (double)zv);
  }
}

// k_resid_sym with the pair distances from quantized coordinates (Xq, the
// exact integer d^2 of mag_math.cuh; pairs with d^2 < tau2 from the FP64
// differences of X), Z = exp(-t d) only: the same entries, products, sums
// and partials, with column q of a thread taken as the outer loop and each
// pair finished on its own.
__global__ void __launch_bounds__(SYM_THREADS, 1)
    k_resid_sym_q(const long long* __restrict__ Xq, const double* __restrict__ X, int64_t n, int m, QuantParams qp,
                  double t, const double* __restrict__ w, double* __restrict__ P, double* __restrict__ rowsum,
                  int64_t N) {
  extern __shared__ double smem[];
  long long* xr = reinterpret_cast<long long*>(smem);  // [TILE][SYM_MC] row points
  long long* xc = xr + TILE * SYM_MC;                  // [SYM_MC][TILE] column points
  __shared__ double colpart[SYM_THREADS / 32][TILE];
  __shared__ float zcol[SYM_THREADS / 32][TILE];
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  __shared__ double s_wr[TILE], s_wc[TILE];
  load_exp_table(exptab);
  int64_t I, J;
  tri_coords((int64_t)blockIdx.x, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = I * TILE, col0 = J * TILE;
  for (int e = threadIdx.x; e < TILE * m; e += SYM_THREADS) {
    const int r = e / m, l = e - r * m;
    const int64_t gr = row0 + r, gc = col0 + r;
    xr[r * SYM_MC + l] = gr < n ? Xq[gr * m + l] : 0ll;
    xc[l * TILE + r] = gc < n ? Xq[gc * m + l] : 0ll;
  }
  if (threadIdx.x < TILE) {
    const int64_t gr = row0 + threadIdx.x, gc = col0 + threadIdx.x;
    s_wr[threadIdx.x] = gr < n ? w[gr] : 0.0;
    s_wc[threadIdx.x] = gc < n ? w[gc] : 0.0;
  }
  __syncthreads();
  const unsigned long long mask = (1ull << qp.L) - 1ull;
  const unsigned long long tau2_bits = (unsigned long long)__double_as_longlong(qp.tau2);
  // d^2 above (kTinyArg / t)^2: t d > kTinyArg, the entry below e^-46
  const double dcut = kTinyArg / t;
  const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(dcut * dcut);
  const float tf = (float)t;
  double v[8];
  float zv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = 0.0;
    zv[i] = 0.0f;
  }
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    const int64_t gc = col0 + c;
    const double wcq = s_wc[c];
    double csq = 0.0;
    float zcq = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = warp + 16 * i;
      const int64_t gr = row0 + r;
      const long long* xrow = xr + r * SYM_MC;
      unsigned long long A = 0ull, Bx = 0ull, C = 0ull;
      for (int l = 0; l < m; ++l) q_accumulate(xrow[l], xc[l * TILE + c], mask, qp.L, A, Bx, C);
      double z = 0.0;
      if (gr < n && gc < n) {
        if (gr == gc) {
          z = 1.0;
        } else {
          double d2 = q128_to_f64(A, Bx, C, qp.L, qp.e);
          if ((unsigned long long)__double_as_longlong(d2) < tau2_bits) {
            d2 = 0.0;
            for (int l = 0; l < m; ++l) {
              const double diff = X[gr * m + l] - X[gc * m + l];
              d2 = fma(diff, diff, d2);
            }
          }
          if ((unsigned long long)__double_as_longlong(d2) > tiny_bits)
            z = f32_to_f64_nonneg(exp_neg_tiny_td2(tf, t, d2));
          else
            z = exp_neg_td(t, sqrt_pos(d2), exptab);
        }
      }
      v[i] = fma(z, wcq, v[i]);
      csq = fma(z, s_wr[r], csq);
      const float zf = f64_to_f32_nonneg(z);
      zv[i] += zf;
      zcq += zf;
    }
    colpart[warp][c] = csq;
    zcol[warp][c] = zcq;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double vi = v[i];
    float zi = zv[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vi += __shfl_xor_sync(0xffffffffu, vi, o);
      zi += __shfl_xor_sync(0xffffffffu, zi, o);
    }
    const int r = warp + 16 * i;
    const int64_t gr = row0 + r;
    if (lane == 0) {
      P[(I * N + J) * TILE + r] = vi;
      if (gr < n) atomicAdd(rowsum + gr, (double)zi);
    }
  }
  if (I == J) return;  // uniform: a diagonal tile's rows cover both triangles
  __syncthreads();
  if (threadIdx.x < TILE) {
    double vc = 0.0;
    float zc = 0.0f;
#pragma unroll
    for (int k = 0; k < SYM_THREADS / 32; ++k) {
      vc += colpart[k][threadIdx.x];
      zc += zcol[k][threadIdx.x];
    }
    P[(J * N + I) * TILE + threadIdx.x] = vc;
    if (col0 + threadIdx.x < n) atomicAdd(rowsum + col0 + threadIdx.x, (double)zc);
  }
}

// r_j = b_j - (the N partials of row j, Neumaier), and the three norms.
__global__ void k_resid_sym_finish(const double* __restrict__ P, int64_t n, int64_t N, int64_t np,
                                   const double* __restrict__ w, const double* __restrict__ b,
                                   const double* __restrict__ rowsum, double* __restrict__ r, DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ra = 0.0, za = 0.0, wa = 0.0;
  if (j < n) {
    const int64_t I = j / TILE, rr = j % TILE;
    double s = 0.0, c = 0.0;
    for (int64_t J = 0; J < N; ++J) {
      const double v = P[(I * N + J) * TILE + rr];
      const double tt = s + v;
      if (fabs(s) >= fabs(v))
        c += (s - tt) + v;
      else
        c += (v - tt) + s;
      s = tt;
    }
    const double bj = b ? b[j] : 1.0;
    const double rj = (bj - s) - c;
    r[j] = rj;
    ra = fabs(rj);
    za = rowsum[j];
    wa = fabs(w[j]);
  } else if (j < np) {
    r[j] = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ra = fmax(ra, __shfl_xor_sync(0xffffffffu, ra, o));
    za = fmax(za, __shfl_xor_sync(0xffffffffu, za, o));
    wa = fmax(wa, __shfl_xor_sync(0xffffffffu, wa, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->r_max_bits, ra);
    atomic_max_nonneg(&st->z_max_bits, za);
    atomic_max_nonneg(&st->w_max_bits, wa);
  }
}

// r_j = b_j - (sum of the partials of row j) with Neumaier compensation: row
// block X holds P[X][J] for J <= X (its tiles' row sums) followed by
// P[X][X+t], t = 1..ceil((N-1-X)/S) (the strips' column sums); with ||r||,
// ||Z|| (from the generator's row sums) and ||w|| maxima.
__global__ void k_resid_stored_finish(const double* __restrict__ P, int64_t n, int64_t N, int64_t np,
                                      const double* __restrict__ w, const double* __restrict__ b,
                                      const double* __restrict__ rowsum, double* __restrict__ r,
                                      DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ra = 0.0, za = 0.0, wa = 0.0;
  if (j < n) {
    const int64_t I = j / TILE, rr = j % TILE;
    const int64_t slots = I + 1 + (N - 1 - I + RS_STRIP - 1) / RS_STRIP;
    double s = 0.0, c = 0.0;
    for (int64_t J = 0; J < slots; ++J) {
      const double v = P[(I * N + J) * TILE + rr];
      const double tt = s + v;
      if (fabs(s) >= fabs(v))
        c += (s - tt) + v;
      else
        c += (v - tt) + s;
      s = tt;
    }
    const double bj = b ? b[j] : 1.0;
    const double rj = (bj - s) - c;
    r[j] = rj;
    ra = fabs(rj);
    za = rowsum[j];
    wa = fabs(w[j]);
  } else if (j < np) {
    r[j] = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ra = fmax(ra, __shfl_xor_sync(0xffffffffu, ra, o));
    za = fmax(za, __shfl_xor_sync(0xffffffffu, za, o));
    wa = fmax(wa, __shfl_xor_sync(0xffffffffu, wa, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->r_max_bits, ra);
    atomic_max_nonneg(&st->z_max_bits, za);
    atomic_max_nonneg(&st->w_max_bits, wa);
  }
}

// Combine the chunk partials of each row (Neumaier), r_j = b_j - (Zw)_j, and
// the three infinity norms.  Rows n <= j < np get r_j = 0.
__global__ void k_resid_finish(const double* __restrict__ part, int chunks, int64_t n, int64_t np,
                               const double* __restrict__ w, const double* __restrict__ b,
                               double* __restrict__ r, DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ra = 0.0, za = 0.0, wa = 0.0;
  if (j < n) {
    double s = 0.0, c = 0.0, zs = 0.0;
    for (int q = 0; q < 2 * chunks; ++q) {
      const double v = part[(int64_t)q * np + j];
      const double tt = s + v;
      if (fabs(s) >= fabs(v))
        c += (s - tt) + v;
      else
        c += (v - tt) + s;
      s = tt;
    }
    for (int q = 0; q < chunks; ++q) zs += part[((int64_t)2 * chunks + q) * np + j];
    const double bj = b ? b[j] : 1.0;
    const double rj = (bj - s) - c;
    r[j] = rj;
    ra = fabs(rj);
    za = zs;
    wa = fabs(w[j]);
  } else if (j < np) {
    r[j] = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ra = fmax(ra, __shfl_xor_sync(0xffffffffu, ra, o));
    za = fmax(za, __shfl_xor_sync(0xffffffffu, za, o));
    wa = fmax(wa, __shfl_xor_sync(0xffffffffu, wa, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&st->r_max_bits, ra);
    atomic_max_nonneg(&st->z_max_bits, za);
    atomic_max_nonneg(&st->w_max_bits, wa);
  }
}

template <typename T>
__global__ void k_scale_rhs(const double* __restrict__ r, int64_t n, int64_t np, T* __restrict__ v,
                            const DevStatus* st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double rm = __longlong_as_double((long long)st->r_max_bits);
  const double inv = rm > 0.0 ? 1.0 / rm : 0.0;
  v[i] = i < n ? (T)(r[i] * inv) : T(0);
}

template <typename T>
__global__ void k_accumulate(double* __restrict__ x, const T* __restrict__ v, int64_t n,
                             const DevStatus* st, int init) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double rm = __longlong_as_double((long long)st->r_max_bits);
  const double d = rm * (double)v[i];
  x[i] = init ? d : x[i] + d;
}

__global__ void k_absmax(const double* __restrict__ v, int64_t n, DevStatus* st) {
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fmax(a, fabs(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->r_max_bits, a);
}

__global__ void k_fill(double* v, int64_t n, double value) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = value;
}

// Error-free sum of two doubles (Knuth's TwoSum).
__device__ inline void two_sum(double a, double b, double* s, double* e) {
  const double x = a + b;
  const double bv = x - a;
  *e = (a - (x - bv)) + (b - bv);
  *s = x;
}

// One CTA: Mag = sum_j w_j with Kahan per thread and TwoSum combination,
// min_j w_j, max_j |w_j|.
__global__ void __launch_bounds__(1024) k_reduce_w(const double* __restrict__ w, int64_t n,
                                                   DevStatus* st) {
  __shared__ double ss[1024], sc[1024], smin[1024], smax[1024];
  double s = 0.0, c = 0.0, mn = INFINITY, mx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = w[i];
    double hi, lo;
    two_sum(s, v, &hi, &lo);
    s = hi;
    c += lo;
    mn = fmin(mn, v);
    mx = fmax(mx, fabs(v));
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double hi, lo;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + h], &hi, &lo);
      ss[threadIdx.x] = hi;
      sc[threadIdx.x] += sc[threadIdx.x + h] + lo;
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + h]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->mag = ss[0] + sc[0];
    st->min_w = smin[0];
    st->w_max_bits = (unsigned long long)__double_as_longlong(smax[0]);
  }
}

// K7: for row i, with u_ik = (x_i - x_k)/d_ik,
//   part_t[i] = sum_{k != i} lam_i d_ik Z_ik w_k          (sum_i part_t[i] = lam^T (d o Z) w)
//   dL_dx[i]  = t sum_{k != i} Z_ik u_ik (lam_i w_k + lam_k w_i).
// One thread per row i, columns staged in shared memory, coordinates in FP64.
template <int MR>
__global__ void __launch_bounds__(RES_THREADS) k_grad(const double* __restrict__ X, int64_t n,
                                                      int m, double t,
                                                      const double* __restrict__ w,
                                                      const double* __restrict__ lam,
                                                      double* __restrict__ dL_dx,
                                                      double* __restrict__ part_t, int ct) {
  extern __shared__ double sm[];
  double* xc = sm;                 // [ct][m]
  double* wc = sm + ct * m;        // [ct]
  double* lc = sm + ct * (m + 1);  // [ct]
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  load_exp_table(exptab);
  const int64_t i = (int64_t)blockIdx.x * RES_THREADS + threadIdx.x;
  const bool live = i < n;
  double xi[MR], g[MR];
#pragma unroll
  for (int l = 0; l < MR; ++l) {
    xi[l] = (live && l < m) ? X[i * m + l] : 0.0;
    g[l] = 0.0;
  }
  const double wi = live ? w[i] : 0.0, li = live ? lam[i] : 0.0;
  double st_s = 0.0, st_c = 0.0;
  for (int64_t k0 = 0; k0 < n; k0 += ct) {
    const int cnt = (int)min((int64_t)ct, n - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * m; e += RES_THREADS) xc[e] = X[k0 * m + e];
    for (int e = threadIdx.x; e < cnt; e += RES_THREADS) {
      wc[e] = w[k0 + e];
      lc[e] = lam[k0 + e];
    }
    __syncthreads();
    if (!live) continue;
    for (int q = 0; q < cnt; ++q) {
      if (k0 + q == i) continue;
      const double* xk = xc + q * m;
      double d2 = 0.0;
#pragma unroll
      for (int l = 0; l < MR; ++l)
        if (l < m) {
          const double diff = xi[l] - xk[l];
          d2 = fma(diff, diff, d2);
        }
      const double d = sqrt_pos(d2);
      const double z = exp_neg_td(t, d, exptab);
      // dL/dt contribution with Kahan compensation
      const double y = fma(li * d * z, wc[q], -st_c);
      const double tt = st_s + y;
      st_c = (tt - st_s) - y;
      st_s = tt;
      const double coef = t * z * (li * wc[q] + lc[q] * wi) / d;
#pragma unroll
      for (int l = 0; l < MR; ++l)
        if (l < m) g[l] = fma(coef, xi[l] - xk[l], g[l]);
    }
  }
  if (live) {
    part_t[i] = st_s - st_c;
#pragma unroll
    for (int l = 0; l < MR; ++l)
      if (l < m) dL_dx[i * m + l] = g[l];
  }
}

__global__ void __launch_bounds__(1024) k_sum_f64(const double* __restrict__ v, int64_t n,
                                                  double* out) {
  __shared__ double ss[1024], sc[1024];
  double s = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double hi, lo;
    two_sum(s, v[i], &hi, &lo);
    s = hi;
    c += lo;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double hi, lo;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + h], &hi, &lo);
      ss[threadIdx.x] = hi;
      sc[threadIdx.x] += sc[threadIdx.x + h] + lo;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = ss[0] + sc[0];
}

// out[0] = min_i v_i, out[1] = max_i v_i (one CTA).
__global__ void __launch_bounds__(1024) k_minmax_f64(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double smin[32], smax[32];
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    lo = fmin(lo, v[i]);
    hi = fmax(hi, v[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = lo, smax[threadIdx.x >> 5] = hi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) lo = fmin(lo, smin[w]), hi = fmax(hi, smax[w]);
    out[0] = lo;
    out[1] = hi;
  }
}

// Checksum: sum over i of a 64-bit mix (splitmix64 finaliser) of the bits of
// v[i] and i, wrapping; one atomic per warp.
__global__ void k_hash_f64(const double* __restrict__ v, int64_t count, unsigned long long* out) {
  unsigned long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)__double_as_longlong(v[i]) + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    acc += z ^ (z >> 31);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// GMRES helpers (FP64): out[i] = <V_i, w> for i < k (V: k rows of length ld),
// one CTA per i; and w -= sum_i h[i] V_i; and x = s * w.
__global__ void __launch_bounds__(256) k_mdot(const double* __restrict__ V, int64_t ld, int k,
                                              const double* __restrict__ w, int64_t n, double* __restrict__ out) {
  __shared__ double ss[256], sc[256];
  const double* v = V + (int64_t)blockIdx.x * ld;
  double s = 0.0, c = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    double hi, lo;
    two_sum(s, v[j] * w[j], &hi, &lo);
    s = hi;
    c += lo;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double hi, lo;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + h], &hi, &lo);
      ss[threadIdx.x] = hi;
      sc[threadIdx.x] += sc[threadIdx.x + h] + lo;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = ss[0] + sc[0];
}

__global__ void k_maxpy(const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ h,
                        double* __restrict__ w, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = w[j];
  for (int i = 0; i < k; ++i) acc -= h[i] * V[(int64_t)i * ld + j];
  w[j] = acc;
}

__global__ void k_scale(const double* __restrict__ w, double s, double* __restrict__ x, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = s * w[j];
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_residual_mf(const double* X, int64_t n, int m, double t, const double* w,
                               const double* b, double* r, double* part, int chunks, int64_t np,
                               DevStatus* st, cudaStream_t s, int kind, double kc) {
  if (m < 1 || m > MAG_MAX_DIM) return cudaErrorInvalidValue;
  int ct = 128;
  while (ct > 8 && (size_t)ct * (m + 1) * sizeof(double) > 44 * 1024) ct /= 2;
  const size_t smem = (size_t)ct * (m + 1) * sizeof(double);
  const dim3 grid(blocks_for(n, RES_THREADS), (unsigned)chunks);
  if (smem > 44 * 1024) {
    // large m: eight column points per stage need more than the default
    // 48 KB of static (4 KB exp table) plus dynamic shared memory; at most
    // 8 x 2049 doubles = 131 KB
    cudaError_t e = cudaFuncSetAttribute(k_resid_mf<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (m <= 8)
    k_resid_mf<8><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, part, chunks, np, ct, kind, kc);
  else if (m <= 16)
    k_resid_mf<16><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, part, chunks, np, ct, kind, kc);
  else if (m <= 32)
    k_resid_mf<32><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, part, chunks, np, ct, kind, kc);
  else
    k_resid_mf<0><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, part, chunks, np, ct, kind, kc);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resid_finish<<<blocks_for(np, 256), 256, 0, s>>>(part, chunks, n, np, w, b, r, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_sym(const double* X, int64_t n, int m, double t, const double* w, const double* b,
                                double* r, double* P, double* rowsum, int64_t np, DevStatus* st, cudaStream_t s,
                                int kind, double kc, const long long* Xq, int qL, int qe, double qtau2) {
  if (m < 1 || m > MAG_MAX_DIM) return cudaErrorInvalidValue;
  const int64_t N = (n + TILE - 1) / TILE;
  const int64_t tiles = num_lower_tiles(N);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)TILE * SYM_MC * sizeof(double);
  cudaError_t e = cudaMemsetAsync(rowsum, 0, (size_t)n * sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (Xq && kind == MAT_EXP && m <= SYM_MC) {
    const QuantParams qp{qL, qe, qtau2};
    // the dimension loop stays a loop: unrolled over eight dimensions the
    // kernel exceeds the 128 registers of its 512-thread launch bound
    e = cudaFuncSetAttribute(k_resid_sym_q, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_resid_sym_q<<<(unsigned)tiles, SYM_THREADS, smem, s>>>(Xq, X, n, m, qp, t, w, P, rowsum, N);
  } else {
    e = cudaFuncSetAttribute(k_resid_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_resid_sym<<<(unsigned)tiles, SYM_THREADS, smem, s>>>(X, n, m, t, w, P, rowsum, N, kind, kc);
  }
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resid_sym_finish<<<blocks_for(np, 256), 256, 0, s>>>(P, n, N, np, w, b, rowsum, r, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_stored(const double* Zd, int64_t n, int64_t N, const double* w,
                                   const double* b, const double* rowsum, double* r, double* P, int64_t np,
                                   DevStatus* st, cudaStream_t s) {
  if (N > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((N - 1 + RS_STRIP - 1) / RS_STRIP + 1), (unsigned)N);
  k_resid_stored<<<grid, 256, 0, s>>>(Zd, n, N, w, P);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resid_stored_finish<<<blocks_for(np, 256), 256, 0, s>>>(P, n, N, np, w, b, rowsum, r, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_stored_ff(const double* Zd, int64_t n, int64_t N, const double* w, void* wsplit,
                                      const double* b, const double* rowsum, double* r, double* P, int64_t np,
                                      DevStatus* st, cudaStream_t s) {
  if (N > 65535 || np < N * TILE) return cudaErrorInvalidValue;
  float2* wf = static_cast<float2*>(wsplit);
  k_split_ff<<<blocks_for(np, 256), 256, 0, s>>>(w, n, np, wf);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((N - 1 + RS_STRIP - 1) / RS_STRIP + 1), (unsigned)N);
  k_resid_stored_ff<<<grid, 256, 0, s>>>(Zd, n, N, wf, P);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resid_stored_finish<<<blocks_for(np, 256), 256, 0, s>>>(P, n, N, np, w, b, rowsum, r, st);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_rhs(const double* r, int64_t n, int64_t np, T* v, const DevStatus* st,
                             cudaStream_t s) {
  k_scale_rhs<T><<<blocks_for(np, 256), 256, 0, s>>>(r, n, np, v, st);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_accumulate(double* x, const T* v, int64_t n, const DevStatus* st, bool init,
                              cudaStream_t s) {
  k_accumulate<T><<<blocks_for(n, 256), 256, 0, s>>>(x, v, n, st, init ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_scale_rhs<float>(const double*, int64_t, int64_t, float*, const DevStatus*,
                                             cudaStream_t);
template cudaError_t launch_scale_rhs<double>(const double*, int64_t, int64_t, double*,
                                              const DevStatus*, cudaStream_t);
template cudaError_t launch_accumulate<float>(double*, const float*, int64_t, const DevStatus*, bool,
                                              cudaStream_t);
template cudaError_t launch_accumulate<double>(double*, const double*, int64_t, const DevStatus*, bool,
                                               cudaStream_t);

cudaError_t launch_absmax(const double* v, int64_t n, DevStatus* st, cudaStream_t s) {
  unsigned blocks = blocks_for(n, 256);
  if (blocks > 1024) blocks = 1024;
  k_absmax<<<blocks, 256, 0, s>>>(v, n, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce_w(const double* w, int64_t n, DevStatus* st, cudaStream_t s) {
  k_reduce_w<<<1, 1024, 0, s>>>(w, n, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mdot(const double* V, int64_t ld, int k, const double* w, int64_t n, double* out,
                        cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_mdot<<<k, 256, 0, s>>>(V, ld, k, w, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_maxpy(const double* V, int64_t ld, int k, const double* h, double* w, int64_t n,
                         cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_maxpy<<<blocks_for(n, 256), 256, 0, s>>>(V, ld, k, h, w, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* w, double sc, double* x, int64_t n, cudaStream_t s) {
  k_scale<<<blocks_for(n, 256), 256, 0, s>>>(w, sc, x, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill(double* v, int64_t n, double value, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<blocks_for(n, 256), 256, 0, s>>>(v, n, value);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_grad(const double* X, int64_t n, int m, double t, const double* w,
                        const double* lam, double* dL_dx, double* part_t, int64_t np,
                        cudaStream_t s) {
  (void)np;
  int ct = 128;
  while (ct > 8 && (size_t)ct * (m + 2) * sizeof(double) > 44 * 1024) ct /= 2;  // + 4 KB exp table
  const size_t smem = (size_t)ct * (m + 2) * sizeof(double);
  const unsigned grid = blocks_for(n, RES_THREADS);
  if (m <= 8)
    k_grad<8><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, lam, dL_dx, part_t, ct);
  else if (m <= 16)
    k_grad<16><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, lam, dL_dx, part_t, ct);
  else if (m <= 32)
    k_grad<32><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, lam, dL_dx, part_t, ct);
  else if (m <= 64)
    k_grad<64><<<grid, RES_THREADS, smem, s>>>(X, n, m, t, w, lam, dL_dx, part_t, ct);
  else
    return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double* v, int64_t n, double* out, cudaStream_t s) {
  k_sum_f64<<<1, 1024, 0, s>>>(v, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_hash(const double* v, int64_t count, unsigned long long* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
  k_hash_f64<<<blocks, 256, 0, s>>>(v, count, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_minmax(const double* v, int64_t n, double* out2, cudaStream_t s) {
  k_minmax_f64<<<1, 1024, 0, s>>>(v, n, out2);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mag

// ------------------------------------------------- allocation-free residual
// Scratch of mag_residual_noalloc: 3 partial-sum rows of up to
// MAG_NOALLOC_MAX_N doubles, then a DevStatus in the last 32 doubles.
namespace mag {
namespace {

constexpr int64_t NOALLOC_STATUS_DOUBLES = 32;
static_assert(sizeof(DevStatus) <= NOALLOC_STATUS_DOUBLES * sizeof(double), "status block fits");
static __device__ __align__(256) double g_noalloc_scratch[3 * (int64_t)MAG_NOALLOC_MAX_N + NOALLOC_STATUS_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace mag

extern "C" int mag_residual_noalloc(const double* points, int64_t n, int32_t m, double t, const double* w,
                                    const double* b, double* r_out, double* norms, void* stream) {
  using namespace mag;
  if (!points || !w || !r_out || !norms || n < 2 || m < 1 || m > MAG_MAX_DIM || !(t > 0.0) || !isfinite(t))
    return MAG_EINVAL;
  if (n > MAG_NOALLOC_MAX_N) return MAG_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return MAG_ECUDA;
  }
  DevStatus* st = reinterpret_cast<DevStatus*>(scratch + 3 * (int64_t)MAG_NOALLOC_MAX_N);
  // the partial sums are written in full; only the norm maxima start at zero
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) {
    cudaGetLastError();
    return MAG_ECUDA;
  }
  // as many column chunks as the scratch holds (at most 8): 3 * chunks * n <= 3 * MAX_N
  int chunks = (int)std::min<int64_t>(8, MAG_NOALLOC_MAX_N / n);
  if (chunks < 1) chunks = 1;
  if (launch_residual_mf(points, n, m, t, w, b, r_out, scratch, chunks, n, st, s, MAT_EXP, 0.0) != cudaSuccess) {
    cudaGetLastError();
    return MAG_ECUDA;
  }
  DevStatus h;
  if (cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MAG_ECUDA;
  }
  double rn, zn, wn;
  std::memcpy(&rn, &h.r_max_bits, sizeof rn);
  std::memcpy(&zn, &h.z_max_bits, sizeof zn);
  std::memcpy(&wn, &h.w_max_bits, sizeof wn);
  norms[0] = (zn > 0 && wn > 0) ? rn / (zn * wn) : INFINITY;
  norms[1] = rn;
  norms[2] = zn;
  norms[3] = wn;
  return MAG_OK;
}
