// K1: fused distance + exp generator of Z = exp[-t d] (Sec. 2), packed lower tiles.
//
// One CTA per lower tile (I, J).  Coordinates of the tile's 128 row points and
// 128 column points are staged in shared memory in chunks of MC coordinates;
// every pair difference x_jl - x_kl is taken in FP64 and squared/accumulated
// with FP64 FMAs (no ||x||^2 + ||y||^2 - 2 x^T y expansion, so close points do
// not cancel).  The FP32 tile (factor input) takes sqrt/exp in FP32 from the
// FP64 d^2; the FP64 tile (FP64 factor or stored residual) takes them in FP64.
//
// Thread layout (512 threads): warp w handles tile rows w + 16 i (i < 8),
// lane l handles tile columns 4 l + q (q < 4), so each thread stores its four
// entries of a row with one 16-byte store (FP32: a float4; FP64: two
// double2) and a warp's stores cover one whole tile row.  The column points
// are staged in shared memory with column 4 l + q at position 32 q + l, so
// the distance loop's reads stay conflict free.
//
// Side outputs, all fused: full row sums of Z (for ||Z||inf and the Gershgorin
// bound used to choose the factor precision), min off-diagonal d^2 (the Sec. 1
// bound), and flags for non-finite coordinates and coincident points.
#include "mag_internal.cuh"
#include "mag_math.cuh"

namespace mag {

namespace {

constexpr int GEN_THREADS = 512;
constexpr int GEN_MC = 32;  // coordinates staged per chunk

__device__ inline void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// Tiles of a slab layout (mag_internal.cuh: tile_index with column cap W)
// whose tile (0, 0) is the global tile (t0, t0); W >= the tile rows and
// t0 = 0 give the whole packed matrix.
template <bool WF, bool WD, bool ROWSUM, bool WDIST>
__global__ void __launch_bounds__(GEN_THREADS, 1)
    k_generate(const double* __restrict__ X, int64_t n, int m, double t, float* __restrict__ Zf,
               double* __restrict__ Zd, double* __restrict__ Dd, double* __restrict__ rowsum, DevStatus* st,
               int kind, double dcut, int64_t t0, int64_t W, double kc) {
  extern __shared__ double smem[];
  double* xr = smem;                   // [TILE][GEN_MC] row points (broadcast reads)
  double* xc = smem + TILE * GEN_MC;   // [GEN_MC][TILE] column points (conflict free)
  __shared__ double colpart[GEN_THREADS / 32][TILE];
  __shared__ unsigned long long warpmin[GEN_THREADS / 32];
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  if (WD) load_exp_table(exptab);

  int64_t I, J;
  tile_coords((int64_t)blockIdx.x, W, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (t0 + I) * TILE, col0 = (t0 + J) * TILE;

  double d2[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) d2[i][q] = 0.0;

  for (int l0 = 0; l0 < m; l0 += GEN_MC) {
    const int mc = min(GEN_MC, m - l0);
    for (int e = threadIdx.x; e < TILE * mc; e += GEN_THREADS) {
      const int r = e / mc, l = e - r * mc;
      const int64_t gr = row0 + r, gc = col0 + r;
      xr[r * GEN_MC + l] = gr < n ? X[gr * m + l0 + l] : 0.0;
      xc[l * TILE + 32 * (r & 3) + (r >> 2)] = gc < n ? X[gc * m + l0 + l] : 0.0;
    }
    __syncthreads();
    for (int l = 0; l < mc; ++l) {
      double a[8], b[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = xr[(warp + 16 * i) * GEN_MC + l];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = xc[l * TILE + 32 * q + lane];  // column 4 lane + q
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

  const int64_t tile_off = tile_index(I, J, W) * TILE_ELEMS;
  // row/column partial sums of a thread cover 4 and 8 entries: FP32 is ample
  // for a norm, and keeps the FP64 pipe for the distances and the exponential
  float rs[8], cs[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) rs[i] = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) cs[q] = 0.0f;
  unsigned long long mind2b = 0x7ff0000000000000ull;  // +inf
  int flags = 0;
  const float tf = (float)t;
  // d > dcut = tiny_arg / t (from the host) on the bit patterns (d >= 0):
  // the FP64 pipe stays on the distances and the exponential
  const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(dcut);

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = warp + 16 * i;
    const int64_t gr = row0 + r;
    float zfv[4];
    double zdv[4], ddv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * lane + q;
      const int64_t gc = col0 + c;
      const double v = d2[i][q];
      double zd = 0.0, dd = 0.0;
      float zf = 0.0f;
      if (gr >= n || gc >= n || gr == gc) {
        zd = (gr == gc) ? 1.0 : 0.0;
        zf = (float)zd;
      } else {
        // v >= 0 or NaN: the checks and the minimum on the bit pattern (integer
        // pipe; non-negative doubles order like their bits)
        const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
        if ((vb >> 52) >= 0x7ffull) flags |= ST_NONFINITE;
        else if (vb == 0ull) flags |= ST_DUPLICATE;
        else mind2b = vb < mind2b ? vb : mind2b;
        if (WD || WDIST) dd = sqrt_pos(v);
        if (WD && !kind && (unsigned long long)__double_as_longlong(dd) > tiny_bits) {
          zf = exp_neg_tiny_td(tf, t, dd);
          zd = f32_to_f64_nonneg(zf);
        } else {
          if (WD) zd = mat_entry(kind, t, kc, dd, exptab);
          if (WF)
            zf = WD ? (kind == MAT_DEFLATED ? __double2float_rn(zd) : f64_to_f32_nonneg(zd))
                    : (kind == MAT_EXP ? expf(-tf * sqrtf((float)v))
                                       : (kind == MAT_SHIFTED_DIST ? 1.0f - tf * sqrtf((float)v)
                                                                   : fmaf((float)kc, expm1f(-tf * sqrtf((float)v)), 1.0f)));
        }
      }
      zfv[q] = zf;
      zdv[q] = zd;
      ddv[q] = dd;
      if (ROWSUM && gr < n && gc < n) {
        const float zs = WF ? zf : (float)zd;
        rs[i] += zs;
        cs[q] += zs;
      }
    }
    // the four entries of row r, columns 4 lane .. 4 lane + 3: 16-byte stores
    const int64_t e = tile_off + (int64_t)r * TILE + 4 * lane;
    if (WF) *reinterpret_cast<float4*>(Zf + e) = make_float4(zfv[0], zfv[1], zfv[2], zfv[3]);
    if (WD) {
      *reinterpret_cast<double2*>(Zd + e) = make_double2(zdv[0], zdv[1]);
      *reinterpret_cast<double2*>(Zd + e + 2) = make_double2(zdv[2], zdv[3]);
    }
    if (WDIST) {
      *reinterpret_cast<double2*>(Dd + e) = make_double2(ddv[0], ddv[1]);
      *reinterpret_cast<double2*>(Dd + e + 2) = make_double2(ddv[2], ddv[3]);
    }
  }

  if (flags) atomicOr(&st->flags, flags);
  // min d^2 over the CTA
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, mind2b, o);
    mind2b = other < mind2b ? other : mind2b;
  }
  if (lane == 0) warpmin[warp] = mind2b;

  if (ROWSUM) {
    // row sums: an FP32 lane tree (a norm: depth 5 adds at most 5 roundings
    // to the 4-entry partials), one FP64 atomic per row
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float v = rs[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int64_t gr = row0 + warp + 16 * i;
      if (lane == 0 && gr < n) atomicAdd(rowsum + gr, (double)v);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) colpart[warp][4 * lane + q] = (double)cs[q];
  }
  __syncthreads();
  if (ROWSUM && I != J && threadIdx.x < TILE) {
    double v = 0.0;
    for (int w = 0; w < GEN_THREADS / 32; ++w) v += colpart[w][threadIdx.x];
    const int64_t gc = col0 + threadIdx.x;
    if (gc < n) atomicAdd(rowsum + gc, v);
  }
  if (threadIdx.x == 0) {
    unsigned long long v = warpmin[0];
    for (int w = 1; w < GEN_THREADS / 32; ++w) v = warpmin[w] < v ? warpmin[w] : v;
    if (v < 0x7ff0000000000000ull) atomicMin(&st->min_d2_bits, v);
  }
}

// Z from stored FP64 distances (same layout): one CTA per lower tile, FP64
// exp only, 16-byte reads and stores (lane l: columns 4 l .. 4 l + 3).
// Tiles of the padding get the identity, as in k_generate.
template <bool WF, bool WD>
__global__ void __launch_bounds__(256) k_generate_from_dist(const double* __restrict__ Dd, int64_t n, double t,
                                                            float* __restrict__ Zf, double* __restrict__ Zd,
                                                            double* __restrict__ rowsum, int kind, double dcut,
                                                            double kc) {
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  __shared__ float colpart[8][TILE];
  load_exp_table(exptab);
  __syncthreads();
  int64_t I, J;
  tri_coords((int64_t)blockIdx.x, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t off = tri_index(I, J) * TILE_ELEMS;
  const float tf = (float)t;
  const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(dcut);
  // row/column partial sums in FP32 (a norm; the FP64 pipe is the limit)
  float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int i = 0; i < 16; ++i) {
    const int r = warp * 16 + i;
    const int64_t gr = I * TILE + r;
    float rs = 0.0f;
    // lane: columns 4 lane .. 4 lane + 3 of row r, read and written with
    // 16-byte accesses
    const int64_t e0 = off + (int64_t)r * TILE + 4 * lane;
    const double2 d01 = *reinterpret_cast<const double2*>(Dd + e0);
    const double2 d23 = *reinterpret_cast<const double2*>(Dd + e0 + 2);
    const double dv[4] = {d01.x, d01.y, d23.x, d23.y};
    float zfv[4];
    double zdv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * lane + q;
      const int64_t gc = J * TILE + c;
      double zd;
      float zf;
      if (gr >= n || gc >= n || gr == gc) {
        zd = (gr == gc) ? 1.0 : 0.0;
        zf = (float)zd;
        if (gr == gc && gr < n) rs += 1.0f;  // the diagonal counts in its row sum
      } else {
        const double d = dv[q];
        if (WD && !kind && (unsigned long long)__double_as_longlong(d) > tiny_bits) {
          zf = exp_neg_tiny_td(tf, t, d);
          zd = f32_to_f64_nonneg(zf);
        } else {
          zd = WD ? mat_entry(kind, t, kc, d, exptab) : 0.0;
          zf = WD ? (kind == MAT_DEFLATED ? __double2float_rn(zd) : f64_to_f32_nonneg(zd))
                  : (kind == MAT_EXP ? expf(-tf * (float)d)
                                     : (kind == MAT_SHIFTED_DIST ? 1.0f - tf * (float)d
                                                                 : fmaf((float)kc, expm1f(-tf * (float)d), 1.0f)));
        }
        rs += zf;
        cs[q] += zf;
      }
      zfv[q] = zf;
      zdv[q] = zd;
    }
    if (WF) *reinterpret_cast<float4*>(Zf + e0) = make_float4(zfv[0], zfv[1], zfv[2], zfv[3]);
    if (WD) {
      *reinterpret_cast<double2*>(Zd + e0) = make_double2(zdv[0], zdv[1]);
      *reinterpret_cast<double2*>(Zd + e0 + 2) = make_double2(zdv[2], zdv[3]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    if (lane == 0 && gr < n) atomicAdd(rowsum + gr, (double)rs);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) colpart[warp][4 * lane + q] = cs[q];
  __syncthreads();
  if (I != J && threadIdx.x < TILE) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += (double)colpart[w][threadIdx.x];
    const int64_t gc = J * TILE + threadIdx.x;
    if (gc < n) atomicAdd(rowsum + gc, v);
  }
}

// max_j ||x_j - x_0||^2 (FP64 differences) into aux_bits: 2 max_j ||x_j - x_0||
// bounds every pairwise distance (triangle inequality through x_0).
__global__ void k_far_from_first(const double* __restrict__ X, int64_t n, int m, DevStatus* st) {
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s2 = 0.0;
    for (int l = 0; l < m; ++l) {
      const double diff = X[i * m + l] - X[l];
      s2 = fma(diff, diff, s2);
    }
    v = fmax(v, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->far_d2_bits, v);
}

__global__ void k_rowsum_max(const double* __restrict__ rowsum, int64_t n, DevStatus* st) {
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v = fmax(v, rowsum[i] - 1.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->off_max_bits, fmax(v, 0.0));
}

// FP64 distances of the packed lower tiles from the quantized coordinates
// (m <= GEN_MC; MQ8: m <= 8, a column's coordinates held in registers),
// with min d^2 and the coincident-point flag as k_generate: one CTA per
// tile, warp w on tile rows w + 16 i (i < 8), lane l on columns 32 q + l
// (q < 4), each pair finished and stored on its own (a warp's store covers
// 32 consecutive entries of a row).  Rows and columns of the padding get
// d = 0 (the generator from distances gives them the identity by index).
template <bool MQ8>
__global__ void __launch_bounds__(GEN_THREADS, 1)
    k_dist_q(const long long* __restrict__ Xq, const double* __restrict__ X, int64_t n, int m, QuantParams qp,
             double* __restrict__ Dd, DevStatus* st) {
  extern __shared__ double smem[];
  long long* xr = reinterpret_cast<long long*>(smem);  // [TILE][GEN_MC] row points (broadcast reads)
  long long* xc = xr + TILE * GEN_MC;                  // [GEN_MC][TILE] column points (conflict free)
  __shared__ unsigned long long warpmin[GEN_THREADS / 32];
  int64_t I, J;
  tri_coords((int64_t)blockIdx.x, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = I * TILE, col0 = J * TILE;
  const int mc = MQ8 ? 8 : m;  // MQ8: dimensions m .. 7 staged as zeros
  for (int e = threadIdx.x; e < TILE * mc; e += GEN_THREADS) {
    const int r = e / mc, l = e - r * mc;
    const int64_t gr = row0 + r, gc = col0 + r;
    xr[r * GEN_MC + l] = gr < n && l < m ? Xq[gr * m + l] : 0ll;
    xc[l * TILE + r] = gc < n && l < m ? Xq[gc * m + l] : 0ll;
  }
  __syncthreads();
  const unsigned long long mask = (1ull << qp.L) - 1ull;
  const unsigned long long tau2_bits = (unsigned long long)__double_as_longlong(qp.tau2);
  const int64_t tile_off = tri_index(I, J) * TILE_ELEMS;
  unsigned long long mind2b = 0x7ff0000000000000ull;  // +inf
  int flags = 0;
  for (int q = 0; q < 4; ++q) {
    const int c = 32 * q + lane;
    const int64_t gc = col0 + c;
    long long cv[8];
    if (MQ8) {
#pragma unroll
      for (int l = 0; l < 8; ++l) cv[l] = xc[l * TILE + c];
    }
#pragma unroll 4
    for (int i = 0; i < 8; ++i) {
      const int r = warp + 16 * i;
      const int64_t gr = row0 + r;
      const long long* xrow = xr + r * GEN_MC;
      unsigned long long A = 0ull, Bx = 0ull, C = 0ull;
      if (MQ8) {
#pragma unroll
        for (int l = 0; l < 8; ++l) q_accumulate(xrow[l], cv[l], mask, qp.L, A, Bx, C);
      } else {
        for (int l = 0; l < m; ++l) q_accumulate(xrow[l], xc[l * TILE + c], mask, qp.L, A, Bx, C);
      }
      double dd = 0.0;
      if (gr < n && gc < n && gr != gc) {
        double v = q128_to_f64(A, Bx, C, qp.L, qp.e);
        unsigned long long vb = (unsigned long long)__double_as_longlong(v);
        if (vb < tau2_bits) {
          // close pair: the FP64 differences of the points, as k_generate
          v = 0.0;
          for (int l = 0; l < m; ++l) {
            const double diff = X[gr * m + l] - X[gc * m + l];
            v = fma(diff, diff, v);
          }
          vb = (unsigned long long)__double_as_longlong(v);
        }
        if (vb == 0ull) flags |= ST_DUPLICATE;
        else mind2b = vb < mind2b ? vb : mind2b;
        dd = sqrt_pos(v);
      }
      Dd[tile_off + (int64_t)r * TILE + c] = dd;
    }
  }
  if (flags) atomicOr(&st->flags, flags);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, mind2b, o);
    mind2b = other < mind2b ? other : mind2b;
  }
  if (lane == 0) warpmin[warp] = mind2b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long v = warpmin[0];
    for (int w = 1; w < GEN_THREADS / 32; ++w) v = warpmin[w] < v ? warpmin[w] : v;
    if (v < 0x7ff0000000000000ull) atomicMin(&st->min_d2_bits, v);
  }
}

// k_generate with the pair distances from the quantized coordinates (the
// exact integer d^2 of mag_math.cuh; pairs with d^2 < tau2 from the FP64
// differences of X), row sums when rowsum is given: the same entries,
// checks and outputs in one pass, each pair finished on its own (row
// r = w + 16 i outer, column 4 l + q inner, so a thread still stores its
// four entries of a row with 16-byte stores), tiles in the slab layout of
// k_generate.  Used where no distances are kept (a single t, the slabs of
// the out-of-core factor); a multi-t call keeps them with k_dist_q, then
// k_generate_from_dist.
template <bool WF, bool WD>
__global__ void __launch_bounds__(GEN_THREADS, 1)
    k_generate_q(const long long* __restrict__ Xq, const double* __restrict__ X, int64_t n, int m, QuantParams qp,
                 double t, float* __restrict__ Zf, double* __restrict__ Zd, double* __restrict__ rowsum,
                 DevStatus* st, int kind, double dcut, double kc, int64_t t0, int64_t W) {
  extern __shared__ double smem[];
  long long* xr = reinterpret_cast<long long*>(smem);  // [TILE][GEN_MC] row points (broadcast reads)
  long long* xc = xr + TILE * GEN_MC;                  // [GEN_MC][TILE] column points (conflict free)
  __shared__ double colpart[GEN_THREADS / 32][TILE];
  __shared__ unsigned long long warpmin[GEN_THREADS / 32];
  __shared__ __align__(16) double exptab[EXPT_SMEM];
  if (WD) load_exp_table(exptab);
  int64_t I, J;
  tile_coords((int64_t)blockIdx.x, W, &I, &J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (t0 + I) * TILE, col0 = (t0 + J) * TILE;
  for (int e = threadIdx.x; e < TILE * m; e += GEN_THREADS) {
    const int r = e / m, l = e - r * m;
    const int64_t gr = row0 + r, gc = col0 + r;
    xr[r * GEN_MC + l] = gr < n ? Xq[gr * m + l] : 0ll;
    xc[l * TILE + 32 * (r & 3) + (r >> 2)] = gc < n ? Xq[gc * m + l] : 0ll;
  }
  __syncthreads();
  const unsigned long long mask = (1ull << qp.L) - 1ull;
  const unsigned long long tau2_bits = (unsigned long long)__double_as_longlong(qp.tau2);
  const int64_t tile_off = tile_index(I, J, W) * TILE_ELEMS;
  float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  unsigned long long mind2b = 0x7ff0000000000000ull;  // +inf
  int flags = 0;
  const float tf = (float)t;
  const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(dcut);
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    const int r = warp + 16 * i;
    const int64_t gr = row0 + r;
    const long long* xrow = xr + r * GEN_MC;
    float rs = 0.0f;
    float zfv[4];
    double zdv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gc = col0 + 4 * lane + q;
      unsigned long long A = 0ull, Bx = 0ull, C = 0ull;
      for (int l = 0; l < m; ++l) q_accumulate(xrow[l], xc[l * TILE + 32 * q + lane], mask, qp.L, A, Bx, C);
      double zd = 0.0;
      float zf = 0.0f;
      if (gr >= n || gc >= n || gr == gc) {
        zd = (gr == gc) ? 1.0 : 0.0;
        zf = (float)zd;
      } else {
        double v = q128_to_f64(A, Bx, C, qp.L, qp.e);
        unsigned long long vb = (unsigned long long)__double_as_longlong(v);
        if (vb < tau2_bits) {
          v = 0.0;
          for (int l = 0; l < m; ++l) {
            const double diff = X[gr * m + l] - X[gc * m + l];
            v = fma(diff, diff, v);
          }
          vb = (unsigned long long)__double_as_longlong(v);
        }
        if (vb == 0ull) flags |= ST_DUPLICATE;
        else mind2b = vb < mind2b ? vb : mind2b;
        if (WD) {
          const double dd = sqrt_pos(v);
          if (!kind && (unsigned long long)__double_as_longlong(dd) > tiny_bits) {
            zf = exp_neg_tiny_td(tf, t, dd);
            zd = f32_to_f64_nonneg(zf);
          } else {
            zd = mat_entry(kind, t, kc, dd, exptab);
            if (WF) zf = kind == MAT_DEFLATED ? __double2float_rn(zd) : f64_to_f32_nonneg(zd);
          }
        } else {
          const float df = sqrtf(f64_to_f32_nonneg(v));
          zf = kind == MAT_EXP ? expf(-tf * df)
                               : (kind == MAT_SHIFTED_DIST ? 1.0f - tf * df
                                                           : fmaf((float)kc, expm1f(-tf * df), 1.0f));
        }
      }
      zfv[q] = zf;
      zdv[q] = zd;
      if (gr < n && gc < n) {
        const float zs = WF ? zf : (float)zd;
        rs += zs;
        cs[q] += zs;
      }
    }
    const int64_t e = tile_off + (int64_t)r * TILE + 4 * lane;
    if (WF) *reinterpret_cast<float4*>(Zf + e) = make_float4(zfv[0], zfv[1], zfv[2], zfv[3]);
    if (WD) {
      *reinterpret_cast<double2*>(Zd + e) = make_double2(zdv[0], zdv[1]);
      *reinterpret_cast<double2*>(Zd + e + 2) = make_double2(zdv[2], zdv[3]);
    }
    // the row's sum: an FP32 lane tree, one FP64 atomic per row
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    if (rowsum && lane == 0 && gr < n) atomicAdd(rowsum + gr, (double)rs);
  }
  if (flags) atomicOr(&st->flags, flags);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, mind2b, o);
    mind2b = other < mind2b ? other : mind2b;
  }
  if (lane == 0) warpmin[warp] = mind2b;
#pragma unroll
  for (int q = 0; q < 4; ++q) colpart[warp][4 * lane + q] = (double)cs[q];
  __syncthreads();
  if (rowsum && I != J && threadIdx.x < TILE) {
    double v = 0.0;
    for (int w = 0; w < GEN_THREADS / 32; ++w) v += colpart[w][threadIdx.x];
    const int64_t gc = col0 + threadIdx.x;
    if (gc < n) atomicAdd(rowsum + gc, v);
  }
  if (threadIdx.x == 0) {
    unsigned long long v = warpmin[0];
    for (int w = 1; w < GEN_THREADS / 32; ++w) v = warpmin[w] < v ? warpmin[w] : v;
    if (v < 0x7ff0000000000000ull) atomicMin(&st->min_d2_bits, v);
  }
}

// Per dimension l < m (one CTA each): min and max of X[:, l] into
// out[2 l], out[2 l + 1]; out[2 m] = 1 if a coordinate is not finite.
__global__ void k_coord_range(const double* __restrict__ X, int64_t n, int m, double* __restrict__ out) {
  const int l = blockIdx.x;
  double lo = INFINITY, hi = -INFINITY;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = X[i * m + l];
    if (!isfinite(v)) bad = 1;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  __shared__ double slo[32], shi[32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (bad) atomicOr(&sbad, 1);
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, slo[w]);
      hi = fmax(hi, shi[w]);
    }
    out[2 * l] = lo;
    out[2 * l + 1] = hi;
    if (sbad) out[2 * m] = 1.0;
  }
}

// q = round(2^e (x - lo_l)) with x - lo_l taken exactly as s + err (TwoSum):
// round(2^e s) + round(2^e err), within one unit of 2^e (x - lo_l).
__global__ void k_quantize(const double* __restrict__ X, int64_t n, int m, const double* __restrict__ range,
                           int e, long long* __restrict__ Xq) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * m) return;
  const int l = (int)(k % m);
  const double x = X[k], b = -range[2 * l];
  const double s = x + b;
  const double bv = s - x;
  const double err = (x - (s - bv)) + (b - bv);
  Xq[k] = __double2ll_rn(ldexp(s, e)) + __double2ll_rn(ldexp(err, e));
}

template <bool WF, bool WD, bool ROWSUM, bool WDIST = false>
cudaError_t launch_gen_t(const double* X, int64_t n, int m, double t, int64_t N, float* Zf,
                         double* Zd, double* rowsum, DevStatus* st, cudaStream_t s, double* Dd = nullptr,
                         int kind = 0, double tiny_arg = INFINITY, int64_t t0 = 0, int64_t W = -1, double kc = 0.0) {
  const size_t smem = 2 * (size_t)TILE * GEN_MC * sizeof(double);
  auto kern = k_generate<WF, WD, ROWSUM, WDIST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // N: tile rows of the (slab) matrix from global tile t0; W < 0: all columns
  if (W < 0) W = N;
  const int64_t tiles = num_slab_tiles(N, W);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  // entries with d > tiny_arg / t leave the FP64 exponential
  const double dcut = tiny_arg / t;
  kern<<<(unsigned)tiles, GEN_THREADS, smem, s>>>(X, n, m, t, Zf, Zd, Dd, rowsum, st, kind, dcut, t0, W, kc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_generate(const double* X, int64_t n, int m, double t, int64_t N, float* Zf,
                            double* Zd, double* rowsum, DevStatus* st, cudaStream_t s, int kind, double tiny_arg,
                            double kc) {
  if (Zf && Zd)
    return launch_gen_t<true, true, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, nullptr, kind, tiny_arg, 0, -1, kc);
  if (Zf) return launch_gen_t<true, false, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, nullptr, kind, INFINITY, 0, -1, kc);
  if (Zd)
    return launch_gen_t<false, true, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, nullptr, kind, tiny_arg, 0, -1, kc);
  return cudaErrorInvalidValue;
}

cudaError_t launch_generate_dist(const double* X, int64_t n, int m, double t, int64_t N, float* Zf,
                                 double* Zd, double* Dd, double* rowsum, DevStatus* st, cudaStream_t s,
                                 int kind, double tiny_arg, double kc) {
  if (Zf && Zd)
    return launch_gen_t<true, true, true, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, Dd, kind, tiny_arg, 0, -1, kc);
  if (Zf) return launch_gen_t<true, false, true, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, Dd, kind, INFINITY, 0, -1, kc);
  if (Zd)
    return launch_gen_t<false, true, true, true>(X, n, m, t, N, Zf, Zd, rowsum, st, s, Dd, kind, tiny_arg, 0, -1, kc);
  return cudaErrorInvalidValue;
}

cudaError_t launch_generate_q(const long long* Xq, const double* X, int64_t n, int m, int L, int e, double tau2,
                              double t, int64_t N, float* Zf, double* Zd, double* rowsum, DevStatus* st,
                              cudaStream_t s, int kind, double tiny_arg, double kc, int64_t t0, int64_t W) {
  if (m < 1 || m > GEN_MC) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)TILE * GEN_MC * sizeof(long long);
  const QuantParams qp{L, e, tau2};
  // N: tile rows of the (slab) matrix from global tile t0; W < 0: all columns
  if (W < 0) W = N;
  const int64_t tiles = num_slab_tiles(N, W);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const double dcut = tiny_arg / t;
  cudaError_t err;
  if (Zf && Zd) {
    err = cudaFuncSetAttribute(k_generate_q<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_generate_q<true, true><<<(unsigned)tiles, GEN_THREADS, smem, s>>>(Xq, X, n, m, qp, t, Zf, Zd, rowsum, st,
                                                                         kind, dcut, kc, t0, W);
  } else if (Zf) {
    err = cudaFuncSetAttribute(k_generate_q<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_generate_q<true, false><<<(unsigned)tiles, GEN_THREADS, smem, s>>>(Xq, X, n, m, qp, t, Zf, Zd, rowsum, st,
                                                                          kind, INFINITY, kc, t0, W);
  } else if (Zd) {
    err = cudaFuncSetAttribute(k_generate_q<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_generate_q<false, true><<<(unsigned)tiles, GEN_THREADS, smem, s>>>(Xq, X, n, m, qp, t, Zf, Zd, rowsum, st,
                                                                          kind, dcut, kc, t0, W);
  } else {
    return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_coord_range(const double* X, int64_t n, int m, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out + 2 * m, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_coord_range<<<m, 1024, 0, s>>>(X, n, m, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_quantize(const double* X, int64_t n, int m, const double* range, int e, long long* Xq,
                            cudaStream_t s) {
  const int64_t k = n * m;
  k_quantize<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(X, n, m, range, e, Xq);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dist_q(const long long* Xq, const double* X, int64_t n, int m, int L, int e, double tau2,
                          int64_t N, double* Dd, DevStatus* st, cudaStream_t s) {
  if (m < 1 || m > GEN_MC) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)TILE * GEN_MC * sizeof(long long);
  const QuantParams qp{L, e, tau2};
  const int64_t tiles = num_lower_tiles(N);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t err;
  if (m <= 8) {
    err = cudaFuncSetAttribute(k_dist_q<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_dist_q<true><<<(unsigned)tiles, GEN_THREADS, smem, s>>>(Xq, X, n, m, qp, Dd, st);
  } else {
    err = cudaFuncSetAttribute(k_dist_q<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_dist_q<false><<<(unsigned)tiles, GEN_THREADS, smem, s>>>(Xq, X, n, m, qp, Dd, st);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_generate_from_dist(const double* Dd, int64_t n, double t, int64_t N, float* Zf, double* Zd,
                                     double* rowsum, cudaStream_t s, int kind, double tiny_arg, double kc) {
  const unsigned tiles = (unsigned)num_lower_tiles(N);
  const double dcut = tiny_arg / t;
  if (Zf && Zd)
    k_generate_from_dist<true, true><<<tiles, 256, 0, s>>>(Dd, n, t, Zf, Zd, rowsum, kind, dcut, kc);
  else if (Zf)
    k_generate_from_dist<true, false><<<tiles, 256, 0, s>>>(Dd, n, t, Zf, Zd, rowsum, kind, INFINITY, kc);
  else if (Zd)
    k_generate_from_dist<false, true><<<tiles, 256, 0, s>>>(Dd, n, t, Zf, Zd, rowsum, kind, dcut, kc);
  else
    return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_generate_slab(const double* X, int64_t n, int m, double t, int64_t t0, int64_t W, float* Zf,
                                 DevStatus* st, cudaStream_t s, double tiny_arg, const long long* Xq, int qL, int qe,
                                 double qtau2) {
  const int64_t N = (n + TILE - 1) / TILE;
  if (t0 < 0 || t0 >= N || W < 1) return cudaErrorInvalidValue;
  if (Xq)
    return launch_generate_q(Xq, X, n, m, qL, qe, qtau2, t, N - t0, Zf, nullptr, nullptr, st, s, MAT_EXP, tiny_arg,
                             0.0, t0, W);
  return launch_gen_t<true, false, false>(X, n, m, t, N - t0, Zf, nullptr, nullptr, st, s, nullptr, MAT_EXP,
                                          tiny_arg, t0, W);
}

cudaError_t launch_min_distance(const double* X, int64_t n, int m, DevStatus* st, cudaStream_t s) {
  const int64_t N = (n + TILE - 1) / TILE;
  return launch_gen_t<false, false, false>(X, n, m, 1.0, N, nullptr, nullptr, nullptr, st, s);
}

cudaError_t launch_far_from_first(const double* X, int64_t n, int m, DevStatus* st, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_far_from_first<<<blocks, 256, 0, s>>>(X, n, m, st);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rowsum_max(const double* rowsum, int64_t n, DevStatus* st, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  k_rowsum_max<<<blocks, 256, 0, s>>>(rowsum, n, st);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mag
