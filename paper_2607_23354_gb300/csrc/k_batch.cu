// K8: many small solves (uneven point clouds x values of t) in one persistent
// launch.  Each CTA pops a problem from a global work queue (problems sorted
// by decreasing n on the host, so the largest start first) and solves it
// alone in its own global scratch:
//
//   Z  = exp(-t d)        FP64 full square (residual) + FP32 lower (factor),
//                         from FP64 distances computed once per cloud
//   Z  = L L^T            FP32 blocked right-looking Cholesky, B x B blocks
//   w  = (L L^T)^{-1} 1   FP32 blocked substitution
//   refinement            r = 1 - Z w in FP64 (compensated), w += solve(r / |r|)
//                         until |r| / (|Z| |w|) <= tol, at most max_iter steps
//   Mag = 1^T w           compensated
//
// A problem whose FP32 factor meets a non-positive pivot, or whose refinement
// stalls, is reported in its status and left to the host to re-solve with the
// single-problem path (which escalates precision).  The factor block is 64;
// the threads per CTA and the CTAs per SM (kBatchShapes) are template
// parameters, chosen per batch size class by the host-side tuner
// (mag_solve_batch).
#include <algorithm>

#include "mag_internal.cuh"
#include "mag_math.cuh"

namespace mag {

namespace {


__device__ __forceinline__ void two_sum_d(double a, double b, double* s, double* e) {
  const double x = a + b;
  const double bv = x - a;
  *e = (a - (x - bv)) + (b - bv);
  *s = x;
}

// Packed lower distances of one cloud: D[i(i-1)/2 + j] = ||x_i - x_j||, j < i.
__global__ void __launch_bounds__(256) k_batch_dist(const double* __restrict__ X, const BatchCloud* clouds,
                                                    int nclouds, double* __restrict__ D, int* cloud_flags) {
  int flags = 0;
  const BatchCloud c = clouds[blockIdx.y];
  const int64_t npairs = (int64_t)c.n * (c.n - 1) / 2;
  const double* P = X + c.point_offset;
  double* out = D + c.dist_offset;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
    while (i * (i - 1) / 2 > q) --i;
    while ((i + 1) * i / 2 <= q) ++i;
    const int64_t j = q - i * (i - 1) / 2;
    double s = 0.0;
    for (int l = 0; l < c.m; ++l) {
      const double d = P[i * c.m + l] - P[j * c.m + l];
      s = fma(d, d, s);
    }
    out[q] = sqrt_pos(s);
    if (!isfinite(s))
      flags |= 1;
    else if (s == 0.0)
      flags |= 2;
  }
  if (flags) atomicOr(cloud_flags + blockIdx.y, flags);
}

// ---------------------------------------------------------- per-CTA pieces
struct Scratch {
  float* Lf;    // n x n row-major, lower triangle used
  double* Zd;   // n x n row-major, full symmetric FP64 Z
  double* w;    // n
  double* r;    // n
  float* v;     // n (FP32 right-hand side / solution)
};

// FP32 Cholesky of the n x n lower triangle of A (row stride n) in place.
// Returns false on a non-positive pivot.
// TF32 split: hi = a rounded to TF32 (10 mantissa bits), lo = the rest
// rounded to TF32; hi*hi + hi*lo + lo*hi recovers the product to about
// 2^-22 relative.
__device__ __forceinline__ void split_tf32(float a, uint32_t* hi, uint32_t* lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
  const float rest = a - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
  *hi = h;
  *lo = l;
}

// d += a b for one m16n8k8 TF32 tile (A row-major 16 x 8, B 8 x 8 column
// fragments, FP32 accumulators; the PTX fragment layout).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// LEFT: left-looking -- before block column kb is factored, all its blocks
// (bi, kb), bi >= kb, take their whole update sum_{k < kb} L_bi,k L_kb,k^T
// in registers (block pairs of L streamed through shared memory, the next
// pair read into registers during the products), and each block of A is
// read and written once instead of once per earlier column: about two
// thirds of the block traffic of the right-looking update (CUDA cores
// only).
template <int B, int NT, bool MMA, bool LEFT>
__device__ bool cta_cholesky(float* A, int n, float* sm, int* flag) {
  static_assert(!(MMA && LEFT), "the left-looking factor runs on the CUDA cores");
  float* D = sm;                    // [B][B+1] diagonal block
  float* Pi = sm + B * (B + 1);     // [B][B+4] panel block of tile row bi (k-major)
  float* Pj = Pi + B * (B + 4);     // [B][B+4] panel block of tile row bj (k-major)
  const int tid = threadIdx.x;
  const int nb = (n + B - 1) / B;
  for (int kb = 0; kb < nb; ++kb) {
    const int k0 = kb * B, kw = min(B, n - k0);
    if constexpr (LEFT) {
      if (kb > 0) {
        constexpr int TR = 4, TC = B * B / (NT * TR), GX = B / TC;
        static_assert(TR * TC * NT == B * B && GX * TC == B && (NT / GX) * TR == B && (TC == 2 || TC == 4),
                      "thread tile of the left-looking update");
        constexpr int LT = B + 4;
        constexpr int PER = B * B / NT;
        const int ty = tid / GX, tx = tid % GX;
        float si[PER], sj[PER];
        // rows r0 .. r0 + rw - 1 of the full column block starting at column c0
        auto fetch_blk = [&](float (&stg)[PER], int r0, int rw, int c0) {
#pragma unroll
          for (int q = 0; q < PER; ++q) {
            const int e = tid + q * NT, r = e / B, c = e % B;
            stg[q] = r < rw ? A[(int64_t)(r0 + r) * n + c0 + c] : 0.0f;
          }
        };
        auto put_blk = [&](const float (&stg)[PER], float* dstT) {
#pragma unroll
          for (int q = 0; q < PER; ++q) {
            const int e = tid + q * NT, r = e / B, c = e % B;
            dstT[c * LT + r] = stg[q];
          }
        };
        for (int bi = kb; bi < nb; ++bi) {
          const int i0 = bi * B, iw = min(B, n - i0);
          const bool diag = bi == kb;
          float acc[TR][TC];
#pragma unroll
          for (int u = 0; u < TR; ++u)
#pragma unroll
            for (int v = 0; v < TC; ++v) acc[u][v] = 0.0f;
          fetch_blk(si, i0, iw, 0);
          if (!diag) fetch_blk(sj, k0, kw, 0);
          for (int k = 0; k < kb; ++k) {
            __syncthreads();  // the previous products are done with PiT / PjT
            put_blk(si, Pi);
            if (!diag) put_blk(sj, Pj);
            __syncthreads();
            if (k + 1 < kb) {  // in flight during the products below
              fetch_blk(si, i0, iw, (k + 1) * B);
              if (!diag) fetch_blk(sj, k0, kw, (k + 1) * B);
            }
            const float* QT = diag ? Pi : Pj;
#pragma unroll 8
            for (int kk = 0; kk < B; ++kk) {
              const float4 a = *reinterpret_cast<const float4*>(Pi + kk * LT + TR * ty);
              float b[TC];
              if constexpr (TC == 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(QT + kk * LT + TC * tx);
                b[0] = b4.x, b[1] = b4.y, b[2] = b4.z, b[3] = b4.w;
              } else {
                const float2 b2 = *reinterpret_cast<const float2*>(QT + kk * LT + TC * tx);
                b[0] = b2.x, b[1] = b2.y;
              }
              const float ar[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
              for (int u = 0; u < TR; ++u)
#pragma unroll
                for (int v = 0; v < TC; ++v) acc[u][v] = fmaf(ar[u], b[v], acc[u][v]);
            }
          }
#pragma unroll
          for (int u = 0; u < TR; ++u) {
            const int r = TR * ty + u;
            if (r >= iw) continue;
#pragma unroll
            for (int v = 0; v < TC; ++v) {
              const int c = TC * tx + v;
              if (c < kw && (!diag || c <= r)) A[(int64_t)(i0 + r) * n + k0 + c] -= acc[u][v];
            }
          }
        }
      }
    }
    // (a) factor the diagonal block in shared memory (unscaled elimination)
    __syncthreads();
    for (int e = tid; e < B * B; e += NT) {
      const int r = e / B, c = e % B;
      D[r * (B + 1) + c] = (r < kw && c < kw && c <= r) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0f;
    }
    __syncthreads();
    for (int c = 0; c < kw - 1; ++c) {
      const float p = D[c * (B + 1) + c];
      const float pinv = p > 0.0f ? 1.0f / p : 0.0f;
      const int w = kw - 1 - c;
      for (int e = tid; e < w * w; e += NT) {
        const int r = c + 1 + e / w, cc = c + 1 + e % w;
        if (cc <= r) D[r * (B + 1) + cc] -= D[r * (B + 1) + c] * D[cc * (B + 1) + c] * pinv;
      }
      __syncthreads();
    }
    if (tid == 0) *flag = 0;
    __syncthreads();
    if (tid < kw) {
      const float p = D[tid * (B + 1) + tid];
      if (!(p > 0.0f)) *flag = 1;
    }
    __syncthreads();
    if (*flag) return false;
    // scale: L[r][c] = D[r][c] / sqrt(p_c), L[c][c] = sqrt(p_c)
    for (int e = tid; e < kw * kw; e += NT) {
      const int r = e / kw, c = e % kw;
      if (c < r) D[r * (B + 1) + c] *= rsqrtf(D[c * (B + 1) + c]);
    }
    __syncthreads();
    if (tid < kw) D[tid * (B + 1) + tid] = sqrtf(D[tid * (B + 1) + tid]);
    __syncthreads();
    for (int e = tid; e < kw * kw; e += NT) {
      const int r = e / kw, c = e % kw;
      if (c <= r) A[(int64_t)(k0 + r) * n + k0 + c] = D[r * (B + 1) + c];
    }
    // (b) panel: rows i >= k0 + kw, x L^T = a (forward substitution per row)
    for (int i = k0 + kw + tid; i < n; i += NT) {
      float x[B];
      float* row = A + (int64_t)i * n + k0;
#pragma unroll
      for (int c = 0; c < B; ++c) x[c] = c < kw ? row[c] : 0.0f;
#pragma unroll
      for (int c = 0; c < B; ++c) {
        if (c < kw) {
          float s = x[c];
#pragma unroll
          for (int cc = 0; cc < c; ++cc) s -= x[cc] * D[c * (B + 1) + cc];
          x[c] = s / D[c * (B + 1) + c];
        }
      }
#pragma unroll
      for (int c = 0; c < B; ++c)
        if (c < kw) row[c] = x[c];
    }
    __syncthreads();
    if constexpr (LEFT) continue;  // the next column's blocks take their updates themselves
    // (c) trailing update of the lower tiles (bi, bj), kb < bj <= bi.  CUDA
    // cores (MMA false): the panel blocks are staged k-major (PiT[k][r],
    // PjT[k][c], row stride B + 4); a thread owns a TR x TC output tile (4 x 2
    // with 512 threads, 4 x 4 with 256) and takes one broadcast float4 of PiT
    // and a TC-wide vector of PjT per k.  Tensor cores (MMA true): the blocks
    // are staged row-major (row stride B + 4, so that the fragment reads
    // below are free of bank conflicts), each warp owns 16 rows x (8 NTW)
    // columns of the output and runs mma.sync m16n8k8 TF32 on split
    // operands (a = a_hi + a_lo, hi*hi + hi*lo + lo*hi: the FP32-class
    // product, error about 2^-22 of |a||b|).  Both: the next panel block is
    // read from global memory into registers while the current one is in
    // use, and the output block's entries of A are read before the products,
    // so the products hide both latencies.
    constexpr int LT = B + 4;
    constexpr int PER = B * B / NT;  // panel entries a thread stages per block
    float* PiT = Pi;  // [B][LT]
    float* PjT = Pj;  // [B][LT]
    float stage[PER];
    auto fetch = [&](int r0, int rw) {  // panel rows r0 .. r0 + rw - 1, columns k0 .. k0 + kw - 1
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = tid + q * NT, r = e / B, c = e % B;
        stage[q] = (r < rw && c < kw) ? A[(int64_t)(r0 + r) * n + k0 + c] : 0.0f;
      }
    };
    auto put = [&](float* dst) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = tid + q * NT, r = e / B, c = e % B;
        if constexpr (MMA)
          dst[r * LT + c] = stage[q];
        else
          dst[c * LT + r] = stage[q];
      }
    };
    for (int bi = kb + 1; bi < nb; ++bi) {
      const int i0 = bi * B, iw = min(B, n - i0);
      __syncthreads();
      fetch(i0, iw);
      put(PiT);
      if (kb + 1 < bi) fetch((kb + 1) * B, B);  // PjT of the first column block
      for (int bj = kb + 1; bj <= bi; ++bj) {
        const int j0 = bj * B, jw = min(B, n - j0);
        __syncthreads();
        if (bj != bi) {
          put(PjT);
          __syncthreads();
          if (bj + 1 < bi) fetch((bj + 1) * B, B);  // in flight during the products below
        }
        const float* QT = bj == bi ? PiT : PjT;
        if constexpr (MMA) {
          static_assert(B == 64 && NT % 128 == 0 && NT <= 512, "warp tiles of the tensor-core update");
          constexpr int W = NT / 32, NTW = 32 / W;  // n8 tiles per warp
          const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
          const int rw0 = 16 * (warp & 3), cw0 = (warp >> 2) * 8 * NTW;
          // the block's entries of A at the accumulator positions, read ahead
          float av[NTW][4];
#pragma unroll
          for (int j = 0; j < NTW; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int r = rw0 + g + 8 * (h >> 1), c = cw0 + 8 * j + 2 * tq + (h & 1);
              av[j][h] = (r < iw && c < jw && (bi != bj || c <= r)) ? A[(int64_t)(i0 + r) * n + j0 + c] : 0.0f;
            }
          float acc[NTW][4];
#pragma unroll
          for (int j = 0; j < NTW; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll 2
          for (int kk = 0; kk < B / 8; ++kk) {
            const int kc = 8 * kk + tq;
            const float ar[4] = {PiT[(rw0 + g) * LT + kc], PiT[(rw0 + g + 8) * LT + kc], PiT[(rw0 + g) * LT + kc + 4],
                                 PiT[(rw0 + g + 8) * LT + kc + 4]};
            uint32_t ahi[4], alo[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) split_tf32(ar[h], &ahi[h], &alo[h]);
#pragma unroll
            for (int j = 0; j < NTW; ++j) {
              const int nn = cw0 + 8 * j + g;
              uint32_t bhi[2], blo[2];
              split_tf32(QT[nn * LT + kc], &bhi[0], &blo[0]);
              split_tf32(QT[nn * LT + kc + 4], &bhi[1], &blo[1]);
              mma_tf32(acc[j], ahi, bhi);
              mma_tf32(acc[j], ahi, blo);
              mma_tf32(acc[j], alo, bhi);
            }
          }
#pragma unroll
          for (int j = 0; j < NTW; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int r = rw0 + g + 8 * (h >> 1), c = cw0 + 8 * j + 2 * tq + (h & 1);
              if (r < iw && c < jw && (bi != bj || c <= r)) A[(int64_t)(i0 + r) * n + j0 + c] = av[j][h] - acc[j][h];
            }
        } else {
          constexpr int TR = 4, TC = B * B / (NT * TR), GX = B / TC;
          static_assert(TR * TC * NT == B * B && GX * TC == B && (NT / GX) * TR == B && (TC == 2 || TC == 4),
                        "thread tile of the trailing update");
          const int ty = tid / GX, tx = tid % GX;  // rows TR ty .., columns TC tx ..
          // the block's entries of A, read ahead of the products
          float av[TR][TC];
#pragma unroll
          for (int u = 0; u < TR; ++u)
#pragma unroll
            for (int v = 0; v < TC; ++v) {
              const int r = TR * ty + u, c = TC * tx + v;
              av[u][v] = (r < iw && c < jw && (bi != bj || c <= r)) ? A[(int64_t)(i0 + r) * n + j0 + c] : 0.0f;
            }
          float acc[TR][TC];
#pragma unroll
          for (int u = 0; u < TR; ++u)
#pragma unroll
            for (int v = 0; v < TC; ++v) acc[u][v] = 0.0f;
#pragma unroll 8
          for (int k = 0; k < B; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(PiT + k * LT + TR * ty);
            float b[TC];
            if constexpr (TC == 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(QT + k * LT + TC * tx);
              b[0] = b4.x, b[1] = b4.y, b[2] = b4.z, b[3] = b4.w;
            } else {
              const float2 b2 = *reinterpret_cast<const float2*>(QT + k * LT + TC * tx);
              b[0] = b2.x, b[1] = b2.y;
            }
            const float ar[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int u = 0; u < TR; ++u)
#pragma unroll
              for (int v = 0; v < TC; ++v) acc[u][v] = fmaf(ar[u], b[v], acc[u][v]);
          }
#pragma unroll
          for (int u = 0; u < TR; ++u) {
            const int r = TR * ty + u;
            if (r >= iw) continue;
#pragma unroll
            for (int v = 0; v < TC; ++v) {
              const int c = TC * tx + v;
              if (c < jw && (bi != bj || c <= r)) A[(int64_t)(i0 + r) * n + j0 + c] = av[u][v] - acc[u][v];
            }
          }
        }
      }
    }
    __syncthreads();
  }
  return true;
}

// v <- (L L^T)^{-1} v with the FP32 factor (blocked).  The diagonal block
// solves run in warp 0 column by column: lane l holds rows l and l + 32 of the
// block's right-hand side; each step divides the pivot row, broadcasts the
// solved unknown by a shuffle and updates the lanes' remaining rows.
template <int B, int NT>
__device__ void cta_solve(const float* L, int n, float* v, float* sm) {
  static_assert(B == 64, "two rows per lane");
  float* blk = sm;                  // [B] block values
  float* Db = sm + B;               // [B][B+1] the diagonal block of L, staged
  const int tid = threadIdx.x;
  const int nb = (n + B - 1) / B;
  // the diagonal block of block row kb into shared memory (all threads), so
  // that warp 0's column-serial solve reads it at shared-memory latency
  auto stage_diag = [&](int k0, int kw) {
    for (int e = tid; e < B * B; e += NT) {
      const int r = e / B, c = e % B;
      if (r < kw && c <= r) Db[r * (B + 1) + c] = L[(int64_t)(k0 + r) * n + k0 + c];
    }
  };
  // forward: L y = v
  for (int kb = 0; kb < nb; ++kb) {
    const int k0 = kb * B, kw = min(B, n - k0);
    __syncthreads();
    stage_diag(k0, kw);
    __syncthreads();
    if (tid < 32) {
      const int r0 = tid, r1 = tid + 32;
      float y0 = r0 < kw ? v[k0 + r0] : 0.0f, y1 = r1 < kw ? v[k0 + r1] : 0.0f;
      const float* L0 = Db + r0 * (B + 1);
      const float* L1 = Db + r1 * (B + 1);
      for (int c = 0; c < kw; ++c) {
        // the owner of row c finishes it, then every lane eliminates it
        const float own = c < 32 ? y0 : y1;
        float xc = __shfl_sync(0xffffffffu, own, c & 31);
        xc /= Db[c * (B + 1) + c];
        if (r0 == c) y0 = xc;
        if (r1 == c) y1 = xc;
        if (r0 > c && r0 < kw) y0 -= L0[c] * xc;
        if (r1 > c && r1 < kw) y1 -= L1[c] * xc;
      }
      if (r0 < kw) blk[r0] = y0;
      if (r1 < kw) blk[r1] = y1;
    }
    __syncthreads();
    for (int e = tid; e < kw; e += NT) v[k0 + e] = blk[e];
    for (int i = k0 + kw + tid; i < n; i += NT) {
      const float* Li = L + (int64_t)i * n + k0;
      float s = 0.0f;
      for (int c = 0; c < kw; ++c) s += Li[c] * blk[c];
      v[i] -= s;
    }
  }
  // backward: L^T x = y
  for (int kb = nb - 1; kb >= 0; --kb) {
    const int k0 = kb * B, kw = min(B, n - k0);
    __syncthreads();
    stage_diag(k0, kw);
    __syncthreads();
    if (tid < 32) {
      const int r0 = tid, r1 = tid + 32;
      float x0 = r0 < kw ? v[k0 + r0] : 0.0f, x1 = r1 < kw ? v[k0 + r1] : 0.0f;
      for (int c = kw - 1; c >= 0; --c) {
        const float own = c < 32 ? x0 : x1;
        float xc = __shfl_sync(0xffffffffu, own, c & 31);
        const float* Lc = Db + c * (B + 1);  // row c: L[c][r] for r < c
        xc /= Lc[c];
        if (r0 == c) x0 = xc;
        if (r1 == c) x1 = xc;
        if (r0 < c) x0 -= Lc[r0] * xc;
        if (r1 < c) x1 -= Lc[r1] * xc;
      }
      if (r0 < kw) blk[r0] = x0;
      if (r1 < kw) blk[r1] = x1;
    }
    __syncthreads();
    for (int e = tid; e < kw; e += NT) v[k0 + e] = blk[e];
    // x_i -= sum_{c in block} L[k0+c][i] x_c for i < k0
    for (int i = tid; i < k0; i += NT) {
      float s = 0.0f;
      for (int c = 0; c < kw; ++c) s += L[(int64_t)(k0 + c) * n + i] * blk[c];
      v[i] -= s;
    }
  }
  __syncthreads();
}

template <int B, int NT, int MINB, bool MMA, bool LEFT>
__global__ void __launch_bounds__(NT, MINB)
    k_batch_solve(const BatchProblem* __restrict__ probs, const int* __restrict__ order, int count,
                  const double* __restrict__ D, const int* __restrict__ cloud_flags, float* scratch_f,
                  double* scratch_d, int64_t nmax,
                  double* __restrict__ w_out, double* __restrict__ mag_out, int* __restrict__ status,
                  int* queue, double tol, int max_iter, unsigned long long* busy_cycles) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_q, s_flag;
  __shared__ double red[NT / 32][3];
  __shared__ double exptab[2 * EXPT_SIZE];
  load_exp_table_d(exptab);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Scratch S;
  S.Lf = scratch_f + (int64_t)blockIdx.x * (nmax * nmax + nmax);
  S.v = S.Lf + nmax * nmax;
  S.Zd = scratch_d + (int64_t)blockIdx.x * (nmax * nmax + 2 * nmax);
  S.w = S.Zd + nmax * nmax;
  S.r = S.w + nmax;
  const long long t_start = clock64();
  for (;;) {
    __syncthreads();
    if (tid == 0) s_q = atomicAdd(queue, 1);
    __syncthreads();
    const int q = s_q;
    if (q >= count) {
      // the tuner's measure: this CTA's busy time (its SM's cycles from the
      // first problem to the last), summed over CTAs
      if (tid == 0 && busy_cycles) atomicAdd(busy_cycles, (unsigned long long)(clock64() - t_start));
      break;
    }
    const int pid = order[q];
    const BatchProblem P = probs[pid];
    const int n = P.n;
    const int cf = cloud_flags[P.cloud];
    if (cf) {  // uniform across the CTA: report and skip the problem
      if (tid == 0) {
        status[pid] = (cf & 1) ? MAG_BATCH_NONFINITE : MAG_BATCH_DUPLICATE;
        mag_out[pid] = 0.0;
      }
      continue;
    }
    const double* Dc = D + P.dist_offset;
    // ---- Z: FP64 full square and FP32 lower, one exp per pair j < i (warp
    // per row, lanes along the row), mirrored into the upper triangle; the
    // row sums of Z (for ||Z||inf) come with the first residual.  Entries
    // below e^-46 in FP32 on the FP32 pipe (exp_neg_tiny_td), as the
    // single-problem solver does.
    const unsigned long long tiny_bits = (unsigned long long)__double_as_longlong(kTinyArg / P.t);
    const float tf = (float)P.t;
    double zmax_p = 0.0;
    for (int i = warp; i < n; i += NT / 32) {
      const double* Di = Dc + (int64_t)i * (i - 1) / 2;
      for (int j = lane; j < i; j += 32) {
        const double d = Di[j];
        const double z = (unsigned long long)__double_as_longlong(d) > tiny_bits
                             ? f32_to_f64_nonneg(exp_neg_tiny_td(tf, P.t, d))
                             : exp_neg_small_d(P.t * d, exptab);
        S.Zd[(int64_t)i * n + j] = z;
        S.Zd[(int64_t)j * n + i] = z;
        S.Lf[(int64_t)i * n + j] = f64_to_f32_nonneg(z);
      }
      if (lane == 0) {
        S.Zd[(int64_t)i * n + i] = 1.0;
        S.Lf[(int64_t)i * n + i] = 1.0f;
      }
    }
    __syncthreads();
    int st = MAG_BATCH_OK;
    if (!cta_cholesky<B, NT, MMA, LEFT>(S.Lf, n, smf, &s_flag)) st = MAG_BATCH_NOTPD;
    double rel = INFINITY;
    if (st == MAG_BATCH_OK) {
      for (int i = tid; i < n; i += NT) S.v[i] = 1.0f;
      cta_solve<B, NT>(S.Lf, n, S.v, smf);
      for (int i = tid; i < n; i += NT) S.w[i] = (double)S.v[i];
      __syncthreads();
      double prev = INFINITY;
      int slow = 0;
      for (int it = 0;; ++it) {
        // r = 1 - Z w (warp per row; per lane FMA chains of 16 terms whose
        // sums are combined with Neumaier compensation, then a plain lane
        // tree: each lane total is within the chains' 16 u of its part of
        // sum |z w|, the tree adds at most 5 u -- both far below the
        // tolerance -- and GB300's FP64 pipe makes a compensated tree (8
        // FP64 operations per level) the bulk of a small row's cost)
        double rmax = 0.0, wmax = 0.0;
        for (int i = warp; i < n; i += NT / 32) {
          const double* Zi = S.Zd + (int64_t)i * n;
          double s = 0.0, c = 0.0;
          float zs = 0.0f;  // row sum of Z, first pass only (a norm: FP32 is ample)
          for (int j0 = lane; j0 < n; j0 += 32 * 16) {
            double part = 0.0;
#pragma unroll 4
            for (int q = 0; q < 16; ++q) {
              const int j = j0 + 32 * q;
              if (j < n) {
                const double z = Zi[j];
                part = fma(z, S.w[j], part);
                if (it == 0) zs += f64_to_f32_nonneg(z);  // integer pipe
              }
            }
            const double tt = s + part;
            c += fabs(s) >= fabs(part) ? (s - tt) + part : (part - tt) + s;
            s = tt;
          }
          double tot = s + c;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
          const double ri = 1.0 - tot;
          if (lane == 0) S.r[i] = ri;
          rmax = fmax(rmax, fabs(ri));
          wmax = fmax(wmax, fabs(S.w[i]));
          if (it == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, o);
            zmax_p = fmax(zmax_p, (double)zs);
          }
        }
        if (lane == 0) {
          red[warp][0] = rmax;
          red[warp][1] = zmax_p;
          red[warp][2] = wmax;
        }
        __syncthreads();
        double rn = 0.0, zn = 0.0, wn = 0.0;
        for (int k = 0; k < NT / 32; ++k) {
          rn = fmax(rn, red[k][0]);
          zn = fmax(zn, red[k][1]);
          wn = fmax(wn, red[k][2]);
        }
        rel = (zn > 0.0 && wn > 0.0) ? rn / (zn * wn) : INFINITY;
        __syncthreads();
        if (rel <= tol) break;
        if (it >= max_iter || !(rel < INFINITY) || (rel > 0.5 * prev && ++slow >= 2)) {
          st = MAG_BATCH_NOCONV;
          break;
        }
        if (!(rel > 0.5 * prev)) slow = 0;
        prev = rel;
        const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
        for (int i = tid; i < n; i += NT) S.v[i] = (float)(S.r[i] * inv);
        cta_solve<B, NT>(S.Lf, n, S.v, smf);
        for (int i = tid; i < n; i += NT) S.w[i] += rn * (double)S.v[i];
        __syncthreads();
      }
    }
    // ---- outputs: w, Mag (compensated), status
    double s = 0.0, c = 0.0;
    for (int i = tid; i < n; i += NT) {
      const double wi = S.w[i];
      w_out[P.w_offset + i] = wi;
      double hi, lo;
      two_sum_d(s, wi, &hi, &lo);
      s = hi;
      c += lo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double hi, lo;
      const double other = __shfl_xor_sync(0xffffffffu, s, o);
      const double oc = __shfl_xor_sync(0xffffffffu, c, o);
      two_sum_d(s, other, &hi, &lo);
      s = hi;
      c += oc + lo;
    }
    if (lane == 0) {
      red[warp][0] = s;
      red[warp][1] = c;
    }
    __syncthreads();
    if (tid == 0) {
      double ss = 0.0, cc = 0.0;
      for (int k = 0; k < NT / 32; ++k) {
        double hi, lo;
        two_sum_d(ss, red[k][0], &hi, &lo);
        ss = hi;
        cc += red[k][1] + lo;
      }
      mag_out[pid] = ss + cc;
      status[pid] = st;
    }
  }
}

template <int B, int NT, int MINB, bool MMA, bool LEFT>
cudaError_t launch_batch_t(const BatchProblem* probs, const int* order, int count, const double* D,
                           const int* cloud_flags, float* scratch_f, double* scratch_d, int64_t nmax,
                           double* w_out, double* mag_out, int* status, int* queue, double tol, int max_iter,
                           int grid, unsigned long long* busy_cycles, cudaStream_t s) {
  const size_t smem = ((size_t)B * (B + 1) + 2 * (size_t)B * (B + 4)) * sizeof(float);
  auto kern = k_batch_solve<B, NT, MINB, MMA, LEFT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, smem, s>>>(probs, order, count, D, cloud_flags, scratch_f, scratch_d, nmax, w_out, mag_out,
                              status, queue, tol, max_iter, busy_cycles);
  note_launch();
  return cudaGetLastError();
}

template <int B, int NT, int MINB, bool MMA, bool LEFT>
int resident_per_sm() {
  const size_t smem = ((size_t)B * (B + 1) + 2 * (size_t)B * (B + 4)) * sizeof(float);
  auto kern = k_batch_solve<B, NT, MINB, MMA, LEFT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per;
}

}  // namespace

cudaError_t launch_batch_dist(const double* X, const BatchCloud* clouds, int nclouds, int64_t max_pairs,
                              double* D, int* cloud_flags, cudaStream_t s) {
  if (nclouds <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min<int64_t>((max_pairs + 255) / 256, 256);
  k_batch_dist<<<dim3(bx > 0 ? bx : 1, (unsigned)nclouds), 256, 0, s>>>(X, clouds, nclouds, D, cloud_flags);
  note_launch();
  return cudaGetLastError();
}

// Launch shapes of the batch kernel (factor block 64): threads per CTA, the
// CTAs per SM the launch bounds are compiled for, and the trailing update on
// CUDA cores (FP32) or on the tensor cores (split TF32, mma.sync).
const BatchShape kBatchShapes[kNumBatchShapes] = {{512, 1, 0, 0}, {256, 2, 0, 0}, {256, 3, 0, 0}, {256, 2, 1, 0},
                                                  {256, 3, 1, 0}, {256, 2, 0, 1}, {256, 3, 0, 1}};

int batch_shape_resident(int shape) {
  switch (shape) {
    case 0: return resident_per_sm<64, 512, 1, false, false>();
    case 1: return resident_per_sm<64, 256, 2, false, false>();
    case 2: return resident_per_sm<64, 256, 3, false, false>();
    case 3: return resident_per_sm<64, 256, 2, true, false>();
    case 4: return resident_per_sm<64, 256, 3, true, false>();
    case 5: return resident_per_sm<64, 256, 2, false, true>();
    case 6: return resident_per_sm<64, 256, 3, false, true>();
    default: return 0;
  }
}

cudaError_t launch_batch_solve(int shape, const BatchProblem* probs, const int* order, int count,
                               const double* D, const int* cloud_flags, float* scratch_f, double* scratch_d,
                               int64_t nmax, double* w_out, double* mag_out, int* status, int* queue, double tol,
                               int max_iter, int grid, unsigned long long* busy_cycles, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
#define MAG_BATCH_LAUNCH(NT_, MINB_, MMA_, LEFT_)                                                              \
  return launch_batch_t<64, NT_, MINB_, MMA_, LEFT_>(probs, order, count, D, cloud_flags, scratch_f, scratch_d, \
                                                      nmax, w_out, mag_out, status, queue, tol, max_iter, grid,   \
                                                      busy_cycles, s)
  switch (shape) {
    case 0: MAG_BATCH_LAUNCH(512, 1, false, false);
    case 1: MAG_BATCH_LAUNCH(256, 2, false, false);
    case 2: MAG_BATCH_LAUNCH(256, 3, false, false);
    case 3: MAG_BATCH_LAUNCH(256, 2, true, false);
    case 4: MAG_BATCH_LAUNCH(256, 3, true, false);
    case 5: MAG_BATCH_LAUNCH(256, 2, false, true);
    case 6: MAG_BATCH_LAUNCH(256, 3, false, true);
    default: return cudaErrorInvalidValue;
  }
#undef MAG_BATCH_LAUNCH
}

}  // namespace mag
