// K2: blocked right-looking Cholesky Z = L L^T on packed lower tiles (Sec. 3.2:
// Z is positive definite for Euclidean d, so the factor exists; a pivot that
// is not positive is reported as the Sec. 4.2 PD-check failure, never trapped).
//
//   potrf  : one CTA factors the diagonal tile in shared memory and also forms
//            inv(L_KK) and its transpose (kept for the panel solve and for the
//            block triangular solves).
//   trsm   : panel tiles L_IK = A_IK inv(L_KK)^T as a small GEMM (in place).
//   syrk   : CUDA-core trailing update C_IJ -= sum_k L_Ik L_Jk^T over a set of
//            tiles (the tensor-core version lives in k_update_tc.cu).
//
// Also K3: block forward/back substitution with the packed factor, using the
// stored inverses of the diagonal blocks so that every step is a GEMV.
//
// All kernels are templated on the element type (float for the mixed
// precision factor, double for the FP64 factor).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "mag_internal.cuh"

namespace mag {

namespace {

template <typename T>
__device__ inline T tsqrt(T x);
template <>
__device__ inline double tsqrt<double>(double x) { return sqrt(x); }

constexpr int LDA = TILE + 1;  // padded shared-memory row stride

// ------------------------------------------------------------------ potrf
// One CTA (512 threads) per diagonal tile.  Thread (ty, tx) = (tid/32, tid%32)
// owns, in registers, the entries (r, c) with r = ty + 16 a (a < 8) and
// c = tx + 32 b (b < 4) of three 128 x 128 arrays: A (becoming L) and
// T (becoming inv(L)).  Each elimination step publishes the one column or row
// it needs through shared memory, so every step costs one barrier and a
// handful of shared loads per thread.
//
// Factor (unscaled elimination, LDL^T form):
//   step c: p = A[c][c];  A[r][cc] -= A[r][c] A[cc][c] / p  for c < cc <= r;
//   then L[r][c] = A[r][c] / sqrt(p_c), L[c][c] = sqrt(p_c).
// Inverse (right-looking sweep over rows of T = inv(L), T starts as I):
//   step k: T[i][c] -= L[i][k] T[k][c] / L[k][k]  for i > k, c <= k;
//   Y[k][c] = T[k][c] / L[k][k].
template <typename T>
__global__ void __launch_bounds__(512) k_potrf_diag(T* __restrict__ Z, T* __restrict__ Dinv,
                                                    T* __restrict__ DinvT, int64_t K, int64_t n,
                                                    DevStatus* st) {
  extern __shared__ unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);  // [TILE][LDA]: L for the inverse phase
  __shared__ T colv[TILE], rowv[TILE], ldiag[TILE], linv[TILE];
  __shared__ int skip;
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  if (tid == 0) skip = (st->flags & (ST_NOTPD | ST_NONFINITE | ST_DUPLICATE)) != 0;  // set by earlier kernels
  __syncthreads();
  if (skip) return;  // uniform across the CTA
  T* tile = Z + tri_index(K, K) * TILE_ELEMS;
  T a[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a[i][j] = tile[(ty + 16 * i) * TILE + tx + 32 * j];
  // publish column 0
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) colv[ty + 16 * i] = a[i][0];
  }
  __syncthreads();
  for (int c = 0; c < TILE - 1; ++c) {
    const T p = colv[c];
    const T pinv = p > T(0) ? T(1) / p : T(0);
    T rc[8], cc4[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) rc[i] = colv[ty + 16 * i] * pinv;
#pragma unroll
    for (int j = 0; j < 4; ++j) cc4[j] = colv[tx + 32 * j];
    if (tid == 0) ldiag[c] = p;  // pivot of step c
    __syncthreads();             // everyone has read column c
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = ty + 16 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = tx + 32 * j;
        if (r > c && cc > c && cc <= r) a[i][j] -= rc[i] * cc4[j];
      }
    }
    // publish column c + 1 (owned by tx == (c+1) % 32, b == (c+1) / 32)
    const int cn = c + 1;
    if (tx == (cn & 31)) {
      const int sel = cn >> 5;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        colv[ty + 16 * i] = sel == 0 ? a[i][0] : (sel == 1 ? a[i][1] : (sel == 2 ? a[i][2] : a[i][3]));
    }
    __syncthreads();
  }
  if (tid == 0) ldiag[TILE - 1] = colv[TILE - 1];
  __syncthreads();
  if (tid < TILE) {
    const T p = ldiag[tid];
    const bool bad = !(p > T(0));
    const T d = bad ? T(1) : tsqrt(p);
    if (bad) {
      atomicOr(&st->flags, ST_NOTPD);
      atomicMin(&st->notpd_index, (int)(K * TILE + tid + 1));
    }
    ldiag[tid] = d;
    linv[tid] = T(1) / d;
  }
  __syncthreads();
  // scale to L, write it to global memory and to shared memory (the inverse
  // phase reads its columns there), and start T = I in registers
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx + 32 * j;
      T l = T(0);
      if (c < r) l = a[i][j] * linv[c];
      else if (c == r) l = ldiag[r];
      tile[r * TILE + c] = l;
      Ls[r * LDA + c] = l;
      a[i][j] = (c == r) ? T(1) : T(0);
    }
  }
  T (&y)[8][4] = a;
  // inverse sweep: needs column k of L (shared) and row k of T each step
  for (int k = 0; k < TILE - 1; ++k) {
    __syncthreads();
    if (ty == (k & 15)) {
      const int sel = k >> 4;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T v = y[0][j];
#pragma unroll
        for (int i = 1; i < 8; ++i) v = sel == i ? y[i][j] : v;
        rowv[tx + 32 * j] = v;  // T[k][.]
      }
    }
    __syncthreads();
    const T lk = linv[k];
    T li[8], tk[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) li[i] = Ls[(ty + 16 * i) * LDA + k] * lk;
#pragma unroll
    for (int j = 0; j < 4; ++j) tk[j] = rowv[tx + 32 * j];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = ty + 16 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = tx + 32 * j;
        if (r > k && c <= k) y[i][j] -= li[i] * tk[j];
      }
    }
  }
  T* Y = Dinv + K * TILE_ELEMS;
  T* YT = DinvT + K * TILE_ELEMS;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx + 32 * j;
      const T v = c <= r ? y[i][j] * linv[r] : T(0);
      Y[r * TILE + c] = v;
      YT[c * TILE + r] = v;
    }
  }
}

// ------------------------------------------------- blocked potrf (FP32)
// The same factor and inverse for the FP32 factor, organised in 32 x 32
// blocks of the tile held in shared memory (A: the tile becoming L; Y: inv(L);
// row stride LDB = 132 floats so that rows are 16-byte aligned for float4
// loads):
//   for kb = 0..3 (o = 32 kb):
//     warp 0 factors the diagonal block A[o:o+32, o:o+32] with lane l owning
//       column l: lane c scales column c (1/sqrt of the pivot from rsqrtf)
//       and publishes it in shared memory, the lanes to its right update
//       their columns from it (broadcast float4 reads, no barrier beyond
//       __syncwarp); then it inverts the block into the diagonal block of Y,
//       lane l solving for column l of the identity right-looking in
//       registers from the published columns;
//     all warps: blocks below it, A_ib,kb <- A_ib,kb Yd_kb^T (panel solve);
//     all warps: trailing blocks A_ib,jb -= A_ib,kb A_jb,kb^T (kb < jb <= ib).
//   Off-diagonal blocks of Y by block diagonals d = ib - jb = 1, 2, 3:
//     Y_ib,jb = -Yd_ib (sum_{kb=jb}^{ib-1} L_ib,kb Y_kb,jb).
// The block products read four consecutive k per float4 (one shared-memory
// wavefront serves the warp's broadcast operand).  A non-positive pivot
// raises ST_NOTPD with its row (1-based, smallest wins) and is replaced by 1
// so the kernel finishes without NaNs.
constexpr int PB = 32;   // block edge
constexpr int LDB = 132; // shared-memory row stride (floats), 16-byte aligned rows

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

__global__ void __launch_bounds__(512, 1) k_potrf_blk(float* __restrict__ Z, float* __restrict__ Dinv,
                                                      float* __restrict__ DinvT, int64_t K, DevStatus* st) {
  extern __shared__ __align__(16) float psm[];
  float* A = psm;                // [TILE][LDB]
  float* Y = psm + TILE * LDB;   // [TILE][LDB]
  __shared__ __align__(16) float colL[PB][PB];  // finished columns of the current diagonal block
  __shared__ int skip;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) skip = (st->flags & (ST_NOTPD | ST_NONFINITE | ST_DUPLICATE)) != 0;  // set by earlier kernels
  __syncthreads();
  if (skip) return;  // uniform across the CTA
  float* tile = Z + tri_index(K, K) * TILE_ELEMS;
  for (int e = tid; e < TILE * TILE / 4; e += 512) {
    const int r = e >> 5, c = (e & 31) * 4;
    *reinterpret_cast<float4*>(A + r * LDB + c) = reinterpret_cast<const float4*>(tile)[e];
  }
  __syncthreads();

  for (int kb = 0; kb < TILE / PB; ++kb) {
    const int o = kb * PB;
    if (w == 0) {
      // lane l owns column l of the diagonal block: a[i] = A[o+i][o+l] (i >= l
      // matter; entries above the diagonal are never read and stored as 0)
      float a[PB];
#pragma unroll
      for (int i = 0; i < PB; ++i) a[i] = A[(o + i) * LDB + o + l];
#pragma unroll
      for (int c = 0; c < PB; ++c) {
        // lane c: column c is final; scale it and publish it in colL[c]
        if (l == c) {
          const float piv = a[c];
          const bool bad = !(piv > 0.f);
          if (bad) {
            atomicOr(&st->flags, ST_NOTPD);
            atomicMin(&st->notpd_index, (int)(K * TILE + o + c + 1));
          }
          const float rs = bad ? 1.f : rsqrtf(piv);
          a[c] = bad ? 1.f : piv * rs;
#pragma unroll
          for (int i = c + 1; i < PB; ++i) a[i] *= rs;
#pragma unroll
          for (int i = 0; i < PB; i += 4)
            *reinterpret_cast<float4*>(&colL[c][i]) =
                make_float4(i >= c ? a[i] : 0.f, i + 1 >= c ? a[i + 1] : 0.f, i + 2 >= c ? a[i + 2] : 0.f,
                            i + 3 >= c ? a[i + 3] : 0.f);
        }
        __syncwarp();
        // lanes l > c: A[i][l] -= L[i][c] L[l][c] (broadcast reads of column c)
        if (l > c) {
          const float llc = colL[c][l];
#pragma unroll
          for (int i4 = (c + 1) & ~3; i4 < PB; i4 += 4) {  // aligned float4 groups from row c+1
            const float4 v = *reinterpret_cast<const float4*>(&colL[c][i4]);
            const float lv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (i4 + q > c) a[i4 + q] -= lv[q] * llc;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < PB; ++i) A[(o + i) * LDB + o + l] = i >= l ? a[i] : 0.f;
      const float myinv = 1.f / colL[l][l];  // every lane its own pivot: one division per lane
      // column l of inv(L_D), right-looking: once y_k is final (scaled by
      // 1/L[k][k]), y_i -= L[i][k] y_k for i > k; L's column k is read from
      // colL by broadcast, so the dependence chain is one multiply and one
      // FMA per k
      float y[PB];
#pragma unroll
      for (int i = 0; i < PB; ++i) y[i] = i == l ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        y[k] *= __shfl_sync(0xffffffffu, myinv, k);
#pragma unroll
        for (int i4 = (k + 1) & ~3; i4 < PB; i4 += 4) {
          const float4 v = *reinterpret_cast<const float4*>(&colL[k][i4]);
          const float lv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (i4 + q > k) y[i4 + q] -= lv[q] * y[k];
        }
      }
#pragma unroll
      for (int i = 0; i < PB; ++i) Y[(o + i) * LDB + o + l] = y[i];
      __syncwarp();  // colL is rewritten by the next block's factor
    }
    __syncthreads();
    // panel solve of the blocks below: X[r][c] = sum_k A[r][o+k] Yd[c][k]
    float xb[3][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int ro = o + PB * (b + 1);
      if (ro < TILE) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = ro + w + 16 * q;
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < PB; k += 4)
            acc = dot4(*reinterpret_cast<const float4*>(A + r * LDB + o + k),
                       *reinterpret_cast<const float4*>(Y + (o + l) * LDB + o + k), acc);
          xb[b][q] = acc;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int ro = o + PB * (b + 1);
      if (ro < TILE) {
#pragma unroll
        for (int q = 0; q < 2; ++q) A[(ro + w + 16 * q) * LDB + o + l] = xb[b][q];
      }
    }
    __syncthreads();
    // trailing blocks
    for (int ib = kb + 1; ib < TILE / PB; ++ib)
      for (int jb = kb + 1; jb <= ib; ++jb) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = ib * PB + w + 16 * q, c = jb * PB + l;
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < PB; k += 4)
            acc = dot4(*reinterpret_cast<const float4*>(A + r * LDB + o + k),
                       *reinterpret_cast<const float4*>(A + c * LDB + o + k), acc);
          A[r * LDB + c] -= acc;
        }
      }
    __syncthreads();
  }

  // off-diagonal blocks of Y = inv(L), one block diagonal at a time
  for (int dd = 1; dd < TILE / PB; ++dd) {
    float tv[3][2];
#pragma unroll
    for (int jb = 0; jb < 3; ++jb) {
      const int ib = jb + dd;
      if (ib < TILE / PB) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = ib * PB + w + 16 * q, c = jb * PB + l;
          float acc = 0.f;
          for (int kb = jb; kb < ib; ++kb) {
#pragma unroll
            for (int k = 0; k < PB; k += 4) {
              const float4 lr = *reinterpret_cast<const float4*>(A + r * LDB + kb * PB + k);
              const float* yc = Y + (kb * PB + k) * LDB + c;
              acc = fmaf(lr.x, yc[0], acc);
              acc = fmaf(lr.y, yc[LDB], acc);
              acc = fmaf(lr.z, yc[2 * LDB], acc);
              acc = fmaf(lr.w, yc[3 * LDB], acc);
            }
          }
          tv[jb][q] = acc;
        }
      }
    }
#pragma unroll
    for (int jb = 0; jb < 3; ++jb) {
      const int ib = jb + dd;
      if (ib < TILE / PB) {
#pragma unroll
        for (int q = 0; q < 2; ++q) Y[(ib * PB + w + 16 * q) * LDB + jb * PB + l] = tv[jb][q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < 3; ++jb) {
      const int ib = jb + dd;
      if (ib < TILE / PB) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = ib * PB + w + 16 * q, c = jb * PB + l;
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < PB; k += 4) {
            const float4 yr = *reinterpret_cast<const float4*>(Y + r * LDB + ib * PB + k);
            const float* tc = Y + (ib * PB + k) * LDB + c;
            acc = fmaf(yr.x, tc[0], acc);
            acc = fmaf(yr.y, tc[LDB], acc);
            acc = fmaf(yr.z, tc[2 * LDB], acc);
            acc = fmaf(yr.w, tc[3 * LDB], acc);
          }
          tv[jb][q] = -acc;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < 3; ++jb) {
      const int ib = jb + dd;
      if (ib < TILE / PB) {
#pragma unroll
        for (int q = 0; q < 2; ++q) Y[(ib * PB + w + 16 * q) * LDB + jb * PB + l] = tv[jb][q];
      }
    }
    __syncthreads();
  }

  float* Yg = Dinv + K * TILE_ELEMS;
  float* YTg = DinvT + K * TILE_ELEMS;
  for (int e = tid; e < TILE * TILE; e += 512) {
    const int r = e >> 7, c = e & 127;
    tile[e] = c <= r ? A[r * LDB + c] : 0.f;
    Yg[e] = c <= r ? Y[r * LDB + c] : 0.f;
    YTg[e] = r <= c ? Y[c * LDB + r] : 0.f;
  }
}

// ------------------------------------------------- CUDA-core tile GEMM (NT)
// C (TILE x TILE) = alpha*C - sign * sum_k A_k B_k^T, A_k/B_k row-major tiles.
constexpr int KC = 16;

template <typename T, bool ASSIGN>
__device__ inline void tile_gemm_nt(T* __restrict__ C, const T* const* Ak, const T* const* Bk,
                                    int nk) {
  __shared__ T As[KC][TILE + 4];
  __shared__ T Bs[KC][TILE + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
  for (int kt = 0; kt < nk; ++kt) {
    const T* A = Ak[kt];
    const T* B = Bk[kt];
    for (int k0 = 0; k0 < TILE; k0 += KC) {
      for (int e = tid; e < TILE * KC; e += 256) {
        const int r = e / KC, k = e % KC;
        As[k][r] = A[r * TILE + k0 + k];
        Bs[k][r] = B[r * TILE + k0 + k];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        T a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = Bs[k][tx + 16 * i];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      T* p = C + (ty + 16 * i) * TILE + tx + 16 * j;
      if (ASSIGN)
        *p = acc[i][j];
      else
        *p -= acc[i][j];
    }
}

// Panel solve of column K: tiles (I, K), I = K+1+blockIdx.x.
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_col(T* __restrict__ Z, const T* __restrict__ Dinv,
                                                  int64_t K, DevStatus* st) {
  if (st->flags & (ST_NOTPD | ST_NONFINITE | ST_DUPLICATE)) return;
  const int64_t I = K + 1 + blockIdx.x;
  T* C = Z + tri_index(I, K) * TILE_ELEMS;
  const T* A[1] = {C};
  const T* B[1] = {Dinv + K * TILE_ELEMS};
  tile_gemm_nt<T, true>(C, A, B, 1);
}

// Trailing update over the trapezoid J in [j0, j1), I in [J, N): the linear
// block index enumerates columns from the right (column J has N - J tiles).
template <typename T>
__global__ void __launch_bounds__(256) k_syrk_simt(T* __restrict__ Z, int64_t N, int64_t k0,
                                                   int64_t k1, int64_t base, DevStatus* st) {
  if (st->flags & (ST_NOTPD | ST_NONFINITE | ST_DUPLICATE)) return;
  int64_t Jp, ii;
  tri_coords((int64_t)blockIdx.x + base, &Jp, &ii);
  const int64_t J = N - 1 - Jp, I = J + ii;
  constexpr int MAXK = 16;
  const T* Ak[MAXK];
  const T* Bk[MAXK];
  T* C = Z + tri_index(I, J) * TILE_ELEMS;
  for (int64_t ks = k0; ks < k1; ks += MAXK) {
    const int nk = (int)((k1 - ks) < MAXK ? (k1 - ks) : MAXK);
    for (int q = 0; q < nk; ++q) {
      Ak[q] = Z + tri_index(I, ks + q) * TILE_ELEMS;
      Bk[q] = Z + tri_index(J, ks + q) * TILE_ELEMS;
    }
    tile_gemm_nt<T, false>(C, Ak, Bk, nk);
    __syncthreads();
  }
}

// ------------------------------------------------------ triangular solves
// Forward step J: y_J = inv(L_JJ) v_J (all CTAs, redundantly), CTA 0 stores
// it in y; CTA b > 0 updates v_I -= L_IJ y_J for I = J + b.
template <typename T>
__global__ void __launch_bounds__(128) k_forward_step(const T* __restrict__ Z,
                                                      const T* __restrict__ DinvT, int64_t J,
                                                      T* __restrict__ v, T* __restrict__ y) {
  __shared__ T ys[TILE];
  const int r = threadIdx.x;
  const T* YT = DinvT + J * TILE_ELEMS;
  const T* vJ = v + J * TILE;
  T s = T(0);
  for (int c = 0; c <= TILE - 1; ++c) s += YT[c * TILE + r] * vJ[c];  // Y[r][c] = YT[c][r]
  ys[r] = s;
  __syncthreads();
  if (blockIdx.x == 0) {
    y[J * TILE + r] = s;
    return;
  }
  const int64_t I = J + blockIdx.x;
  const T* L = Z + tri_index(I, J) * TILE_ELEMS;
  const int warp = r >> 5, lane = r & 31;
  for (int rr = warp; rr < TILE; rr += 4) {
    const T* row = L + rr * TILE;
    T p = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) p += row[lane + 32 * q] * ys[lane + 32 * q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) v[I * TILE + rr] -= p;
  }
}

// Backward step J: x_J = inv(L_JJ)^T v_J (all CTAs), CTA 0 stores it in x;
// CTA b > 0 updates v_I -= L_JI^T x_J for I = J - b.
template <typename T>
__global__ void __launch_bounds__(128) k_backward_step(const T* __restrict__ Z,
                                                       const T* __restrict__ Dinv, int64_t J,
                                                       T* __restrict__ v, T* __restrict__ x) {
  __shared__ T xs[TILE];
  const int c = threadIdx.x;
  const T* Y = Dinv + J * TILE_ELEMS;
  const T* vJ = v + J * TILE;
  T s = T(0);
  for (int r = 0; r < TILE; ++r) s += Y[r * TILE + c] * vJ[r];  // (Y^T v)[c]
  xs[c] = s;
  __syncthreads();
  if (blockIdx.x == 0) {
    x[J * TILE + c] = s;
    return;
  }
  const int64_t I = J - blockIdx.x;
  const T* L = Z + tri_index(J, I) * TILE_ELEMS;
  T p = T(0);
  for (int r = 0; r < TILE; ++r) p += L[r * TILE + c] * xs[r];
  v[I * TILE + c] -= p;
}

template <typename T>
__global__ void k_unpack(const T* __restrict__ Z, int64_t n, int symmetric, T* __restrict__ out) {
  const int64_t r = blockIdx.y;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = r >= c ? r : c, b = r >= c ? c : r;  // lower-triangle coordinates
    T v = Z[tri_index(a / TILE, b / TILE) * TILE_ELEMS + (a % TILE) * TILE + (b % TILE)];
    if (r < c && !symmetric) v = T(0);
    out[r * n + c] = v;
  }
}

// Panel copy of tile column K for the tensor-core update (one CTA per tile).
__global__ void __launch_bounds__(256) k_split_col(const float* __restrict__ Z, int64_t K, int64_t k0,
                                                   int64_t width, int mode, void* __restrict__ hi,
                                                   void* __restrict__ lo) {
  const int64_t I = K + 1 + blockIdx.x;
  const float* src = Z + tri_index(I, K) * TILE_ELEMS;
  const int64_t row0 = (I - k0) * TILE, col0 = (K - k0) * TILE;
  for (int e = threadIdx.x; e < TILE * TILE / 4; e += blockDim.x) {
    const int r = e / (TILE / 4), c = (e % (TILE / 4)) * 4;
    const float4 x = reinterpret_cast<const float4*>(src)[e];
    const int64_t off = (row0 + r) * width + col0 + c;
    if (mode == UPD_BF16) {
      __nv_bfloat162 a = __floats2bfloat162_rn(x.x, x.y), b = __floats2bfloat162_rn(x.z, x.w);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(hi) + off) = u;
    } else if (mode == UPD_FP16X3 || mode == UPD_FP16) {
      const float sc = (float)(1 << FP16_SCALE_LOG2);
      const float ys[4] = {x.x * sc, x.y * sc, x.z * sc, x.w * sc};
      __half h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h[q] = __float2half_rn(ys[q]);
        l[q] = __float2half_rn(ys[q] - __half2float(h[q]));
      }
      uint2 uh, ul;
      __half2 h01 = __halves2half2(h[0], h[1]), h23 = __halves2half2(h[2], h[3]);
      __half2 l01 = __halves2half2(l[0], l[1]), l23 = __halves2half2(l[2], l[3]);
      uh.x = *reinterpret_cast<uint32_t*>(&h01);
      uh.y = *reinterpret_cast<uint32_t*>(&h23);
      ul.x = *reinterpret_cast<uint32_t*>(&l01);
      ul.y = *reinterpret_cast<uint32_t*>(&l23);
      *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(hi) + off) = uh;
      if (mode == UPD_FP16X3) *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(lo) + off) = ul;
    } else {
      float xs[4] = {x.x, x.y, x.z, x.w}, h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t hb, lb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(xs[q]));
        h[q] = __uint_as_float(hb);
        const float rem = xs[q] - h[q];
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(rem));
        l[q] = __uint_as_float(lb);
      }
      *reinterpret_cast<float4*>(reinterpret_cast<float*>(hi) + off) = make_float4(h[0], h[1], h[2], h[3]);
      if (mode == UPD_TF32X3)
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(lo) + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

}  // namespace

cudaError_t launch_split_col(const float* Z, int64_t K, int64_t N, int64_t k0, int64_t width, int mode,
                             void* hi, void* lo, cudaStream_t s) {
  if (K + 1 >= N) return cudaSuccess;
  k_split_col<<<(unsigned)(N - K - 1), 256, 0, s>>>(Z, K, k0, width, mode, hi, lo);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(const T* Z, int64_t n, int64_t N, bool symmetric, T* out, cudaStream_t s) {
  (void)N;
  if (n > 65535) return cudaErrorInvalidValue;
  const unsigned bx = (unsigned)std::min<int64_t>((n + 255) / 256, 64);
  k_unpack<T><<<dim3(bx, (unsigned)n), 256, 0, s>>>(Z, n, symmetric ? 1 : 0, out);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_potrf_diag(T* Z, T* Dinv, int64_t K, int64_t n, DevStatus* st, cudaStream_t s) {
  const int64_t N = (n + TILE - 1) / TILE;
  // Dinv holds N tiles of inv(L_KK) followed by N tiles of inv(L_KK)^T.
  if constexpr (sizeof(T) == 4) {
    const size_t smem = (size_t)2 * TILE * LDB * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_potrf_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_potrf_blk<<<1, 512, smem, s>>>(Z, Dinv, Dinv + N * TILE_ELEMS, K, st);
  } else {
    const size_t smem = (size_t)TILE * LDA * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_potrf_diag<T><<<1, 512, smem, s>>>(Z, Dinv, Dinv + N * TILE_ELEMS, K, n, st);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trsm_col(T* Z, const T* Dinv, int64_t K, int64_t N, DevStatus* st,
                            cudaStream_t s) {
  if (K + 1 >= N) return cudaSuccess;
  k_trsm_col<T><<<(unsigned)(N - K - 1), 256, 0, s>>>(Z, Dinv, K, st);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_syrk_simt(T* Z, int64_t N, int64_t k0, int64_t k1, int64_t j0, int64_t j1,
                             DevStatus* st, cudaStream_t s) {
  if (j0 >= j1 || k0 >= k1) return cudaSuccess;
  const int64_t base = (N - j1) * (N - j1 + 1) / 2;
  const int64_t count = (N - j0) * (N - j0 + 1) / 2 - base;
  k_syrk_simt<T><<<(unsigned)count, 256, 0, s>>>(Z, N, k0, k1, base, st);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward(const T* Z, const T* Dinv, int64_t N, T* v, T* y, cudaStream_t s) {
  const T* DinvT = Dinv + N * TILE_ELEMS;
  for (int64_t J = 0; J < N; ++J) {
    k_forward_step<T><<<(unsigned)(N - J), TILE, 0, s>>>(Z, DinvT, J, v, y);
    note_launch();
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const T* Z, const T* Dinv, int64_t N, T* v, T* x, cudaStream_t s) {
  for (int64_t J = N - 1; J >= 0; --J) {
    k_backward_step<T><<<(unsigned)(J + 1), TILE, 0, s>>>(Z, Dinv, J, v, x);
    note_launch();
  }
  return cudaGetLastError();
}

#define MAG_INST(T)                                                                              \
  template cudaError_t launch_potrf_diag<T>(T*, T*, int64_t, int64_t, DevStatus*, cudaStream_t); \
  template cudaError_t launch_trsm_col<T>(T*, const T*, int64_t, int64_t, DevStatus*,            \
                                          cudaStream_t);                                         \
  template cudaError_t launch_syrk_simt<T>(T*, int64_t, int64_t, int64_t, int64_t, int64_t,      \
                                           DevStatus*, cudaStream_t);                            \
  template cudaError_t launch_forward<T>(const T*, const T*, int64_t, T*, T*, cudaStream_t);     \
  template cudaError_t launch_backward<T>(const T*, const T*, int64_t, T*, T*, cudaStream_t);    \
  template cudaError_t launch_unpack<T>(const T*, int64_t, int64_t, bool, T*, cudaStream_t);
MAG_INST(float)
MAG_INST(double)
#undef MAG_INST

}  // namespace mag
