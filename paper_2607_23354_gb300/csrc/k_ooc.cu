// Kernels of the out-of-core factor: the Cholesky factor of a matrix whose
// packed tiles do not fit in device memory is computed slab by slab (a slab =
// a range of tile columns with every row below; the slabs partition the lower
// triangle), each slab generated, updated with the finished slabs to its
// left, factored on the device and then kept in device memory or moved to
// (pinned, mapped) host memory.  These kernels read finished slabs wherever
// they live -- a device pointer or a host pointer the GPU reads over the
// CPU-GPU link -- with plain coalesced loads:
//
//   k_gather_split : the FP16 panel copies of a K chunk of a finished slab,
//                    restricted to the rows of a later slab (the operands of
//                    that slab's tensor-core update);
//   k_rect_gemv    : v -= A y over the rectangular part of a slab (the forward
//                    substitution's update of the rows below the slab);
//   k_rect_gemv_t  : y -= A^T x over the same part (the backward one).
#include <cuda_fp16.h>

#include "mag_internal.cuh"

namespace mag {

namespace {

constexpr int GS_THREADS = 256;

__global__ void __launch_bounds__(GS_THREADS) k_gather_split(const float* __restrict__ Lq, int64_t q0, int64_t Sq,
                                                             int64_t c0, int64_t k0, __half* __restrict__ hi,
                                                             __half* __restrict__ lo, int64_t width, int split) {
  const int64_t Ip = blockIdx.x;  // local tile row of the later slab
  const int k = blockIdx.y;       // tile column of the chunk
  const int64_t I = c0 + Ip, K = k0 + k;
  const float* src = Lq + tile_index(I - q0, K - q0, Sq) * TILE_ELEMS;
  const float pscale = (float)(1 << FP16_SCALE_LOG2);
  // a warp reads one 512-byte row of the tile per step and writes its 256
  // bytes of FP16 into the panel row
  for (int e = threadIdx.x; e < TILE * TILE / 4; e += GS_THREADS) {
    const int r = e >> 5, c = (e & 31) * 4;
    const float4 x = *reinterpret_cast<const float4*>(src + r * TILE + c);
    const float y[4] = {x.x * pscale, x.y * pscale, x.z * pscale, x.w * pscale};
    __align__(8) __half h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = __float2half_rn(y[q]);
      l[q] = __float2half_rn(y[q] - __half2float(h[q]));
    }
    const int64_t off = (Ip * TILE + r) * width + (int64_t)k * TILE + c;
    *reinterpret_cast<uint2*>(hi + off) = *reinterpret_cast<const uint2*>(h);
    if (split) *reinterpret_cast<uint2*>(lo + off) = *reinterpret_cast<const uint2*>(l);
  }
}

// One CTA per tile row i of the rectangle; thread (warp w, lane l) covers tile
// rows w * 32 + ii and columns 4 l .. 4 l + 3 of every tile (j) of the row.
__global__ void __launch_bounds__(128) k_rect_gemv(const float* __restrict__ A, int64_t S,
                                                   const float* __restrict__ y, float* __restrict__ v) {
  const int64_t i = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float part[32];
#pragma unroll
  for (int ii = 0; ii < 32; ++ii) part[ii] = 0.0f;
  const float* row = A + i * S * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
  for (int64_t j = 0; j < S; ++j) {
    const float* tile = row + j * TILE_ELEMS;
    const float4 yj = *reinterpret_cast<const float4*>(y + j * TILE + 4 * l);
#pragma unroll
    for (int ii = 0; ii < 32; ++ii) {
      const float4 a = *reinterpret_cast<const float4*>(tile + (int64_t)ii * TILE);
      part[ii] += a.x * yj.x + a.y * yj.y + a.z * yj.z + a.w * yj.w;
    }
  }
#pragma unroll
  for (int ii = 0; ii < 32; ++ii) {
    float sum = part[ii];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (l == ii) v[i * TILE + w * 32 + ii] -= sum;
  }
}

// One CTA per tile column j of the rectangle; thread (warp w, lane l) covers
// tile rows w * 32 + ii and columns 4 l .. 4 l + 3 of every tile (i) of the
// column; the four warps' column sums meet in shared memory.
__global__ void __launch_bounds__(128) k_rect_gemv_t(const float* __restrict__ A, int64_t R, int64_t S,
                                                     const float* __restrict__ x, float* __restrict__ y) {
  __shared__ float accw[4][TILE];
  const int64_t j = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  for (int64_t i = 0; i < R; ++i) {
    const float* tile = A + (i * S + j) * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
    const float xl = x[i * TILE + w * 32 + l];
#pragma unroll 8
    for (int ii = 0; ii < 32; ++ii) {
      const float4 a = *reinterpret_cast<const float4*>(tile + (int64_t)ii * TILE);
      const float xi = __shfl_sync(0xffffffffu, xl, ii);
      p0 += a.x * xi;
      p1 += a.y * xi;
      p2 += a.z * xi;
      p3 += a.w * xi;
    }
  }
  accw[w][4 * l + 0] = p0;
  accw[w][4 * l + 1] = p1;
  accw[w][4 * l + 2] = p2;
  accw[w][4 * l + 3] = p3;
  __syncthreads();
  const int c = threadIdx.x;
  y[j * TILE + c] -= accw[0][c] + accw[1][c] + accw[2][c] + accw[3][c];
}

}  // namespace

cudaError_t launch_gather_split(const float* Lq, int64_t q0, int64_t Sq, int64_t c0, int64_t rows, int64_t k0,
                                int kw, void* hi, void* lo, int64_t width, bool split, cudaStream_t s) {
  if (rows <= 0 || kw <= 0) return cudaSuccess;
  if (rows > 0x7fffffffLL || kw > 65535 || k0 < q0 || k0 + kw > q0 + Sq || c0 < q0 + Sq ||
      (int64_t)kw * TILE > width)
    return cudaErrorInvalidValue;
  k_gather_split<<<dim3((unsigned)rows, (unsigned)kw), GS_THREADS, 0, s>>>(
      Lq, q0, Sq, c0, k0, static_cast<__half*>(hi), static_cast<__half*>(lo), width, split ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rect_gemv(const float* A, int64_t R, int64_t S, const float* y, float* v, cudaStream_t s) {
  if (R <= 0 || S <= 0) return cudaSuccess;
  if (R > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_rect_gemv<<<(unsigned)R, 128, 0, s>>>(A, S, y, v);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rect_gemv_t(const float* A, int64_t R, int64_t S, const float* x, float* y, cudaStream_t s) {
  if (R <= 0 || S <= 0) return cudaSuccess;
  if (S > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_rect_gemv_t<<<(unsigned)S, 128, 0, s>>>(A, R, S, x, y);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mag
