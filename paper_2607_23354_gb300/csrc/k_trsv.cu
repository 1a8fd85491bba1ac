// K3: block forward/back substitution with the packed Cholesky factor in one
// persistent (cooperative) launch each.
//
//   forward : L y = v,   y_I = inv(L_II) (v_I - sum_{J<I} L_IJ y_J)
//   backward: L^T x = y, x_I = inv(L_II)^T (y_I - sum_{J>I} L_JI^T x_J)
//
// CTA b owns the row tiles I = b, b + G, ... (ascending for the forward
// sweep, descending for the backward one).  Finished tiles are published
// through a per-tile flag written with release semantics after the tile's
// values are in global memory; consumers acquire the flag before reading.
// Each CTA streams the tiles it needs as soon as their right-hand sides are
// published, so the whole sweep is one launch: its critical path is N small
// GEMVs with the stored inverse of the diagonal blocks, and its bandwidth
// cost one read of the factor.
//
// Waits are bounded (%globaltimer deadline); on expiry the kernel raises
// ST_TIMEOUT and stops waiting.  The grid never exceeds the co-resident
// block count (cooperative launch), so every producer is running.
#include "mag_internal.cuh"

namespace mag {

namespace {

constexpr int TS_THREADS = 128;

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp-level wait for flags[J] == epoch (lane 0 spins, every lane then
// acquires once so its own later loads are ordered after the publication).
__device__ __forceinline__ bool warp_wait(const unsigned* flags, int64_t J, unsigned epoch, uint64_t deadline,
                                          int* abort_flag) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    uint32_t it = 0;
    while (ld_acquire(flags + J) != epoch) {
      if ((++it & 63u) == 0 && (*(volatile int*)abort_flag || gtimer() > deadline)) {
        ok = 0;
        *(volatile int*)abort_flag = 1;
        break;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) (void)ld_acquire(flags + J);
  return ok != 0;
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4;
};

template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ldv(const T* p) {
  return *reinterpret_cast<const typename Vec4<T>::type*>(p);
}
template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ldv_cg(const T* p);
template <>
__device__ __forceinline__ float4 ldv_cg<float>(const float* p) {
  return __ldcg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ double4 ldv_cg<double>(const double* p) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

// Forward: thread (warp w, lane l) covers tile rows w*32 + i, columns 4l..4l+3.
template <typename T>
__global__ void __launch_bounds__(TS_THREADS) k_forward_persistent(const T* __restrict__ Z,
                                                                   const T* __restrict__ DinvT, int64_t N,
                                                                   const T* __restrict__ v, T* __restrict__ y,
                                                                   unsigned* flags, unsigned epoch,
                                                                   DevStatus* st, uint64_t timeout_ns) {
  __shared__ T accs[TILE];
  __shared__ T rhs[TILE];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  for (int64_t I = blockIdx.x; I < N; I += gridDim.x) {
    T part[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) part[i] = T(0);
    for (int64_t J = 0; J < I; ++J) {
      if (!warp_wait(flags, J, epoch, deadline, &abort_flag)) break;
      const auto yj = ldv_cg<T>(y + J * TILE + 4 * l);
      const T* tile = Z + tri_index(I, J) * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const auto a = ldv<T>(tile + (int64_t)i * TILE);
        part[i] += a.x * yj.x + a.y * yj.y + a.z * yj.z + a.w * yj.w;
      }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      T s = part[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == i) accs[w * 32 + i] = s;
    }
    __syncthreads();
    rhs[tid] = v[I * TILE + tid] - accs[tid];
    __syncthreads();
    const T* YT = DinvT + I * TILE_ELEMS;
    T s = T(0);
#pragma unroll 8
    for (int c = 0; c < TILE; ++c) s += YT[c * TILE + tid] * rhs[c];  // (inv(L_II) rhs)[tid]
    y[I * TILE + tid] = s;
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flags + I, epoch);
    }
  }
  if (tid == 0 && abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

// Backward: thread (warp w, lane l) covers tile rows w*32 + i, columns 4l..4l+3
// of the tiles L_JI (J > I); the four warps' column sums are combined in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(TS_THREADS) k_backward_persistent(const T* __restrict__ Z,
                                                                    const T* __restrict__ Dinv, int64_t N,
                                                                    const T* __restrict__ yv, T* __restrict__ x,
                                                                    unsigned* flags, unsigned epoch,
                                                                    DevStatus* st, uint64_t timeout_ns) {
  __shared__ T accw[4][TILE];
  __shared__ T rhs[TILE];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  // descending ownership: CTA b takes I = N-1-b, N-1-b-G, ...
  for (int64_t I = N - 1 - blockIdx.x; I >= 0; I -= gridDim.x) {
    T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
    for (int64_t J = N - 1; J > I; --J) {
      if (!warp_wait(flags, J, epoch, deadline, &abort_flag)) break;
      const T* tile = Z + tri_index(J, I) * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
      const T* xj = x + J * TILE + w * 32;
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const auto a = ldv<T>(tile + (int64_t)i * TILE);
        const T xi = __ldcg(xj + i);
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
    rhs[tid] = yv[I * TILE + tid] - (accw[0][tid] + accw[1][tid] + accw[2][tid] + accw[3][tid]);
    __syncthreads();
    const T* Y = Dinv + I * TILE_ELEMS;
    T s = T(0);
#pragma unroll 8
    for (int r = 0; r < TILE; ++r) s += Y[r * TILE + tid] * rhs[r];  // (inv(L_II)^T rhs)[tid]
    x[I * TILE + tid] = s;
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flags + I, epoch);
    }
  }
  if (tid == 0 && abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

template <typename K>
int coop_grid(K kern, int64_t N) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, TS_THREADS, 0);
  int64_t g = (int64_t)sms * (per > 0 ? per : 1);
  if (g > N) g = N;
  return (int)g;
}

}  // namespace

template <typename T>
cudaError_t launch_forward_persistent(const T* Z, const T* Dinv, int64_t N, const T* v, T* y, unsigned* flags,
                                      DevStatus* st, cudaStream_t s) {
  const T* DinvT = Dinv + N * TILE_ELEMS;
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)N * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  auto kern = k_forward_persistent<T>;
  const int grid = coop_grid(kern, N);
  unsigned epoch = 1;
  uint64_t timeout = 10000000000ull;
  void* args[] = {(void*)&Z, (void*)&DinvT, (void*)&N, (void*)&v, (void*)&y, (void*)&flags, (void*)&epoch,
                  (void*)&st, (void*)&timeout};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(TS_THREADS), args, 0, s);
  note_launch();
  return e;
}

template <typename T>
cudaError_t launch_backward_persistent(const T* Z, const T* Dinv, int64_t N, const T* yv, T* x, unsigned* flags,
                                       DevStatus* st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)N * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  auto kern = k_backward_persistent<T>;
  const int grid = coop_grid(kern, N);
  unsigned epoch = 1;
  uint64_t timeout = 10000000000ull;
  void* args[] = {(void*)&Z, (void*)&Dinv, (void*)&N, (void*)&yv, (void*)&x, (void*)&flags, (void*)&epoch,
                  (void*)&st, (void*)&timeout};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(TS_THREADS), args, 0, s);
  note_launch();
  return e;
}

template cudaError_t launch_forward_persistent<float>(const float*, const float*, int64_t, const float*, float*,
                                                      unsigned*, DevStatus*, cudaStream_t);
template cudaError_t launch_forward_persistent<double>(const double*, const double*, int64_t, const double*,
                                                       double*, unsigned*, DevStatus*, cudaStream_t);
template cudaError_t launch_backward_persistent<float>(const float*, const float*, int64_t, const float*, float*,
                                                       unsigned*, DevStatus*, cudaStream_t);
template cudaError_t launch_backward_persistent<double>(const double*, const double*, int64_t, const double*,
                                                        double*, unsigned*, DevStatus*, cudaStream_t);

}  // namespace mag
