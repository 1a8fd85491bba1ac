// K3: block forward/back substitution with the packed Cholesky factor in one
// persistent (cooperative) launch each.
//
//   forward : L y = v,   y_I = inv(L_II) (v_I - sum_{J<I} L_IJ y_J)
//   backward: L^T x = y, x_I = inv(L_II)^T (y_I - sum_{J>I} L_JI^T x_J)
//
// CTA b owns the row tiles I = b, b + G, ... (ascending for the forward
// sweep, descending for the backward one).  Tiles finish strictly in sweep
// order (tile I needs its predecessor), so one progress counter -- the number
// of finished tiles, raised with release semantics by the owner of each tile
// after its values are in global memory -- tells every consumer which right-
// hand sides are ready.  A CTA re-reads the counter (acquire) only when it
// reaches a tile beyond the last value it saw, so the products with long-
// finished tiles stream without a round trip per tile.  While it waits it
// prefetches its rows of the next tile into L2; the inverse of its own
// diagonal block is staged in shared memory (cp.async) meanwhile, so the
// critical path per tile is one tile product, one reduction and one
// shared-memory GEMV.
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
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Warp-level wait for *progress >= target (lane 0 spins, every lane then
// acquires once so its own later loads are ordered after the publication).
// Returns the value seen, or 0 if the wait gave up (deadline or abort).  The
// deadline and the CTA's abort flag are checked when a wait starts and then
// every 64 reads, so a wait that begins after the deadline gives up at once.
__device__ __forceinline__ unsigned warp_wait_progress(const unsigned* progress, unsigned target,
                                                       uint64_t deadline, int* abort_flag) {
  unsigned seen = 0;
  if ((threadIdx.x & 31) == 0) {
    uint32_t it = 0;
    while ((seen = ld_acquire(progress)) < target) {
      if ((it++ & 63u) == 0 && (*(volatile int*)abort_flag || gtimer() > deadline)) {
        seen = 0;
        *(volatile int*)abort_flag = 1;
        break;
      }
    }
  }
  seen = __shfl_sync(0xffffffffu, seen, 0);
  if (seen) (void)ld_acquire(progress);
  return seen;
}

// Stage one TILE x TILE block of T into shared memory (asynchronous).
template <typename T>
__device__ __forceinline__ void stage_tile(T* sdst, const T* gsrc) {
  constexpr int CHUNKS = TILE_ELEMS * (int)sizeof(T) / 16;
  for (int e = threadIdx.x; e < CHUNKS; e += TS_THREADS)
    cp_async16(reinterpret_cast<char*>(sdst) + 16 * e, reinterpret_cast<const char*>(gsrc) + 16 * e);
  cp_async_commit();
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_16a;
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
__device__ __forceinline__ double4_16a ldv_cg<double>(const double* p) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  return make_double4_16a(a.x, a.y, b.x, b.y);
}

// Forward: thread (warp w, lane l) covers tile rows w*32 + i, columns 4l..4l+3.
template <typename T>
__global__ void __launch_bounds__(TS_THREADS, 1) k_forward_persistent(const T* __restrict__ Z,
                                                                      const T* __restrict__ DinvT, int64_t N,
                                                                      const T* __restrict__ v, T* __restrict__ y,
                                                                      unsigned* progress, DevStatus* st,
                                                                      uint64_t timeout_ns, int prefetch) {
  extern __shared__ __align__(16) unsigned char ts_smem[];
  T* Ds = reinterpret_cast<T*>(ts_smem);  // inv(L_II)^T
  __shared__ T accs[TILE];
  __shared__ T rhs[TILE];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  unsigned known = 0;  // finished tiles this warp has seen
  for (int64_t I = blockIdx.x; I < N; I += gridDim.x) {
    stage_tile(Ds, DinvT + I * TILE_ELEMS);
    T part[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) part[i] = T(0);
    for (int64_t J = 0; J < I; ++J) {
      const T* tile = Z + tri_index(I, J) * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
      if ((unsigned)J >= known) {
        if (prefetch) {
#pragma unroll 4
          for (int i = 0; i < 32; ++i) prefetch_l2(tile + (int64_t)i * TILE);
        }
        known = warp_wait_progress(progress, (unsigned)J + 1u, deadline, &abort_flag);
        if (!known) break;
      }
      const auto yj = ldv_cg<T>(y + J * TILE + 4 * l);
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
    cp_async_wait_all();
    __syncthreads();
    rhs[tid] = v[I * TILE + tid] - accs[tid];
    __syncthreads();
    T s = T(0);
#pragma unroll 8
    for (int c = 0; c < TILE; ++c) s += Ds[c * TILE + tid] * rhs[c];  // (inv(L_II) rhs)[tid]
    y[I * TILE + tid] = s;
    __syncthreads();  // y_I stored; Ds and rhs free for the next tile
    if (tid == 0) {
      __threadfence();
      st_release(progress, (unsigned)(I + 1));
    }
  }
  if (tid == 0 && abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

// Backward: thread (warp w, lane l) covers tile rows w*32 + i, columns 4l..4l+3
// of the tiles L_JI (J > I); the four warps' column sums are combined in
// shared memory.  Tile J is finished once N - J tiles are.
template <typename T>
__global__ void __launch_bounds__(TS_THREADS, 1) k_backward_persistent(const T* __restrict__ Z,
                                                                       const T* __restrict__ Dinv, int64_t N,
                                                                       const T* __restrict__ yv, T* __restrict__ x,
                                                                       unsigned* progress, DevStatus* st,
                                                                       uint64_t timeout_ns, int prefetch) {
  extern __shared__ __align__(16) unsigned char ts_smem[];
  T* Ds = reinterpret_cast<T*>(ts_smem);  // inv(L_II)
  __shared__ T accw[4][TILE];
  __shared__ T rhs[TILE];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  unsigned known = 0;
  // descending ownership: CTA b takes I = N-1-b, N-1-b-G, ...
  for (int64_t I = N - 1 - blockIdx.x; I >= 0; I -= gridDim.x) {
    stage_tile(Ds, Dinv + I * TILE_ELEMS);
    T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
    for (int64_t J = N - 1; J > I; --J) {
      const T* tile = Z + tri_index(J, I) * TILE_ELEMS + (int64_t)(w * 32) * TILE + 4 * l;
      const unsigned need = (unsigned)(N - J);
      if (need > known) {
        if (prefetch) {
#pragma unroll 4
          for (int i = 0; i < 32; ++i) prefetch_l2(tile + (int64_t)i * TILE);
        }
        known = warp_wait_progress(progress, need, deadline, &abort_flag);
        if (!known) break;
      }
      // lane l holds x_J[32 w + l]; row i's value comes by shuffle
      const T xl = __ldcg(x + J * TILE + w * 32 + l);
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const auto a = ldv<T>(tile + (int64_t)i * TILE);
        const T xi = __shfl_sync(0xffffffffu, xl, i);
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
    cp_async_wait_all();
    __syncthreads();
    rhs[tid] = yv[I * TILE + tid] - (accw[0][tid] + accw[1][tid] + accw[2][tid] + accw[3][tid]);
    __syncthreads();
    T s = T(0);
#pragma unroll 8
    for (int r = 0; r < TILE; ++r) s += Ds[r * TILE + tid] * rhs[r];  // (inv(L_II)^T rhs)[tid]
    x[I * TILE + tid] = s;
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(progress, (unsigned)(N - I));
    }
  }
  if (tid == 0 && abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

template <typename K>
int coop_grid(K kern, int64_t N, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, TS_THREADS, smem);
  int64_t g = (int64_t)sms * (per > 0 ? per : 1);
  if (g > N) g = N;
  return (int)g;
}

template <typename T, typename K>
cudaError_t launch_sweep(K kern, const T* Z, const T* D, int64_t N, const T* in, T* out, unsigned* progress,
                         DevStatus* st, uint64_t timeout, cudaStream_t s, int prefetch = 1) {
  cudaError_t e = cudaMemsetAsync(progress, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)TILE_ELEMS * sizeof(T);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = coop_grid(kern, N, smem);
  void* args[] = {(void*)&Z, (void*)&D, (void*)&N, (void*)&in, (void*)&out, (void*)&progress, (void*)&st,
                  (void*)&timeout, (void*)&prefetch};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(TS_THREADS), args, smem, s);
  note_launch();
  return e;
}

}  // namespace

template <typename T>
cudaError_t launch_forward_persistent(const T* Z, const T* Dinv, int64_t N, const T* v, T* y, unsigned* flags,
                                      DevStatus* st, uint64_t timeout_ns, cudaStream_t s) {
  return launch_sweep<T>(k_forward_persistent<T>, Z, Dinv + N * TILE_ELEMS, N, v, y, flags, st, timeout_ns, s);
}

template <typename T>
cudaError_t launch_backward_persistent(const T* Z, const T* Dinv, int64_t N, const T* yv, T* x, unsigned* flags,
                                       DevStatus* st, uint64_t timeout_ns, cudaStream_t s) {
  return launch_sweep<T>(k_backward_persistent<T>, Z, Dinv, N, yv, x, flags, st, timeout_ns, s);
}

template <typename T>
cudaError_t launch_forward_sweep(const T* Z, const T* DinvT, int64_t N, const T* v, T* y, unsigned* progress,
                                 DevStatus* st, uint64_t timeout_ns, bool z_on_host, cudaStream_t s) {
  return launch_sweep<T>(k_forward_persistent<T>, Z, DinvT, N, v, y, progress, st, timeout_ns, s, z_on_host ? 0 : 1);
}

template <typename T>
cudaError_t launch_backward_sweep(const T* Z, const T* Dinv, int64_t N, const T* yv, T* x, unsigned* progress,
                                  DevStatus* st, uint64_t timeout_ns, bool z_on_host, cudaStream_t s) {
  return launch_sweep<T>(k_backward_persistent<T>, Z, Dinv, N, yv, x, progress, st, timeout_ns, s, z_on_host ? 0 : 1);
}

template cudaError_t launch_forward_sweep<float>(const float*, const float*, int64_t, const float*, float*,
                                                 unsigned*, DevStatus*, uint64_t, bool, cudaStream_t);
template cudaError_t launch_backward_sweep<float>(const float*, const float*, int64_t, const float*, float*,
                                                  unsigned*, DevStatus*, uint64_t, bool, cudaStream_t);

template cudaError_t launch_forward_persistent<float>(const float*, const float*, int64_t, const float*, float*,
                                                      unsigned*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_forward_persistent<double>(const double*, const double*, int64_t, const double*,
                                                       double*, unsigned*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_backward_persistent<float>(const float*, const float*, int64_t, const float*, float*,
                                                       unsigned*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_backward_persistent<double>(const double*, const double*, int64_t, const double*,
                                                        double*, unsigned*, DevStatus*, uint64_t, cudaStream_t);

}  // namespace mag
