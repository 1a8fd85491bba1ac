// K3, in-core form: block forward and backward substitution with the packed
// Cholesky factor, with the tile-to-tile dependency reduced to one 128 x 128
// product per tile.
//
//   forward : L y = v,    y_I = inv(L_II) (v_I - sum_{J<I} L_IJ y_J)
//             = a_I - B_I y_{I-1},        B_I  = inv(L_II) L_{I,I-1},
//               a_I = inv(L_II) (v_I - sum_{J<I-1} L_IJ y_J)
//   backward: L^T x = y,  x_I = inv(L_II)^T (y_I - sum_{J>I} L_JI^T x_J)
//             = a_I - B'_I x_{I+1},       B'_I = inv(L_II)^T L_{I+1,I}^T
//
// Tile I becomes ready only once tile I-1 (I+1) is, so a sweep is a chain of
// N steps.  Here the step is: wait for the 128 values of the previous tile,
// one product with B_I (held in registers), one store.  a_I, which needs
// the tiles up to I-2 only, is formed meanwhile from the row's tile products
// (the bulk of the bytes) and one product with inv(L_II).  The B_I of a
// factor are formed once (k_chain_prep) and serve every sweep with it.
//
// Readiness travels with the data: before a sweep the output vector holds a
// signalling-NaN pattern that no arithmetic produces, each value is stored
// once (relaxed), and a consumer re-reads a value until it differs from the
// pattern.  Every wait is bounded (%globaltimer deadline); on expiry the
// kernel raises ST_TIMEOUT, stops waiting (the results are then invalid) and
// still stores values, so no other block waits past the deadline either.
// Waits only go to lower (forward) or higher (backward) tiles, each block
// takes its tiles in sweep order and the launch is cooperative, so the
// lowest unfinished tile always has a running block that can finish it.
//
// The off-diagonal tiles are read as FP32 (the factor itself) or as FP16
// (the 2^12-scaled FP16 copy the panel solve of the one-product factor
// writes: the operands its updates used); products accumulate in FP32.
#include <cuda_fp16.h>

#include "mag_internal.cuh"

namespace mag {

namespace {

constexpr int CH_THREADS = 256;
constexpr unsigned kUnset = 0x7FA5A5A5u;  // a signalling NaN: never the result of arithmetic

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool unset(float x) { return __float_as_uint(x) == kUnset; }
__device__ __forceinline__ float ld_volatile(const float* p) {
  float v;
  asm volatile("ld.volatile.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage one FP32 TILE x TILE block into shared memory (asynchronous).
__device__ __forceinline__ void stage_tile(float* sdst, const float* gsrc) {
  constexpr int CHUNKS = TILE_ELEMS * (int)sizeof(float) / 16;
  for (int e = threadIdx.x; e < CHUNKS; e += CH_THREADS)
    cp_async16(reinterpret_cast<char*>(sdst) + 16 * e, reinterpret_cast<const char*>(gsrc) + 16 * e);
  cp_async_commit();
}

// Re-read *p until it is set; the deadline and the block's abort flag are
// checked every 64 reads.  Returns 0 once the wait gave up.
__device__ __noinline__ float spin_value(const float* p, uint64_t deadline, int* abort_flag) {
  uint32_t it = 0;
  for (;;) {
    const float v = ld_volatile(p);
    if (!unset(v)) return v;
    if ((it++ & 63u) == 0 && (*(volatile int*)abort_flag || gtimer() > deadline)) {
      *(volatile int*)abort_flag = 1;
      return 0.0f;
    }
  }
}
__device__ __forceinline__ float wait_value(const float* p, uint64_t deadline, int* abort_flag) {
  const float v = __ldcg(p);
  return unset(v) ? spin_value(p, deadline, abort_flag) : v;
}
__device__ __forceinline__ float4 wait_value4(const float* p, uint64_t deadline, int* abort_flag) {
  float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  if (unset(v.x)) v.x = spin_value(p, deadline, abort_flag);
  if (unset(v.y)) v.y = spin_value(p + 1, deadline, abort_flag);
  if (unset(v.z)) v.z = spin_value(p + 2, deadline, abort_flag);
  if (unset(v.w)) v.w = spin_value(p + 3, deadline, abort_flag);
  return v;
}

// Four consecutive tile entries as FP32.
template <typename TL>
struct Row4;
template <>
struct Row4<float> {
  using raw = float4;
  static __device__ __forceinline__ raw load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ float4 cvt(raw r) { return r; }
};
template <>
struct Row4<__half> {
  using raw = uint2;
  static __device__ __forceinline__ raw load(const __half* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
  static __device__ __forceinline__ float4 cvt(raw r) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

// The rows of B (forward: B_I^T, backward: B'_I^T, both [c][t] row-major)
// that thread (t, h) needs: entries (64 h + c, t), c < 64.
__device__ __forceinline__ void load_b(const float* __restrict__ S, int t, int h, float* b) {
#pragma unroll
  for (int c = 0; c < 64; ++c) b[c] = __ldg(S + (int64_t)(64 * h + c) * TILE + t);
}

// Shared state of one block.
struct ChainSmem {
  float red[TILE];      // row (forward) / column (backward) sums of the streamed tiles
  float rhs[TILE];
  float prev[TILE];     // the previous tile's values
  float pa[2][TILE];    // halves of inv(L_II) rhs
  float pq[2][TILE];    // halves of B prev
  float accw[CH_THREADS / 32][TILE];  // backward: the warps' column sums
  int abort_flag;
};

// Warp w streams tile rows 16 w + i (i < 16), lane l columns 4 l .. 4 l + 3.
template <typename TL>
__global__ void __launch_bounds__(CH_THREADS, 1)
    k_fwd_chain(const TL* __restrict__ Lt, float lscale, const float* __restrict__ DinvT,
                const float* __restrict__ Sf, int64_t N, float* __restrict__ v, float* __restrict__ y,
                DevStatus* st, uint64_t timeout_ns) {
  extern __shared__ __align__(16) unsigned char ch_smem[];
  float* D = reinterpret_cast<float*>(ch_smem);  // inv(L_II)^T
  __shared__ ChainSmem sh;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31, t = tid & (TILE - 1), h = tid >> 7;
  if (tid == 0) sh.abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  using R4 = Row4<TL>;
  for (int64_t I = blockIdx.x; I < N; I += gridDim.x) {
    stage_tile(D, DinvT + I * TILE_ELEMS);
    float part[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) part[i] = 0.0f;
    const TL* row = Lt + tri_index(I, 0) * TILE_ELEMS + (int64_t)(16 * w) * TILE + 4 * l;
    for (int64_t J = 0; J + 1 < I; ++J) {
      const TL* tile = row + J * TILE_ELEMS;
      typename R4::raw a[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] = R4::load(tile + i * TILE);
      const float4 yj = wait_value4(y + J * TILE + 4 * l, deadline, &sh.abort_flag);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float4 x = R4::cvt(a[i]);
        part[i] = fmaf(x.x, yj.x, fmaf(x.y, yj.y, fmaf(x.z, yj.z, fmaf(x.w, yj.w, part[i]))));
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float s = part[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == i) sh.red[16 * w + i] = s;
    }
    float b[64];
    if (I > 0) load_b(Sf + I * TILE_ELEMS, t, h, b);
    cp_async_wait_all();
    __syncthreads();
    if (tid < TILE) {
      const int64_t g = I * TILE + tid;
      sh.rhs[tid] = v[g] - lscale * sh.red[tid];
      v[g] = __uint_as_float(kUnset);  // v receives the backward sweep's output next
    }
    __syncthreads();
    {
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 8
      for (int c = 64 * h; c < 64 * h + 64; c += 2) {
        s0 = fmaf(D[c * TILE + t], sh.rhs[c], s0);
        s1 = fmaf(D[(c + 1) * TILE + t], sh.rhs[c + 1], s1);
      }
      sh.pa[h][t] = s0 + s1;
    }
    if (I > 0 && tid < TILE) sh.prev[tid] = wait_value(y + (I - 1) * TILE + tid, deadline, &sh.abort_flag);
    __syncthreads();
    if (I > 0) {
      float q0 = 0.0f, q1 = 0.0f;
#pragma unroll
      for (int c = 0; c < 64; c += 2) {
        q0 = fmaf(b[c], sh.prev[64 * h + c], q0);
        q1 = fmaf(b[c + 1], sh.prev[64 * h + c + 1], q1);
      }
      sh.pq[h][t] = q0 + q1;
    } else {
      sh.pq[h][t] = 0.0f;
    }
    __syncthreads();
    if (tid < TILE) st_relaxed(y + I * TILE + tid, (sh.pa[0][tid] + sh.pa[1][tid]) - (sh.pq[0][tid] + sh.pq[1][tid]));
    __syncthreads();  // D, rhs and prev are rewritten for the next tile
  }
  if (tid == 0 && sh.abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

// Warp w streams rows 16 w + i (i < 16) of the tiles L_JI, lane l columns
// 4 l .. 4 l + 3; x_J[16 w + i] comes from lane i by shuffle.
template <typename TL>
__global__ void __launch_bounds__(CH_THREADS, 1)
    k_bwd_chain(const TL* __restrict__ Lt, float lscale, const float* __restrict__ Dinv,
                const float* __restrict__ Sb, int64_t N, const float* __restrict__ yv, float* __restrict__ x,
                DevStatus* st, uint64_t timeout_ns) {
  extern __shared__ __align__(16) unsigned char ch_smem[];
  float* D = reinterpret_cast<float*>(ch_smem);  // inv(L_II)
  __shared__ ChainSmem sh;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31, t = tid & (TILE - 1), h = tid >> 7;
  if (tid == 0) sh.abort_flag = 0;
  __syncthreads();
  const uint64_t deadline = gtimer() + timeout_ns;
  using R4 = Row4<TL>;
  for (int64_t I = N - 1 - blockIdx.x; I >= 0; I -= gridDim.x) {
    stage_tile(D, Dinv + I * TILE_ELEMS);
    float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
    for (int64_t J = N - 1; J > I + 1; --J) {
      const TL* tile = Lt + tri_index(J, I) * TILE_ELEMS + (int64_t)(16 * w) * TILE + 4 * l;
      typename R4::raw a[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] = R4::load(tile + i * TILE);
      const float xl = l < 16 ? wait_value(x + J * TILE + 16 * w + l, deadline, &sh.abort_flag) : 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float4 q = R4::cvt(a[i]);
        const float xi = __shfl_sync(0xffffffffu, xl, i);
        p0 = fmaf(q.x, xi, p0);
        p1 = fmaf(q.y, xi, p1);
        p2 = fmaf(q.z, xi, p2);
        p3 = fmaf(q.w, xi, p3);
      }
    }
    *reinterpret_cast<float4*>(&sh.accw[w][4 * l]) = make_float4(p0, p1, p2, p3);
    float b[64];
    if (I + 1 < N) load_b(Sb + I * TILE_ELEMS, t, h, b);
    cp_async_wait_all();
    __syncthreads();
    if (tid < TILE) {
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < CH_THREADS / 32; ++k) s += sh.accw[k][tid];
      sh.rhs[tid] = yv[I * TILE + tid] - lscale * s;
    }
    __syncthreads();
    {
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 8
      for (int r = 64 * h; r < 64 * h + 64; r += 2) {
        s0 = fmaf(D[r * TILE + t], sh.rhs[r], s0);
        s1 = fmaf(D[(r + 1) * TILE + t], sh.rhs[r + 1], s1);
      }
      sh.pa[h][t] = s0 + s1;
    }
    if (I + 1 < N && tid < TILE) sh.prev[tid] = wait_value(x + (I + 1) * TILE + tid, deadline, &sh.abort_flag);
    __syncthreads();
    if (I + 1 < N) {
      float q0 = 0.0f, q1 = 0.0f;
#pragma unroll
      for (int c = 0; c < 64; c += 2) {
        q0 = fmaf(b[c], sh.prev[64 * h + c], q0);
        q1 = fmaf(b[c + 1], sh.prev[64 * h + c + 1], q1);
      }
      sh.pq[h][t] = q0 + q1;
    } else {
      sh.pq[h][t] = 0.0f;
    }
    __syncthreads();
    if (tid < TILE) st_relaxed(x + I * TILE + tid, (sh.pa[0][tid] + sh.pa[1][tid]) - (sh.pq[0][tid] + sh.pq[1][tid]));
    __syncthreads();
  }
  if (tid == 0 && sh.abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
}

// B tiles of a factor, as the sweeps read them ([c][t] row-major):
//   block q <  N - 1, I = q + 1:  Sf_I = L_{I,I-1}^T inv(L_II)^T   (= B_I^T)
//   block q >= N - 1, I = q - N + 1:  Sb_I = L_{I+1,I} inv(L_II)  (= B'_I^T)
// C = op(A) B with A, B row-major FP32 tiles, in FP32 on the CUDA cores:
// K in chunks of 32 through shared memory, 8 x 8 outputs per thread.
constexpr int PREP_KC = 32;
constexpr int PREP_LD = TILE + 4;

__global__ void __launch_bounds__(256) k_chain_prep(const float* __restrict__ Z, const float* __restrict__ Dinv,
                                                    int64_t N, float* __restrict__ Sf, float* __restrict__ Sb) {
  __shared__ __align__(16) float As[PREP_KC][PREP_LD];  // op(A)^T chunk: As[k][c] = op(A)[c][k]
  __shared__ __align__(16) float Bs[PREP_KC][TILE];     // B chunk: Bs[k][t]
  const int64_t q = blockIdx.x;
  const bool fwd = q < N - 1;
  const int64_t I = fwd ? q + 1 : q - (N - 1);
  const float* A = Z + (fwd ? tri_index(I, I - 1) : tri_index(I + 1, I)) * TILE_ELEMS;
  const float* B = Dinv + (fwd ? (N + I) : I) * TILE_ELEMS;  // inv(L_II)^T or inv(L_II)
  float* C = (fwd ? Sf : Sb) + I * TILE_ELEMS;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < TILE; k0 += PREP_KC) {
    for (int e = tid; e < PREP_KC * TILE; e += 256) {
      const int k = e / TILE, c = e % TILE;
      Bs[k][c] = B[(int64_t)(k0 + k) * TILE + c];
      // forward: op(A) = A^T, op(A)[c][k] = A[k][c] (row k0 + k, coalesced);
      // backward: op(A)[c][k] = A[c][k] (column read, 32 k per row)
      if (fwd) {
        As[k][c] = A[(int64_t)(k0 + k) * TILE + c];
      } else {
        const int cc = e / PREP_KC, kk = e % PREP_KC;
        As[kk][cc] = A[(int64_t)cc * TILE + k0 + kk];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < PREP_KC; ++k) {
      float a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[k][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[k][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) C[(int64_t)(ty * 8 + i) * TILE + tx * 8 + j] = acc[i][j];
}

__global__ void k_scale_rhs_unset(const double* __restrict__ r, int64_t n, int64_t np, float* __restrict__ v,
                                  float* __restrict__ y, const DevStatus* st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double rm = __longlong_as_double((long long)st->r_max_bits);
  const double inv = rm > 0.0 ? 1.0 / rm : 0.0;
  v[i] = i < n ? (float)(r[i] * inv) : 0.0f;
  y[i] = __uint_as_float(kUnset);
}

template <typename K>
cudaError_t launch_chain(K kern, int64_t N, void** args, cudaStream_t s) {
  const size_t smem = (size_t)TILE_ELEMS * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, CH_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const int64_t grid = std::min<int64_t>((int64_t)sms * per, N);
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(CH_THREADS), args, smem, s);
  note_launch();
  return e;
}

}  // namespace

cudaError_t launch_chain_prep(const float* Z, const float* Dinv, int64_t N, float* Sf, float* Sb, cudaStream_t s) {
  if (N < 2) return cudaSuccess;
  k_chain_prep<<<(unsigned)(2 * (N - 1)), 256, 0, s>>>(Z, Dinv, N, Sf, Sb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_rhs_unset(const double* r, int64_t n, int64_t np, float* v, float* y, const DevStatus* st,
                                   cudaStream_t s) {
  k_scale_rhs_unset<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(r, n, np, v, y, st);
  note_launch();
  return cudaGetLastError();
}

template <typename TL>
cudaError_t launch_forward_chain(const TL* Lt, float lscale, const float* Dinv, const float* Sf, int64_t N, float* v,
                                 float* y, DevStatus* st, uint64_t timeout_ns, cudaStream_t s) {
  const float* DinvT = Dinv + N * TILE_ELEMS;
  void* args[] = {(void*)&Lt, (void*)&lscale, (void*)&DinvT, (void*)&Sf, (void*)&N, (void*)&v, (void*)&y,
                  (void*)&st, (void*)&timeout_ns};
  return launch_chain(k_fwd_chain<TL>, N, args, s);
}

template <typename TL>
cudaError_t launch_backward_chain(const TL* Lt, float lscale, const float* Dinv, const float* Sb, int64_t N,
                                  const float* y, float* x, DevStatus* st, uint64_t timeout_ns, cudaStream_t s) {
  void* args[] = {(void*)&Lt, (void*)&lscale, (void*)&Dinv, (void*)&Sb, (void*)&N, (void*)&y, (void*)&x,
                  (void*)&st, (void*)&timeout_ns};
  return launch_chain(k_bwd_chain<TL>, N, args, s);
}

template cudaError_t launch_forward_chain<float>(const float*, float, const float*, const float*, int64_t, float*,
                                                 float*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_forward_chain<__half>(const __half*, float, const float*, const float*, int64_t, float*,
                                                  float*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_backward_chain<float>(const float*, float, const float*, const float*, int64_t,
                                                  const float*, float*, DevStatus*, uint64_t, cudaStream_t);
template cudaError_t launch_backward_chain<__half>(const __half*, float, const float*, const float*, int64_t,
                                                   const float*, float*, DevStatus*, uint64_t, cudaStream_t);

}  // namespace mag
