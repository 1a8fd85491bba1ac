// K2c: the Cholesky trailing update on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA).
//
//   C_IJ -= sum_{k in K-range} L_Ik L_Jk^T     for J in [j0, j1), I in [J, N)
//
// Operands come from the panel buffer P: a row-major matrix whose row block
// (I - k0) holds [L_{I,k0} | L_{I,k0+1} | ...] for the current panel, already
// split for the product kind (TF32 hi/lo pairs, TF32, or BF16).  Each CTA task
// is a 128 x 256 output block: tile (I, J) and, when it is in the trapezoid,
// tile (I, J+1) -- A = 128 rows of P (row block I), B = 256 rows of P (row
// blocks J, J+1), both K-major with the 128-byte swizzle, so one
// M=128 x N=256 MMA per K step covers both tiles.
//
// Products (FP32 accumulation in TMEM):
//   TF32X3: A_hi B_hi + A_hi B_lo + A_lo B_hi with hi = rna_tf32(x),
//           lo = rna_tf32(x - hi): about 2^-21 relative per product (the
//           split-TF32 scheme of Markidis et al., IPDPSW 2018).
//   TF32  : A_hi B_hi.        BF16: one product of BF16-rounded operands.
//   FP16X3: the split with FP16 hi/lo of the panel scaled by 2^12 (FP16 has
//           TF32's significand at twice the TF32 tensor rate; the scale keeps
//           |L| <= 1 in range and small entries normal); the epilogue
//           multiplies the accumulator by 2^-24.   FP16: A_hi B_hi of that.
//
// Structure: persistent CTAs (one per SM, 6 warps), warp-specialized:
//   warp 0     : TMA producer (one thread), S-stage shared-memory ring;
//   warp 1     : TMEM owner and MMA issuer (one thread); two 128x256 FP32
//                accumulators (all 512 TMEM columns) so the epilogue of one
//                task overlaps the MMAs of the next;
//   warps 2..5 : epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//                lanes 32*(w%4)..+31), C -= acc on the packed tiles.
// Tasks come from a host-built table in 16x16-tile super-block order (so the
// CTAs running concurrently share panel rows through L2); the producer thread
// claims the next table entry with an atomic counter of the launch and hands
// it to the MMA and epilogue roles through a small mbarrier ring.  CTAs that
// start late (their SMs busy with other streams' kernels) find the queue
// drained and exit, so a launch never waits for SMs it cannot get.
//
// Every mbarrier wait is bounded (wall-clock deadline via %globaltimer); on
// expiry the CTA raises ST_TIMEOUT, stops issuing work, drains its own TMA
// loads with a bounded wait, frees its TMEM and returns.
#include <cuda.h>

#include <cuda_fp16.h>

#include "mag_internal.cuh"

namespace mag {

namespace {

constexpr int UPD_THREADS = 192;
constexpr int A_ROWS = 128, B_ROWS = 256;
constexpr uint32_t TMEM_COLS = 512;
constexpr int SUPER = 16;  // super-block edge in tiles
constexpr int TQ = 4;      // depth of the task hand-off ring

template <int MODE>
struct ModeCfg;
template <>
struct ModeCfg<UPD_TF32X3> {  // hi/lo pairs, 3 MMAs per K step
  static constexpr int ELEM = 4;
  static constexpr bool SPLIT = true;
  static constexpr uint32_t FMT = 2;  // TF32
  static constexpr int CHUNK = 128;
};
template <>
struct ModeCfg<UPD_TF32> {
  static constexpr int ELEM = 4;
  static constexpr bool SPLIT = false;
  static constexpr uint32_t FMT = 2;
  static constexpr int CHUNK = 128;
};
template <>
struct ModeCfg<UPD_BF16> {
  static constexpr int ELEM = 2;
  static constexpr bool SPLIT = false;
  static constexpr uint32_t FMT = 1;  // BF16 (kind::f16)
  static constexpr int CHUNK = 128;
};
template <>
struct ModeCfg<UPD_FP16X3> {  // scaled FP16 hi/lo pairs, 3 MMAs per K step
  static constexpr int ELEM = 2;
  static constexpr bool SPLIT = true;
  static constexpr uint32_t FMT = 0;  // F16 (kind::f16)
  static constexpr int CHUNK = 128;
};
template <>
struct ModeCfg<UPD_FP16> {
  static constexpr int ELEM = 2;
  static constexpr bool SPLIT = false;
  static constexpr uint32_t FMT = 0;
  static constexpr int CHUNK = 128;
};
// 128-byte stage rows everywhere (measured faster than 64-byte rows with twice
// the stages for the split kinds): 2 stages of 96 KB for split kinds, 4 of 48 KB
// otherwise.
template <int MODE>
constexpr int stages_of() {
  return ModeCfg<MODE>::SPLIT ? 2 : 4;
}
__host__ __device__ constexpr int chunk_bytes_of(int mode) {
  return (mode == UPD_TF32X3 || mode == UPD_FP16X3) ? 128 : 128;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with `parity` to complete.  Returns false if the
// deadline passed (then raises the CTA abort flag) or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t deadline) {
  uint32_t it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 255u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() > deadline) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// The same load into this CTA's shared memory, completing on an mbarrier of
// the peer CTA of a CTA pair (cluster address), as the pair's MMA issuer waits
// on its own barrier for both CTAs' operands.
__device__ __forceinline__ void tma_load_2d_peer_bar(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                     int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor, K-major, version 1, base offset 0:
// 128-byte rows -> SWIZZLE_128B (layout 2), 8-row groups 1024 B apart;
// 64-byte rows  -> SWIZZLE_64B (layout 4), 8-row groups 512 B apart.
template <int CHUNK>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);         // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * CHUNK) >> 4) << 32;          // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)(CHUNK == 128 ? 2 : 4) << 61;      // SWIZZLE_128B / SWIZZLE_64B
  return d;
}
// Instruction descriptor: D = F32, A/B format `fmt`, both K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(B_ROWS >> 3) << 17) |
         ((uint32_t)(A_ROWS >> 4) << 24);
}
template <int MODE>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = instr_desc(ModeCfg<MODE>::FMT);
  if constexpr (ModeCfg<MODE>::ELEM == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Bulk reduce-add of a 32 x 32 FP32 box from shared memory into global
// memory (the L2 performs the read-modify-write), tracked by bulk groups.
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap* map, uint32_t saddr, int x, int y, int z) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          (uint64_t)map),
      "r"(x), "r"(y), "r"(z), "r"(saddr)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Epilogue of one accumulator for one warp: its 32 rows (TMEM lanes of the
// warp's quadrant) of the 128 x 256 block, `nchunks` column chunks of 32
// (4: tile J only, 8: tiles J and J+1).  Each chunk is read from TMEM,
// scaled by -scale, written to a 4 KB staging box (row = lane, 16-byte chunks
// XOR-swizzled by row as the 128-byte TMA swizzle expects: no bank
// conflicts) and added to C_{Ir, J+cc/4} by the TMA; two boxes alternate.
// Returns once the TMEM reads are done and the boxes may be reused.
__device__ __forceinline__ void epilogue_reduce(const CUtensorMap* cmap, uint32_t tmem_addr, int64_t Ir, int64_t J,
                                                int64_t wcap, int nchunks, int quad, int lane, float* stg,
                                                float scale) {
  for (int cc = 0; cc < nchunks; ++cc) {
    float* sb = stg + (cc & 1) * 1024;
    if (cc >= 2) {
      if (lane == 0) bulk_wait_read<1>();  // the box of chunk cc-2 has been read
      __syncwarp();
    }
    float v[32];
    tmem_ld32(tmem_addr + cc * 32, v);
    float4* row = reinterpret_cast<float4*>(sb + lane * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      row[j ^ (lane & 7)] =
          make_float4(-scale * v[4 * j], -scale * v[4 * j + 1], -scale * v[4 * j + 2], -scale * v[4 * j + 3]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      tma_reduce_add_3d(cmap, smem_u32(sb), (cc & 3) * 32, quad * 32, (int)tile_index(Ir, J + (cc >> 2), wcap));
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_read<0>();
  __syncwarp();
}

// Task q -> output block (I, J) from the task table.
__device__ __forceinline__ void decode_task(int64_t q, const UpdParams& p, int64_t* I, int64_t* J) {
  const uint32_t v = __ldg(p.tasks + q);
  *I = (int64_t)(v >> 16);
  *J = (int64_t)(v & 0xFFFFu);
}

template <int MODE>
__global__ void __launch_bounds__(UPD_THREADS, 1)
    k_update_tc(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mB_hi,
                const __grid_constant__ CUtensorMap mA_lo, const __grid_constant__ CUtensorMap mB_lo,
                const __grid_constant__ CUtensorMap mC, const UpdParams p) {
  using Cfg = ModeCfg<MODE>;
  constexpr int S = stages_of<MODE>();
  constexpr int CHUNK_BYTES = Cfg::CHUNK;                  // K bytes per stage row
  constexpr int A_BYTES = A_ROWS * CHUNK_BYTES;
  constexpr int B_BYTES = B_ROWS * CHUNK_BYTES;
  constexpr int OPS = Cfg::SPLIT ? 2 : 1;                 // hi (+ lo) copies per operand
  constexpr int STAGE_BYTES = OPS * (A_BYTES + B_BYTES);  // 48 KB
  constexpr int KSTEP_BYTES = 32;                          // K per MMA: 8 tf32 / 16 fp16
  constexpr int KSTEPS = CHUNK_BYTES / KSTEP_BYTES;        // 2 or 4
  constexpr int ELEMS_PER_CHUNK = CHUNK_BYTES / Cfg::ELEM;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], tfull_bar[2], tempty_bar[2];
  __shared__ __align__(8) uint64_t tq_full[TQ], tq_empty[TQ];
  __shared__ int64_t tq_val[TQ];  // task index, or -1 once the queue is exhausted
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);
    }
    for (int i = 0; i < TQ; ++i) {
      mbar_init(&tq_full[i], 1);
      mbar_init(&tq_empty[i], 5);  // the MMA thread + one thread per epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  const uint64_t deadline = globaltimer() + p.timeout_ns;
  const int chunk_lo = p.kc_lo * (TILE * Cfg::ELEM / CHUNK_BYTES);
  const int chunk_hi = p.kc_hi * (TILE * Cfg::ELEM / CHUNK_BYTES);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      uint32_t issued_parity[S];
      bool issued[S];
      for (int s = 0; s < S; ++s) issued[s] = false, issued_parity[s] = 0;
      bool ok = true;
      uint32_t ts = 0, tph = 0;
      int claimed = 0;
      while (ok) {
        // claim the next task and hand it to the MMA and epilogue roles (at
        // most p.max_tasks per CTA when that is set)
        if (!mbar_wait(&tq_empty[ts], tph ^ 1u, &abort_flag, deadline)) break;
        const bool capped = p.max_tasks > 0 && claimed >= p.max_tasks;
        const int64_t q = capped ? p.ntasks : (int64_t)atomicAdd(p.counter, 1u);
        ++claimed;
        const bool end = q >= p.ntasks;
        tq_val[ts] = end ? -1 : q;
        mbar_arrive(&tq_full[ts]);
        if (++ts == TQ) ts = 0, tph ^= 1u;
        if (end) break;
        int64_t I, J;
        decode_task(q, p, &I, &J);
        const int ya = (int)((I - p.k0) * TILE), yb = (int)((J - p.k0) * TILE);
        for (int c = chunk_lo; c < chunk_hi; ++c) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, deadline)) {
            ok = false;
            break;
          }
          unsigned char* sbase = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full_bar[stage], STAGE_BYTES);
          const int x = c * ELEMS_PER_CHUNK;
          tma_load_2d(sbase, &mA_hi, &full_bar[stage], x, ya);
          tma_load_2d(sbase + A_BYTES, &mB_hi, &full_bar[stage], x, yb);
          if (Cfg::SPLIT) {
            tma_load_2d(sbase + A_BYTES + B_BYTES, &mA_lo, &full_bar[stage], x, ya);
            tma_load_2d(sbase + 2 * A_BYTES + B_BYTES, &mB_lo, &full_bar[stage], x, yb);
          }
          issued[stage] = true;
          issued_parity[stage] = phase;
          if (++stage == S) stage = 0, phase ^= 1u;
        }
      }
      if (!ok) {
        // drain our own loads in flight (bounded), so no TMA lands after exit
        const uint64_t dl = globaltimer() + 200000000ull;
        for (int s = 0; s < S; ++s)
          if (issued[s])
            while (!mbar_try_wait(&full_bar[s], issued_parity[s]) && globaltimer() < dl) {
            }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
      bool ok = true;
      uint32_t ts = 0, tph = 0;
      while (ok) {
        if (!mbar_wait(&tq_full[ts], tph, &abort_flag, deadline)) break;
        const int64_t q = tq_val[ts];
        mbar_arrive(&tq_empty[ts]);
        if (++ts == TQ) ts = 0, tph ^= 1u;
        if (q < 0) break;
        if (!mbar_wait(&tempty_bar[acc], acc_phase ^ 1u, &abort_flag, deadline)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + acc * (uint32_t)B_ROWS;
        for (int c = chunk_lo; c < chunk_hi; ++c) {
          if (!mbar_wait(&full_bar[stage], phase, &abort_flag, deadline)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k) {
            const uint64_t ahi = smem_desc<CHUNK_BYTES>(sb + k * KSTEP_BYTES);
            const uint64_t bhi = smem_desc<CHUNK_BYTES>(sb + A_BYTES + k * KSTEP_BYTES);
            const uint32_t accum = (c > chunk_lo || k > 0) ? 1u : 0u;
            mma<MODE>(d, ahi, bhi, accum);
            if (Cfg::SPLIT) {
              const uint64_t alo = smem_desc<CHUNK_BYTES>(sb + A_BYTES + B_BYTES + k * KSTEP_BYTES);
              const uint64_t blo = smem_desc<CHUNK_BYTES>(sb + 2 * A_BYTES + B_BYTES + k * KSTEP_BYTES);
              mma<MODE>(d, ahi, blo, 1u);
              mma<MODE>(d, alo, bhi, 1u);
            }
          }
          mma_commit(&empty_bar[stage]);  // stage free once these MMAs have read it
          if (++stage == S) stage = 0, phase ^= 1u;
        }
        if (!ok) break;
        mma_commit(&tfull_bar[acc]);  // accumulator ready once all MMAs finished
        if (++acc == 2) acc = 0, acc_phase ^= 1u;
      }
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    float* stg = reinterpret_cast<float*>(smem + S * STAGE_BYTES + (warp - 2) * 8192);
    uint32_t acc = 0, acc_phase = 0, ts = 0, tph = 0;
    for (;;) {
      if (!mbar_wait(&tq_full[ts], tph, &abort_flag, deadline)) break;
      const int64_t q = tq_val[ts];
      __syncwarp();
      if (lane == 0) mbar_arrive(&tq_empty[ts]);
      if (++ts == TQ) ts = 0, tph ^= 1u;
      if (q < 0) break;
      int64_t I, J;
      decode_task(q, p, &I, &J);
      if (!mbar_wait(&tfull_bar[acc], acc_phase, &abort_flag, deadline)) break;
      tc_fence_after();
      const bool second = (J + 1 < p.j1) && (J + 1 <= I);
      // FP16 panels are stored scaled by 2^s, so products carry 2^(2s)
      constexpr float acc_scale =
          (MODE == UPD_FP16X3 || MODE == UPD_FP16) ? 1.0f / (float)(1u << (2 * FP16_SCALE_LOG2)) : 1.0f;
      epilogue_reduce(&mC, tmem_base + ((uint32_t)(quad * 32) << 16) + acc * (uint32_t)B_ROWS, I, J, p.wcap,
                      second ? 8 : 4, quad, lane, stg, acc_scale);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[acc]);
      if (++acc == 2) acc = 0, acc_phase ^= 1u;
    }
    if (lane == 0) bulk_wait_all();  // reduce-adds complete before the CTA ends
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(&p.st->flags, ST_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ====================================================== CTA-pair version
// The same update with tcgen05 MMAs of cta_group::2: a cluster of two CTAs on
// two SMs computes a 256 x 256 block -- rows of tile I (CTA rank 0) and tile
// I+1 (rank 1), columns of tiles J, J+1 -- as one M=256, N=256 MMA per K
// step.  Each CTA stages only its own 128 rows of A and its 128-row half of
// B (rank 0: tile J, rank 1: tile J+1); the MMA reads the peer's halves, so
// per SM the L2 -> shared-memory traffic per flop is two thirds of the single-
// CTA kernel's and the stage ring is 1.5x deeper.  Each CTA's TMEM receives
// its own 128 rows x 256 columns of the accumulator.
//
// Roles (6 warps per CTA):
//   warp 0 : TMA producer of this CTA's halves (local mbarrier); in rank 0 it
//            also claims tasks and hands them to both CTAs (remote stores +
//            remote mbarrier arrivals);
//   warp 1 : TMEM allocation (both CTAs, cta_group::2); rank 0 issues the MMAs
//            once both CTAs' stages are full; rank 1 forwards "stage full" of
//            its own loads to rank 0's barrier (so each CTA can always wait
//            for the loads it issued itself);
//   warps 2..5 : epilogue on this CTA's rows.
// MMA completion is committed to the barrier of both CTAs (multicast), the
// epilogues of both CTAs report "accumulator drained" to rank 0.
// Every wait is bounded as in the single-CTA kernel; both CTAs meet at a
// cluster barrier before TMEM is released and before either exits.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void st_remote_s64(uint32_t cluster_addr, int64_t v) {
  asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(cluster_addr), "l"(v) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                  uint64_t deadline) {
  uint32_t it = 0;
  while (!mbar_try_wait_cluster(bar, parity)) {
    if ((++it & 255u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() > deadline) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  return true;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Instruction descriptor for the pair: D = F32, M = 256, N = 256, K-major A/B.
__host__ __device__ constexpr uint32_t instr_desc2(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}
template <int MODE>
__device__ __forceinline__ void mma2(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = instr_desc2(ModeCfg<MODE>::FMT);
  if constexpr (ModeCfg<MODE>::ELEM == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
// Arrive on the barrier at this offset in both CTAs once the MMAs issued so
// far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// K chunks (128-byte rows) per stage: the one-product kinds take two, so that
// every stage hand-off carries as much MMA work as a split stage.
template <int MODE>
constexpr int chunks2_of() {
  return ModeCfg<MODE>::SPLIT ? 1 : 2;
}
template <int MODE>
constexpr int stages2_of() {
  return 3;  // x 64 KB
}
constexpr uint32_t TMEM_COLS2 = 512;  // two 128 x 256 FP32 accumulators per CTA
constexpr int NACC2 = (int)(TMEM_COLS2 / 256);

template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(UPD_THREADS, 1)
    k_update_tc2(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_lo,
                 const __grid_constant__ CUtensorMap mC, const UpdParams p) {
  using Cfg = ModeCfg<MODE>;
  constexpr int S = stages2_of<MODE>();
  constexpr int CHUNK_BYTES = Cfg::CHUNK;
  constexpr int HALF_BYTES = 128 * CHUNK_BYTES;           // 128 rows of one operand copy
  constexpr int OPS = Cfg::SPLIT ? 2 : 1;
  constexpr int CPS = chunks2_of<MODE>();
  constexpr int STAGE_BYTES = OPS * CPS * 2 * HALF_BYTES;  // A half + B half (x hi/lo or x chunks)
  constexpr int KSTEP_BYTES = 32;
  constexpr int KSTEPS = CHUNK_BYTES / KSTEP_BYTES;
  constexpr int ELEMS_PER_CHUNK = CHUNK_BYTES / Cfg::ELEM;
  // stage layout: [A_hi | B_hi | A_lo | B_lo] for the split kinds,
  // [A_c | B_c | A_c+1 | B_c+1] (two K chunks) for the one-product kinds
  constexpr int OFF_BHI = HALF_BYTES, OFF_ALO = 2 * HALF_BYTES, OFF_BLO = 3 * HALF_BYTES;
  static_assert(OPS * CPS == 2, "64 KB stages");

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // full_bar (rank 0's is used): both CTAs' loads of a stage landed
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], tfull_bar[NACC2], tempty_bar[NACC2];
  __shared__ __align__(8) uint64_t tq_full[TQ], tq_empty[TQ];
  __shared__ int64_t tq_val[TQ];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < NACC2; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 8);  // four epilogue warps of each CTA (rank 0's barrier is used)
    }
    for (int i = 0; i < TQ; ++i) {
      mbar_init(&tq_full[i], 1);
      // rank 0: its MMA thread + 4 epilogue warps + rank 1's producer and 4 epilogue warps
      mbar_init(&tq_empty[i], 10);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS2)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  const uint64_t deadline = globaltimer() + p.timeout_ns;
  // both CTAs must hold the accumulator at the same TMEM address; after an
  // earlier launch gave up waiting, this one does no work either
  if (threadIdx.x == 0) {
    const uint32_t peer = map_to_rank(smem_u32(&tmem_base_sh), rank ^ 1u);
    uint32_t other;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(peer) : "memory");
    if (other != tmem_base) {
      abort_flag = 1;
      atomicOr(&p.st->flags, ST_TIMEOUT);
    }
    if (*(volatile int*)&p.st->flags & ST_TIMEOUT) abort_flag = 1;
  }
  cluster_sync_all();  // both decisions made; the pair works only if both CTAs will
  if (threadIdx.x == 0) {
    int other;
    asm volatile("ld.shared::cluster.s32 %0, [%1];"
                 : "=r"(other)
                 : "r"(map_to_rank(smem_u32(&abort_flag), rank ^ 1u))
                 : "memory");
    if (other) abort_flag = 1;
  }
  cluster_sync_all();  // the peer has read this CTA's flag before it can change
  const bool run = abort_flag == 0;
  const int chunk_lo = p.kc_lo * (TILE * Cfg::ELEM / CHUNK_BYTES);
  const int chunk_hi = p.kc_hi * (TILE * Cfg::ELEM / CHUNK_BYTES);
  // rank-0 addresses of the shared hand-off barriers, as seen from this CTA
  const uint32_t r0_tq_empty = map_to_rank(smem_u32(&tq_empty[0]), 0);
  const uint32_t r0_tempty = map_to_rank(smem_u32(&tempty_bar[0]), 0);
  const uint32_t r0_full = map_to_rank(smem_u32(&full_bar[0]), 0);
  const uint32_t r1_tq_full = map_to_rank(smem_u32(&tq_full[0]), 1);
  const uint32_t r1_tq_val = map_to_rank(smem_u32(&tq_val[0]), 1);

  if (run && warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, ts = 0, tph = 0;
      uint32_t issued_parity[S];
      bool issued[S];
      for (int s = 0; s < S; ++s) issued[s] = false, issued_parity[s] = 0;
      bool ok = true;
      int claimed = 0;
      while (ok) {
        int64_t q;
        if (rank == 0) {
          if (!mbar_wait_cluster(&tq_empty[ts], tph ^ 1u, &abort_flag, deadline)) break;
          // at most p.max_tasks per CTA pair when that is set
          const bool capped = p.max_tasks > 0 && claimed >= p.max_tasks;
          q = capped ? -1 : (int64_t)atomicAdd(p.counter, 1u);
          ++claimed;
          if (q >= p.ntasks) q = -1;
          tq_val[ts] = q;
          st_remote_s64(r1_tq_val + ts * 8u, q);
          mbar_arrive(&tq_full[ts]);
          mbar_arrive_remote(r1_tq_full + ts * 8u);
        } else {
          if (!mbar_wait_cluster(&tq_full[ts], tph, &abort_flag, deadline)) break;
          q = tq_val[ts];
          mbar_arrive_remote(r0_tq_empty + ts * 8u);
        }
        if (++ts == TQ) ts = 0, tph ^= 1u;
        if (q < 0) break;
        int64_t I, J;
        decode_task(q, p, &I, &J);
        const int ya = (int)((I + rank - p.k0) * TILE), yb = (int)((J + rank - p.k0) * TILE);
        for (int c = chunk_lo; c < chunk_hi; c += CPS) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, deadline)) {
            ok = false;
            break;
          }
          unsigned char* sbase = smem + stage * STAGE_BYTES;
          const int x = c * ELEMS_PER_CHUNK;
          // second copy: the lo operands (split kinds) or the next K chunk
          const CUtensorMap* m2 = Cfg::SPLIT ? &m_lo : &m_hi;
          const int x2 = Cfg::SPLIT ? x : x + ELEMS_PER_CHUNK;
          if (rank == 0) {
            // rank 0's barrier counts the bytes of both CTAs' loads of this stage
            mbar_expect_tx(&full_bar[stage], 2 * STAGE_BYTES);
            tma_load_2d(sbase, &m_hi, &full_bar[stage], x, ya);
            tma_load_2d(sbase + OFF_BHI, &m_hi, &full_bar[stage], x, yb);
            tma_load_2d(sbase + OFF_ALO, m2, &full_bar[stage], x2, ya);
            tma_load_2d(sbase + OFF_BLO, m2, &full_bar[stage], x2, yb);
          } else {
            const uint32_t bar = r0_full + stage * 8u;
            tma_load_2d_peer_bar(sbase, &m_hi, bar, x, ya);
            tma_load_2d_peer_bar(sbase + OFF_BHI, &m_hi, bar, x, yb);
            tma_load_2d_peer_bar(sbase + OFF_ALO, m2, bar, x2, ya);
            tma_load_2d_peer_bar(sbase + OFF_BLO, m2, bar, x2, yb);
          }
          issued[stage] = true;
          issued_parity[stage] = phase;
          if (++stage == S) stage = 0, phase ^= 1u;
        }
      }
      if (!ok || abort_flag) {
        // wait (bounded) for this CTA's loads in flight: rank 0 on its
        // barriers; rank 1, whose loads complete on rank 0's barriers, for
        // the same bound
        const uint64_t dl = globaltimer() + 200000000ull;
        bool any = false;
        for (int s = 0; s < S; ++s) any = any || issued[s];
        if (rank == 0) {
          for (int s = 0; s < S; ++s)
            if (issued[s])
              while (!mbar_try_wait(&full_bar[s], issued_parity[s]) && globaltimer() < dl) {
              }
        } else if (any) {
          while (globaltimer() < dl) {
          }
        }
      }
    }
  } else if (run && warp == 1) {
    if (lane == 0) {
      uint32_t ts = 0, tph = 0, stage = 0, phase = 0;
      if (rank == 0) {
        // ------------------------------------------------------- MMA issuer
        uint32_t acc = 0, acc_phase = 0;
        bool ok = true;
        while (ok) {
          if (!mbar_wait_cluster(&tq_full[ts], tph, &abort_flag, deadline)) break;
          const int64_t q = tq_val[ts];
          mbar_arrive(&tq_empty[ts]);
          if (++ts == TQ) ts = 0, tph ^= 1u;
          if (q < 0) break;
          if (!mbar_wait_cluster(&tempty_bar[acc], acc_phase ^ 1u, &abort_flag, deadline)) break;
          tc_fence_after();
          const uint32_t d = tmem_base + acc * 256u;
          for (int c = chunk_lo; c < chunk_hi; c += CPS) {
            if (!mbar_wait_cluster(&full_bar[stage], phase, &abort_flag, deadline)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
            for (int k = 0; k < KSTEPS; ++k) {
              const uint64_t ahi = smem_desc<CHUNK_BYTES>(sb + k * KSTEP_BYTES);
              const uint64_t bhi = smem_desc<CHUNK_BYTES>(sb + OFF_BHI + k * KSTEP_BYTES);
              const uint32_t accum = (c > chunk_lo || k > 0) ? 1u : 0u;
              mma2<MODE>(d, ahi, bhi, accum);
              if (Cfg::SPLIT) {
                const uint64_t alo = smem_desc<CHUNK_BYTES>(sb + OFF_ALO + k * KSTEP_BYTES);
                const uint64_t blo = smem_desc<CHUNK_BYTES>(sb + OFF_BLO + k * KSTEP_BYTES);
                mma2<MODE>(d, ahi, blo, 1u);
                mma2<MODE>(d, alo, bhi, 1u);
              }
            }
            if (!Cfg::SPLIT) {
#pragma unroll
              for (int k = 0; k < KSTEPS; ++k)
                mma2<MODE>(d, smem_desc<CHUNK_BYTES>(sb + OFF_ALO + k * KSTEP_BYTES),
                           smem_desc<CHUNK_BYTES>(sb + OFF_BLO + k * KSTEP_BYTES), 1u);
            }
            mma_commit_pair(&empty_bar[stage]);  // stage of both CTAs free once read
            if (++stage == S) stage = 0, phase ^= 1u;
          }
          if (!ok) break;
          mma_commit_pair(&tfull_bar[acc]);  // both halves of the accumulator ready
          if (++acc == NACC2) acc = 0, acc_phase ^= 1u;
        }
      }
    }
  } else if (run) {
    // --------------------------------------------------------------- epilogue
    const int quad = warp & 3;
    float* stg = reinterpret_cast<float*>(smem + S * STAGE_BYTES + (warp - 2) * 8192);
    uint32_t acc = 0, acc_phase = 0, ts = 0, tph = 0;
    constexpr float acc_scale =
        (MODE == UPD_FP16X3 || MODE == UPD_FP16) ? 1.0f / (float)(1u << (2 * FP16_SCALE_LOG2)) : 1.0f;
    for (;;) {
      if (!mbar_wait_cluster(&tq_full[ts], tph, &abort_flag, deadline)) break;
      const int64_t q = tq_val[ts];
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          mbar_arrive(&tq_empty[ts]);
        else
          mbar_arrive_remote(r0_tq_empty + ts * 8u);
      }
      if (++ts == TQ) ts = 0, tph ^= 1u;
      if (q < 0) break;
      int64_t I, J;
      decode_task(q, p, &I, &J);
      const int64_t Ir = I + rank;  // this CTA's row tile
      if (!mbar_wait_cluster(&tfull_bar[acc], acc_phase, &abort_flag, deadline)) break;
      tc_fence_after();
      if (Ir < p.N) {
        // tile (Ir, J) is always in the trapezoid; (Ir, J+1) only below j1 and the diagonal
        const int nchunks = (J + 1 < p.j1 && J + 1 <= Ir) ? 8 : 4;
        epilogue_reduce(&mC, tmem_base + ((uint32_t)(quad * 32) << 16) + acc * 256u, Ir, J, p.wcap, nchunks, quad,
                        lane, stg, acc_scale);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          mbar_arrive(&tempty_bar[acc]);
        else
          mbar_arrive_remote(r0_tempty + acc * 8u);
      }
      if (++acc == NACC2) acc = 0, acc_phase ^= 1u;
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(&p.st->flags, ST_TIMEOUT);
  cluster_sync_all();  // no CTA leaves while its peer may still signal it or read its stages
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS2)
                 : "memory");
  }
}

// ------------------------------------------------------------ panel solve
// L_IK = Z_IK inv(L_KK)^T for the tiles I in (K, N) of column K on the
// tensor cores, with the panel copies of the tensor-core update written from
// the same result.  Both operands are split into FP16 hi + lo after a
// power-of-two scale per row (so that no row overflows or sinks into FP16
// subnormals whatever the size of inv(L_KK)); three products hi*hi + hi*lo +
// lo*hi with FP32 accumulation give about 2^-22 per product, the accuracy of
// the FP32 solve it replaces.  Row r of A scaled by 2^a_r and row c of B by
// 2^b_c scale the result's (r, c) by 2^(a_r + b_c), removed exactly in the
// epilogue.  Persistent CTAs (one per SM: 129 KB of shared memory) claim
// tiles from a counter; the next tile's loads run during the current MMA.
constexpr int TRSM_THREADS = 256;
constexpr uint32_t TRSM_TMEM_COLS = 128;
constexpr int TRSM_OP_BYTES = 2 * 128 * 128;  // one FP16 copy of a 128 x 128 operand: two 16 KB K chunks

// A 128-row x 128-column FP16 operand in the layout the K-major SWIZZLE_128B
// descriptors read: two chunks of 64 columns (16 KB each), row r at byte
// 128 r of its chunk, 16-byte unit u (columns 8u .. 8u + 7 of the chunk) at
// unit u ^ (r & 7).
__device__ __forceinline__ uint32_t trsm_unit_offset(int r, int u16) {
  const int chunk = u16 >> 3, u = u16 & 7;
  return (uint32_t)(chunk * 16384 + r * 128 + ((u ^ (r & 7)) << 4));
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Power-of-two exponent e with max |x| * 2^e in [2^13, 2^14): 0 for a row of
// zeros, subnormals or non-finite values.
__device__ __forceinline__ int row_scale_exp(float m) {
  const int ex = (int)((__float_as_uint(m) >> 23) & 0xffu);
  if (ex == 0 || ex == 255) return 0;
  const int e = 14 - (ex - 126);
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// 128 x 128 FP32 tile (row-major) in registers: warp w holds rows
// 2 (w + 8 i) + (lane >> 4), i = 0..7, lane & 15 holds its columns
// 8 (lane & 15) .. + 7.
__device__ __forceinline__ void trsm_load(const float* __restrict__ src, float4 (&x)[16]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = 2 * (warp + 8 * i) + (lane >> 4);
    const float4* p = reinterpret_cast<const float4*>(src + r * TILE + 8 * (lane & 15));
    x[2 * i] = __ldcg(p);
    x[2 * i + 1] = __ldcg(p + 1);
  }
}

// Split the register tile into scaled FP16 hi / lo operands and the row
// exponents.
__device__ __forceinline__ void trsm_split(const float4 (&x)[16], unsigned char* hi, unsigned char* lo, int* rexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = 2 * (warp + 8 * i) + (lane >> 4);
    const float4 a = x[2 * i], b = x[2 * i + 1];
    float m = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                    fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = row_scale_exp(m);
    const float sc = pow2f(e);
    const float v[8] = {a.x * sc, a.y * sc, a.z * sc, a.w * sc, b.x * sc, b.y * sc, b.z * sc, b.w * sc};
    __align__(16) __half h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] = __float2half_rn(v[q]);
      l[q] = __float2half_rn(v[q] - __half2float(h[q]));
    }
    const uint32_t off = trsm_unit_offset(r, lane & 15);
    *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
    if ((lane & 15) == 0) rexp[r] = e;
  }
}

__device__ __forceinline__ void mma_f16_128x128(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  // D = F32, A = B = F16, both K-major, M = 128, N = 128
  constexpr uint32_t idesc = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(TRSM_THREADS, 1)
    k_trsm_tc(float* __restrict__ Z, const float* __restrict__ Dinv, int64_t K, int64_t N, int64_t k0,
              int64_t width, int split, __half* __restrict__ phi, __half* __restrict__ plo,
              unsigned* __restrict__ counter, DevStatus* st, uint64_t timeout_ns, int64_t wcap,
              __half* __restrict__ lh) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* b_hi = smem;
  unsigned char* b_lo = smem + TRSM_OP_BYTES;
  unsigned char* a_hi = smem + 2 * TRSM_OP_BYTES;
  unsigned char* a_lo = smem + 3 * TRSM_OP_BYTES;
  float* stage = reinterpret_cast<float*>(a_hi);  // the result, once the MMA has read A
  __shared__ int aexp[TILE], bexp[TILE];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_next, s_skip, abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = N - K - 1;
  if (tid == 0) {
    s_skip = (*(volatile int*)&st->flags & (ST_NOTPD | ST_NONFINITE | ST_DUPLICATE | ST_TIMEOUT)) != 0;
    s_next = (int)atomicAdd(counter, 1u);
    abort_flag = 0;
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s_skip || s_next >= ntiles) return;  // uniform: nothing claimed, nothing allocated
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TRSM_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  float4 x[16];
  trsm_load(Dinv + K * TILE_ELEMS, x);
  trsm_split(x, b_hi, b_lo, bexp);
  int64_t tile = s_next;
  trsm_load(Z + tile_index(K + 1 + tile, K, wcap) * TILE_ELEMS, x);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint64_t deadline = globaltimer() + timeout_ns;
  uint32_t phase = 0;
  const float pscale = (float)(1 << FP16_SCALE_LOG2);
  while (tile < ntiles) {
    const int64_t I = K + 1 + tile;
    trsm_split(x, a_hi, a_lo, aexp);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) s_next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t o = c * 16384 + k * 32;
          const uint64_t ah = smem_desc<128>(smem_u32(a_hi + o)), al = smem_desc<128>(smem_u32(a_lo + o));
          const uint64_t bh = smem_desc<128>(smem_u32(b_hi + o)), bl = smem_desc<128>(smem_u32(b_lo + o));
          mma_f16_128x128(tmem, ah, bh, (c | k) != 0);
          mma_f16_128x128(tmem, ah, bl, 1u);
          mma_f16_128x128(tmem, al, bh, 1u);
        }
      }
      mma_commit(&done_bar);
    }
    const int64_t next = s_next;
    if (next < ntiles) trsm_load(Z + tile_index(K + 1 + next, K, wcap) * TILE_ELEMS, x);
    const bool waited = mbar_wait(&done_bar, phase, &abort_flag, deadline);
    phase ^= 1u;
    const bool ok = __syncthreads_and(waited ? 1 : 0) != 0;  // one decision for the whole CTA
    tc_fence_after();
    if (ok) {
      // TMEM lanes 32 (warp & 3) .. + 31 are the rows, warp >> 2 picks 64 columns
      const int r = 32 * (warp & 3) + lane, c0 = 64 * (warp >> 2);
      const float ra = pow2f(-aexp[r]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 32 * j), v);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = c0 + 32 * j + 4 * q;
          const float4 o = make_float4(v[4 * q] * ra * pow2f(-bexp[c]), v[4 * q + 1] * ra * pow2f(-bexp[c + 1]),
                                       v[4 * q + 2] * ra * pow2f(-bexp[c + 2]),
                                       v[4 * q + 3] * ra * pow2f(-bexp[c + 3]));
          reinterpret_cast<float4*>(stage + r * TILE)[(c >> 2) ^ (r & 31)] = o;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    if (!ok) break;
    // row-major write-out: warp w, rows w + 8 i; lane l, columns 4 l .. 4 l + 3
    float* out = Z + tile_index(I, K, wcap) * TILE_ELEMS;
    __half* lout = lh ? lh + tile_index(I, K, wcap) * TILE_ELEMS : nullptr;
    const int64_t prow = (I - k0) * TILE, pcol = (K - k0) * TILE + 4 * lane;
    for (int i = 0; i < 16; ++i) {
      const int r = warp + 8 * i;
      const float4 o = reinterpret_cast<const float4*>(stage + r * TILE)[lane ^ (r & 31)];
      reinterpret_cast<float4*>(out + r * TILE)[lane] = o;
      const float y[4] = {o.x * pscale, o.y * pscale, o.z * pscale, o.w * pscale};
      __align__(8) __half h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        h[q] = __float2half_rn(y[q]);
        l[q] = __float2half_rn(y[q] - __half2float(h[q]));
      }
      const int64_t off = (prow + r) * width + pcol;
      *reinterpret_cast<uint2*>(phi + off) = *reinterpret_cast<const uint2*>(h);
      if (split) *reinterpret_cast<uint2*>(plo + off) = *reinterpret_cast<const uint2*>(l);
      if (lout) *reinterpret_cast<uint2*>(lout + r * TILE + 4 * lane) = *reinterpret_cast<const uint2*>(h);
    }
    __syncthreads();
    tile = next;
  }
  if (tid == 0 && abort_flag) atomicOr(&st->flags, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TRSM_TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  }
  return fn;
}

bool encode_2d(CUtensorMap* m, const void* base, int mode, int64_t cols, int64_t rows, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  const bool bf16 = mode == UPD_BF16, f16 = mode == UPD_FP16X3 || mode == UPD_FP16;
  const int elem = (bf16 || f16) ? 2 : 4;
  const int chunk = chunk_bytes_of(mode);
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                      : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * elem)};
  cuuint32_t box[2] = {(cuuint32_t)(chunk / elem), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dt, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   chunk == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

constexpr size_t EPI_STAGING = 4 * 8192;  // two 4 KB boxes per epilogue warp

template <int MODE>
cudaError_t launch_mode(const UpdMaps& maps, const CMap& cmap, const UpdParams& p, int grid, cudaStream_t s) {
  constexpr int OPS = ModeCfg<MODE>::SPLIT ? 2 : 1;
  constexpr int CH = ModeCfg<MODE>::CHUNK;
  const size_t smem = (size_t)stages_of<MODE>() * OPS * (A_ROWS + B_ROWS) * CH + EPI_STAGING + 1024;
  auto kern = k_update_tc<MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps.m);
  const CUtensorMap* c = reinterpret_cast<const CUtensorMap*>(cmap.m);
  kern<<<grid, UPD_THREADS, smem, s>>>(m[0], m[1], m[2], m[3], *c, p);
  note_launch();
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode2(const UpdMaps& maps, const CMap& cmap, const UpdParams& p, int grid, cudaStream_t s) {
  constexpr int OPS = ModeCfg<MODE>::SPLIT ? 2 : 1;
  constexpr int CH = ModeCfg<MODE>::CHUNK;
  const size_t smem = (size_t)stages2_of<MODE>() * OPS * chunks2_of<MODE>() * 2 * 128 * CH + EPI_STAGING + 1024;
  auto kern = k_update_tc2<MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps.m);
  grid &= ~1;  // whole clusters
  if (grid < 2) grid = 2;
  const CUtensorMap* c = reinterpret_cast<const CUtensorMap*>(cmap.m);
  kern<<<grid, UPD_THREADS, smem, s>>>(m[0], m[2], *c, p);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap layout");

bool make_update_maps(UpdMaps* maps, const void* hi, const void* lo, int mode, int64_t cols, int64_t rows) {
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(maps->m);
  if (!encode_2d(&m[0], hi, mode, cols, rows, A_ROWS)) return false;
  if (!encode_2d(&m[1], hi, mode, cols, rows, B_ROWS)) return false;
  const void* l = lo ? lo : hi;
  if (!encode_2d(&m[2], l, mode, cols, rows, A_ROWS)) return false;
  if (!encode_2d(&m[3], l, mode, cols, rows, B_ROWS)) return false;
  return true;
}

bool make_c_map(CMap* map, float* Z, int64_t tiles) {
  EncodeTiledFn enc = get_encode();
  if (!enc || tiles < 1 || tiles > 0x7fffffffLL) return false;
  cuuint64_t dims[3] = {(cuuint64_t)TILE, (cuuint64_t)TILE, (cuuint64_t)tiles};
  cuuint64_t strides[2] = {(cuuint64_t)TILE * sizeof(float), (cuuint64_t)TILE_ELEMS * sizeof(float)};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map->m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Z, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t update_tasks(int64_t N, int64_t j0, int64_t j1, bool pairs, std::vector<uint32_t>* out) {
  if (j0 >= j1 || j0 >= N || N >= 65536) return 0;
  const int rstep = pairs ? 2 : 1;                    // rows of tiles per task
  const int SRB = SUPER / rstep;                      // tasks per super-block row
  const int64_t SR = (N - j0 + SUPER - 1) / SUPER;   // super-block rows
  const int64_t SC = (j1 - j0 + SUPER - 1) / SUPER;  // super-block columns
  const int64_t n_super = SR <= SC ? SR * (SR + 1) / 2 : SC * (SC + 1) / 2 + (SR - SC) * SC;
  const size_t before = out->size();
  for (int64_t sb = 0; sb < n_super; ++sb) {
    int64_t sr, sc;
    const int64_t tri = SC * (SC + 1) / 2;
    if (sb < tri) {
      tri_coords(sb, &sr, &sc);
    } else {
      sr = SC + (sb - tri) / SC;
      sc = (sb - tri) % SC;
    }
    for (int r = 0; r < SRB; ++r)
      for (int c = 0; c < SUPER / 2; ++c) {
        const int64_t I = j0 + sr * SUPER + rstep * r, J = j0 + sc * SUPER + 2 * c;
        if (I < N && J < j1 && J <= I) out->push_back((uint32_t)(I << 16) | (uint32_t)J);
      }
  }
  return (int64_t)(out->size() - before);
}

cudaError_t launch_update_tc(const UpdMaps& maps, const CMap& cmap, UpdParams p, int mode, int grid, bool pairs,
                             cudaStream_t s) {
  if (p.ntasks <= 0 || p.kc_hi <= p.kc_lo) return cudaSuccess;
  if (p.wcap <= 0) p.wcap = p.N;
  if (pairs) {
    if ((int64_t)grid > 2 * p.ntasks) grid = (int)(2 * p.ntasks);
    switch (mode) {
      case UPD_TF32X3: return launch_mode2<UPD_TF32X3>(maps, cmap, p, grid, s);
      case UPD_TF32: return launch_mode2<UPD_TF32>(maps, cmap, p, grid, s);
      case UPD_BF16: return launch_mode2<UPD_BF16>(maps, cmap, p, grid, s);
      case UPD_FP16X3: return launch_mode2<UPD_FP16X3>(maps, cmap, p, grid, s);
      case UPD_FP16: return launch_mode2<UPD_FP16>(maps, cmap, p, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if ((int64_t)grid > p.ntasks) grid = (int)p.ntasks;
  switch (mode) {
    case UPD_TF32X3: return launch_mode<UPD_TF32X3>(maps, cmap, p, grid, s);
    case UPD_TF32: return launch_mode<UPD_TF32>(maps, cmap, p, grid, s);
    case UPD_BF16: return launch_mode<UPD_BF16>(maps, cmap, p, grid, s);
    case UPD_FP16X3: return launch_mode<UPD_FP16X3>(maps, cmap, p, grid, s);
    case UPD_FP16: return launch_mode<UPD_FP16>(maps, cmap, p, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_trsm_tc(float* Z, const float* Dinv, int64_t K, int64_t N, int64_t k0, int64_t width, int mode,
                           void* hi, void* lo, unsigned* counter, DevStatus* st, int grid, cudaStream_t s,
                           int64_t wcap, void* lh) {
  if (wcap < 0) wcap = N;
  if (K >= wcap) return cudaErrorInvalidValue;
  const int64_t ntiles = N - K - 1;
  if (ntiles <= 0) return cudaSuccess;
  if (mode != UPD_FP16 && mode != UPD_FP16X3) return cudaErrorInvalidValue;
  const size_t smem = 4 * (size_t)TRSM_OP_BYTES + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_trsm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((int64_t)grid > ntiles) grid = (int)ntiles;
  if (grid < 1) grid = 1;
  k_trsm_tc<<<grid, TRSM_THREADS, smem, s>>>(Z, Dinv, K, N, k0, width, mode == UPD_FP16X3 ? 1 : 0,
                                              static_cast<__half*>(hi), static_cast<__half*>(lo), counter, st,
                                              10000000000ull, wcap,
                                              mode == UPD_FP16 ? static_cast<__half*>(lh) : nullptr);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mag
