// Internal declarations shared by the CUDA translation units of the magnitude
// solver.  Nothing here is part of the public C ABI (include/magnitude.h).
//
// Data layout in HBM (one solve of size n, N = ceil(n / TILE) tiles a side):
//   * Z and its Cholesky factor live in "packed lower tiles": tile (I, J) with
//     I >= J is a contiguous TILE x TILE row-major block at tile index
//     I (I + 1) / 2 + J.  Rows/columns >= n are padding and hold the identity,
//     so the factor of the padded matrix is blockdiag(L, I) and padded
//     solution entries are zero.
//   * Diagonal tiles are stored in full (both triangles) by the generator; the
//     factor keeps L in their lower triangle and zeros above.
//   * Inverses of the diagonal factor blocks, inv(L_KK), live in a separate
//     array of N full tiles (used by the panel solve and the triangular solves).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

namespace mag {

// Number of kernels enqueued by this library (all contexts), for the
// per-call kernel_launches diagnostic.
extern std::atomic<long long> g_kernel_launches;
inline void note_launch(long long k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr int TILE = 128;
constexpr int64_t TILE_ELEMS = (int64_t)TILE * TILE;

__host__ __device__ inline int64_t tri_index(int64_t I, int64_t J) { return I * (I + 1) / 2 + J; }
__host__ __device__ inline int64_t num_lower_tiles(int64_t N) { return N * (N + 1) / 2; }

// Inverse of tri_index restricted to a triangle of tiles: linear index q over
// the lower triangle {(I, J) : J <= I}, row-major by I.
__host__ __device__ inline void tri_coords(int64_t q, int64_t* I, int64_t* J) {
  int64_t i = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > q) --i;
  while ((i + 1) * (i + 2) / 2 <= q) ++i;
  *I = i;
  *J = q - i * (i + 1) / 2;
}

// Packed lower tiles with at most W tile columns (a "slab": the first W
// columns of a lower-triangular tile matrix).  Rows I < W are packed like
// tri_index; rows I >= W hold W tiles each, row-major after them.  W >= the
// number of rows gives tri_index exactly, so the full matrix is the case
// W = N.  Tile (I, J) needs J <= min(I, W - 1).
__host__ __device__ inline int64_t tile_index(int64_t I, int64_t J, int64_t W) {
  return I < W ? I * (I + 1) / 2 + J : W * (W + 1) / 2 + (I - W) * W + J;
}
__host__ __device__ inline int64_t num_slab_tiles(int64_t rows, int64_t W) {
  return rows <= W ? rows * (rows + 1) / 2 : W * (W + 1) / 2 + (rows - W) * W;
}
__host__ __device__ inline void tile_coords(int64_t q, int64_t W, int64_t* I, int64_t* J) {
  const int64_t tri = W * (W + 1) / 2;
  if (q < tri) {
    tri_coords(q, I, J);
  } else {
    *I = W + (q - tri) / W;
    *J = (q - tri) % W;
  }
}

// Device-side status and scalar results of the kernels of one solve.  Reset
// (memset 0 plus the min fields) before each solve, read back by the host.
enum StatusFlags : int {
  ST_NONFINITE = 1,   // a coordinate is NaN/Inf (some d^2 is not finite)
  ST_DUPLICATE = 2,   // d_jk = 0 for j != k
  ST_NOTPD = 4,       // a Cholesky pivot was not positive
  ST_TIMEOUT = 8,     // a bounded device wait gave up
  ST_BADLAUNCH = 16   // a kernel got a launch shape it does not support
};

struct DevStatus {
  int flags;
  int notpd_index;                 // 1 + first failing pivot row, valid if ST_NOTPD
  unsigned long long min_d2_bits;  // min off-diagonal d^2 (non-negative double bits)
  unsigned long long r_max_bits;   // max_j |r_j|
  unsigned long long z_max_bits;   // max_j sum_k Z_jk
  unsigned long long w_max_bits;   // max_j |w_j|
  unsigned long long off_max_bits; // max_j sum_{k != j} Z_jk (from the generator)
  unsigned long long far_d2_bits;  // max_j ||x_j - x_0||^2 (k_far_from_first)
  double mag;                      // 1^T w (compensated)
  double min_w;                    // min_j w_j
  double aux[6];                   // scratch scalars (GMRES dot products, grad sums)
  unsigned long long hash_bits;    // checksum of the points (launch_hash)
};

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `s` and returns cudaGetLastError().

// K1: fused distance + exp generator of the packed lower tiles.
// Writes Zf (FP32 tiles, may be null) and/or Zd (FP64 tiles, may be null),
// accumulates full row sums of Z into rowsum (n doubles, must be zeroed),
// min off-diagonal d^2, and non-finite/duplicate flags.  kind selects the
// matrix: MAT_EXP, Z_jk = exp(-t d_jk) (Eq. weighting); MAT_SHIFTED_DIST,
// Z_jk = 1 - t d_jk (the scale-zero system with t = 1/c).  With tiny_arg
// finite, MAT_EXP entries with t d_jk > tiny_arg are evaluated in FP32
// (exp_neg_tiny_td); +inf keeps every entry FP64-exact.
// MAT_DEFLATED: Z_jk = 1 + expm1(-t d_jk) / (c t), unit diagonal (the
// small-t system (Z - (1 - c t) 1 1^T) / (c t) with its rank-one part
// deflated; kc = 1 / (c t)).
enum MatKind : int { MAT_EXP = 0, MAT_SHIFTED_DIST = 1, MAT_DEFLATED = 2 };
// Entries exp(-t d) with t d above this (below e^-46 < 2^-66) are evaluated in
// FP32 on the solve path: their error cannot reach one FP64 rounding of a row
// sum that holds the unit diagonal (exp_neg_tiny_td in mag_math.cuh).
constexpr double kTinyArg = 46.0;
cudaError_t launch_generate(const double* X, int64_t n, int m, double t, int64_t N, float* Zf,
                            double* Zd, double* rowsum, DevStatus* st, cudaStream_t s, int kind = MAT_EXP,
                            double tiny_arg = INFINITY, double kc = 0.0);
// The same, also writing the FP64 distances d_jk into Dd (packed tiles like Z).
cudaError_t launch_generate_dist(const double* X, int64_t n, int m, double t, int64_t N, float* Zf,
                                 double* Zd, double* Dd, double* rowsum, DevStatus* st, cudaStream_t s,
                                 int kind = MAT_EXP, double tiny_arg = INFINITY, double kc = 0.0);
// Exact pair distances from quantized coordinates (k_generate.cu).
// launch_coord_range: per dimension min and max of X into out[2l], out[2l+1]
// and out[2m] = 1 if a coordinate is not finite (2m + 1 doubles).
// launch_quantize: Xq[i m + l] = round(2^e (X[i m + l] - out[2l])) (int64).
// launch_dist_q: FP64 distances Dd of the packed lower tiles (m <= 32) from
// Xq (limb bits L, scale 2^e; pairs with d^2 < tau2 from the FP64
// differences of X), min d^2 and ST_DUPLICATE into st as the generator.
cudaError_t launch_coord_range(const double* X, int64_t n, int m, double* out, cudaStream_t s);
cudaError_t launch_quantize(const double* X, int64_t n, int m, const double* range, int e, long long* Xq,
                            cudaStream_t s);
cudaError_t launch_dist_q(const long long* Xq, const double* X, int64_t n, int m, int L, int e, double tau2,
                          int64_t N, double* Dd, DevStatus* st, cudaStream_t s);
// launch_generate (row sums, min d^2, flags) with the distances of
// launch_dist_q, in one pass (no distances kept).
// rowsum may be null (none); t0, W: the slab layout of launch_generate_slab.
cudaError_t launch_generate_q(const long long* Xq, const double* X, int64_t n, int m, int L, int e, double tau2,
                              double t, int64_t N, float* Zf, double* Zd, double* rowsum, DevStatus* st,
                              cudaStream_t s, int kind = MAT_EXP, double tiny_arg = INFINITY, double kc = 0.0,
                              int64_t t0 = 0, int64_t W = -1);
// FP32 tiles of one slab for the out-of-core factor: global tile columns
// [t0, t0 + W) of rows [t0, N), in the slab layout (tile_index with column
// cap W, tile (0, 0) = global (t0, t0)); no row sums; min d^2 and flags as
// above (the slabs of a factor partition the lower triangle's pairs).
// Xq (optional): the quantized coordinates (launch_quantize), the pairs'
// distances from their exact integer d^2 (launch_generate_q).
cudaError_t launch_generate_slab(const double* X, int64_t n, int m, double t, int64_t t0, int64_t W, float* Zf,
                                 DevStatus* st, cudaStream_t s, double tiny_arg = INFINITY,
                                 const long long* Xq = nullptr, int qL = 0, int qe = 0, double qtau2 = 0.0);
// Z from stored FP64 distance tiles: Zf (may be null) and Zd (may be null), row sums.
cudaError_t launch_generate_from_dist(const double* Dd, int64_t n, double t, int64_t N, float* Zf, double* Zd,
                                     double* rowsum, cudaStream_t s, int kind = MAT_EXP,
                                     double tiny_arg = INFINITY, double kc = 0.0);
// max_j ||x_j - x_0||^2 into st->far_d2_bits (st->far_d2_bits must start at 0).
cudaError_t launch_far_from_first(const double* X, int64_t n, int m, DevStatus* st, cudaStream_t s);
// min_{j != k} d^2 over all pairs (FP64) into st->min_d2_bits.
cudaError_t launch_min_distance(const double* X, int64_t n, int m, DevStatus* st, cudaStream_t s);
// off-diagonal row-sum maximum (Gershgorin) from rowsum into st->off_max_bits.
cudaError_t launch_rowsum_max(const double* rowsum, int64_t n, DevStatus* st, cudaStream_t s);

// K2: blocked right-looking Cholesky pieces (T = float or double).
template <typename T>
cudaError_t launch_potrf_diag(T* Z, T* Dinv, int64_t K, int64_t n, DevStatus* st, cudaStream_t s);
// Panel solve: tiles (I, K) for I in [K+1, N): A_IK <- A_IK inv(L_KK)^T.
template <typename T>
cudaError_t launch_trsm_col(T* Z, const T* Dinv, int64_t K, int64_t N, DevStatus* st,
                            cudaStream_t s);
// CUDA-core trailing update: C_IJ -= sum_{k in [k0,k1)} L_Ik L_Jk^T for all
// tiles with j0 <= J < j1, J <= I < N.
template <typename T>
cudaError_t launch_syrk_simt(T* Z, int64_t N, int64_t k0, int64_t k1, int64_t j0, int64_t j1,
                             DevStatus* st, cudaStream_t s);

// Dense n x n row-major copy of the packed tiles: symmetric (Z) or lower (L).
template <typename T>
cudaError_t launch_unpack(const T* Z, int64_t n, int64_t N, bool symmetric, T* out, cudaStream_t s);

// K2c on tensor cores (k_update_tc.cu).  Product kinds of the trailing update.
enum UpdMode { UPD_TF32X3 = 0, UPD_TF32 = 1, UPD_BF16 = 2, UPD_FP16X3 = 3, UPD_FP16 = 4 };
// FP16 modes store the panel scaled by 2^FP16_SCALE_LOG2 (|L| <= 1 stays far
// below the FP16 maximum; entries down to ~1e-8 stay normal); the update
// multiplies the accumulator by 2^(-2 FP16_SCALE_LOG2), exactly.
constexpr int FP16_SCALE_LOG2 = 12;

struct UpdParams {
  float* Z;            // packed FP32 tiles (updated in place)
  int64_t N;           // tiles per side
  int64_t k0;          // first tile column of the panel = row block 0 of the panel buffer
  int kc_lo, kc_hi;    // K range in panel-local tile columns [kc_lo, kc_hi)
  int64_t j1;          // output tile columns end before j1 (tile J+1 is skipped at j1)
  const uint32_t* tasks;  // output blocks (I << 16) | J, in processing order
  int64_t ntasks;
  unsigned* counter;      // zero before the launch; CTAs claim tasks from it
  DevStatus* st;
  uint64_t timeout_ns; // bound on every barrier wait inside the kernel
  int max_tasks;       // > 0: a CTA (pair) leaves after that many tasks, so that
                       // SMs come free during the launch; 0: until the queue is empty
  int64_t wcap;        // column cap of Z's tile layout (tile_index); <= 0: N (the whole matrix)
};

// Four TMA descriptors (A/B boxes of the hi and lo panel copies), 128 B each.
struct alignas(64) UpdMaps {
  unsigned char m[4][128];
};

bool make_update_maps(UpdMaps* maps, const void* hi, const void* lo, int mode, int64_t cols, int64_t rows);

// TMA descriptor of the packed FP32 tiles Z seen as [tiles][128][128] with
// 32 x 32 boxes and the 128-byte swizzle: the target of the update
// epilogue's bulk reduce-add C += (-acc).
struct alignas(64) CMap {
  unsigned char m[128];
};
bool make_c_map(CMap* map, float* Z, int64_t tiles);
// Appends the output blocks of one update to `out`: tiles (I, J), (I, J+1)
// for J = j0, j0+2, ... < j1 -- and, with `pairs` (the CTA-pair kernel),
// also (I+1, J), (I+1, J+1) with I = j0, j0+2, ... -- for the rows I in
// [J, N), in 16-row x 8-column-pair super-block order (rows of super-blocks
// top-down, lower triangle of the super-block grid first), skipping blocks
// outside the trapezoid.  Returns the number appended.  Requires N < 65536.
int64_t update_tasks(int64_t N, int64_t j0, int64_t j1, bool pairs, std::vector<uint32_t>* out);
// pairs: the CTA-pair (cta_group::2) kernel with a pair task table; grid is
// rounded down to whole clusters of two CTAs.
cudaError_t launch_update_tc(const UpdMaps& maps, const CMap& cmap, UpdParams p, int mode, int grid, bool pairs,
                             cudaStream_t s);

// Panel copy of column K (tiles I in (K, N)) for the tensor-core update:
// row (I - k0)*TILE + r, column (K - k0)*TILE + c of the row-major panel
// buffer with `width` columns.  TF32X3: hi = rna_tf32(x), lo = rna_tf32(x - hi);
// TF32: hi only; BF16: round-to-nearest BF16 into hi (as 16-bit words);
// FP16X3: y = 2^12 x, hi = rn_fp16(y), lo = rn_fp16(y - hi); FP16: hi only.
cudaError_t launch_split_col(const float* Z, int64_t K, int64_t N, int64_t k0, int64_t width, int mode,
                             void* hi, void* lo, cudaStream_t s);
// Panel solve + panel copy of column K on the tensor cores (FP16 and FP16X3
// factors): L_IK = Z_IK inv(L_KK)^T from the split-FP16 products hi*hi +
// hi*lo + lo*hi of row-scaled operands, written over Z_IK, then copied into
// the panel buffer as launch_split_col does (lo only for FP16X3).  At most
// `grid` persistent CTAs (129 KB of shared memory each) claim the N - K - 1
// tiles from *counter, which must be zero before the launch.
// wcap: column cap of Z's tile layout (tile_index), -1 for the whole matrix.
// lh (FP16 mode only, may be null): also writes the panel copy's FP16
// values (2^12 L_IK) to tile tile_index(I, K, wcap) of lh, row-major: the
// FP16 copy of the factor that the in-core sweeps read.
cudaError_t launch_trsm_tc(float* Z, const float* Dinv, int64_t K, int64_t N, int64_t k0, int64_t width, int mode,
                           void* hi, void* lo, unsigned* counter, DevStatus* st, int grid, cudaStream_t s,
                           int64_t wcap = -1, void* lh = nullptr);

// K3: triangular solves with the packed factor, in place on v (np = N*TILE
// entries of type T).  tmp: np entries of scratch.
template <typename T>
cudaError_t launch_forward(const T* Z, const T* Dinv, int64_t N, T* v, T* tmp, cudaStream_t s);
template <typename T>
cudaError_t launch_backward(const T* Z, const T* Dinv, int64_t N, T* v, T* tmp, cudaStream_t s);

// K3, persistent single-launch versions (cooperative; one progress counter,
// flags[0]).  Same arguments as above; y/x must not alias v/yv.  Every wait
// for another CTA's tile gives up timeout_ns after the launch started and
// raises ST_TIMEOUT (the results are then invalid).
template <typename T>
cudaError_t launch_forward_persistent(const T* Z, const T* Dinv, int64_t N, const T* v, T* y, unsigned* flags,
                                      DevStatus* st, uint64_t timeout_ns, cudaStream_t s);
template <typename T>
cudaError_t launch_backward_persistent(const T* Z, const T* Dinv, int64_t N, const T* yv, T* x, unsigned* flags,
                                       DevStatus* st, uint64_t timeout_ns, cudaStream_t s);
// K3, in-core sweeps with one 128 x 128 product per tile on the critical
// path (k_chain.cu).  After a factor: launch_chain_prep forms Sf (N tiles,
// tile I = (inv(L_II) L_{I,I-1})^T) and Sb (N tiles, tile I =
// L_{I+1,I} inv(L_II)) from the FP32 factor Z and Dinv (2N tiles: inv(L_II),
// then the transposes).  Per correction: launch_scale_rhs_unset (v = r /
// r_max as launch_scale_rhs, y = the "not yet written" pattern), the forward
// sweep v -> y (v is reset to the pattern), the backward sweep y -> x (x = v
// of the forward sweep).  Lt: the off-diagonal tiles (packed, FP32 or FP16
// scaled by 1/lscale).  Waits give up timeout_ns after the launch started
// and raise ST_TIMEOUT (the results are then invalid).
cudaError_t launch_chain_prep(const float* Z, const float* Dinv, int64_t N, float* Sf, float* Sb, cudaStream_t s);
cudaError_t launch_scale_rhs_unset(const double* r, int64_t n, int64_t np, float* v, float* y, const DevStatus* st,
                                   cudaStream_t s);
template <typename TL>
cudaError_t launch_forward_chain(const TL* Lt, float lscale, const float* Dinv, const float* Sf, int64_t N, float* v,
                                 float* y, DevStatus* st, uint64_t timeout_ns, cudaStream_t s);
template <typename TL>
cudaError_t launch_backward_chain(const TL* Lt, float lscale, const float* Dinv, const float* Sb, int64_t N,
                                  const float* y, float* x, DevStatus* st, uint64_t timeout_ns, cudaStream_t s);

// The same sweeps with the transposed inverses given directly (DinvT: N tiles
// of inv(L_II)^T), for the triangle of one slab of the out-of-core factor;
// z_on_host: Z is host memory read in place (no L2 prefetch hints).
template <typename T>
cudaError_t launch_forward_sweep(const T* Z, const T* DinvT, int64_t N, const T* v, T* y, unsigned* progress,
                                 DevStatus* st, uint64_t timeout_ns, bool z_on_host, cudaStream_t s);
template <typename T>
cudaError_t launch_backward_sweep(const T* Z, const T* Dinv, int64_t N, const T* yv, T* x, unsigned* progress,
                                  DevStatus* st, uint64_t timeout_ns, bool z_on_host, cudaStream_t s);

// Out-of-core factor (k_ooc.cu).  A slab of tile columns [q0, q0 + Sq) is
// stored in the slab layout (tile_index with cap Sq, tile (0, 0) = global
// (q0, q0)), in device or (mapped) host memory.
// Panel copy for the updates of a later slab: for local tile rows I' in
// [0, rows) (global c0 + I') and the global tile columns [k0, k0 + kw) of
// slab (Lq, q0, Sq), writes 2^12 x rounded to FP16 (hi) and the rounded
// remainder (lo, when split) at row I' * TILE + r, column (K - k0) * TILE + c
// of the row-major panel buffers with `width` columns -- the values the
// panel solve writes for the same entries of L.
cudaError_t launch_gather_split(const float* Lq, int64_t q0, int64_t Sq, int64_t c0, int64_t rows, int64_t k0,
                                int kw, void* hi, void* lo, int64_t width, bool split, cudaStream_t s);
// v[r] -= sum_c A[r][c] y[c] for the rectangle part of a slab (R tile rows x
// S tile columns, tile (i, j) at A + (i S + j) TILE^2): r < R TILE, c < S TILE.
cudaError_t launch_rect_gemv(const float* A, int64_t R, int64_t S, const float* y, float* v, cudaStream_t s);
// y[c] -= sum_r A[r][c] x[r] (the transposed product) for the same rectangle.
cudaError_t launch_rect_gemv_t(const float* A, int64_t R, int64_t S, const float* x, float* y, cudaStream_t s);

// K4: FP64 residual r = b - Z w (b == null means all ones), Z regenerated
// from the points (matrix free) or read from FP64 packed tiles (stored).
// part: scratch of 3 * chunks * np doubles.  Norms go to st (r_max, z_max, w_max).
cudaError_t launch_residual_mf(const double* X, int64_t n, int m, double t, const double* w,
                               const double* b, double* r, double* part, int chunks, int64_t np,
                               DevStatus* st, cudaStream_t s, int kind = MAT_EXP, double kc = 0.0);
// Matrix free over the lower triangle (each Z entry computed once, used for
// its row and its column): P is scratch of N * N * 128 doubles, rowsum of n
// doubles (overwritten with the row sums of Z).  Same outputs as above.
// Xq (optional, Z = exp(-t d) with m <= 32): the quantized coordinates of
// launch_quantize (limb bits qL, scale 2^qe, FP64 differences below qtau2),
// the pair distances from their exact integer d^2.
cudaError_t launch_residual_sym(const double* X, int64_t n, int m, double t, const double* w, const double* b,
                                double* r, double* P, double* rowsum, int64_t np, DevStatus* st, cudaStream_t s,
                                int kind = MAT_EXP, double kc = 0.0, const long long* Xq = nullptr, int qL = 0,
                                int qe = 0, double qtau2 = 0.0);
// Stored: P is scratch of N * N * 128 doubles (one partial per row block,
// tile and row); rowsum holds the row sums of Z from the generator.
cudaError_t launch_residual_stored(const double* Zd, int64_t n, int64_t N, const double* w,
                                   const double* b, const double* rowsum, double* r, double* P, int64_t np,
                                   DevStatus* st, cudaStream_t s);
// The same product in float-float on the FP32 pipe (entries of exp(-t d) in
// [0, 1] only): r = b - Z w to a few units of 2^-46 of sum |Z| |w|, for the
// inner iterations of GMRES-IR.  wsplit: np float2 of scratch (w split into
// FP32 leading and trailing parts); np >= N * TILE.
cudaError_t launch_residual_stored_ff(const double* Zd, int64_t n, int64_t N, const double* w, void* wsplit,
                                      const double* b, const double* rowsum, double* r, double* P, int64_t np,
                                      DevStatus* st, cudaStream_t s);

// K5/K6 helpers.  r_max below is max_j |r_j| as kept in st->r_max_bits.
// v[i] = r[i] / r_max for i < n, 0 for n <= i < np (right-hand side of a correction).
template <typename T>
cudaError_t launch_scale_rhs(const double* r, int64_t n, int64_t np, T* v, const DevStatus* st,
                             cudaStream_t s);
// x[i] = (init ? 0 : x[i]) + r_max * v[i], in FP64 (the refinement update).
template <typename T>
cudaError_t launch_accumulate(double* x, const T* v, int64_t n, const DevStatus* st, bool init,
                              cudaStream_t s);
// st->r_max_bits = max(st->r_max_bits, max_i |v[i]|).
cudaError_t launch_absmax(const double* v, int64_t n, DevStatus* st, cudaStream_t s);
// Mag = 1^T w (compensated), min w, max |w| into st.
cudaError_t launch_reduce_w(const double* w, int64_t n, DevStatus* st, cudaStream_t s);
cudaError_t launch_fill(double* v, int64_t n, double value, cudaStream_t s);
// GMRES helpers: out[i] = <V_i, w> (i < k, compensated); w -= sum_i h[i] V_i; x = sc * w.
cudaError_t launch_mdot(const double* V, int64_t ld, int k, const double* w, int64_t n, double* out,
                        cudaStream_t s);
cudaError_t launch_maxpy(const double* V, int64_t ld, int k, const double* h, double* w, int64_t n,
                         cudaStream_t s);
cudaError_t launch_scale(const double* w, double sc, double* x, int64_t n, cudaStream_t s);

// K8 batch (k_batch.cu).
struct BatchCloud {
  int64_t point_offset;  // doubles into the points array
  int64_t dist_offset;   // doubles into the packed-distance array
  int32_t n, m;
};
struct BatchProblem {
  int64_t dist_offset;   // of its cloud
  int64_t w_offset;      // doubles into w_out
  int32_t n, cloud;
  double t;
};
enum BatchStatus { MAG_BATCH_OK = 0, MAG_BATCH_NOTPD = 1, MAG_BATCH_NOCONV = 2, MAG_BATCH_DUPLICATE = 3,
                   MAG_BATCH_NONFINITE = 4 };
constexpr int BATCH_NMAX = 2048;  // largest n solved inside one CTA
// Also sets cloud_flags[c] |= 1 (non-finite coordinate) / 2 (coincident points);
// cloud_flags must be zeroed.
cudaError_t launch_batch_dist(const double* X, const BatchCloud* clouds, int nclouds, int64_t max_pairs,
                              double* D, int* cloud_flags, cudaStream_t s);
// block = 32 or 64 (factor block size); scratch_f: grid * (nmax^2 + nmax) floats,
// scratch_d: grid * (nmax^2 + 2 nmax) doubles; queue: one zeroed int.
// Launch shapes of k_batch_solve: threads per CTA, CTAs per SM its launch
// bounds target, trailing update on the tensor cores (split TF32) or not,
// right- or left-looking factor;
// batch_shape_resident(i) = CTAs of shape i one SM holds.
// busy_cycles (or null) receives the sum over CTAs of their busy time in SM
// cycles (the tuner's measure).
struct BatchShape {
  int threads, ctas_per_sm, tensor_cores, left_looking;
};
constexpr int kNumBatchShapes = 7;
extern const BatchShape kBatchShapes[kNumBatchShapes];
int batch_shape_resident(int shape);
cudaError_t launch_batch_solve(int shape, const BatchProblem* probs, const int* order, int count,
                               const double* D, const int* cloud_flags, float* scratch_f, double* scratch_d,
                               int64_t nmax, double* w_out, double* mag_out, int* status, int* queue, double tol,
                               int max_iter, int grid, unsigned long long* busy_cycles, cudaStream_t s);

// K7 gradients: dL/dt partial sums and dL/dx.
cudaError_t launch_grad(const double* X, int64_t n, int m, double t, const double* w,
                        const double* lam, double* dL_dx, double* part_t, int64_t np,
                        cudaStream_t s);
cudaError_t launch_sum_f64(const double* v, int64_t n, double* out, cudaStream_t s);
// *out += an order-independent 64-bit mix of the bits of v[0..count) and
// their positions (a checksum: *out must be zeroed first).
cudaError_t launch_hash(const double* v, int64_t count, unsigned long long* out, cudaStream_t s);
// out2[0] = min_i v_i, out2[1] = max_i v_i (device).
cudaError_t launch_minmax(const double* v, int64_t n, double* out2, cudaStream_t s);

}  // namespace mag
