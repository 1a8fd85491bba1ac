// Host side of the C ABI declared in include/magnitude.h: context, workspace,
// and the stream-ordered pipelines of mag_solve (generate -> factor -> solve
// -> FP64 iterative refinement -> magnitude), mag_sweep_tplus (bisection),
// mag_grad (adjoint) and mag_solve_batch.
//
// Iterative refinement follows the classical mixed-precision scheme (Wilkinson;
// Carson & Higham, SIAM J. Sci. Comput. 40 (2018)): the factor is computed in a
// low precision, the residual r = 1 - Zw and the update w += e in FP64, and
// the correction e solves with the low-precision factor applied to r scaled by
// 1/||r||inf.  When the residual stagnates the solve escalates to GMRES-IR
// (FGMRES preconditioned by the same factor, all vectors FP64) and then to an
// FP64 factor.
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "../../include/magnitude.h"
#include "mag_internal.cuh"

using namespace mag;

std::atomic<long long> mag::g_kernel_launches{0};

namespace {

struct Layout {
  int64_t n = 0, N = 0, np = 0, tiles = 0;
  int chunks = 1;
  bool f32 = false, f64 = false;
  size_t off_zf = 0, off_zd = 0, off_dinvf = 0, off_dinvd = 0, off_vec = 0, off_part = 0,
         off_status = 0, off_panel = 0, off_flags = 0, off_spart = 0, off_dist = 0, off_ctr = 0, total = 0;
  bool dist = false;   // FP64 distance tiles present
  int nb = 24;         // panel buffer capacity in tiles (the widest panel a factor may use)
  int64_t W = 0;       // panel buffer row length in columns (nb * TILE)
  int64_t nctr = 0;    // task counters of one factor: update launches, then one per panel solve
  int64_t nctr_upd = 0;  // the update launches' share (at the front)
  int64_t zf_tiles = 0;  // FP32 tiles of the zf region: all lower tiles, or the slab pool
};

// One slab of the out-of-core factor: tile columns [c0, c0 + S) of every row
// below, in the slab layout (tile_index with cap S); generated and factored
// at dev (device pool), then kept there or copied to host (pinned, mapped).
struct Slab {
  int64_t c0 = 0, S = 0, tiles = 0;
  int64_t pool_off = 0;    // tile offset of its device location in the pool
  bool host = false;       // finished slab lives in host memory
  int64_t host_off = 0;    // tile offset in the host buffer
};

constexpr int NVEC_D = 6;   // FP64 vectors of np entries
constexpr int NVEC_F = 3;   // FP32 vectors of np entries

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct mag_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  mag_options opt{};
  std::string err;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Layout lay;
  DevStatus* h_st = nullptr;  // pinned host copy
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int sm_count = 152;
  double* aux = nullptr;  // vectors that must survive workspace re-plans
  int64_t aux_np = 0;
  std::vector<cudaEvent_t> prof_ev;  // event pairs around profiled launches
  std::vector<int> prof_cat;         // category of each used pair
  int prof_used = 0;
  double* gm = nullptr;              // GMRES basis, zeros and small vectors
  size_t gm_bytes = 0;
  bool dist_active = false;          // inside a call that reuses distances
  bool dist_valid = false;           // dist() holds the distances of dist_pts
  const double* dist_pts = nullptr;
  int64_t dist_n = 0;
  int32_t dist_m = 0;
  double dist_dmin = 0, dist_gersh_unused = 0;
  bool dist_exact = false;           // the stored distances came from the exact integer pass
  void* bws = nullptr;               // batch workspace
  size_t bws_bytes = 0;
  int batch_tuned[12] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};  // launch shape per
                                     // size class ceil(log2 nmax) of the batch kernel (-1: not tuned)
  int batch_shape_used = 0;
  UpdMaps maps[2];                   // TMA descriptors of the two panel buffers
  const void* maps_base[2] = {nullptr, nullptr};
  int maps_mode[2] = {-1, -1};
  int64_t maps_W[2] = {0, 0}, maps_np[2] = {0, 0};
  CMap cmap;                         // TMA descriptor of the FP32 tiles (update epilogue)
  const void* cmap_base = nullptr;
  int64_t cmap_tiles = 0;
  // task tables of the update launches of one factor, per (N, panel width,
  // look-ahead, CTA pairs): device table and (j0, j1) -> (offset, count)
  struct TaskTable {
    uint32_t* d = nullptr;
    std::map<std::pair<int64_t, int64_t>, std::pair<int64_t, int64_t>> rng;
  };
  std::map<std::tuple<int64_t, int, int, int, int64_t>, TaskTable> task_tables;
  TaskTable* tasks = nullptr;        // the table of the factor in progress
  cudaStream_t side = nullptr;       // panel stream of the look-ahead factor
  int kind = MAT_EXP;                // matrix the solve path generates (MatKind)
  double kind_c = 0.0;               // its parameter c (MAT_DEFLATED)
  cudaEvent_t ev_la[3] = {nullptr, nullptr, nullptr};  // start, panel done, trailing done
  // the factor left in the workspace by the last in-core solve of Z =
  // exp[-t d], reusable by a later solve with the same points and t (the
  // adjoint solve of mag_grad): key and how to refine with it
  bool fac_valid = false;
  const double* fac_pts = nullptr;
  int64_t fac_n = 0;
  int32_t fac_m = 0;
  double fac_t = 0.0;
  unsigned long long fac_hash = 0;
  int fac_prec = 0;
  bool fac_stored = false;
  bool fac_gmres = false;  // the solve that made it needed GMRES-IR
  // out-of-core factor (slabs); empty when the solve runs in core
  std::vector<Slab> slabs;
  bool ooc = false;                  // the current solve factors out of core
  float* host_L = nullptr;           // pinned host memory of the host slabs (mapped)
  size_t host_L_bytes = 0;
  CMap slab_cmap;                    // TMA descriptor of the slab being updated
  const void* slab_cmap_base = nullptr;
  int64_t slab_cmap_tiles = 0;
  // in-core sweeps (k_chain.cu): the B tiles of the factor in the workspace
  // (Sf: N tiles, then Sb: N tiles) and the FP16 copy of its off-diagonal
  // tiles that the panel solve of the one-product factor writes
  float* chain_s = nullptr;
  size_t chain_s_bytes = 0;
  // quantized coordinates of the exact distance pass: 2m + 1 doubles of
  // ranges (and a flag), then n m int64
  void* xq = nullptr;
  size_t xq_bytes = 0;
  bool xq_ok = false;                // xq holds the quantization of (xq_pts, xq_n, xq_m) for this solve
  const double* xq_pts = nullptr;
  int64_t xq_n = 0;
  int32_t xq_m = 0;
  int xq_L = 0, xq_e = 0;
  double xq_tau2 = 0.0;
  const long long* xq_q = nullptr;
  void* lh = nullptr;
  size_t lh_bytes = 0;
  bool chain_ready = false;          // chain_s holds the B tiles of the current factor
  bool lh_ready = false;             // lh holds its FP16 tiles
  int64_t chain_N = 0;
  float* probe_z = nullptr;          // FP32 tiles of the leading block the precision probe factors
  size_t probe_bytes = 0;
  CMap probe_cmap;                   // TMA descriptor of those tiles (update epilogue)
  const void* probe_cmap_base = nullptr;
  int64_t probe_cmap_tiles = 0;

  // typed views of the workspace
  float* zf() { return (float*)((char*)ws + lay.off_zf); }
  float* slab_dev(const Slab& sl) { return zf() + sl.pool_off * TILE_ELEMS; }
  // where a finished slab is read: its device location, or its host copy
  const float* slab_data(const Slab& sl) {
    return sl.host ? host_L + sl.host_off * TILE_ELEMS : slab_dev(sl);
  }
  double* zd() { return (double*)((char*)ws + lay.off_zd); }
  float* dinvf() { return (float*)((char*)ws + lay.off_dinvf); }
  double* dinvd() { return (double*)((char*)ws + lay.off_dinvd); }
  double* vd(int i) { return (double*)((char*)ws + lay.off_vec) + (size_t)i * lay.np; }
  float* vf(int i) {
    return (float*)((double*)((char*)ws + lay.off_vec) + (size_t)NVEC_D * lay.np) + (size_t)i * lay.np;
  }
  double* part() { return (double*)((char*)ws + lay.off_part); }
  double* spart() { return (double*)((char*)ws + lay.off_spart); }
  double* dist() { return (double*)((char*)ws + lay.off_dist); }
  float* panel_hi(int b) { return (float*)((char*)ws + lay.off_panel) + (size_t)b * 2 * lay.np * lay.W; }
  float* panel_lo(int b) { return panel_hi(b) + (size_t)lay.np * lay.W; }
  unsigned* counters() { return (unsigned*)((char*)ws + lay.off_ctr); }
  DevStatus* st() { return (DevStatus*)((char*)ws + lay.off_status); }
  unsigned* flags() { return (unsigned*)((char*)ws + lay.off_flags); }
};

// FP64 vector slots
enum { V_ROWSUM = 0, V_R = 1, V_X = 2, V_E = 3, V_BEST = 4, V_T2 = 5 };
enum { F_V = 0, F_Y = 1, F_T = 2 };
// FP64 vectors of the aux buffer (sweep probes, gradients)
enum { A_W = 0, A_LAM = 1, A_G = 2, A_PART = 3, A_COUNT = 4 };

namespace {

int fail(mag_ctx* c, int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return status;
}

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MAG_ENOMEM : MAG_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

#define TRY(expr)           \
  do {                      \
    int s_ = (expr);        \
    if (s_ != MAG_OK) return s_; \
  } while (0)

// Refinement stops once its own FP64 residual is below this fraction of the
// tolerance, so that an independent FP64 evaluation of the same residual
// (which differs in rounding by far less than 10%) also meets the tolerance.
constexpr double kStopMargin = 0.9;

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

Layout plan(const mag_ctx* ctx, int64_t n, bool f32, bool f64, bool dist = false, int64_t zf_tiles = -1) {
  Layout L;
  L.n = n;
  L.N = (n + TILE - 1) / TILE;
  L.np = L.N * TILE;
  L.tiles = num_lower_tiles(L.N);
  L.f32 = f32;
  L.f64 = f64;
  const int64_t rowblocks = (n + 127) / 128;
  int64_t chunks = (4 * (int64_t)ctx->sm_count * 4 + rowblocks - 1) / rowblocks;
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, std::max<int64_t>(1, L.N)));
  L.chunks = (int)chunks;
  size_t off = 0;
  L.off_status = off;
  off = align_up(off + sizeof(DevStatus));
  L.off_flags = off;
  off = align_up(off + (size_t)L.N * sizeof(unsigned));
  L.off_ctr = off;  // at most N - 1 in-panel + 2 per panel update launches, one per column solve
  L.nctr_upd = 2 * L.N + 16;
  L.nctr = L.nctr_upd + L.N;
  off = align_up(off + (size_t)L.nctr * sizeof(unsigned));
  L.off_vec = off;
  off = align_up(off + (size_t)L.np * (NVEC_D * sizeof(double) + NVEC_F * sizeof(float)));
  L.off_part = off;
  off = align_up(off + (size_t)3 * L.chunks * L.np * sizeof(double));
  L.dist = dist;
  L.off_dist = off;  // placed before every precision-dependent region: stable offset
  if (dist) off = align_up(off + (size_t)L.tiles * TILE_ELEMS * sizeof(double));
  // panel buffers sized for the widest default panel, so that factors of
  // different precisions in one call share the workspace
  L.nb = ctx->opt.panel_tiles > 0 ? ctx->opt.panel_tiles : 32;
  L.W = (int64_t)L.nb * TILE;
  L.off_panel = off;
  // two panel buffers (hi + lo copies each): the next panel is written while
  // the trailing update still reads the current one
  if (f32) off = align_up(off + (size_t)L.np * L.W * 4 * sizeof(float));
  L.off_dinvf = off;
  if (f32) off = align_up(off + (size_t)2 * L.N * TILE_ELEMS * sizeof(float));
  L.off_dinvd = off;
  if (f64) off = align_up(off + (size_t)2 * L.N * TILE_ELEMS * sizeof(double));
  L.off_zf = off;
  L.zf_tiles = zf_tiles >= 0 ? zf_tiles : L.tiles;
  if (f32) off = align_up(off + (size_t)L.zf_tiles * TILE_ELEMS * sizeof(float));
  L.off_zd = off;
  if (f64) off = align_up(off + (size_t)L.tiles * TILE_ELEMS * sizeof(double));
  L.off_spart = off;  // partials of the stored and the symmetric matrix-free residual: N * N * 128 doubles
  if (f32 || f64) off = align_up(off + (size_t)L.N * L.N * TILE * sizeof(double));
  L.total = off;
  return L;
}

int ensure_workspace(mag_ctx* ctx, int64_t n, bool f32, bool f64, int64_t zf_tiles = -1) {
  Layout L = plan(ctx, n, f32, f64, ctx->dist_active && zf_tiles < 0, zf_tiles);
  if (ctx->opt.workspace_limit_bytes > 0 && (double)L.total > ctx->opt.workspace_limit_bytes)
    return fail(ctx, MAG_ENOMEM, "workspace of %.3g bytes exceeds the limit %.3g", (double)L.total,
                ctx->opt.workspace_limit_bytes);
  if (L.total > ctx->ws_bytes) {
    if (ctx->ws) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    ctx->dist_valid = false;  // any stored distances are gone with the old buffer
    ctx->fac_valid = false;   // and the factor
    ctx->chain_ready = ctx->lh_ready = false;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, MAG_ENOMEM, "cudaMalloc(%.3g GB) failed: %s", L.total / 1e9,
                  cudaGetErrorString(e));
    }
    ctx->ws = p;
    ctx->ws_bytes = L.total;
  }
  ctx->lay = L;
  return MAG_OK;
}

// A device buffer of at least `need` bytes at *p (*have: its size), grown
// only while at least `margin` bytes of device memory stay free beside it.
// false (and no buffer change) when that does not hold or cudaMalloc fails:
// the caller then takes a path without the buffer.
bool grow_buffer(mag_ctx* ctx, void** p, size_t* have, size_t need, size_t margin) {
  if (need <= *have) return true;
  size_t fre = 0, tot = 0;
  if (cudaMemGetInfo(&fre, &tot) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if ((double)fre + (double)*have < (double)need + (double)margin) return false;
  if (*p) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
  }
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  *have = need;
  return true;
}

int ensure_aux(mag_ctx* ctx, int64_t n) {
  const int64_t np = ((n + TILE - 1) / TILE) * TILE;
  if (np <= ctx->aux_np) return MAG_OK;
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->aux);
    ctx->aux = nullptr;
    ctx->aux_np = 0;
  }
  cudaError_t e = cudaMalloc((void**)&ctx->aux, (size_t)A_COUNT * np * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->aux = nullptr;
    return fail(ctx, MAG_ENOMEM, "cudaMalloc(aux) failed: %s", cudaGetErrorString(e));
  }
  ctx->aux_np = np;
  return MAG_OK;
}

int reset_status(mag_ctx* ctx) {
  DevStatus init;
  std::memset(&init, 0, sizeof init);
  const double inf = INFINITY;
  std::memcpy(&init.min_d2_bits, &inf, sizeof inf);
  init.notpd_index = 0x7fffffff;  // atomicMin target
  *ctx->h_st = init;
  CU(cudaMemcpyAsync(ctx->st(), ctx->h_st, sizeof(DevStatus), cudaMemcpyHostToDevice, ctx->stream));
  return MAG_OK;
}

// Copy the device status to the pinned host copy and wait.
int read_status(mag_ctx* ctx) {
  CU(cudaMemcpyAsync(ctx->h_st, ctx->st(), sizeof(DevStatus), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return MAG_OK;
}

// Clear only the three norm maxima before a residual evaluation.
int reset_norms(mag_ctx* ctx) {
  CU(cudaMemsetAsync(&ctx->st()->r_max_bits, 0, 3 * sizeof(unsigned long long), ctx->stream));
  return MAG_OK;
}

int check_args(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t) {
  if (!ctx) return MAG_EINVAL;
  if (!points) return fail(ctx, MAG_EINVAL, "points is NULL");
  if (n < 2) return fail(ctx, MAG_EINVAL, "n = %lld < 2", (long long)n);
  if (m < 1 || m > MAG_MAX_DIM) return fail(ctx, MAG_EINVAL, "m = %d outside [1, %d]", (int)m, MAG_MAX_DIM);
  if (n > (int64_t)1 << 31) return fail(ctx, MAG_EINVAL, "n = %lld too large", (long long)n);
  if (!(t > 0.0) || !std::isfinite(t)) return fail(ctx, MAG_EINVAL, "t = %g must be finite and > 0", t);
  return MAG_OK;
}

// ---------------------------------------------------------------- factor
// Optional CUDA-event timing of factor launches by category (profile = 1).
enum { PC_UPDATE = 0, PC_UPDATE_PANEL = 1, PC_POTRF = 2, PC_TRSM = 3, PC_SPLIT = 4, PC_HOST_READ = 5, PC_COUNT = 6 };
int prof_begin(mag_ctx* ctx, int cat = PC_UPDATE, cudaStream_t st = nullptr) {
  if (!ctx->opt.profile) return MAG_OK;
  const size_t need = 2 * (size_t)(ctx->prof_used + 1);
  while (ctx->prof_ev.size() < need) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    ctx->prof_ev.push_back(e);
  }
  if (ctx->prof_cat.size() < (size_t)ctx->prof_used + 1) ctx->prof_cat.resize(ctx->prof_used + 1);
  ctx->prof_cat[ctx->prof_used] = cat;
  CU(cudaEventRecord(ctx->prof_ev[2 * ctx->prof_used], st ? st : ctx->stream));
  return MAG_OK;
}
int prof_end(mag_ctx* ctx, cudaStream_t st = nullptr) {
  if (!ctx->opt.profile) return MAG_OK;
  CU(cudaEventRecord(ctx->prof_ev[2 * ctx->prof_used + 1], st ? st : ctx->stream));
  ctx->prof_used++;
  return MAG_OK;
}
// Per-category sums of the recorded intervals (after the stream has been
// synchronized); returns the update total (trailing + panel updates).
// *busy (if given) receives the length of the union of the update
// intervals: launches on the two look-ahead streams overlap in time, so the
// sum counts the shared stretches twice while the union is the time during
// which at least one update launch was in flight.
double prof_collect(mag_ctx* ctx, double* per_cat, double* busy = nullptr) {
  for (int c = 0; c < PC_COUNT; ++c) per_cat[c] = 0;
  std::vector<std::pair<float, float>> upd;
  for (int i = 0; i < ctx->prof_used; ++i) {
    float v = 0, a = 0, b = 0;
    if (cudaEventElapsedTime(&v, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]) == cudaSuccess) {
      per_cat[ctx->prof_cat[i]] += v;
      if (busy && (ctx->prof_cat[i] == PC_UPDATE || ctx->prof_cat[i] == PC_UPDATE_PANEL) &&
          cudaEventElapsedTime(&a, ctx->prof_ev[0], ctx->prof_ev[2 * i]) == cudaSuccess &&
          cudaEventElapsedTime(&b, ctx->prof_ev[0], ctx->prof_ev[2 * i + 1]) == cudaSuccess)
        upd.emplace_back(a, b);
      cudaGetLastError();
    } else {
      cudaGetLastError();  // an interval cut short by an error: drop it, leave no pending error
    }
  }
  if (busy) {
    std::sort(upd.begin(), upd.end());
    double total = 0, lo = 0, hi = -INFINITY;
    for (const auto& iv : upd) {
      if (iv.first > hi) {
        if (hi > lo) total += hi - lo;
        lo = iv.first;
        hi = iv.second;
      } else if (iv.second > hi) {
        hi = iv.second;
      }
    }
    if (hi > lo) total += hi - lo;
    *busy = total;
  }
  ctx->prof_used = 0;
  return per_cat[PC_UPDATE] + per_cat[PC_UPDATE_PANEL];
}

// Algorithmic flops of C_IJ -= sum_k L_Ik L_Jk^T over the tiles J in [j0, j1),
// I in [J, N), k in [k0, k1): 2 * 128^3 per (output tile, k tile).
double update_flops(int64_t N, int64_t k0, int64_t k1, int64_t j0, int64_t j1) {
  const double tiles = (double)((N - j0) * (N - j0 + 1) / 2 - (N - j1) * (N - j1 + 1) / 2);
  return tiles * (double)(k1 - k0) * 2.0 * TILE * TILE * TILE;
}

template <typename T>
int factor_blocked(mag_ctx* ctx, T* Z, T* Dinv, int* launches, double* flops) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  for (int64_t K = 0; K < L.N; ++K) {
    CU(launch_potrf_diag<T>(Z, Dinv, K, L.n, ctx->st(), s));
    CU(launch_trsm_col<T>(Z, Dinv, K, L.N, ctx->st(), s));
    if (K + 1 < L.N) {
      TRY(prof_begin(ctx));
      CU(launch_syrk_simt<T>(Z, L.N, K, K + 1, K + 1, L.N, ctx->st(), s));
      TRY(prof_end(ctx));
      ++*launches;
      *flops += update_flops(L.N, K, K + 1, K + 1, L.N);
    }
  }
  return MAG_OK;
}

int upd_mode(int prec) {
  switch (prec) {
    case MAG_PREC_BF16: return UPD_BF16;
    case MAG_PREC_TF32: return UPD_TF32;
    case MAG_PREC_FP16X3: return UPD_FP16X3;
    case MAG_PREC_FP16: return UPD_FP16;
    default: return UPD_TF32X3;
  }
}

// Two-level blocked Cholesky with the trailing update on tensor cores.  For
// each panel of nb tile columns [k0, k1): potrf + panel solve per column
// with the column's copy into the panel buffer (one tensor-core pass for the
// FP16 kinds), recursive tensor-core updates inside the panel; then one
// tensor-core update of the whole trailing matrix with K = (k1 - k0) * 128.
// Task tables of every tensor-core update launch of one factor with the
// current N, panel width nb and schedule (built on the host once and kept).
int ensure_tasks(mag_ctx* ctx, int64_t N, int nb, bool la, bool pairs, int64_t ncol = -1, bool slab = false) {
  // ncol: tile columns factored (a slab of the out-of-core factor); -1 = N.
  // slab: also the range [0, ncol) (the update of a slab by earlier slabs)
  if (ncol < 0) ncol = N;
  const auto key = std::make_tuple(N, nb, (int)la + 2 * (int)slab, (int)pairs, ncol);
  auto found = ctx->task_tables.find(key);
  if (found != ctx->task_tables.end()) {
    ctx->tasks = &found->second;
    return MAG_OK;
  }
  if (N >= 65536) return fail(ctx, MAG_EINVAL, "%lld tiles too many for the tensor-core factor", (long long)N);
  std::vector<uint32_t> t;
  mag_ctx::TaskTable tab;
  auto add = [&](int64_t j0, int64_t j1) {
    const auto k = std::make_pair(j0, j1);
    if (j0 >= j1 || tab.rng.count(k)) return;
    const int64_t off = (int64_t)t.size();
    const int64_t cnt = update_tasks(N, j0, j1, pairs, &t);
    tab.rng[k] = std::make_pair(off, cnt);
  };
  // the in-panel updates of the recursive panel factor (tc_panel_range)
  std::function<void(int64_t, int64_t)> panel = [&](int64_t a, int64_t b) {
    if (b - a <= 1) return;
    const int64_t mid = a + (b - a) / 2;
    panel(a, mid);
    add(mid, b);
    panel(mid, b);
  };
  for (int64_t k0 = 0; k0 < ncol; k0 += nb) {
    const int64_t k1 = std::min<int64_t>(ncol, k0 + nb), k2 = std::min<int64_t>(ncol, k1 + nb);
    panel(k0, k1);
    if (la) {
      add(k1, k2);
      add(k2, ncol);
    } else {
      add(k1, ncol);
    }
  }
  if (slab) add(0, ncol);  // a whole slab: the updates from earlier slabs
  cudaError_t e = cudaMalloc((void**)&tab.d, std::max<size_t>(1, t.size()) * sizeof(uint32_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MAG_ENOMEM, "cudaMalloc(task table) failed: %s", cudaGetErrorString(e));
  }
  if (!t.empty()) {
    e = cudaMemcpy(tab.d, t.data(), t.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(tab.d);
      return fail(ctx, MAG_ECUDA, "task table upload: %s", cudaGetErrorString(e));
    }
  }
  auto ins = ctx->task_tables.emplace(key, std::move(tab));
  ctx->tasks = &ins.first->second;
  return MAG_OK;
}

int ensure_maps(mag_ctx* ctx, int mode, int b) {
  const Layout& L = ctx->lay;
  void* hi = ctx->panel_hi(b);
  if (ctx->maps_base[b] == hi && ctx->maps_mode[b] == mode && ctx->maps_W[b] == L.W && ctx->maps_np[b] == L.np)
    return MAG_OK;
  if (!make_update_maps(&ctx->maps[b], hi, ctx->panel_lo(b), mode, L.W, L.np))
    return fail(ctx, MAG_ECUDA, "cuTensorMapEncodeTiled failed for the panel buffer");
  ctx->maps_base[b] = hi;
  ctx->maps_mode[b] = mode;
  ctx->maps_W[b] = L.W;
  ctx->maps_np[b] = L.np;
  return MAG_OK;
}

// State of one tensor-core factorization: the matrix (packed FP32 tiles of
// n rows = N tile rows, their diagonal inverses, the epilogue's descriptor of
// the tiles), launch parameters and counters.
struct TcFactor {
  mag_ctx* ctx;
  int mode;
  bool pairs;
  int nb;  // panel width in tiles of this factor
  int* launches;
  double* flops;
  int64_t next_ctr;
  float* Z;
  float* Dinv;
  const CMap* cmap;
  int64_t n, N;
  // CTAs of the panel factor's launches: all SMs, or the SMs the trailing
  // update leaves free while it runs beside them (a launch whose CTAs cannot
  // all be resident ends only when the trailing update does)
  int panel_grid;
  // tile columns of Z's layout (tile_index column cap): N for the whole
  // matrix, the slab width for a slab of the out-of-core factor
  int64_t W = 0;
  // FP16 copy of the factor's off-diagonal tiles (one-product factor in
  // core), written by the panel solves; null: none
  void* lh = nullptr;
};

// C_IJ -= sum_{k in [kc_lo, kc_hi)} P_Ik P_Jk^T for J in [j0, j1) with the
// panel of tile column k0 in buffer b, on stream st with at most `grid` CTAs.
int tc_update(TcFactor& F, int b, int64_t k0, int kc_lo, int kc_hi, int64_t j0, int64_t j1, int grid,
              cudaStream_t st, int cat, int max_tasks = 0) {
  mag_ctx* ctx = F.ctx;
  const Layout& L = ctx->lay;
  auto it = ctx->tasks->rng.find(std::make_pair(j0, j1));
  if (it == ctx->tasks->rng.end() || it->second.second == 0) return MAG_OK;
  if (F.next_ctr >= L.nctr_upd) return fail(ctx, MAG_ECUDA, "update launch counters exhausted");
  UpdParams up;
  std::memset(&up, 0, sizeof up);
  up.Z = F.Z;
  up.N = F.N;
  up.k0 = k0;
  up.kc_lo = kc_lo;
  up.kc_hi = kc_hi;
  up.j1 = j1;
  up.tasks = ctx->tasks->d + it->second.first;
  up.ntasks = it->second.second;
  up.counter = ctx->counters() + F.next_ctr++;
  up.st = ctx->st();
  up.timeout_ns = 20000000000ull;
  up.max_tasks = max_tasks;
  up.wcap = F.W > 0 ? F.W : F.N;
  if (max_tasks > 0) {
    // enough CTAs (pairs) for every task at max_tasks each; they start as SMs come free
    const int64_t units = (up.ntasks + max_tasks - 1) / max_tasks;
    grid = (int)std::min<int64_t>(units * (F.pairs ? 2 : 1), 1 << 30);
  }
  TRY(prof_begin(ctx, cat, st));
  CU(launch_update_tc(ctx->maps[b], *F.cmap, up, F.mode, grid, F.pairs, st));
  TRY(prof_end(ctx, st));
  ++*F.launches;
  *F.flops += update_flops(F.N, k0 + kc_lo, k0 + kc_hi, j0, j1);
  return MAG_OK;
}

// Tile columns [a, b) of the panel that starts at k0 (copies go to panel
// buffer `buf`), factored recursively: the left half, then one update of the
// right half with all columns of the left half (K = 128 (mid - a)), then the
// right half; a single column is its diagonal factor + inverse, its panel
// solve and its copy.  Every output tile of the panel is read and written
// once per recursion level instead of once per earlier column.
int tc_panel_range(TcFactor& F, int64_t k0, int64_t a, int64_t b, int buf, cudaStream_t st) {
  mag_ctx* ctx = F.ctx;
  const Layout& L = ctx->lay;
  float* Z = F.Z;
  float* Dinv = F.Dinv;
  if (b - a == 1) {
    TRY(prof_begin(ctx, PC_POTRF, st));
    CU(launch_potrf_diag<float>(Z, Dinv, a, F.n, ctx->st(), st));
    TRY(prof_end(ctx, st));
    if (F.mode == UPD_FP16 || F.mode == UPD_FP16X3) {
      // solve and panel copy in one tensor-core pass
      TRY(prof_begin(ctx, PC_TRSM, st));
      CU(launch_trsm_tc(Z, Dinv, a, F.N, k0, L.W, F.mode, ctx->panel_hi(buf), ctx->panel_lo(buf),
                        ctx->counters() + L.nctr_upd + a, ctx->st(), F.panel_grid, st, F.W > 0 ? F.W : F.N, F.lh));
      TRY(prof_end(ctx, st));
      return MAG_OK;
    }
    TRY(prof_begin(ctx, PC_TRSM, st));
    CU(launch_trsm_col<float>(Z, Dinv, a, F.N, ctx->st(), st));
    TRY(prof_end(ctx, st));
    if (a + 1 < F.N) {
      TRY(prof_begin(ctx, PC_SPLIT, st));
      CU(launch_split_col(Z, a, F.N, k0, L.W, F.mode, ctx->panel_hi(buf), ctx->panel_lo(buf), st));
      TRY(prof_end(ctx, st));
    }
    return MAG_OK;
  }
  const int64_t mid = a + (b - a) / 2;
  TRY(tc_panel_range(F, k0, a, mid, buf, st));
  TRY(tc_update(F, buf, k0, (int)(a - k0), (int)(mid - k0), mid, b, F.panel_grid, st, PC_UPDATE_PANEL));
  return tc_panel_range(F, k0, mid, b, buf, st);
}

// The panel of tile columns [k0, min(N, k0 + nb)) into panel buffer b.
int tc_panel(TcFactor& F, int64_t k0, int b, cudaStream_t st) {
  // a slab's last panel ends at its column cap
  const int64_t k1 = std::min<int64_t>(F.W > 0 ? F.W : F.N, k0 + F.nb);
  return tc_panel_range(F, k0, k0, k1, b, st);
}

// Two-level right-looking Cholesky with the tensor-core updates.  Without
// look-ahead every step runs on the solver's stream.  With look-ahead the
// panel stream updates the next panel's columns with the current panel and
// factors it (into the other panel buffer) while the solver's stream applies
// the current panel to the remaining columns; CTAs of the trailing update are
// capped so that some SMs stay free for the panel stream.
// Two-level right-looking Cholesky of the packed FP32 tiles at Z (N tile
// rows; the first W tile columns are factored, the slab layout tile_index
// with cap W -- W = N is the whole matrix) with the tensor-core updates.
// Dinv receives inv(L_KK) of its diagonal tiles (and the transposes N_global
// tiles further, see launch_potrf_diag).
int factor_tc_on(mag_ctx* ctx, int mode, float* Z, float* Dinv, const CMap* cmap, int64_t N, int64_t W,
                 int* launches, double* flops, bool slab = false, void* lh = nullptr) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  const bool split = mode == UPD_FP16X3 || mode == UPD_TF32X3;
  // panel width by product count (measured at n = 1e5): one-product updates
  // are short and gain from K = 4096 per launch (32 tiles); the split
  // products refine in fewer steps with 16-tile panels
  int nb = std::max(1, std::min(L.nb, ctx->opt.panel_tiles > 0 ? ctx->opt.panel_tiles : (split ? 16 : 32)));
  nb = (int)std::min<int64_t>(nb, W);
  const int64_t npanels = (W + nb - 1) / nb;
  const bool la = ctx->opt.lookahead != 0 && npanels > 2;
  const bool pairs = ctx->opt.cta_pairs == 1 || (ctx->opt.cta_pairs == 2 && split);
  TRY(ensure_tasks(ctx, N, nb, la, pairs, W, slab));
  TRY(ensure_maps(ctx, mode, 0));
  TRY(ensure_maps(ctx, mode, 1));
  CU(cudaMemsetAsync(ctx->counters(), 0, (size_t)L.nctr * sizeof(unsigned), s));
  TcFactor F{ctx, mode, pairs, nb, launches, flops, 0, Z, Dinv, cmap, L.n, N, ctx->sm_count};
  F.W = W;
  F.lh = lh;
  if (!la) {
    for (int64_t k0 = 0; k0 < W; k0 += nb) {
      const int64_t k1 = std::min<int64_t>(W, k0 + nb);
      TRY(tc_panel(F, k0, 0, s));
      if (k1 < W) TRY(tc_update(F, 0, k0, 0, (int)(k1 - k0), k1, W, ctx->sm_count, s, PC_UPDATE));
    }
    return MAG_OK;
  }
  if (!ctx->side) {
    // the panel stream outranks the solver's stream: CTAs of its launches
    // are placed on SMs before pending CTAs of the trailing update
    int least = 0, greatest = 0;
    CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CU(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest));
    for (int i = 0; i < 3; ++i) CU(cudaEventCreateWithFlags(&ctx->ev_la[i], cudaEventDisableTiming));
  }
  cudaStream_t side = ctx->side;
  cudaEvent_t ev_start = ctx->ev_la[0], ev_panel = ctx->ev_la[1], ev_trail = ctx->ev_la[2];
  // Two ways to share the GPU between the streams.  lookahead_sms > 0: the
  // trailing update is a persistent launch on all but that many SMs, and
  // the panel factor's launches beside it are capped at the rest.  Else
  // (default): every trailing CTA (pair) leaves after `tpc` 256 x 256 output
  // blocks (4: measured at n = 1e5 against 5 to 20, and 16 to 32 reserved
  // SMs; -lookahead_sms sets it), so SMs come free all the time and the
  // panel stream's launches, on the higher-priority stream, take them first.
  const bool reserved = ctx->opt.lookahead_sms > 0;
  const int reserve = reserved ? ctx->opt.lookahead_sms : 0;
  const int tpc = ctx->opt.lookahead_sms < 0 ? -ctx->opt.lookahead_sms : 4;
  const int trail_grid = reserved ? std::max(1, ctx->sm_count - reserve) : ctx->sm_count;
  const int trail_tasks = reserved ? 0 : tpc;
  CU(cudaEventRecord(ev_start, s));
  CU(cudaStreamWaitEvent(side, ev_start, 0));
  TRY(tc_panel(F, 0, 0, side));  // nothing runs beside the first panel: all SMs
  CU(cudaEventRecord(ev_panel, side));
  const int beside = reserved ? std::max(1, std::min(ctx->sm_count, reserve)) : ctx->sm_count;
  int64_t p = 0;
  for (int64_t k0 = 0;; k0 += nb, ++p) {
    const int64_t k1 = std::min<int64_t>(W, k0 + nb);
    if (k1 >= W) break;
    const int64_t k2 = std::min<int64_t>(W, k1 + nb);
    const int b = (int)(p & 1);
    CU(cudaStreamWaitEvent(s, ev_panel, 0));  // panel p factored and copied
    // panel stream: next panel's columns, then the next panel itself
    TRY(tc_update(F, b, k0, 0, (int)(k1 - k0), k1, k2, ctx->sm_count, side, PC_UPDATE));
    F.panel_grid = k2 < W ? beside : ctx->sm_count;  // the last panel runs alone
    TRY(tc_panel(F, k1, b ^ 1, side));
    CU(cudaEventRecord(ev_panel, side));
    // solver stream: the rest of the trailing matrix
    if (k2 < W) TRY(tc_update(F, b, k0, 0, (int)(k1 - k0), k2, W, trail_grid, s, PC_UPDATE, trail_tasks));
    CU(cudaEventRecord(ev_trail, s));
    CU(cudaStreamWaitEvent(side, ev_trail, 0));  // columns of panel p+2 and buffer b are free
  }
  CU(cudaStreamWaitEvent(s, ev_panel, 0));
  return MAG_OK;
}

// The in-core factor: the whole packed matrix of the workspace.
int factor_tc(mag_ctx* ctx, int mode, int* launches, double* flops, void* lh = nullptr) {
  const Layout& L = ctx->lay;
  if (ctx->cmap_base != ctx->zf() || ctx->cmap_tiles != L.tiles) {
    if (!make_c_map(&ctx->cmap, ctx->zf(), L.tiles))
      return fail(ctx, MAG_ECUDA, "cuTensorMapEncodeTiled failed for the factor tiles");
    ctx->cmap_base = ctx->zf();
    ctx->cmap_tiles = L.tiles;
  }
  return factor_tc_on(ctx, mode, ctx->zf(), ctx->dinvf(), &ctx->cmap, L.N, L.N, launches, flops, false, lh);
}

// ------------------------------------------------------------ out of core
// When the packed FP32 tiles of Z do not fit in device memory (or the
// workspace limit), the factor runs slab by slab (mag_internal.cuh: slab
// layout).  The device keeps a pool of tiles: the first slab, as wide as
// two thirds of the pool allows, is generated, factored and kept there; the
// remaining columns go through a working buffer (the last third) one slab
// at a time, each copied to pinned host memory once factored, except the
// last, which stays.  Slab s is first updated with every earlier slab q
// (C -= L_q L_q^T restricted to its rows and columns): the FP16 panel copies
// of q's columns are gathered K chunk by K chunk (from device or host memory)
// into the panel buffers and applied by the tensor-core update kernel; then
// its columns are factored by the right-looking two-level factor.

// Widest slab (tile columns) of `rows` tile rows in `cap` tiles (0 if none).
int64_t slab_width(int64_t rows, int64_t cap) {
  int64_t lo = 0, hi = rows;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (num_slab_tiles(rows, mid) <= cap) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Host memory the host slabs may take: options.host_limit_bytes, else half
// of the machine's physical memory.
double host_limit(const mag_ctx* ctx) {
  if (ctx->opt.host_limit_bytes > 0) return ctx->opt.host_limit_bytes;
  const long pages = sysconf(_SC_PHYS_PAGES), psz = sysconf(_SC_PAGE_SIZE);
  return pages > 0 && psz > 0 ? 0.5 * (double)pages * (double)psz : 0.0;
}

// Decide whether the solve of size n factors out of core and, if so, plan
// the slabs and the device pool (pool_tiles > 0 on return).  In core: 0.
int plan_out_of_core(mag_ctx* ctx, int64_t n, int prec, int64_t* pool_tiles) {
  *pool_tiles = 0;
  ctx->slabs.clear();
  const mag_options& o = ctx->opt;
  if (o.out_of_core < 0) return MAG_OK;
  // the slab generator forms Z = exp[-t d]; the scale-zero and the deflated
  // systems are solved in core
  if (ctx->kind != MAT_EXP) return MAG_OK;
  const bool fp16_kind = prec == MAG_PREC_AUTO || prec == MAG_PREC_FP16 || prec == MAG_PREC_FP16X3;
  if (!fp16_kind) {
    if (o.out_of_core > 0)
      return fail(ctx, MAG_EINVAL, "the out-of-core factor runs the FP16 and FP16X3 (or AUTO) precisions");
    return MAG_OK;
  }
  size_t fre = 0, tot = 0;
  if (cudaMemGetInfo(&fre, &tot) != cudaSuccess) {
    cudaGetLastError();
    fre = 0;
  }
  double avail = 0.95 * ((double)fre + (double)ctx->ws_bytes);
  if (o.workspace_limit_bytes > 0) avail = std::min(avail, o.workspace_limit_bytes);
  const Layout incore = plan(ctx, n, true, false);
  if (o.out_of_core == 0 && (double)incore.total <= avail) return MAG_OK;
  const Layout base = plan(ctx, n, true, false, false, 0);
  const double tile_bytes = (double)TILE_ELEMS * sizeof(float);
  const int64_t pool = (int64_t)std::floor((avail - (double)base.total - 4096.0) / tile_bytes);
  const int64_t N = incore.N;
  if (pool < 1) return fail(ctx, MAG_ENOMEM, "no device memory left for the out-of-core factor's tiles");
  std::vector<Slab> sl;
  int64_t host_tiles = 0;
  if (num_lower_tiles(N) <= pool) {
    Slab a;
    a.c0 = 0;
    a.S = N;
    a.tiles = num_lower_tiles(N);
    sl.push_back(a);
  } else {
    const int64_t work = pool / 3, resident = pool - work;
    int64_t c0 = slab_width(N, resident), used = 0;
    if (c0 > 0) {
      Slab a;
      a.c0 = 0;
      a.S = c0;
      a.tiles = num_slab_tiles(N, c0);
      sl.push_back(a);
      used = a.tiles;
    }
    while (c0 < N) {
      Slab b;
      b.c0 = c0;
      b.S = slab_width(N - c0, work);
      if (b.S < 1) return fail(ctx, MAG_ENOMEM, "device pool of %lld tiles too small for a slab", (long long)pool);
      b.tiles = num_slab_tiles(N - c0, b.S);
      b.pool_off = used;
      c0 += b.S;
      b.host = c0 < N;  // the last slab stays on the device
      if (b.host) {
        b.host_off = host_tiles;
        host_tiles += b.tiles;
      }
      sl.push_back(b);
    }
  }
  const double host_bytes = (double)host_tiles * tile_bytes;
  if (host_bytes > host_limit(ctx))
    return fail(ctx, MAG_ENOMEM, "out-of-core factor needs %.3g GB of host memory (limit %.3g GB)", host_bytes / 1e9,
                host_limit(ctx) / 1e9);
  if (host_tiles > 0 && (size_t)host_bytes > ctx->host_L_bytes) {
    if (ctx->host_L) {
      cudaStreamSynchronize(ctx->stream);
      cudaFreeHost(ctx->host_L);
      ctx->host_L = nullptr;
      ctx->host_L_bytes = 0;
    }
    void* h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, (size_t)host_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, MAG_ENOMEM, "pinned host memory of %.3g GB: %s", host_bytes / 1e9, cudaGetErrorString(e));
    }
    void* d = nullptr;
    e = cudaHostGetDevicePointer(&d, h, 0);
    if (e != cudaSuccess || d != h) {
      cudaGetLastError();
      cudaFreeHost(h);
      return fail(ctx, MAG_ECUDA, "host memory is not addressed alike on the device");
    }
    ctx->host_L = static_cast<float*>(h);
    ctx->host_L_bytes = (size_t)host_bytes;
  }
  int64_t need = 0;
  for (const Slab& x : sl) need = std::max(need, x.pool_off + x.tiles);
  ctx->slabs = sl;
  *pool_tiles = need;
  return MAG_OK;
}

// The quantized coordinates of this solve's points (defined with generate).
const long long* quantized(mag_ctx* ctx, const double* X, int64_t n, int32_t m);

// The out-of-core factor of Z = exp[-t d] in an FP16 kind (UPD_FP16X3 or
// UPD_FP16).  slab0_ready: slab 0 is already generated (the precision probe
// read its leading block).
int factor_ooc(mag_ctx* ctx, const double* X, int32_t m, double t, int mode, bool slab0_ready, int* launches,
               double* flops, double* host_read_bytes) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  const bool split = mode == UPD_FP16X3;
  const bool pairs = ctx->opt.cta_pairs != 0;
  for (size_t si = 0; si < ctx->slabs.size(); ++si) {
    const Slab& sl = ctx->slabs[si];
    float* Zs = ctx->slab_dev(sl);
    const int64_t rows = L.N - sl.c0;
    if (!(si == 0 && slab0_ready)) {
      const long long* q = quantized(ctx, X, L.n, m);
      CU(launch_generate_slab(X, L.n, m, t, sl.c0, sl.S, Zs, ctx->st(), s, INFINITY, q, ctx->xq_L, ctx->xq_e,
                              ctx->xq_tau2));
    }
    if (ctx->slab_cmap_base != Zs || ctx->slab_cmap_tiles != sl.tiles) {
      if (!make_c_map(&ctx->slab_cmap, Zs, sl.tiles))
        return fail(ctx, MAG_ECUDA, "cuTensorMapEncodeTiled failed for a slab");
      ctx->slab_cmap_base = Zs;
      ctx->slab_cmap_tiles = sl.tiles;
    }
    if (si > 0) {
      // C -= L_q L_q^T from every earlier slab, K chunks of at most L.nb
      // tiles gathered into the two panel buffers in turn
      const int nb = (int)std::min<int64_t>(L.nb, 32);
      TRY(ensure_tasks(ctx, rows, nb, false, pairs, sl.S, true));
      TRY(ensure_maps(ctx, mode, 0));
      TRY(ensure_maps(ctx, mode, 1));
      CU(cudaMemsetAsync(ctx->counters(), 0, (size_t)L.nctr_upd * sizeof(unsigned), s));
      TcFactor F{ctx, mode, pairs, nb, launches, flops, 0, Zs, ctx->dinvf(), &ctx->slab_cmap, L.n, rows,
                 ctx->sm_count};
      F.W = sl.S;
      int buf = 0;
      for (size_t qi = 0; qi < si; ++qi) {
        const Slab& q = ctx->slabs[qi];
        for (int64_t k = q.c0; k < q.c0 + q.S; k += nb) {
          const int kw = (int)std::min<int64_t>(nb, q.c0 + q.S - k);
          if (F.next_ctr >= L.nctr_upd) {
            CU(cudaMemsetAsync(ctx->counters(), 0, (size_t)L.nctr_upd * sizeof(unsigned), s));
            F.next_ctr = 0;
          }
          // gathers from host slabs are timed (profile = 1): the reads over
          // the CPU-GPU link
          if (q.host) TRY(prof_begin(ctx, PC_HOST_READ, s));
          CU(launch_gather_split(ctx->slab_data(q), q.c0, q.S, sl.c0, rows, k, kw, ctx->panel_hi(buf),
                                 ctx->panel_lo(buf), L.W, split, s));
          if (q.host) {
            TRY(prof_end(ctx, s));
            *host_read_bytes += (double)rows * kw * TILE_ELEMS * sizeof(float);
          }
          TRY(tc_update(F, buf, 0, 0, kw, 0, sl.S, ctx->sm_count, s, PC_UPDATE));
          buf ^= 1;
        }
      }
    }
    TRY(factor_tc_on(ctx, mode, Zs, ctx->dinvf() + sl.c0 * TILE_ELEMS, &ctx->slab_cmap, rows, sl.S, launches,
                     flops, true));
    if (sl.host)
      CU(cudaMemcpyAsync(ctx->host_L + sl.host_off * TILE_ELEMS, Zs, (size_t)sl.tiles * TILE_ELEMS * sizeof(float),
                         cudaMemcpyDeviceToHost, s));
  }
  return MAG_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

const char* mag_status_string(int status) {
  switch (status) {
    case MAG_OK: return "MAG_OK";
    case MAG_EINVAL: return "MAG_EINVAL";
    case MAG_EDUPLICATE: return "MAG_EDUPLICATE";
    case MAG_ENOTPD: return "MAG_ENOTPD";
    case MAG_ENOCONV: return "MAG_ENOCONV";
    case MAG_ENOBRACKET: return "MAG_ENOBRACKET";
    case MAG_ENOMEM: return "MAG_ENOMEM";
    case MAG_ECUDA: return "MAG_ECUDA";
    case MAG_ETIMEOUT: return "MAG_ETIMEOUT";
    default: return "MAG_UNKNOWN";
  }
}

int mag_options_default(mag_options* opt) {
  if (!opt) return MAG_EINVAL;
  std::memset(opt, 0, sizeof *opt);
  opt->precision = MAG_PREC_AUTO;
  opt->residual_mode = MAG_RESID_AUTO;
  opt->ir_tol = 1e-14;
  opt->ir_max_iters = 12;
  opt->gmres_max_iters = 30;
  opt->allow_fallback = 1;
  opt->panel_tiles = 0;
  opt->workspace_limit_bytes = 0.0;
  opt->profile = 0;
  opt->reuse_distances = 1;
  opt->lookahead = 1;
  opt->lookahead_sms = 0;
  opt->cta_pairs = 1;
  opt->tplus_method = 0;
  opt->wait_timeout_ns = 10000000000ll;
  opt->out_of_core = 0;
  opt->deflate = 0;
  opt->host_limit_bytes = 0.0;
  opt->gmres_matvec = 0;
  opt->fp16_gmres = 0;
  opt->batch_shape = 0;
  opt->sweep_kind = 0;
  opt->exact_distances = 1;
  opt->reserved4 = 0;
  return MAG_OK;
}

int mag_ctx_create(mag_ctx** out, void* stream, const mag_options* opt) {
  if (!out) return MAG_EINVAL;
  *out = nullptr;
  mag_ctx* ctx = new (std::nothrow) mag_ctx();
  if (!ctx) return MAG_ENOMEM;
  ctx->stream = (cudaStream_t)stream;
  if (opt && opt->wait_timeout_ns <= 0) {
    delete ctx;
    return MAG_EINVAL;
  }
  if (opt)
    ctx->opt = *opt;
  else
    mag_options_default(&ctx->opt);
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_st, sizeof(DevStatus));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (int i = 0; i < 4; ++i)
      if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    delete ctx;
    return MAG_ECUDA;
  }
  *out = ctx;
  return MAG_OK;
}

int mag_ctx_set_options(mag_ctx* ctx, const mag_options* opt) {
  if (!ctx || !opt) return MAG_EINVAL;
  if (opt->wait_timeout_ns <= 0) return fail(ctx, MAG_EINVAL, "wait_timeout_ns must be > 0");
  ctx->opt = *opt;
  return MAG_OK;
}

int mag_ctx_destroy(mag_ctx* ctx) {
  if (!ctx) return MAG_OK;
  if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->bws) cudaFree(ctx->bws);
  if (ctx->gm) cudaFree(ctx->gm);
  if (ctx->probe_z) cudaFree(ctx->probe_z);
  if (ctx->chain_s) cudaFree(ctx->chain_s);
  if (ctx->xq) cudaFree(ctx->xq);
  if (ctx->lh) cudaFree(ctx->lh);
  if (ctx->host_L) cudaFreeHost(ctx->host_L);
  for (auto& kv : ctx->task_tables)
    if (kv.second.d) cudaFree(kv.second.d);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  for (int i = 0; i < 3; ++i)
    if (ctx->ev_la[i]) cudaEventDestroy(ctx->ev_la[i]);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  for (int i = 0; i < 4; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  delete ctx;
  return MAG_OK;
}

const char* mag_last_error(const mag_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int mag_workspace_bytes(const mag_ctx* ctx, int64_t n, int32_t m, double* bytes) {
  (void)m;
  if (!ctx || !bytes || n < 1) return MAG_EINVAL;
  const int prec = ctx->opt.precision;
  const bool f64 = prec == MAG_PREC_FP64 || ctx->opt.residual_mode != MAG_RESID_MATRIX_FREE;
  const bool f32 = prec != MAG_PREC_FP64;
  *bytes = (double)plan(ctx, n, f32, f64).total;
  return MAG_OK;
}

int mag_min_distance(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double* dmin,
                     double* t_bound) {
  TRY(check_args(ctx, points, n, m, 1.0));
  if (!dmin || !t_bound) return fail(ctx, MAG_EINVAL, "NULL output");
  ctx->err.clear();
  // Only the status block and vectors are needed; reuse whatever layout fits.
  if (!ctx->ws || ctx->lay.np < ((n + TILE - 1) / TILE) * TILE) TRY(ensure_workspace(ctx, n, false, false));
  TRY(reset_status(ctx));
  CU(launch_min_distance(points, n, m, ctx->st(), ctx->stream));
  TRY(read_status(ctx));
  const int fl = ctx->h_st->flags;
  const double d2 = bits_to_double(ctx->h_st->min_d2_bits);
  if (fl & ST_NONFINITE) return fail(ctx, MAG_EINVAL, "non-finite coordinate");
  *dmin = std::sqrt(d2);
  if (fl & ST_DUPLICATE || !(d2 > 0.0)) {
    *dmin = 0.0;
    *t_bound = INFINITY;
    return fail(ctx, MAG_EDUPLICATE, "two points coincide");
  }
  *t_bound = std::log((double)(n - 1)) / *dmin;
  return MAG_OK;
}

int mag_scale_zero(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double* w0, double* s,
                   mag_info* info) {
  TRY(check_args(ctx, points, n, m, 1.0));
  if (!w0 || !s) return fail(ctx, MAG_EINVAL, "NULL output");
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  // c >= 2 max d from 2 max_j ||x_j - x_0|| (triangle inequality through x_0)
  if (!ctx->ws || ctx->lay.np < ((n + TILE - 1) / TILE) * TILE) TRY(ensure_workspace(ctx, n, false, false));
  TRY(reset_status(ctx));
  CU(launch_far_from_first(points, n, m, ctx->st(), ctx->stream));
  TRY(read_status(ctx));
  const double far = std::sqrt(bits_to_double(ctx->h_st->far_d2_bits));
  if (!std::isfinite(far)) return fail(ctx, MAG_EINVAL, "non-finite coordinate");
  if (!(far > 0.0)) return fail(ctx, MAG_EDUPLICATE, "all points coincide");
  double c = 4.0 * far;
  // M = 1 1^T - d / c is positive definite for c large enough; d^{-1} 1 is
  // proportional to M^{-1} 1 (Sherman-Morrison), so w0 = z / 1^T z with M z = 1
  double sz = 0.0;
  mag_info zi;
  int st = MAG_ENOTPD;
  for (int attempt = 0; attempt < 8 && st == MAG_ENOTPD; ++attempt) {
    ctx->kind = MAT_SHIFTED_DIST;
    st = mag_solve(ctx, points, n, m, 1.0 / c, w0, &sz, &zi);
    ctx->kind = MAT_EXP;
    if (st == MAG_ENOTPD) c *= 2.0;
  }
  if (info) *info = zi;
  if (st != MAG_OK && st != MAG_ENOCONV) return st;
  if (!(sz > 0.0) || !std::isfinite(sz)) return fail(ctx, MAG_ENOCONV, "1^T z = %g is not positive", sz);
  CU(launch_scale(w0, 1.0 / sz, w0, n, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  // M z = 1  =>  d z = c (1^T z - 1) 1  =>  1^T d^{-1} 1 = 1^T z / (c (1^T z - 1))
  *s = sz / (c * (sz - 1.0));
  if (info) info->min_w = zi.min_w / sz;
  return st;
}

}  // extern "C"

// ------------------------------------------------------------ the solve
namespace {

struct SolveResult {
  int prec_used = 0, ir_iters = 0, gmres_iters = 0, fallback = 0;
  double rel = INFINITY, znorm = 0, wnorm = 0, gersh = 0, dmin = 0;
  double ms_gen = 0, ms_fac = 0, ms_solve = 0, ms_res = 0;
  int residual_evals = 0, update_launches = 0;
  bool stored = false;
  double ms_update = 0, update_flops = 0, ms_update_panel = 0, ms_potrf = 0, ms_trsm = 0, ms_split = 0;
  double ms_update_busy = 0;
  int residual_evals_ff = 0;
  int sweeps_used = -1;
  int exact_distances = 0;
  double probe_rho = 0, ms_probe = 0;
  int slabs = 0, host_slabs = 0;
  double host_bytes = 0, host_read_bytes = 0, ms_host_read = 0;
  double deflation_c = 0;
  int factor_reused = 0;
};

float elapsed(mag_ctx* ctx, int a, int b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) != cudaSuccess) {
    cudaGetLastError();  // an event not recorded on this path: no time, no pending error
    ms = 0.f;
  }
  return ms;
}

// Generate the tiles for the given precision into the current layout.
// tiny_fp32: entries below e^-46 in FP32 (exp_neg_tiny_td), for the solve path;
// the entry points that return Z or differentiate it keep FP64 everywhere.
// Coordinates quantized for the exact distance pass (launch_dist_q): per
// dimension the minimum lo_l, the largest span S < 2^E, limbs of L bits with
// m 2^(2L) <= 2^63 (the kernel's 64-bit sums cannot wrap), B = 2L - 1 bits
// per coordinate, scale 2^e with e = B - E (every coordinate offset below
// 2^B), and tau2 = m 2^(106 - 2e): at d >= sqrt(tau2) the quantization
// (at most 2 sqrt(m) 2^-e in d) is below 2^-52 d.  false: FP64 differences
// instead (a non-finite coordinate, every dimension constant, m > 32, a
// scale beyond 2^+-400, or no memory for the copy).
bool quantize_points(mag_ctx* ctx, const double* X, int64_t n, int32_t m, int* L, int* e, double* tau2,
                     const long long** Xq) {
  ctx->xq_ok = false;
  if (!ctx->opt.exact_distances || m > 32 || m < 1) return false;
  const size_t head = ((size_t)(2 * m + 1) * sizeof(double) + 255) & ~(size_t)255;
  if (!grow_buffer(ctx, &ctx->xq, &ctx->xq_bytes, head + (size_t)n * m * sizeof(long long), 0)) return false;
  double* range = (double*)ctx->xq;
  long long* q = (long long*)((char*)ctx->xq + head);
  cudaStream_t s = ctx->stream;
  std::vector<double> h(2 * m + 1);
  if (launch_coord_range(X, n, m, range, s) != cudaSuccess ||
      cudaMemcpyAsync(h.data(), range, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (h[2 * m] != 0.0) return false;
  double S = 0.0;
  for (int l = 0; l < m; ++l) S = std::max(S, h[2 * l + 1] - h[2 * l]);
  if (!(S > 0.0) || !std::isfinite(S)) return false;
  const int E = std::ilogb(S) + 1;  // S < 2^E
  int mb = 0;
  while ((1 << mb) < m) ++mb;
  *L = (63 - mb) / 2;
  *e = (2 * *L - 1) - E;
  if (*e < -400 || *e > 400) return false;
  *tau2 = std::ldexp((double)m, 106 - 2 * *e);
  if (launch_quantize(X, n, m, range, *e, q, s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *Xq = q;
  ctx->xq_ok = true;
  ctx->xq_pts = X;
  ctx->xq_n = n;
  ctx->xq_m = m;
  ctx->xq_L = *L;
  ctx->xq_e = *e;
  ctx->xq_tau2 = *tau2;
  ctx->xq_q = q;
  return true;
}

// The quantized coordinates of this solve's points for the matrix-free
// residual (quantize_points on first use; null: FP64 differences).
const long long* quantized(mag_ctx* ctx, const double* X, int64_t n, int32_t m) {
  if (ctx->xq_ok && ctx->xq_pts == X && ctx->xq_n == n && ctx->xq_m == m) return ctx->xq_q;
  int L = 0, e = 0;
  double tau2 = 0.0;
  const long long* q = nullptr;
  if (!quantize_points(ctx, X, n, m, &L, &e, &tau2, &q)) {
    ctx->xq_ok = false;
    return nullptr;
  }
  return q;
}

int generate(mag_ctx* ctx, const double* X, int32_t m, double t, bool f32, bool f64, SolveResult* R,
             bool tiny_fp32 = false) {
  const double tiny_arg = tiny_fp32 ? kTinyArg : INFINITY;
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  TRY(reset_status(ctx));
  CU(cudaMemsetAsync(ctx->vd(V_ROWSUM), 0, L.np * sizeof(double), s));
  CU(cudaEventRecord(ctx->ev[0], s));
  const bool reuse = ctx->dist_active && L.dist && ctx->dist_valid && ctx->dist_pts == X && ctx->dist_n == L.n &&
                     ctx->dist_m == m;
  if (reuse) {
    CU(launch_generate_from_dist(ctx->dist(), L.n, t, L.N, f32 ? ctx->zf() : nullptr, f64 ? ctx->zd() : nullptr,
                                 ctx->vd(V_ROWSUM), s, ctx->kind, tiny_arg, ctx->kind_c));
  } else if (ctx->dist_active && L.dist) {
    int qL = 0, qe = 0;
    double qtau2 = 0.0;
    const long long* Xq = nullptr;
    if (quantize_points(ctx, X, L.n, m, &qL, &qe, &qtau2, &Xq)) {
      // exact d^2 on the integer pipe, then Z from the distances
      CU(launch_dist_q(Xq, X, L.n, m, qL, qe, qtau2, L.N, ctx->dist(), ctx->st(), s));
      CU(launch_generate_from_dist(ctx->dist(), L.n, t, L.N, f32 ? ctx->zf() : nullptr, f64 ? ctx->zd() : nullptr,
                                   ctx->vd(V_ROWSUM), s, ctx->kind, tiny_arg, ctx->kind_c));
      R->exact_distances = 1;
    } else {
      CU(launch_generate_dist(X, L.n, m, t, L.N, f32 ? ctx->zf() : nullptr, f64 ? ctx->zd() : nullptr,
                              ctx->dist(), ctx->vd(V_ROWSUM), ctx->st(), s, ctx->kind, tiny_arg, ctx->kind_c));
    }
  } else {
    int qL = 0, qe = 0;
    double qtau2 = 0.0;
    const long long* Xq = nullptr;
    if (quantize_points(ctx, X, L.n, m, &qL, &qe, &qtau2, &Xq)) {
      CU(launch_generate_q(Xq, X, L.n, m, qL, qe, qtau2, t, L.N, f32 ? ctx->zf() : nullptr,
                           f64 ? ctx->zd() : nullptr, ctx->vd(V_ROWSUM), ctx->st(), s, ctx->kind, tiny_arg,
                           ctx->kind_c));
      R->exact_distances = 1;
    } else {
      CU(launch_generate(X, L.n, m, t, L.N, f32 ? ctx->zf() : nullptr, f64 ? ctx->zd() : nullptr,
                         ctx->vd(V_ROWSUM), ctx->st(), s, ctx->kind, tiny_arg, ctx->kind_c));
    }
  }
  CU(launch_rowsum_max(ctx->vd(V_ROWSUM), L.n, ctx->st(), s));
  CU(cudaEventRecord(ctx->ev[1], s));
  TRY(read_status(ctx));
  R->ms_gen += elapsed(ctx, 0, 1);
  if (reuse) {
    R->dmin = ctx->dist_dmin;
    R->exact_distances = ctx->dist_exact ? 1 : 0;
    R->gersh = 1.0 - bits_to_double(ctx->h_st->off_max_bits);
    return MAG_OK;
  }
  const int fl = ctx->h_st->flags;
  if (fl & ST_NONFINITE) return fail(ctx, MAG_EINVAL, "non-finite coordinate in points");
  const double d2 = bits_to_double(ctx->h_st->min_d2_bits);
  R->dmin = std::sqrt(d2);
  if ((fl & ST_DUPLICATE) || !(d2 > 0.0)) return fail(ctx, MAG_EDUPLICATE, "two points coincide (min d = 0)");
  R->gersh = 1.0 - bits_to_double(ctx->h_st->off_max_bits);
  if (ctx->dist_active && L.dist) {
    ctx->dist_valid = true;
    ctx->dist_pts = X;
    ctx->dist_n = L.n;
    ctx->dist_m = m;
    ctx->dist_dmin = R->dmin;
    ctx->dist_exact = R->exact_distances != 0;
  }
  return MAG_OK;
}

// Turn distance reuse on for one call when it is allowed and the FP64
// distance tiles fit next to the largest workspace the solve may need.
void begin_dist_reuse(mag_ctx* ctx, int64_t n) {
  ctx->dist_valid = false;
  ctx->dist_active = false;
  if (!ctx->opt.reuse_distances) return;
  size_t fre = 0, tot = 0;
  if (cudaMemGetInfo(&fre, &tot) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const Layout with = plan(ctx, n, true, true, true);
  ctx->dist_active = (double)with.total <= 0.8 * ((double)fre + (double)ctx->ws_bytes);
}
void end_dist_reuse(mag_ctx* ctx) {
  ctx->dist_active = false;
  ctx->dist_valid = false;
}

int run_factor(mag_ctx* ctx, int prec, SolveResult* R) {
  cudaStream_t s = ctx->stream;
  const Layout& L = ctx->lay;
  ctx->chain_ready = ctx->lh_ready = false;
  const bool chain = prec != MAG_PREC_FP64 && ctx->opt.sweep_kind != 2 &&
                     grow_buffer(ctx, (void**)&ctx->chain_s, &ctx->chain_s_bytes,
                                 (size_t)2 * L.N * TILE_ELEMS * sizeof(float), 0);
  void* lh = nullptr;
  if (chain && ctx->opt.sweep_kind == 0 && prec != MAG_PREC_FP32 && upd_mode(prec) == UPD_FP16 &&
      grow_buffer(ctx, &ctx->lh, &ctx->lh_bytes, (size_t)L.tiles * TILE_ELEMS * 2, 1u << 30))
    lh = ctx->lh;
  CU(cudaEventRecord(ctx->ev[0], s));
  ctx->prof_used = 0;
  if (prec == MAG_PREC_FP64)
    TRY(factor_blocked<double>(ctx, ctx->zd(), ctx->dinvd(), &R->update_launches, &R->update_flops));
  else if (prec == MAG_PREC_FP32)
    TRY(factor_blocked<float>(ctx, ctx->zf(), ctx->dinvf(), &R->update_launches, &R->update_flops));
  else
    TRY(factor_tc(ctx, upd_mode(prec), &R->update_launches, &R->update_flops, lh));
  if (chain) CU(launch_chain_prep(ctx->zf(), ctx->dinvf(), L.N, ctx->chain_s, ctx->chain_s + L.N * TILE_ELEMS, s));
  CU(cudaEventRecord(ctx->ev[1], s));
  TRY(read_status(ctx));
  R->ms_fac += elapsed(ctx, 0, 1);
  double pc[PC_COUNT], busy = 0;
  R->ms_update += prof_collect(ctx, pc, &busy);
  R->ms_update_busy += busy;
  R->ms_update_panel += pc[PC_UPDATE_PANEL];
  R->ms_potrf += pc[PC_POTRF];
  R->ms_trsm += pc[PC_TRSM];
  R->ms_split += pc[PC_SPLIT];
  if (ctx->h_st->flags & ST_TIMEOUT)
    return fail(ctx, MAG_ETIMEOUT, "a bounded device wait in the tensor-core update expired");
  if (ctx->h_st->flags & ST_NOTPD)
    return fail(ctx, MAG_ENOTPD, "non-positive pivot at row %d (precision %d)", ctx->h_st->notpd_index - 1,
                prec);
  ctx->chain_ready = chain;
  ctx->lh_ready = chain && lh != nullptr;
  ctx->chain_N = L.N;
  return MAG_OK;
}

// x = (init ? 0 : x) + r_max * (L L^T)^{-1} (r / r_max) with the current
// factor; r_max = max|r| must already be in the status block.
// The factor is that of the leading n rows (N tile rows, np = 128 N).
template <typename T>
int correction_t(mag_ctx* ctx, T* Z, T* Dinv, T* v, T* y, const double* r, double* x, bool init, int64_t n,
                 int64_t np, int64_t N) {
  cudaStream_t s = ctx->stream;
  CU(launch_scale_rhs<T>(r, n, np, v, ctx->st(), s));
  const uint64_t tmo = (uint64_t)ctx->opt.wait_timeout_ns;
  CU(launch_forward_persistent<T>(Z, Dinv, N, v, y, ctx->flags(), ctx->st(), tmo, s));
  CU(launch_backward_persistent<T>(Z, Dinv, N, y, v, ctx->flags(), ctx->st(), tmo, s));
  CU(launch_accumulate<T>(x, v, n, ctx->st(), init, s));
  return MAG_OK;
}

// The same correction with the out-of-core factor: forward and backward
// substitution slab by slab (each slab's triangle by the persistent sweeps,
// its rectangle below by a product with the rows that follow), reading every
// slab where it lives.
int correction_ooc(mag_ctx* ctx, const double* r, double* x, bool init) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  const uint64_t tmo = (uint64_t)ctx->opt.wait_timeout_ns;
  float* v = ctx->vf(F_V);
  float* y = ctx->vf(F_Y);
  float* Dinv = ctx->dinvf();
  float* DinvT = Dinv + L.N * TILE_ELEMS;
  CU(launch_scale_rhs<float>(r, L.n, L.np, v, ctx->st(), s));
  for (const Slab& sl : ctx->slabs) {  // L y = v
    const float* Ls = ctx->slab_data(sl);
    const int64_t o = sl.c0 * TILE, below = L.N - sl.c0 - sl.S;
    CU(launch_forward_sweep<float>(Ls, DinvT + sl.c0 * TILE_ELEMS, sl.S, v + o, y + o, ctx->flags(), ctx->st(), tmo,
                                   sl.host, s));
    CU(launch_rect_gemv(Ls + num_lower_tiles(sl.S) * TILE_ELEMS, below, sl.S, y + o, v + o + sl.S * TILE, s));
  }
  for (size_t i = ctx->slabs.size(); i-- > 0;) {  // L^T x = y, x into v
    const Slab& sl = ctx->slabs[i];
    const float* Ls = ctx->slab_data(sl);
    const int64_t o = sl.c0 * TILE, below = L.N - sl.c0 - sl.S;
    CU(launch_rect_gemv_t(Ls + num_lower_tiles(sl.S) * TILE_ELEMS, below, sl.S, v + o + sl.S * TILE, y + o, s));
    CU(launch_backward_sweep<float>(Ls, Dinv + sl.c0 * TILE_ELEMS, sl.S, y + o, v + o, ctx->flags(), ctx->st(), tmo,
                                    sl.host, s));
  }
  CU(launch_accumulate<float>(x, v, L.n, ctx->st(), init, s));
  return MAG_OK;
}

// The same correction with the in-core sweeps of k_chain.cu (the B tiles
// formed after the factor; FP16 off-diagonal tiles when the one-product
// factor wrote them).
int correction_chain(mag_ctx* ctx, const double* r, double* x, bool init) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  const uint64_t tmo = (uint64_t)ctx->opt.wait_timeout_ns;
  float* v = ctx->vf(F_V);
  float* y = ctx->vf(F_Y);
  const float* Sf = ctx->chain_s;
  const float* Sb = ctx->chain_s + L.N * TILE_ELEMS;
  CU(launch_scale_rhs_unset(r, L.n, L.np, v, y, ctx->st(), s));
  if (ctx->lh_ready) {
    const __half* lh = (const __half*)ctx->lh;
    const float sc = 1.0f / (float)(1 << FP16_SCALE_LOG2);
    CU(launch_forward_chain<__half>(lh, sc, ctx->dinvf(), Sf, L.N, v, y, ctx->st(), tmo, s));
    CU(launch_backward_chain<__half>(lh, sc, ctx->dinvf(), Sb, L.N, y, v, ctx->st(), tmo, s));
  } else {
    CU(launch_forward_chain<float>(ctx->zf(), 1.0f, ctx->dinvf(), Sf, L.N, v, y, ctx->st(), tmo, s));
    CU(launch_backward_chain<float>(ctx->zf(), 1.0f, ctx->dinvf(), Sb, L.N, y, v, ctx->st(), tmo, s));
  }
  CU(launch_accumulate<float>(x, v, L.n, ctx->st(), init, s));
  return MAG_OK;
}

int correction(mag_ctx* ctx, int prec, const double* r, double* x, bool init, SolveResult* R) {
  cudaStream_t s = ctx->stream;
  CU(cudaEventRecord(ctx->ev[2], s));
  const Layout& L = ctx->lay;
  R->sweeps_used = 2;
  if (ctx->ooc)
    TRY(correction_ooc(ctx, r, x, init));
  else if (prec != MAG_PREC_FP64 && ctx->chain_ready && ctx->chain_N == L.N) {
    TRY(correction_chain(ctx, r, x, init));
    R->sweeps_used = ctx->lh_ready ? 0 : 1;
  } else if (prec == MAG_PREC_FP64)
    TRY(correction_t<double>(ctx, ctx->zd(), ctx->dinvd(), ctx->vd(V_T2), ctx->vd(V_E), r, x, init, L.n, L.np,
                             L.N));
  else
    TRY(correction_t<float>(ctx, ctx->zf(), ctx->dinvf(), ctx->vf(F_V), ctx->vf(F_Y), r, x, init, L.n, L.np,
                            L.N));
  CU(cudaEventRecord(ctx->ev[3], s));
  CU(cudaEventSynchronize(ctx->ev[3]));
  R->ms_solve += elapsed(ctx, 2, 3);
  return MAG_OK;
}

// Residual r = b - Zw and the norms; returns relres through *rel.
// ff: the float-float product from the stored tiles (Z = exp(-t d) only;
// V_T2 holds the split of w), for refinement steps whose residual is far
// above the tolerance -- its error, a few units of 2^-46 of ||Z|| ||w||,
// does not limit their corrections; the residual that decides convergence
// is always FP64.
int residual(mag_ctx* ctx, const double* X, int32_t m, double t, const double* w, const double* b,
             double* r, double* rel, bool stored, SolveResult* R, bool ff = false) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  TRY(reset_norms(ctx));
  CU(cudaEventRecord(ctx->ev[0], s));
  if (stored && ff)
    CU(launch_residual_stored_ff(ctx->zd(), L.n, L.N, w, ctx->vd(V_T2), b, ctx->vd(V_ROWSUM), r, ctx->spart(),
                                 L.np, ctx->st(), s));
  else if (stored)
    CU(launch_residual_stored(ctx->zd(), L.n, L.N, w, b, ctx->vd(V_ROWSUM), r, ctx->spart(), L.np,
                              ctx->st(), s));
  else {
    const long long* q = ctx->kind == MAT_EXP ? quantized(ctx, X, L.n, m) : nullptr;
    CU(launch_residual_sym(X, L.n, m, t, w, b, r, ctx->spart(), ctx->vd(V_ROWSUM), L.np, ctx->st(), s, ctx->kind,
                           ctx->kind_c, q, ctx->xq_L, ctx->xq_e, ctx->xq_tau2));
  }
  CU(cudaEventRecord(ctx->ev[1], s));
  TRY(read_status(ctx));
  if (ctx->h_st->flags & ST_TIMEOUT)
    return fail(ctx, MAG_ETIMEOUT, "a bounded wait of a triangular sweep expired (wait_timeout_ns = %lld)",
                (long long)ctx->opt.wait_timeout_ns);
  R->ms_res += elapsed(ctx, 0, 1);
  if (stored && ff)
    R->residual_evals_ff++;
  else
    R->residual_evals++;
  const double rn = bits_to_double(ctx->h_st->r_max_bits);
  const double zn = bits_to_double(ctx->h_st->z_max_bits);
  const double wn = bits_to_double(ctx->h_st->w_max_bits);
  R->znorm = zn;
  R->wnorm = wn;
  *rel = (zn > 0 && wn > 0) ? rn / (zn * wn) : INFINITY;
  if (!std::isfinite(*rel)) *rel = INFINITY;
  return MAG_OK;
}

// Tile rows of the precision probe's leading block (3072 points).
constexpr int64_t kProbeTiles = 24;

// Refinement steps after the first solve until a relative residual that
// starts near rho and shrinks by rho per step is below tol.
double ir_steps(double rho, double tol) {
  if (!(rho < 1.0)) return INFINITY;
  if (!(rho > 0.0)) return 0.0;
  return std::max(0.0, std::ceil(std::log(tol) / std::log(rho)) - 1.0);
}

// Precision probe of the AUTO policy: the contraction of refinement with the
// one-product FP16 factor, measured on the leading K x K tile block (K = 24,
// or the panel width when that is smaller).  The packed index of a tile does not depend on N, so
// the first K(K+1)/2 tiles are the packed matrix of the first 128 K points:
// a copy of their FP32 tiles is factored with FP16 updates (one panel of K
// tiles), then x_0 = F^{-1} 1, r_0 = 1 - Z_K x_0, x_1 = x_0 + F^{-1} r_0,
// r_1 = 1 - Z_K x_1 in FP64 give the block's contraction rho_K.  The
// full system's contraction is predicted as rho_K n / (128 K): the error of
// an FP16 operand grows with the row norms (about sqrt(n) for a flat kernel)
// and lambda_min shrinks with the point density (about n^{-1/m} in m
// dimensions), both bounded by that linear factor for m >= 2.  *rho =
// +inf when the block's FP16 factor breaks down.  The full workspace's
// vectors r and x, the FP32 diagonal inverses and panel buffer 0 are used as
// scratch; the solve that follows rewrites them.
int probe_fp16(mag_ctx* ctx, const double* X, int32_t m, double t, bool stored, SolveResult* R, double* rho) {
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  const int64_t K = std::min<int64_t>(L.nb, kProbeTiles), ns = K * TILE, tiles = K * (K + 1) / 2;
  const size_t bytes = (size_t)tiles * TILE_ELEMS * sizeof(float);
  if (bytes > ctx->probe_bytes) {
    if (ctx->probe_z) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->probe_z);
      ctx->probe_z = nullptr;
      ctx->probe_bytes = 0;
    }
    cudaError_t e = cudaMalloc((void**)&ctx->probe_z, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->probe_z = nullptr;
      return fail(ctx, MAG_ENOMEM, "precision probe tiles: %s", cudaGetErrorString(e));
    }
    ctx->probe_bytes = bytes;
  }
  if (ctx->probe_cmap_base != ctx->probe_z || ctx->probe_cmap_tiles != tiles) {
    if (!make_c_map(&ctx->probe_cmap, ctx->probe_z, tiles))
      return fail(ctx, MAG_ECUDA, "cuTensorMapEncodeTiled failed for the probe tiles");
    ctx->probe_cmap_base = ctx->probe_z;
    ctx->probe_cmap_tiles = tiles;
  }
  CU(cudaEventRecord(ctx->ev[0], s));
  CU(cudaMemcpyAsync(ctx->probe_z, ctx->zf(), bytes, cudaMemcpyDeviceToDevice, s));
  const bool pairs = ctx->opt.cta_pairs == 1;
  TRY(ensure_tasks(ctx, K, (int)K, false, pairs));
  TRY(ensure_maps(ctx, UPD_FP16, 0));
  CU(cudaMemsetAsync(ctx->counters(), 0, (size_t)L.nctr * sizeof(unsigned), s));
  int launches = 0;
  double flops = 0;
  TcFactor F{ctx, UPD_FP16, pairs, (int)K, &launches, &flops, 0, ctx->probe_z, ctx->dinvf(), &ctx->probe_cmap,
             ns, K, ctx->sm_count};
  TRY(tc_panel_range(F, 0, 0, K, 0, s));
  TRY(read_status(ctx));
  const int fl = ctx->h_st->flags;
  if (fl & ST_TIMEOUT) return fail(ctx, MAG_ETIMEOUT, "a bounded device wait in the precision probe expired");
  if (fl & ST_NOTPD) {
    // breakdown of the FP16 block factor: clear the flag for the real factor
    ctx->h_st->flags = 0;
    ctx->h_st->notpd_index = 0x7fffffff;
    CU(cudaMemcpyAsync(ctx->st(), ctx->h_st, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    *rho = INFINITY;
    R->probe_rho = INFINITY;
    return MAG_OK;
  }
  double* r = ctx->vd(V_R);
  double* x = ctx->vd(V_X);
  CU(launch_fill(r, ns, 1.0, s));
  TRY(reset_norms(ctx));
  CU(launch_absmax(r, ns, ctx->st(), s));
  TRY(correction_t<float>(ctx, ctx->probe_z, ctx->dinvf(), ctx->vf(F_V), ctx->vf(F_Y), r, x, true, ns, ns, K));
  // r_0 = (I - Z F^{-1}) 1 and r_1 = (I - Z F^{-1}) r_0: two samples of the
  // operator that multiplies the residual in each refinement step
  // (||r_0||inf / ||1||inf and ||r_1||inf / ||r_0||inf); rho_K is the larger.
  // A residual at the FP64 rounding level of ||Z|| ||x|| cannot shrink
  // further: r_0 there ends the probe (the FP16 factor solved the block to
  // full accuracy), r_1 there is counted at that level.
  const int chunks = (int)std::min<int64_t>(L.chunks, K);
  auto block_residual = [&](double* rn, double* floor) -> int {
    TRY(reset_norms(ctx));
    if (stored)
      CU(launch_residual_stored(ctx->zd(), ns, K, x, nullptr, ctx->vd(V_ROWSUM), r, ctx->spart(), ns, ctx->st(),
                                s));
    else
      CU(launch_residual_mf(X, ns, m, t, x, nullptr, r, ctx->part(), chunks, ns, ctx->st(), s, ctx->kind,
                            ctx->kind_c));
    TRY(read_status(ctx));
    *rn = bits_to_double(ctx->h_st->r_max_bits);
    *floor = 32.0 * 0x1p-52 * bits_to_double(ctx->h_st->z_max_bits) * bits_to_double(ctx->h_st->w_max_bits);
    return MAG_OK;
  };
  double rn0 = 0.0, rn1 = 0.0, floor0 = 0.0, floor1 = 0.0, rk = 0.0;
  TRY(block_residual(&rn0, &floor0));
  if (!(rn0 <= floor0)) {
    TRY(correction_t<float>(ctx, ctx->probe_z, ctx->dinvf(), ctx->vf(F_V), ctx->vf(F_Y), r, x, false, ns, ns, K));
    TRY(block_residual(&rn1, &floor1));
    rk = std::max(rn0, std::max(rn1, floor1) / rn0);
  } else {
    rk = rn0;
  }
  CU(cudaEventRecord(ctx->ev[1], s));
  CU(cudaEventSynchronize(ctx->ev[1]));
  R->ms_probe += elapsed(ctx, 0, 1);
  if (ctx->h_st->flags & ST_TIMEOUT)
    return fail(ctx, MAG_ETIMEOUT, "a bounded device wait in the precision probe expired");
  *rho = std::isfinite(rk) ? rk * (double)L.n / (double)ns : INFINITY;
  R->probe_rho = *rho;
  return MAG_OK;
}

// GMRES-IR (Carson & Higham, SIAM J. Sci. Comput. 40 (2018)): refinement whose
// correction equation Z d = r is solved by GMRES(k) in FP64, left-preconditioned
// by the low-precision factor M = L L^T (M^{-1} Z is close to I even when
// kappa(Z) u_factor is not small), with classical Gram-Schmidt applied twice.
// x is the FP64 iterate (updated in place); returns the best relative residual.
int gmres_ir(mag_ctx* ctx, int prec, const double* X, int32_t m, double t, const double* b, double* x,
             bool stored, SolveResult* R, double* rel_out, bool planned = false) {
  const Layout& L = ctx->lay;
  const int64_t n = L.n, np = L.np;
  cudaStream_t s = ctx->stream;
  const int k = std::max(2, std::min(ctx->opt.gmres_max_iters, 200));
  const size_t need = ((size_t)(k + 1) * np + 3 * np + 2 * (size_t)(k + 2)) * sizeof(double);
  if (need > ctx->gm_bytes) {
    if (ctx->gm) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->gm);
      ctx->gm = nullptr;
      ctx->gm_bytes = 0;
    }
    cudaError_t e = cudaMalloc((void**)&ctx->gm, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->gm = nullptr;
      return fail(ctx, MAG_ENOMEM, "GMRES basis: %s", cudaGetErrorString(e));
    }
    ctx->gm_bytes = need;
  }
  double* V = ctx->gm;                         // (k+1) x np
  double* zeros = V + (size_t)(k + 1) * np;    // np
  double* wv = zeros + np;                     // np
  double* dh = wv + np;                        // k+2
  double* dh2 = dh + (k + 2);                  // k+2
  double* vsplit = dh2 + (k + 2);              // np float2 (the float-float product's split of v)
  double* r = ctx->vd(V_R);
  double* tmp = ctx->vd(V_E);
  CU(cudaMemsetAsync(zeros, 0, np * sizeof(double), s));
  // the inner products Z v in float-float from the stored tiles of exp(-t d)
  const bool ff = stored && ctx->kind == MAT_EXP && ctx->opt.gmres_matvec == 0;
  auto precond_matvec = [&](const double* v, double* out) -> int {
    // out = M^{-1} (Z v):  the residual kernel with b = 0 gives -Z v
    TRY(reset_norms(ctx));
    if (ff)
      CU(launch_residual_stored_ff(ctx->zd(), n, L.N, v, vsplit, zeros, ctx->vd(V_ROWSUM), tmp, ctx->spart(), np,
                                   ctx->st(), s));
    else if (stored)
      CU(launch_residual_stored(ctx->zd(), n, L.N, v, zeros, ctx->vd(V_ROWSUM), tmp, ctx->spart(), np, ctx->st(), s));
    else {
      const long long* q = ctx->kind == MAT_EXP ? quantized(ctx, X, n, m) : nullptr;
      CU(launch_residual_sym(X, n, m, t, v, zeros, tmp, ctx->spart(), ctx->vd(V_ROWSUM), np, ctx->st(), s,
                             ctx->kind, ctx->kind_c, q, ctx->xq_L, ctx->xq_e, ctx->xq_tau2));
    }
    TRY(correction(ctx, prec, tmp, out, /*init=*/true, R));
    CU(launch_scale(out, -1.0, out, n, s));
    return MAG_OK;
  };
  double best = INFINITY, prev_rel = INFINITY, prev2_rel = INFINITY, rel = INFINITY;
  bool fresh = false;  // rel is the residual of the current x
  std::vector<double> H((size_t)(k + 1) * k), cs(k), sn(k), g(k + 1), y(k), h(k + 1), h2(k + 1);
  // outer residuals in float-float while they are predicted well above the
  // tolerance (the rule of refine's loop); the deciding ones in FP64
  const bool ff_ok = ff && prec != MAG_PREC_FP64;
  for (int outer = 0; outer < 8; ++outer) {
    bool ffr = false;
    if (ff_ok) {
      const double rho_est =
          (std::isfinite(prev2_rel) && prev2_rel > 0.0) ? std::min(1.0, prev_rel / prev2_rel) : 1e-3;
      ffr = outer == 0 || prev_rel * rho_est > 1e-10;
    }
    TRY(residual(ctx, X, m, t, x, b, r, &rel, stored, R, ffr));
    if (ffr && !(rel > 1e-10)) TRY(residual(ctx, X, m, t, x, b, r, &rel, stored, R, false));
    fresh = true;
    best = std::min(best, rel);
    if (rel <= kStopMargin * ctx->opt.ir_tol) break;
    // planned (the probe's FP16 choice): an outer step that gains less than
    // two digits leaves the rest to the split factor
    if (planned && !(rel <= 1e-2 * prev_rel)) break;
    prev2_rel = prev_rel;
    prev_rel = rel;
    // V_0 = M^{-1} r / beta
    TRY(correction(ctx, prec, r, wv, /*init=*/true, R));
    CU(launch_mdot(wv, np, 1, wv, n, dh, s));
    double beta2 = 0;
    CU(cudaMemcpyAsync(&beta2, dh, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const double beta = std::sqrt(beta2);
    if (!(beta > 0) || !std::isfinite(beta)) break;
    CU(launch_scale(wv, 1.0 / beta, V, n, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < k; ++j) {
      TRY(precond_matvec(V + (size_t)j * np, wv));
      // classical Gram-Schmidt, twice
      CU(launch_mdot(V, np, j + 1, wv, n, dh, s));
      CU(launch_maxpy(V, np, j + 1, dh, wv, n, s));
      CU(launch_mdot(V, np, j + 1, wv, n, dh2, s));
      CU(launch_maxpy(V, np, j + 1, dh2, wv, n, s));
      CU(launch_mdot(wv, np, 1, wv, n, dh2 + j + 1, s));
      CU(cudaMemcpyAsync(h.data(), dh, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(h2.data(), dh2, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      R->gmres_iters++;
      double* col = &H[(size_t)j * (k + 1)];
      for (int i = 0; i <= j; ++i) col[i] = h[i] + h2[i];
      col[j + 1] = std::sqrt(std::max(h2[j + 1], 0.0));
      // apply previous rotations, then a new one to zero col[j+1]
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = a;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0 ? col[j] / den : 1.0;
      sn[j] = den > 0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      const double hj1 = std::sqrt(std::max(h2[j + 1], 0.0));
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      const bool last = j + 1 == k || std::fabs(g[j + 1]) <= 1e-6 * beta || !(hj1 > 0);
      if (!last) CU(launch_scale(wv, 1.0 / hj1, V + (size_t)(j + 1) * np, n, s));
      if (last) {
        ++j;
        break;
      }
    }
    // y = H^{-1} g (upper triangular j x j), x += V y
    for (int i = j - 1; i >= 0; --i) {
      double acc = g[i];
      for (int c = i + 1; c < j; ++c) acc -= H[(size_t)c * (k + 1) + i] * y[c];
      y[i] = acc / H[(size_t)i * (k + 1) + i];
    }
    for (int i = 0; i < j; ++i) y[i] = -y[i];
    CU(cudaMemcpyAsync(dh, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, s));
    CU(launch_maxpy(V, np, j, dh, x, n, s));
    fresh = false;
    R->ir_iters++;
  }
  if (!fresh) TRY(residual(ctx, X, m, t, x, b, r, &rel, stored, R));
  *rel_out = rel;
  return MAG_OK;
}

// Full solve of Z x = b (b == null: ones) into x (device, n).  The iterate
// lives in the workspace; x receives the best iterate (lowest relative
// residual) over all precisions tried.
// Checksum of the points (order-independent mix of their bits), the part of
// the factor's key that sees changes made in place.
int points_hash(mag_ctx* ctx, const double* X, int64_t n, int32_t m, unsigned long long* h) {
  CU(cudaMemsetAsync(&ctx->st()->hash_bits, 0, sizeof(unsigned long long), ctx->stream));
  CU(launch_hash(X, n * m, &ctx->st()->hash_bits, ctx->stream));
  unsigned long long v = 0;
  CU(cudaMemcpyAsync(&v, &ctx->st()->hash_bits, sizeof v, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  *h = v;
  return MAG_OK;
}

int keep_factor(mag_ctx* ctx, const double* X, int64_t n, int32_t m, double t, int prec, bool stored,
                bool gmres) {
  unsigned long long h = 0;
  TRY(points_hash(ctx, X, n, m, &h));
  ctx->fac_valid = true;
  ctx->fac_pts = X;
  ctx->fac_n = n;
  ctx->fac_m = m;
  ctx->fac_t = t;
  ctx->fac_hash = h;
  ctx->fac_prec = prec;
  ctx->fac_stored = stored && prec != MAG_PREC_FP64;
  ctx->fac_gmres = gmres;
  return MAG_OK;
}

// FP16 factor chosen on the probe's prediction rho: its extra refinement
// steps over the split factor cost less than the factor time saved (n / 9500
// steps with stored FP64 tiles, a quarter of that matrix free).
bool probe_takes_fp16(double rho, double tol, int64_t n, bool stored) {
  const double saved = (double)n / 9500.0 * (stored ? 1.0 : 0.25);
  return rho < 1.0 && ir_steps(rho, tol) - ir_steps(rho * 0x1p-12, tol) <= saved;
}

// The FP16 factor with GMRES-IR where plain refinement with it would not
// do (probe_takes_fp16 false): preconditioned by an FP16 factor whose
// refinement contraction is predicted at most 16, GMRES-IR took 10-15 inner
// iterations from n = 16384 to 1e5 (t = 1 on [0,1]^8, rho 0.87 to 5.3).  An
// inner iteration is a float-float product with the stored tiles (8 ms at
// n = 1e5) and a correction through the chain sweeps with the FP16 tiles
// (4.5 ms).  Measured against the split factor: 0.859 against 1.012 s at
// n = 1e5 (factor 285 against 632 ms, 15 inner iterations), 0.356 against
// 0.360 s at n = 65,536: taken from n = 72,000 (options.fp16_gmres = 1: at
// any n).
bool probe_takes_fp16_gmres(const mag_ctx* ctx, double rho, int64_t n, bool stored) {
  const int mode = ctx->opt.fp16_gmres;
  if (mode < 0 || !stored || ctx->kind != MAT_EXP || ctx->opt.gmres_max_iters < 2 || !ctx->opt.allow_fallback)
    return false;
  return rho <= 16.0 && (mode > 0 || n >= 72000);
}

// Refinement of Z x = b (b == null: ones) with the factor in the workspace
// (precision prec): x0 = factor^{-1} b, then r = b - Z x in FP64 and
// x += factor^{-1} r until the relative residual is below kStopMargin times
// the tolerance; on stagnation (two steps each reducing it by less than 2x)
// or after ir_max_iters steps, GMRES-IR with the same factor from the best
// iterate, unless the probe chose FP16 (probed16: the caller replaces the
// factor instead).  *overall keeps the lowest relative residual over calls,
// with its iterate in x; *escalate reports a factor that did not get there.
int refine(mag_ctx* ctx, int prec, const double* X, int64_t n, int32_t m, double t, const double* b, double* x,
           bool stored, bool probed16, SolveResult* R, double* overall, bool* escalate, bool gm_direct = false) {
  const mag_options& o = ctx->opt;
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  double* r = ctx->vd(V_R);
  double* xw = ctx->vd(V_X);
  double* best = ctx->vd(V_BEST);
  double best_rel = INFINITY;
  *escalate = false;
  R->prec_used = prec;
  // initial solve x0 = factor^{-1} b: the correction from x = 0 with r = b.
  if (b)
    CU(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    CU(launch_fill(r, n, 1.0, s));
  CU(launch_fill(r + n, L.np - n, 0.0, s));
  TRY(reset_norms(ctx));
  CU(launch_absmax(r, n, ctx->st(), s));
  TRY(correction(ctx, prec, r, xw, /*init=*/true, R));
  if (gm_direct) {
    // the probe's FP16 factor with GMRES-IR from x0 at once: plain
    // refinement was predicted to diverge or crawl
    double grel = INFINITY;
    R->fallback = 4;
    TRY(gmres_ir(ctx, prec, X, m, t, b, xw, stored, R, &grel, /*planned=*/true));
    if (grel < *overall) {
      *overall = grel;
      CU(cudaMemcpyAsync(x, xw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(cudaStreamSynchronize(s));
    }
    *escalate = !(grel <= kStopMargin * o.ir_tol);
    return MAG_OK;
  }
  double rel = INFINITY, prev = INFINITY, prev2 = INFINITY;
  int slow = 0;
  // float-float residuals (FP32 pipe) while the residual is predicted well
  // above the tolerance: the first one, then while the last residual times
  // the observed contraction (10^-3 before two are known) stays above
  // 1e-10; a float-float residual at or below 1e-10 is evaluated again in
  // FP64, which decides the stopping test and feeds the next correction
  const bool ff_ok = stored && prec != MAG_PREC_FP64 && ctx->kind == MAT_EXP && o.gmres_matvec == 0;
  for (int it = 0;; ++it) {
    bool ff = false;
    if (ff_ok) {
      const double rho_est = (std::isfinite(prev2) && prev2 > 0.0) ? std::min(1.0, prev / prev2) : 1e-3;
      ff = it == 0 || prev * rho_est > 1e-10;
    }
    // The FP64 factor overwrites the FP64 tiles, so it refines matrix free.
    TRY(residual(ctx, X, m, t, xw, b, r, &rel, stored && prec != MAG_PREC_FP64, R, ff));
    if (ff && !(rel > 1e-10)) TRY(residual(ctx, X, m, t, xw, b, r, &rel, stored, R, false));
    if (rel < best_rel) {
      best_rel = rel;
      CU(cudaMemcpyAsync(best, xw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (rel <= kStopMargin * o.ir_tol) break;
    if (it >= o.ir_max_iters || (rel > 0.5 * prev && ++slow >= 2)) {
      *escalate = true;
      break;
    }
    if (!(rel > 0.5 * prev)) slow = 0;
    prev2 = prev;
    prev = rel;
    TRY(correction(ctx, prec, r, xw, /*init=*/false, R));
    R->ir_iters++;
  }
  if (best_rel < *overall) {
    *overall = best_rel;
    CU(cudaMemcpyAsync(x, best, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(cudaStreamSynchronize(s));
  }
  // a mispredicted FP16 choice goes to the split factor instead of GMRES-IR
  const bool to_split = *escalate && probed16 && prec == MAG_PREC_FP16 && o.allow_fallback;
  if (*escalate && !to_split && prec != MAG_PREC_FP64 && o.allow_fallback && o.gmres_max_iters > 0) {
    // GMRES-IR with the same factor, from the best iterate so far
    CU(cudaMemcpyAsync(xw, best, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double grel = INFINITY;
    R->fallback = 1;
    TRY(gmres_ir(ctx, prec, X, m, t, b, xw, stored, R, &grel));
    if (grel < *overall) {
      *overall = grel;
      CU(cudaMemcpyAsync(x, xw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(cudaStreamSynchronize(s));
    }
    if (grel <= kStopMargin * o.ir_tol) *escalate = false;
  }
  return MAG_OK;
}

// The solve with the out-of-core factor (plan_out_of_core set the slabs; the
// device pool holds pool_tiles tiles).  The residual is matrix free, the
// generation happens inside the factor slab by slab, the AUTO policy has no
// Gershgorin shortcut (no full row sums before the factor) and runs the probe
// on the first slab's leading block; refinement and GMRES-IR as in core, but
// no FP64 factor (it would not fit either).
int solve_ooc(mag_ctx* ctx, const double* X, int64_t n, int32_t m, double t, const double* b, double* x,
              int64_t pool_tiles, SolveResult* R) {
  const mag_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  R->stored = false;
  R->gersh = NAN;
  TRY(ensure_workspace(ctx, n, true, false, pool_tiles));
  ctx->ooc = true;
  struct OocOff {
    mag_ctx* c;
    ~OocOff() { c->ooc = false; }
  } ooc_off{ctx};
  R->slabs = (int)ctx->slabs.size();
  for (const Slab& sl : ctx->slabs)
    if (sl.host) {
      R->host_slabs++;
      R->host_bytes += (double)sl.tiles * TILE_ELEMS * sizeof(float);
    }
  const Layout& L = ctx->lay;
  const double tol = kStopMargin * o.ir_tol;
  int prec = o.precision;
  bool slab0_ready = false, probed16 = false;
  TRY(reset_status(ctx));
  if (prec == MAG_PREC_AUTO) {
    prec = MAG_PREC_FP16X3;
    const int64_t K = std::min<int64_t>(L.nb, kProbeTiles);
    if (ctx->slabs[0].S >= K && L.N >= 3 * K) {
      CU(cudaEventRecord(ctx->ev[0], s));
      const long long* q = quantized(ctx, X, n, m);
      CU(launch_generate_slab(X, n, m, t, 0, ctx->slabs[0].S, ctx->slab_dev(ctx->slabs[0]), ctx->st(), s, INFINITY,
                              q, ctx->xq_L, ctx->xq_e, ctx->xq_tau2));
      CU(cudaEventRecord(ctx->ev[1], s));
      TRY(read_status(ctx));
      R->ms_gen += elapsed(ctx, 0, 1);
      if (ctx->h_st->flags & ST_NONFINITE) return fail(ctx, MAG_EINVAL, "non-finite coordinate in points");
      if (ctx->h_st->flags & ST_DUPLICATE) return fail(ctx, MAG_EDUPLICATE, "two points coincide (min d = 0)");
      slab0_ready = true;
      double rho = INFINITY;
      TRY(probe_fp16(ctx, X, m, t, false, R, &rho));
      if (probe_takes_fp16(rho, tol, n, false)) {
        prec = MAG_PREC_FP16;
        probed16 = true;
      }
    }
  }
  if (prec != MAG_PREC_FP16 && prec != MAG_PREC_FP16X3)
    return fail(ctx, MAG_EINVAL, "the out-of-core factor runs the FP16 and FP16X3 (or AUTO) precisions");
  double overall = INFINITY;
  for (int attempt = 0; attempt < 2; ++attempt) {
    double* r = ctx->vd(V_R);
    double* xw = ctx->vd(V_X);
    double* best = ctx->vd(V_BEST);
    double best_rel = INFINITY;
    bool escalate = false;
    if (!slab0_ready) TRY(reset_status(ctx));
    CU(cudaEventRecord(ctx->ev[0], s));
    ctx->prof_used = 0;
    TRY(factor_ooc(ctx, X, m, t, upd_mode(prec), slab0_ready, &R->update_launches, &R->update_flops,
                   &R->host_read_bytes));
    slab0_ready = false;
    CU(cudaEventRecord(ctx->ev[1], s));
    TRY(read_status(ctx));
    R->ms_fac += elapsed(ctx, 0, 1);
    double pc[PC_COUNT], busy = 0;
    R->ms_update += prof_collect(ctx, pc, &busy);
    R->ms_update_busy += busy;
    R->ms_update_panel += pc[PC_UPDATE_PANEL];
    R->ms_potrf += pc[PC_POTRF];
    R->ms_trsm += pc[PC_TRSM];
    R->ms_host_read += pc[PC_HOST_READ];
    const int fl = ctx->h_st->flags;
    if (fl & ST_NONFINITE) return fail(ctx, MAG_EINVAL, "non-finite coordinate in points");
    if (fl & ST_DUPLICATE) return fail(ctx, MAG_EDUPLICATE, "two points coincide (min d = 0)");
    R->dmin = std::sqrt(bits_to_double(ctx->h_st->min_d2_bits));
    if (fl & ST_TIMEOUT) return fail(ctx, MAG_ETIMEOUT, "a bounded device wait in the tensor-core update expired");
    if (fl & ST_NOTPD) {
      if (probed16 && o.allow_fallback) {
        prec = MAG_PREC_FP16X3;
        probed16 = false;
        R->fallback = 3;
        continue;
      }
      return fail(ctx, MAG_ENOTPD, "non-positive pivot at row %d of a slab (precision %d)",
                  ctx->h_st->notpd_index - 1, prec);
    }
    R->prec_used = prec;
    if (b)
      CU(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else
      CU(launch_fill(r, n, 1.0, s));
    CU(launch_fill(r + n, L.np - n, 0.0, s));
    TRY(reset_norms(ctx));
    CU(launch_absmax(r, n, ctx->st(), s));
    TRY(correction(ctx, prec, r, xw, /*init=*/true, R));
    double rel = INFINITY, prev = INFINITY;
    int slow = 0;
    for (int it = 0;; ++it) {
      TRY(residual(ctx, X, m, t, xw, b, r, &rel, false, R));
      if (rel < best_rel) {
        best_rel = rel;
        CU(cudaMemcpyAsync(best, xw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
      if (rel <= tol) break;
      if (it >= o.ir_max_iters || (rel > 0.5 * prev && ++slow >= 2)) {
        escalate = true;
        break;
      }
      if (!(rel > 0.5 * prev)) slow = 0;
      prev = rel;
      TRY(correction(ctx, prec, r, xw, /*init=*/false, R));
      R->ir_iters++;
    }
    if (best_rel < overall) {
      overall = best_rel;
      CU(cudaMemcpyAsync(x, best, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(cudaStreamSynchronize(s));
    }
    if (!escalate || !o.allow_fallback) break;
    if (probed16 && prec == MAG_PREC_FP16) {
      prec = MAG_PREC_FP16X3;
      probed16 = false;
      R->fallback = 3;
      continue;
    }
    if (o.gmres_max_iters > 0) {
      CU(cudaMemcpyAsync(xw, best, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      double grel = INFINITY;
      R->fallback = 1;
      TRY(gmres_ir(ctx, prec, X, m, t, b, xw, false, R, &grel));
      if (grel < overall) {
        overall = grel;
        CU(cudaMemcpyAsync(x, xw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CU(cudaStreamSynchronize(s));
      }
    }
    break;
  }
  R->rel = overall;
  if (!(overall < INFINITY)) return fail(ctx, MAG_ENOTPD, "no factor succeeded");
  if (!(overall <= o.ir_tol))
    return fail(ctx, MAG_ENOCONV, "refinement stopped at relative residual %.3e > %.3e", overall, o.ir_tol);
  return MAG_OK;
}

int solve_impl(mag_ctx* ctx, const double* X, int64_t n, int32_t m, double t, const double* b,
               double* x, SolveResult* R) {
  const mag_options& o = ctx->opt;
  int prec = o.precision;
  ctx->fac_valid = false;  // the workspace's tiles are about to be rewritten
  ctx->chain_ready = ctx->lh_ready = false;
  ctx->xq_ok = false;      // the points may have changed in place since the last call
  {
    int64_t pool_tiles = 0;
    TRY(plan_out_of_core(ctx, n, prec, &pool_tiles));
    if (pool_tiles > 0) return solve_ooc(ctx, X, n, m, t, b, x, pool_tiles, R);
  }
  bool stored = o.residual_mode == MAG_RESID_STORED;
  if (o.residual_mode == MAG_RESID_AUTO && prec != MAG_PREC_FP64) {
    // Stored FP64 tiles cost one FP64 exp per pair once instead of once per
    // refinement step; use them when they fit comfortably.
    size_t fre = 0, tot = 0;
    const Layout with = plan(ctx, n, true, true);
    if (cudaMemGetInfo(&fre, &tot) == cudaSuccess) {
      const double avail = (double)fre + (double)ctx->ws_bytes;
      stored = (double)with.total <= 0.5 * avail;
    } else {
      cudaGetLastError();
    }
  }
  R->stored = stored;
  bool f64 = prec == MAG_PREC_FP64 || stored;
  bool f32 = prec != MAG_PREC_FP64;
  TRY(ensure_workspace(ctx, n, f32, f64));
  TRY(generate(ctx, X, m, t, f32, f64, R, true));
  // AUTO: one scaled-FP16 product when the Gershgorin bound keeps
  // lambda_min(Z) >= 1/2 (then kappa(Z) <= 2 ||Z|| and an 11-bit factor still
  // contracts refinement quickly).  Otherwise the probe predicts the
  // contraction rho of refinement with the FP16 factor; FP16 is taken when
  // the extra refinement steps it needs over the split factor (whose error,
  // and so its rho, is about 2^-12 times smaller) cost less than the half of
  // the factor it saves.  With the FP64 tiles stored that half is worth about
  // n / 9500 refinement steps at the GB300's rates (311 ms of factor against
  // 29 ms per step at n = 1e5); a matrix-free residual step costs about four
  // times more.  Else the scaled-FP16 split (FP32-like factor accuracy at the
  // FP16 tensor rate).
  bool probed16 = false;  // FP16 chosen on the probe's prediction
  bool gm_direct = false;  // ... with GMRES-IR from the first solve on
  if (prec == MAG_PREC_AUTO) {
    prec = MAG_PREC_FP16X3;
    if (R->gersh >= 0.5) {
      prec = MAG_PREC_FP16;
    } else if (ctx->lay.N >= 3 * std::min<int64_t>(ctx->lay.nb, kProbeTiles)) {
      double rho = INFINITY;
      TRY(probe_fp16(ctx, X, m, t, stored, R, &rho));
      if (probe_takes_fp16(rho, kStopMargin * o.ir_tol, n, stored)) {
        prec = MAG_PREC_FP16;
        probed16 = true;
      } else if (probe_takes_fp16_gmres(ctx, rho, n, stored)) {
        prec = MAG_PREC_FP16;
        probed16 = true;
        gm_direct = true;
      }
    }
  }

  double overall = INFINITY;
  for (int attempt = 0; attempt < 3; ++attempt) {
    bool escalate = false;
    int st = run_factor(ctx, prec, R);
    if (st == MAG_ENOTPD && prec != MAG_PREC_FP64 && o.allow_fallback) {
      escalate = true;
    } else {
      TRY(st);
      TRY(refine(ctx, prec, X, n, m, t, b, x, stored, probed16, R, &overall, &escalate,
                 gm_direct && prec == MAG_PREC_FP16));
    }
    if (!escalate || prec == MAG_PREC_FP64 || !o.allow_fallback) break;
    if (probed16 && prec == MAG_PREC_FP16) {
      // the FP16 factor overwrote the FP32 tiles: generate them again
      prec = MAG_PREC_FP16X3;
      probed16 = false;
      R->fallback = 3;
      TRY(generate(ctx, X, m, t, true, false, R, true));
      continue;
    }
    // escalate to the FP64 factor (re-plans the workspace: pointers re-fetched above)
    prec = MAG_PREC_FP64;
    R->fallback = 2;
    TRY(ensure_workspace(ctx, n, true, true));
    TRY(generate(ctx, X, m, t, false, true, R, true));
  }
  R->rel = overall;
  if (overall < INFINITY && ctx->kind == MAT_EXP)
    TRY(keep_factor(ctx, X, n, m, t, R->prec_used, stored, R->fallback == 1 || R->fallback == 4));
  if (!(overall < INFINITY)) return fail(ctx, MAG_ENOTPD, "no factor succeeded");
  if (!(overall <= o.ir_tol))
    return fail(ctx, MAG_ENOCONV, "refinement stopped at relative residual %.3e > %.3e", overall, o.ir_tol);
  return MAG_OK;
}

void fill_info(mag_ctx* ctx, const SolveResult& R, int64_t n, mag_info* info) {
  if (!info) return;
  info->precision_used = R.prec_used;
  info->ir_iters = R.ir_iters;
  info->gmres_iters = R.gmres_iters;
  info->fallback = R.fallback;
  info->residual_mode = R.stored ? MAG_RESID_STORED : MAG_RESID_MATRIX_FREE;
  info->rel_residual = R.rel;
  info->z_norm_inf = R.znorm;
  info->w_norm_inf = R.wnorm;
  info->min_w = ctx->h_st->min_w;
  info->gershgorin_lmin = R.gersh;
  info->min_distance = R.dmin;
  info->ms_generate = R.ms_gen;
  info->ms_factor = R.ms_fac;
  info->ms_solve = R.ms_solve;
  info->ms_residual = R.ms_res;
  const double nn = (double)n;
  info->useful_flops = nn * nn * nn / 3.0 + 2.0 * nn * nn * (double)R.ir_iters;
  info->residual_evals = R.residual_evals;
  info->update_launches = R.update_launches;
  info->ms_update = R.ms_update;
  info->update_flops = R.update_flops;
  info->ms_update_panel = R.ms_update_panel;
  info->ms_potrf = R.ms_potrf;
  info->ms_trsm = R.ms_trsm;
  info->ms_split = R.ms_split;
  info->probe_rho = R.probe_rho;
  info->ms_probe = R.ms_probe;
  info->slabs = R.slabs;
  info->host_slabs = R.host_slabs;
  info->host_bytes = R.host_bytes;
  info->host_read_bytes = R.host_read_bytes;
  info->ms_host_read = R.ms_host_read;
  info->deflation_c = R.deflation_c;
  info->factor_reused = R.factor_reused;
  info->ms_update_busy = R.ms_update_busy;
  info->residual_evals_ff = R.residual_evals_ff;
  info->sweeps_used = R.sweeps_used;
  info->exact_distances = R.exact_distances;
}

// The small-t end (Z close to 1 1^T, kappa(Z) growing like 1/t): with
// alpha = 1 - c t, Z = c t A + alpha 1 1^T where A = (Z - alpha 1 1^T) / (c t)
// has entries 1 + expm1(-t d_jk) / (c t) and a unit diagonal (no
// cancellation: expm1).  A = 1 1^T - D_t / c with D_t = (1 1^T - Z) / t
// conditionally negative definite (Z is positive definite), so A is positive
// definite for c large enough -- the t > 0 form of the scale-zero system M of
// App. C -- and has Z's structure (unit diagonal, entries in [1/2, 1] for
// c >= 2 max d), with a condition number that stays bounded as t -> 0, where
// that of Z grows like 1/t.  The solver refines u = A^{-1} 1 to the tolerance
// on A's system, and by Sherman-Morrison w = Z^{-1} 1 = u / (c t + alpha
// 1^T u).  Then 1 - Z w = c t (1 - A u) / (c t + alpha 1^T u) exactly, so
// Z's relative residual is A's times c t ||A|| / ||Z|| (||Z||inf = c t
// ||A||inf + alpha n): below the tolerance as well.  c starts at
// 4 max_j ||x_j - x_0|| >= 2 max d and doubles on a non-positive pivot while
// c t <= 1 (alpha >= 0: no cancellation in c t + alpha 1^T u).  Returns
// MAG_ENOTPD when no such c gave a positive definite A (the caller then
// solves Z directly).
int solve_deflated(mag_ctx* ctx, const double* X, int64_t n, int32_t m, double t, double* w, double c,
                   SolveResult* R) {
  cudaStream_t s = ctx->stream;
  int st = MAG_ENOTPD;
  for (; c * t <= 1.0 && st == MAG_ENOTPD; c *= 2.0) {
    SolveResult Ra;
    const double ct = c * t;
    ctx->kind = MAT_DEFLATED;
    ctx->kind_c = 1.0 / ct;
    st = solve_impl(ctx, X, n, m, t, nullptr, w, &Ra);
    ctx->kind = MAT_EXP;
    ctx->kind_c = 0.0;
    *R = Ra;
    if (st != MAG_OK && st != MAG_ENOCONV) continue;
    CU(launch_reduce_w(w, n, ctx->st(), s));  // 1^T u (compensated)
    TRY(read_status(ctx));
    const double alpha = 1.0 - ct, su = ctx->h_st->mag, den = ct + alpha * su;
    if (!(den > 0.0) || !std::isfinite(den)) return fail(ctx, MAG_ENOCONV, "deflated solve: c t + alpha 1^T u = %g", den);
    CU(launch_scale(w, 1.0 / den, w, n, s));
    const double za = R->znorm;
    R->znorm = ct * za + alpha * (double)n;
    R->rel = R->rel * ct * za / R->znorm;
    R->wnorm = R->wnorm / den;
    R->deflation_c = c;
    return st;
  }
  return st;
}

}  // namespace

extern "C" {

int mag_similarity_matrix(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                          int32_t precision, void* Z_out) {
  TRY(check_args(ctx, points, n, m, t));
  if (!Z_out) return fail(ctx, MAG_EINVAL, "NULL output");
  ctx->err.clear();
  const bool f64 = precision == MAG_PREC_FP64;
  SolveResult R;
  ctx->fac_valid = false;
  TRY(ensure_workspace(ctx, n, !f64, f64));
  TRY(generate(ctx, points, m, t, !f64, f64, &R));
  const Layout& L = ctx->lay;
  if (f64)
    CU(launch_unpack<double>(ctx->zd(), n, L.N, true, (double*)Z_out, ctx->stream));
  else
    CU(launch_unpack<float>(ctx->zf(), n, L.N, true, (float*)Z_out, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return MAG_OK;
}

int mag_cholesky_factor(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                        int32_t precision, void* L_out) {
  TRY(check_args(ctx, points, n, m, t));
  if (!L_out) return fail(ctx, MAG_EINVAL, "NULL output");
  ctx->err.clear();
  const bool f64 = precision == MAG_PREC_FP64;
  int prec = f64 ? MAG_PREC_FP64 : (precision == MAG_PREC_AUTO ? MAG_PREC_FP16X3 : precision);
  SolveResult R;
  ctx->fac_valid = false;
  TRY(ensure_workspace(ctx, n, !f64, f64));
  TRY(generate(ctx, points, m, t, !f64, f64, &R));
  TRY(run_factor(ctx, prec, &R));
  const Layout& L = ctx->lay;
  if (f64)
    CU(launch_unpack<double>(ctx->zd(), n, L.N, false, (double*)L_out, ctx->stream));
  else
    CU(launch_unpack<float>(ctx->zf(), n, L.N, false, (float*)L_out, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return MAG_OK;
}

int mag_solve(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t, double* w,
              double* mag, mag_info* info) {
  TRY(check_args(ctx, points, n, m, t));
  if (!w || !mag) return fail(ctx, MAG_EINVAL, "NULL output");
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  SolveResult R;
  const long long l0 = g_kernel_launches.load();
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, ctx->stream);
  int st = MAG_ENOTPD;
  bool deflated = false;
  if (ctx->kind == MAT_EXP && ctx->opt.deflate >= 0) {
    // the deflated form when t max d <= 1/4: every entry of Z at least
    // e^-1/4, kappa(Z) dominated by the rank-one 1 1^T part
    if (!ctx->ws || ctx->lay.np < ((n + TILE - 1) / TILE) * TILE) st = ensure_workspace(ctx, n, false, false);
    if (st == MAG_ENOTPD || st == MAG_OK) st = reset_status(ctx);
    if (st == MAG_OK) {
      cudaError_t e = launch_far_from_first(points, n, m, ctx->st(), ctx->stream);
      st = e == cudaSuccess ? read_status(ctx) : fail(ctx, MAG_ECUDA, "far: %s", cudaGetErrorString(e));
    }
    if (st != MAG_OK) {
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      return st;
    }
    const double far = std::sqrt(bits_to_double(ctx->h_st->far_d2_bits));
    if (std::isfinite(far) && far > 0.0 && (ctx->opt.deflate > 0 || t * far <= 0.125)) {
      st = solve_deflated(ctx, points, n, m, t, w, 4.0 * far, &R);
      deflated = st != MAG_ENOTPD;
    }
  }
  if (!deflated) st = solve_impl(ctx, points, n, m, t, nullptr, w, &R);
  bool timed = false;
  if (st == MAG_OK || st == MAG_ENOCONV) {
    cudaStream_t s = ctx->stream;
    cudaError_t e = launch_reduce_w(w, n, ctx->st(), s);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    timed = e == cudaSuccess;
    if (e == cudaSuccess) {
      int rs = read_status(ctx);
      if (rs != MAG_OK) st = rs;
      *mag = ctx->h_st->mag;
    } else {
      st = fail(ctx, MAG_ECUDA, "reduce: %s", cudaGetErrorString(e));
    }
  }
  fill_info(ctx, R, n, info);
  if (info) {
    info->t = t;
    float ms = 0;
    if (!timed || cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) {
      cudaGetLastError();  // the end event was not recorded (failed solve): no total time
      ms = 0;
    }
    info->ms_total = ms;
    info->kernel_launches = g_kernel_launches.load() - l0;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return st;
}

int mag_solve_multi(mag_ctx* ctx, const double* points, int64_t n, int32_t m, const double* ts, int32_t nt,
                    double* W, double* mags, mag_info* infos) {
  TRY(check_args(ctx, points, n, m, 1.0));
  if (!ts || nt < 1 || !W || !mags) return fail(ctx, MAG_EINVAL, "bad multi-t arguments");
  for (int32_t i = 0; i < nt; ++i)
    if (!std::isfinite(ts[i])) return fail(ctx, MAG_EINVAL, "t[%d] = %g", (int)i, ts[i]);
  // explicit t first (their solves find min d), then the Sec. 1 bound entries
  std::vector<int32_t> order;
  for (int32_t i = 0; i < nt; ++i)
    if (ts[i] > 0.0) order.push_back(i);
  for (int32_t i = 0; i < nt; ++i)
    if (!(ts[i] > 0.0)) order.push_back(i);
  begin_dist_reuse(ctx, n);
  int first = MAG_OK;
  std::string first_err;
  double dmin = -1.0;  // min d from a solve of this call (-1: none yet)
  for (int32_t i : order) {
    mag_info inf;
    std::memset(&inf, 0, sizeof inf);
    double t = ts[i];
    int st = MAG_OK;
    if (!(t > 0.0)) {
      if (dmin < 0.0) {
        double bound = 0.0;
        st = mag_min_distance(ctx, points, n, m, &dmin, &bound);
        if (st != MAG_OK) dmin = -1.0;
      }
      if (st == MAG_OK && !(dmin > 0.0)) st = fail(ctx, MAG_EDUPLICATE, "two points coincide (min d = 0)");
      if (st == MAG_OK) t = std::log((double)(n - 1)) / dmin;
    }
    if (st == MAG_OK) {
      st = mag_solve(ctx, points, n, m, t, W + (size_t)i * n, &mags[i], &inf);
      if (dmin < 0.0 && (st == MAG_OK || st == MAG_ENOCONV || st == MAG_ENOTPD)) dmin = inf.min_distance;
    }
    inf.t = t;
    if (infos) infos[i] = inf;
    if (st != MAG_OK && first == MAG_OK) {
      first = st;
      first_err = ctx->err;
    }
  }
  end_dist_reuse(ctx);
  if (first != MAG_OK) ctx->err = first_err;
  return first;
}

int mag_solve_rhs(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                  const double* b, double* x, mag_info* info) {
  TRY(check_args(ctx, points, n, m, t));
  if (!b || !x) return fail(ctx, MAG_EINVAL, "NULL vector");
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  SolveResult R;
  int st = MAG_ENOCONV;
  if (ctx->fac_valid && ctx->fac_pts == points && ctx->fac_n == n && ctx->fac_m == m && ctx->fac_t == t &&
      ctx->kind == MAT_EXP) {
    // the factor of the last solve with these points and t is still in the
    // workspace: refine with it (the adjoint solve of mag_grad after the
    // forward solve); a new factor only if that does not converge
    unsigned long long h = 0;
    TRY(points_hash(ctx, points, n, m, &h));
    if (h == ctx->fac_hash) {
      TRY(reset_status(ctx));
      double overall = INFINITY;
      bool escalate = false;
      R.stored = ctx->fac_stored;
      R.factor_reused = 1;
      TRY(refine(ctx, ctx->fac_prec, points, n, m, t, b, x, ctx->fac_stored, false, &R, &overall, &escalate,
                 ctx->fac_gmres));
      R.rel = overall;
      st = overall <= ctx->opt.ir_tol ? MAG_OK : MAG_ENOCONV;
    }
  }
  if (st != MAG_OK) {
    R = SolveResult();
    st = solve_impl(ctx, points, n, m, t, b, x, &R);
  }
  fill_info(ctx, R, n, info);
  return st;
}

int mag_residual(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t, const double* w,
                 const double* b, double* r_out, double* norms) {
  TRY(check_args(ctx, points, n, m, t));
  if (!w || !norms) return fail(ctx, MAG_EINVAL, "NULL w or norms");
  ctx->err.clear();
  if (!ctx->ws || ctx->lay.np < ((n + TILE - 1) / TILE) * TILE) TRY(ensure_workspace(ctx, n, false, false));
  const Layout& L = ctx->lay;
  cudaStream_t s = ctx->stream;
  TRY(reset_status(ctx));
  // r_out holds exactly n entries, so the residual kernel gets n as its row
  // stride and padding length.
  double* r = r_out ? r_out : ctx->vd(V_R);
  CU(launch_residual_mf(points, n, m, t, w, b, r, ctx->part(), L.chunks, n, ctx->st(), s));
  TRY(read_status(ctx));
  const double rn = bits_to_double(ctx->h_st->r_max_bits);
  const double zn = bits_to_double(ctx->h_st->z_max_bits);
  const double wn = bits_to_double(ctx->h_st->w_max_bits);
  norms[0] = (zn > 0 && wn > 0) ? rn / (zn * wn) : INFINITY;
  norms[1] = rn;
  norms[2] = zn;
  norms[3] = wn;
  return MAG_OK;
}

int mag_sweep_tplus(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t_lo,
                    double t_hi, double rel_tol, double* t_plus, double* t_bracket, double* w,
                    double* mag, mag_info* info) {
  TRY(check_args(ctx, points, n, m, 1.0));
  if (!t_plus || !t_bracket || !w || !mag) return fail(ctx, MAG_EINVAL, "NULL output");
  if (!(rel_tol > 0.0)) return fail(ctx, MAG_EINVAL, "rel_tol must be > 0");
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  double dmin = 0, bound = 0;
  if (t_hi <= 0.0) {
    TRY(mag_min_distance(ctx, points, n, m, &dmin, &bound));
    t_hi = bound;
  }
  if (!(t_lo > 0.0) || !(t_hi > t_lo) || !std::isfinite(t_hi))
    return fail(ctx, MAG_EINVAL, "bad bracket [%g, %g]", t_lo, t_hi);
  // Probes solve into the aux vector A_W (it survives workspace re-plans); w
  // receives the solution at the feasible end.
  mag_info pi;
  double pm = 0;
  int probes = 0, iters = 0;
  TRY(ensure_aux(ctx, n));
  double* wp = ctx->aux + (size_t)A_W * ctx->aux_np;
  begin_dist_reuse(ctx, n);
  struct EndReuse {
    mag_ctx* c;
    ~EndReuse() { end_dist_reuse(c); }
  } end_reuse{ctx};
  auto probe = [&](double t, bool* feas) -> int {
    int st = mag_solve(ctx, points, n, m, t, wp, &pm, &pi);
    ++probes;
    iters += pi.ir_iters;
    if (st != MAG_OK) return st;
    *feas = pi.min_w >= 0.0;
    return MAG_OK;
  };
  const bool ridders = ctx->opt.tplus_method == 1;
  bool feas = false;
  TRY(probe(t_hi, &feas));
  if (!feas) {
    if (info) info->probes = probes;
    return fail(ctx, MAG_ENOBRACKET, "min w = %.3e < 0 at the upper end t = %.17g", pi.min_w, t_hi);
  }
  cudaStream_t s = ctx->stream;
  CU(cudaMemcpyAsync(w, wp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double mag_hi = pm;
  mag_info info_hi = pi;
  TRY(probe(t_lo, &feas));
  double lo = t_lo, hi = t_hi;
  int below = 0;
  if (feas) {
    below = 1;
    hi = t_lo;
    CU(cudaMemcpyAsync(w, wp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    mag_hi = pm;
    info_hi = pi;
  } else if (!ridders) {
    while (hi - lo > rel_tol * hi) {
      const double mid = lo + (hi - lo) / 2.0;
      TRY(probe(mid, &feas));
      if (feas) {
        hi = mid;
        CU(cudaMemcpyAsync(w, wp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        mag_hi = pm;
        info_hi = pi;
      } else {
        lo = mid;
      }
    }
  } else {
    // Ridders' method (Ridders, IEEE Trans. Circuits Syst. 26 (1979)) on
    // f(t) = min_j w_j(t) with the bracket kept on feasibility: each
    // iteration evaluates the midpoint x3, then Ridders' point
    // x4 = x3 + (x3 - x1) sign(f1 - f2) f3 / sqrt(f3^2 - f1 f2) when it lies
    // inside the bracket; once two successive x4 agree to within
    // delta = rel_tol hi / 2, one evaluation at x4 -/+ delta closes the
    // bracket.  Every evaluation moves the bracket end of its class.
    double flo = pi.min_w, fhi = info_hi.min_w;
    auto eval = [&](double t, double* f) -> int {
      TRY(probe(t, &feas));
      *f = pi.min_w;
      if (feas) {
        hi = t;
        fhi = pi.min_w;
        CU(cudaMemcpyAsync(w, wp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        mag_hi = pm;
        info_hi = pi;
      } else {
        lo = t;
        flo = pi.min_w;
      }
      return MAG_OK;
    };
    double prev_x4 = NAN;
    while (hi - lo > rel_tol * hi) {
      const double x1 = lo, f1 = flo, f2 = fhi;
      const double x3 = lo + (hi - lo) / 2.0;
      double f3 = 0, f4 = 0;
      TRY(eval(x3, &f3));
      if (hi - lo <= rel_tol * hi) break;
      const double sq = std::sqrt(f3 * f3 - f1 * f2);
      if (!(sq > 0.0)) continue;
      const double x4 = x3 + (x3 - x1) * (f1 >= f2 ? 1.0 : -1.0) * f3 / sq;
      if (!(x4 > lo && x4 < hi)) {
        prev_x4 = NAN;
        continue;
      }
      TRY(eval(x4, &f4));
      if (hi - lo <= rel_tol * hi) break;
      const double delta = 0.5 * rel_tol * hi;
      if (std::fabs(x4 - prev_x4) <= delta) {
        const double xc = (hi == x4) ? x4 - delta : x4 + delta;
        double fc = 0;
        if (xc > lo && xc < hi) TRY(eval(xc, &fc));
      }
      prev_x4 = x4;
    }
  }
  CU(cudaStreamSynchronize(s));
  *t_plus = hi;
  t_bracket[0] = below ? hi : lo;
  t_bracket[1] = hi;
  *mag = mag_hi;
  if (info) {
    *info = info_hi;
    info->below_bracket = below;
    info->probes = probes;
    info->ir_iters = iters;
  }
  return MAG_OK;
}

int mag_grad(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t, const double* w,
             const double* dL_dw, double* dL_dt, double* dL_dx, mag_info* info) {
  TRY(check_args(ctx, points, n, m, t));
  if (!dL_dt || !dL_dx) return fail(ctx, MAG_EINVAL, "NULL output");
  if (m > 64) return fail(ctx, MAG_EINVAL, "mag_grad supports m <= 64 (m = %d)", (int)m);
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  mag_info si;
  std::memset(&si, 0, sizeof si);
  TRY(ensure_aux(ctx, n));
  cudaStream_t s = ctx->stream;
  double* wv = ctx->aux + (size_t)A_W * ctx->aux_np;
  double* lam = ctx->aux + (size_t)A_LAM * ctx->aux_np;
  double* g = ctx->aux + (size_t)A_G * ctx->aux_np;
  if (w) {
    CU(cudaMemcpyAsync(wv, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    double mg = 0;
    TRY(mag_solve(ctx, points, n, m, t, wv, &mg, &si));
  }
  bool constant_g = false;
  double gc = 0.0;
  if (dL_dw) {
    // a constant g = c 1 (the loss c Mag) needs no adjoint solve: lambda = c w
    if (!ctx->ws) TRY(ensure_workspace(ctx, n, false, false));
    CU(launch_minmax(dL_dw, n, &ctx->st()->aux[1], s));
    TRY(read_status(ctx));
    constant_g = ctx->h_st->aux[1] == ctx->h_st->aux[2];
    gc = ctx->h_st->aux[1];
  }
  if (dL_dw && constant_g) {
    CU(launch_scale(wv, gc, lam, n, s));
  } else if (dL_dw) {
    // adjoint solve lambda = Z^{-1} g
    CU(cudaMemcpyAsync(g, dL_dw, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    mag_info ai;
    TRY(mag_solve_rhs(ctx, points, n, m, t, g, lam, &ai));
    si.ir_iters += ai.ir_iters;
    si.rel_residual = std::max(si.rel_residual, ai.rel_residual);
    si.factor_reused = ai.factor_reused;
  } else {
    CU(cudaMemcpyAsync(lam, wv, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (!ctx->ws) TRY(ensure_workspace(ctx, n, false, false));
  double* part_t = ctx->aux + (size_t)A_PART * ctx->aux_np;
  CU(launch_grad(points, n, m, t, wv, lam, dL_dx, part_t, ctx->aux_np, s));
  CU(launch_sum_f64(part_t, n, &ctx->st()->aux[0], s));
  TRY(read_status(ctx));
  *dL_dt = ctx->h_st->aux[0];
  if (info) *info = si;
  return MAG_OK;
}

int mag_solve_batch(mag_ctx* ctx, const mag_batch_desc* desc, int32_t count, const double* points,
                    double* w_out, double* mag_out, int32_t* status_out, mag_info* info) {
  if (!ctx) return MAG_EINVAL;
  if (!desc || count < 0 || !points || !w_out || !mag_out) return fail(ctx, MAG_EINVAL, "bad batch arguments");
  ctx->err.clear();
  if (info) std::memset(info, 0, sizeof *info);
  if (count == 0) return MAG_OK;
  for (int32_t i = 0; i < count; ++i) {
    const mag_batch_desc& d = desc[i];
    if (d.n < 2 || d.m < 1 || d.m > MAG_MAX_DIM || !(d.t > 0.0) || !std::isfinite(d.t) || d.point_offset < 0 || d.w_offset < 0)
      return fail(ctx, MAG_EINVAL, "bad descriptor %d (n=%d m=%d t=%g)", (int)i, (int)d.n, (int)d.m, d.t);
  }
  cudaStream_t s = ctx->stream;
  const long long l0 = g_kernel_launches.load();
  // group problems by cloud (same points, n, m): distances are shared across t
  std::vector<BatchCloud> clouds;
  std::vector<BatchProblem> probs(count);
  std::vector<int> small, large;
  int64_t dist_total = 0, max_pairs = 0, nmax = 0;
  {
    std::vector<std::pair<std::pair<int64_t, int64_t>, int>> keys;  // ((offset, n*65536+m), cloud)
    for (int32_t i = 0; i < count; ++i) {
      const mag_batch_desc& d = desc[i];
      probs[i].w_offset = d.w_offset;
      probs[i].n = d.n;
      probs[i].t = d.t;
      if (d.n > BATCH_NMAX) {
        large.push_back(i);
        probs[i].cloud = -1;
        continue;
      }
      const std::pair<int64_t, int64_t> key(d.point_offset, (int64_t)d.n * 65536 + d.m);
      int cid = -1;
      for (auto& k : keys)
        if (k.first == key) cid = k.second;
      if (cid < 0) {
        BatchCloud c;
        c.point_offset = d.point_offset;
        c.dist_offset = dist_total;
        c.n = d.n;
        c.m = d.m;
        cid = (int)clouds.size();
        clouds.push_back(c);
        keys.push_back({key, cid});
        const int64_t pairs = (int64_t)d.n * (d.n - 1) / 2;
        dist_total += pairs;
        max_pairs = std::max(max_pairs, pairs);
      }
      probs[i].cloud = cid;
      probs[i].dist_offset = clouds[cid].dist_offset;
      nmax = std::max<int64_t>(nmax, d.n);
      small.push_back(i);
    }
  }
  std::vector<int> st_host(count, MAG_BATCH_OK);
  if (!small.empty()) {
    std::sort(small.begin(), small.end(), [&](int a, int b) { return probs[a].n > probs[b].n; });
    // launch shape (threads per CTA, CTAs per SM): options.batch_shape, else
    // the one tuned for this size class, else tuned below on a sample
    int cls = 0;
    while ((int64_t)1 << cls < nmax) ++cls;
    cls = std::min(cls, 11);
    int grids[kNumBatchShapes];
    for (int i = 0; i < kNumBatchShapes; ++i)
      grids[i] = std::min<int>(ctx->sm_count * std::max(1, batch_shape_resident(i)), (int)small.size());
    int shape = ctx->opt.batch_shape > 0 ? std::min(ctx->opt.batch_shape, kNumBatchShapes) - 1 : ctx->batch_tuned[cls];
    const int maxgrid = *std::max_element(grids, grids + kNumBatchShapes);
    // tuning needs a batch that fills every shape's grid twice
    const bool tune = shape < 0 && (int64_t)small.size() >= 2 * (int64_t)maxgrid && ctx->opt.batch_shape == 0;
    if (shape < 0 && !tune) shape = 0;
    int grid = 0;
    for (int i = 0; i < kNumBatchShapes; ++i)
      if (tune || i == shape) grid = std::max(grid, grids[i]);
    // batch workspace: clouds | problems | order | sample order | status | queue (+ tuner cycle count) | D |
    // scratch_f | scratch_d
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_cl = take(clouds.size() * sizeof(BatchCloud));
    const size_t o_pr = take((size_t)count * sizeof(BatchProblem));
    const size_t o_or = take(small.size() * sizeof(int));
    const size_t o_sa = take(small.size() * sizeof(int));
    const size_t o_st = take((size_t)count * sizeof(int));
    const size_t o_q = take(2 * sizeof(int));
    const size_t o_cy = take(sizeof(unsigned long long));
    const size_t o_cf = take(clouds.size() * sizeof(int));
    const size_t o_d = take((size_t)dist_total * sizeof(double));
    const size_t o_sf = take((size_t)grid * (nmax * nmax + nmax) * sizeof(float));
    const size_t o_sd = take((size_t)grid * (nmax * nmax + 2 * nmax) * sizeof(double));
    if (off > ctx->bws_bytes) {
      if (ctx->bws) {
        cudaStreamSynchronize(s);
        cudaFree(ctx->bws);
        ctx->bws = nullptr;
        ctx->bws_bytes = 0;
      }
      cudaError_t e = cudaMalloc(&ctx->bws, off);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->bws = nullptr;
        return fail(ctx, MAG_ENOMEM, "batch workspace of %.3g GB: %s", off / 1e9, cudaGetErrorString(e));
      }
      ctx->bws_bytes = off;
    }
    char* base = (char*)ctx->bws;
    BatchCloud* d_cl = (BatchCloud*)(base + o_cl);
    BatchProblem* d_pr = (BatchProblem*)(base + o_pr);
    int* d_or = (int*)(base + o_or);
    int* d_sa = (int*)(base + o_sa);
    int* d_st = (int*)(base + o_st);
    int* d_q = (int*)(base + o_q);
    unsigned long long* d_cy = (unsigned long long*)(base + o_cy);
    int* d_cf = (int*)(base + o_cf);
    double* d_D = (double*)(base + o_d);
    float* d_sf = (float*)(base + o_sf);
    double* d_sd = (double*)(base + o_sd);
    CU(cudaMemcpyAsync(d_cl, clouds.data(), clouds.size() * sizeof(BatchCloud), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_pr, probs.data(), (size_t)count * sizeof(BatchProblem), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_or, small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(d_cf, 0, clouds.size() * sizeof(int), s));
    CU(launch_batch_dist(points, d_cl, (int)clouds.size(), max_pairs, d_D, d_cf, s));
    const double tol = kStopMargin * ctx->opt.ir_tol;
    const int max_iter = std::max(ctx->opt.ir_max_iters, 1);
    if (tune) {
      // every k-th problem of the size-sorted order (the batch's size mix),
      // about twice the largest grid; each shape solves it once.  The measure
      // is the CTAs' summed busy cycles over the grid -- the time of a batch
      // whose load balances, as the full one does with several problems per
      // CTA -- not the sample's makespan, which one large problem can set.
      // The fastest shape is kept for this size class; the sample's outputs
      // are overwritten by the full run below.
      const int64_t want = 2 * (int64_t)maxgrid;
      const int64_t stride = std::max<int64_t>(1, (int64_t)small.size() / want);
      std::vector<int> sample;
      for (int64_t i = 0; i < (int64_t)small.size() && (int64_t)sample.size() < want; i += stride)
        sample.push_back(small[i]);
      CU(cudaMemcpyAsync(d_sa, sample.data(), sample.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      double best = INFINITY;
      for (int i = 0; i < kNumBatchShapes; ++i) {
        const int g = std::min<int>(grids[i], (int)sample.size());
        CU(cudaMemsetAsync(d_q, 0, sizeof(int), s));
        CU(cudaMemsetAsync(d_cy, 0, sizeof(unsigned long long), s));
        CU(launch_batch_solve(i, d_pr, d_sa, (int)sample.size(), d_D, d_cf, d_sf, d_sd, nmax, w_out, mag_out,
                              d_st, d_q, tol, max_iter, g, d_cy, s));
        unsigned long long cyc = 0;
        CU(cudaMemcpyAsync(&cyc, d_cy, sizeof cyc, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        const double est = (double)cyc / g;
        if (est < best) {
          best = est;
          shape = i;
        }
      }
      ctx->batch_tuned[cls] = shape;
    }
    ctx->batch_shape_used = shape;
    CU(cudaMemsetAsync(d_q, 0, sizeof(int), s));
    CU(cudaMemsetAsync(d_st, 0, (size_t)count * sizeof(int), s));
    CU(launch_batch_solve(shape, d_pr, d_or, (int)small.size(), d_D, d_cf, d_sf, d_sd, nmax, w_out,
                          mag_out, d_st, d_q, tol, max_iter, grids[shape], nullptr, s));
    CU(cudaMemcpyAsync(st_host.data(), d_st, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
  }
  // problems too large for one CTA, or that the FP32 batch path could not
  // finish, go through the single-problem solver (which escalates precision)
  int first = MAG_OK, fallbacks = 0;
  std::vector<int32_t> final_st(count, MAG_OK);
  for (int32_t i = 0; i < count; ++i) {
    if (probs[i].cloud >= 0 && (st_host[i] == MAG_BATCH_DUPLICATE || st_host[i] == MAG_BATCH_NONFINITE)) {
      final_st[i] = st_host[i] == MAG_BATCH_DUPLICATE ? MAG_EDUPLICATE : MAG_EINVAL;
      if (first == MAG_OK) first = final_st[i];
      continue;
    }
    const bool redo = probs[i].cloud < 0 || st_host[i] != MAG_BATCH_OK;
    if (!redo) continue;
    ++fallbacks;
    double mg = 0;
    const mag_batch_desc& d = desc[i];
    int st = mag_solve(ctx, points + d.point_offset, d.n, d.m, d.t, w_out + d.w_offset, &mg, nullptr);
    CU(cudaMemcpyAsync(mag_out + i, &mg, sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    final_st[i] = st;
    if (st != MAG_OK && first == MAG_OK) first = st;
  }
  if (status_out) {
    CU(cudaMemcpyAsync(status_out, final_st.data(), (size_t)count * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
  }
  if (info) {
    info->fallback = fallbacks;
    info->kernel_launches = g_kernel_launches.load() - l0;
    info->batch_threads = kBatchShapes[ctx->batch_shape_used].threads;
    info->batch_ctas_per_sm = kBatchShapes[ctx->batch_shape_used].ctas_per_sm;
    info->batch_tensor_cores = kBatchShapes[ctx->batch_shape_used].tensor_cores;
    info->batch_left_looking = kBatchShapes[ctx->batch_shape_used].left_looking;
  }
  return first;
}

}  // extern "C"
