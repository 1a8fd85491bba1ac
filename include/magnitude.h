/*
 * magnitude.h -- C ABI of the GB300 metric-magnitude solver.
 *
 * Paper: "Scalably computing metric magnitude" (arXiv 2607.23354).
 *
 * For points x_1..x_n in R^m (Sec. 2):
 *   d_jk = ||x_j - x_k||          (Euclidean distance, from coordinate differences)
 *   Z    = exp[-t d]              (similarity matrix, componentwise exp, t > 0)
 *   Z w  = 1                      (Eq. weighting; Z is positive definite, w unique)
 *   Mag  = 1^T w                  (magnitude)
 *   t_+  = least t with w >= 0    (cutoff, Sec. 2), bounded by
 *          t_+ <= log(n-1) / min_{j != k} d_jk   (Sec. 1)
 *
 * Conventions for every entry point:
 *   - Every function returns an int status (enum mag_status).  On an error
 *     mag_last_error(ctx) gives a one-line message for that context.
 *   - Array arguments are DEVICE pointers owned by the caller (for example
 *     PyTorch tensors on the context's device), FP64, C-contiguous.  Points
 *     are an n x m row-major array.  Scalars come back through HOST pointers.
 *   - Work is ordered on the stream given to mag_ctx_create; every entry
 *     point returns after its results (device arrays and host scalars) are
 *     complete on that stream (the host waits on the stream).
 *   - The library owns only the workspace inside a context (device memory it
 *     allocates and grows on demand, freed by mag_ctx_destroy).  A context is
 *     used by one host thread at a time; use one context per thread/stream.
 *   - Invalid arguments (n < 2, m < 1 or m > MAG_MAX_DIM, t <= 0 or not
 *     finite, NULL pointers) give MAG_EINVAL before any device work.
 *     Non-finite coordinates give MAG_EINVAL and coincident points
 *     MAG_EDUPLICATE (Z is then singular), both detected on the device while
 *     Z is generated.
 */
#ifndef MAGNITUDE_H
#define MAGNITUDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest dimension m of the points accepted by every entry point (the
 * matrix-free residual stages at least eight points of m + 1 doubles in
 * shared memory).  mag_grad accepts m <= 64. */
#define MAG_MAX_DIM 2048

/* Status codes. */
enum mag_status {
  MAG_OK = 0,
  MAG_EINVAL = 1,        /* bad argument or non-finite coordinate            */
  MAG_EDUPLICATE = 2,    /* two points coincide: min d = 0, Z singular        */
  MAG_ENOTPD = 3,        /* every precision tried hit a non-positive pivot    */
  MAG_ENOCONV = 4,       /* refinement did not reach the tolerance; the best
                            w found is returned with its residual in info    */
  MAG_ENOBRACKET = 5,    /* sweep: w is not nonnegative at the upper end     */
  MAG_ENOMEM = 6,        /* workspace allocation failed or exceeds the limit */
  MAG_ECUDA = 7,         /* a CUDA call failed (message in mag_last_error)   */
  MAG_ETIMEOUT = 8       /* a bounded device wait gave up                    */
};

/* Precision of the Cholesky factor (Zw = 1 is always refined in FP64). */
enum mag_precision {
  MAG_PREC_AUTO = 0,     /* FP16 if the Gershgorin bound gives lambda_min(Z) >= 1/2;
                            else (n >= 384 K, K = min(24, panel width)) FP16
                            when a probe (FP16 factor + two refinement steps
                            on the leading 128 K points) predicts that its
                            extra refinement steps cost less than the factor
                            time saved; else FP16X3.  A mispredicted FP16
                            factor that refines slowly is replaced by FP16X3
                            (mag_info.fallback = 3).                        */
  MAG_PREC_BF16 = 1,     /* BF16 tensor-core products, FP32 accumulation      */
  MAG_PREC_TF32 = 2,     /* one TF32 tensor-core product, FP32 accumulation   */
  MAG_PREC_TF32X3 = 3,   /* split TF32 (hi*hi + hi*lo + lo*hi), FP32 accum.   */
  MAG_PREC_FP32 = 4,     /* FP32 CUDA-core products (no tensor cores)          */
  MAG_PREC_FP64 = 5,     /* full FP64 factor (the plain dense method)          */
  MAG_PREC_FP16X3 = 6,   /* split FP16 of the panel scaled by 2^12 (hi*hi +
                            hi*lo + lo*hi), FP32 accumulation: split-TF32
                            accuracy at the FP16 tensor rate                   */
  MAG_PREC_FP16 = 7      /* one FP16 product of that scaled panel              */
};

/* How the FP64 residual r = 1 - Zw of iterative refinement is formed. */
enum mag_residual_mode {
  MAG_RESID_MATRIX_FREE = 0, /* Z_jk regenerated in FP64 from the points      */
  MAG_RESID_STORED = 1,      /* Z kept in FP64 tiles, residual reads them      */
  MAG_RESID_AUTO = 2         /* STORED when its extra n^2/2 FP64 tiles fit in
                                half of the free device memory, else MATRIX_FREE */
};

typedef struct mag_options {
  int32_t precision;      /* enum mag_precision, default MAG_PREC_AUTO           */
  int32_t residual_mode;  /* enum mag_residual_mode, default MAG_RESID_AUTO      */
  double ir_tol;          /* target ||1-Zw||inf/(||Z||inf ||w||inf), default 1e-14 */
  int32_t ir_max_iters;   /* refinement steps before escalating, default 12     */
  int32_t gmres_max_iters;/* inner GMRES iterations of GMRES-IR, default 30     */
  int32_t allow_fallback; /* 1: escalate to GMRES-IR then FP64 factor (default)  */
  int32_t panel_tiles;    /* outer panel width in 128-wide tiles (0: 16 for the
                             split precisions, 32 for one-product factors)     */
  double workspace_limit_bytes; /* 0 = no limit; larger requests give ENOMEM     */
  int32_t profile;        /* 1: time the trailing-update kernel with CUDA events */
  int32_t reuse_distances;/* 1 (default): inside one mag_solve_multi or
                             mag_sweep_tplus call, keep the FP64 distances in
                             device memory (n^2/2 doubles) and regenerate Z for
                             each t from them when they fit; 0: recompute      */
  int32_t lookahead;      /* 1 (default): the tensor-core factor runs the next
                             panel (its update, diagonal factor, panel solve
                             and copy) on a second stream alongside the
                             trailing update of the current panel; 0: one
                             stream, step after step (same arithmetic)        */
  int32_t lookahead_sms;  /* how the look-ahead streams share the GPU.  > 0:
                             that many SMs kept free of the (persistent)
                             trailing update for the panel stream, whose
                             launches beside it use that many CTAs.  0
                             (default): the panel stream has the higher
                             stream priority and every trailing CTA (pair)
                             leaves after 4 output blocks of 256 x 256,
                             so the panel stream's CTAs take
                             SMs as they come free; < 0: the same with
                             -lookahead_sms blocks per CTA                   */
  int32_t cta_pairs;      /* tensor-core updates on clusters of two CTAs
                             sharing each 256 x 256 MMA (cta_group::2):
                             1 (default) always, 0 never, 2 for the split
                             precisions (FP16X3, TF32X3) only                 */
  int32_t tplus_method;   /* mag_sweep_tplus root-finder on min_j w_j(t):
                             0 (default) bisection, 1 Ridders' method        */
  int64_t wait_timeout_ns;/* the persistent triangular sweeps wait for
                             tiles that other CTAs solve; each wait gives up
                             this long after the sweep started and the solve
                             returns MAG_ETIMEOUT (default 1e10 = 10 s; must be
                             > 0).  The context stays usable.  The
                             tensor-core update keeps a fixed 20 s bound on
                             its barrier waits.                               */
  int32_t out_of_core;    /* 0 (default): when the packed FP32 tiles of Z do
                             not fit in device memory (or in
                             workspace_limit_bytes), factor slab by slab:
                             slabs of tile columns generated, updated by the
                             earlier slabs and factored on the device, then
                             kept in device memory while it has room, else in
                             pinned host memory; the triangular solves read
                             each slab where it lives.  1: always (slabs
                             sized by workspace_limit_bytes or the free device
                             memory); -1: never.  FP16, FP16X3 and AUTO only;
                             the residual is then matrix free.             */
  int32_t deflate;        /* mag_solve at the small-t end, where Z nears the
                             all-ones matrix: 0 (default) when t max d <= 1/4
                             (judged from max_j ||x_j - x_0||), solve instead
                             A u = 1 with A = (Z - (1 - c t) 1 1^T) / (c t)
                             (entries 1 + expm1(-t d_jk) / (c t), unit
                             diagonal), positive definite and well
                             conditioned for c large enough, and return
                             w = u / (c t + (1 - c t) 1^T u) = Z^{-1} 1
                             (Sherman-Morrison); 1: whenever c t <= 1 allows
                             it; -1: never.  Reported in
                             mag_info.deflation_c.                          */
  double host_limit_bytes;/* pinned host memory the out-of-core factor may
                             take (0: half of the host's physical memory);
                             more gives MAG_ENOMEM                          */
  int32_t gmres_matvec;   /* products Z v of GMRES-IR's inner iterations
                             and the residuals of refinement steps far
                             above the tolerance: 0 (default) float-float on
                             the FP32 pipe from the stored FP64 tiles of
                             exp(-t d) (a few units of 2^-46 of sum |Z||v|;
                             the residuals that decide convergence stay
                             FP64), else FP64 as the residual               */
  int32_t fp16_gmres;     /* AUTO: 0 (default) the one-product FP16 factor
                             with GMRES-IR straight after the first solve
                             when the probe predicts plain refinement to
                             diverge or crawl (contraction <= 16) and the
                             factor saved outweighs the inner iterations
                             (n >= 72,000 with stored tiles); a GMRES-IR that
                             stalls is replaced by the split factor
                             (mag_info.fallback = 3); -1 never; 1 whenever
                             the contraction is <= 16 (any n)              */
  int32_t batch_shape;    /* mag_solve_batch launch shape: 0 (default) tuned
                             per size class (ceil(log2 max n)) on the first
                             batch of that class with at least twice the
                             largest grid of problems -- each shape solves a
                             sample of the batch once, the fastest is kept
                             (smaller batches use shape 1 until then); 1:
                             512 threads x 1 CTA per SM, 2: 256 x 2, 3: 256
                             x 3, all with the factor's trailing update on
                             the CUDA cores in FP32; 4: 256 x 2, 5: 256 x 3
                             with it on the tensor cores in split TF32; 6:
                             256 x 2, 7: 256 x 3 with a left-looking factor
                             (each block of A updated once, with all earlier
                             columns; CUDA cores) (mag_info.batch_threads /
                             _ctas_per_sm / _tensor_cores / _left_looking)  */
  int32_t sweep_kind;     /* triangular sweeps of the refinement corrections
                             (in core): 0 (default) one product with a
                             precomputed B_I = inv(L_II) L_{I,I-1} per tile on
                             the sweep's critical path, the off-diagonal tiles
                             read as FP16 for the one-product FP16 factor (the
                             operands its updates used) and as FP32 otherwise;
                             1 the same with FP32 tiles always; 2 the sweeps
                             with one progress counter and the full tile
                             product per step                               */
  int32_t exact_distances;  /* distances of a multi-t call (mag_solve_multi,
                             mag_sweep_tplus) from coordinates quantized to
                             a common grid, as exact integer sums on the
                             integer pipe (1, default; pairs closer than
                             sqrt(m) 2^53 times the grid step take FP64
                             differences), or FP64 differences for all
                             pairs (0).  Either way within the FP64
                             differences' rounding of d; m <= 32 and finite
                             coordinates, else FP64                          */
  int32_t reserved4;
} mag_options;

/* Diagnostics of one call (all fields written when info != NULL). */
typedef struct mag_info {
  int32_t precision_used;  /* enum mag_precision of the factor that succeeded  */
  int32_t ir_iters;        /* refinement steps taken (all precisions)          */
  int32_t gmres_iters;     /* total inner GMRES iterations (0 if not used)     */
  int32_t fallback;        /* 0 none, 1 GMRES-IR, 2 FP64 factor, 3 the probe's
                              FP16 choice refined slowly: split factor,
                              4 the probe chose the FP16 factor with
                              GMRES-IR (options.fp16_gmres)                  */
  int32_t residual_mode;   /* enum mag_residual_mode actually used (0 or 1)    */
  int32_t reserved0;
  double rel_residual;     /* final ||1-Zw||inf / (||Z||inf ||w||inf)          */
  double z_norm_inf;       /* ||Z||inf = max row sum                           */
  double w_norm_inf;       /* max |w_j|                                       */
  double min_w;            /* min w_j                                         */
  double gershgorin_lmin;  /* 1 - max_j sum_{k != j} Z_jk (lower bound on
                              lambda_min); NaN for out-of-core solves, which
                              do not form the row sums before the factor     */
  double min_distance;     /* min_{j != k} d_jk                                */
  int32_t below_bracket;   /* sweep: feasible already at t_lo                  */
  int32_t probes;          /* sweep: number of solves                           */
  double ms_generate, ms_factor, ms_solve, ms_residual, ms_total;
  double useful_flops;     /* n^3/3 + 2 n^2 ir_iters (factor + refinement steps)   */
  int64_t kernel_launches; /* kernels this call launched                        */
  int32_t residual_evals;  /* FP64 residual evaluations                         */
  int32_t update_launches; /* trailing-update kernel launches                   */
  double ms_update;        /* their total device time (profile = 1), else 0     */
  double update_flops;     /* algorithmic flops of those launches: 2*128^3 per
                              (output tile, panel tile) product                 */
  double ms_update_panel;  /* part of ms_update spent inside panels (profile = 1) */
  double ms_potrf;         /* diagonal-tile factors (profile = 1)              */
  double ms_trsm;          /* panel solves (profile = 1)                        */
  double ms_split;         /* panel copies for the tensor cores (profile = 1)   */
  double probe_rho;        /* AUTO precision probe: predicted contraction per
                              refinement step of the one-product FP16 factor
                              (0 = no probe, +inf = its block factor broke down) */
  double ms_probe;         /* device time of the probe                          */
  double t;                /* the t of this solve (the Sec. 1 bound where the
                              call asked for it with t <= 0)                   */
  int32_t slabs;           /* slabs of the out-of-core factor (0: in core)     */
  int32_t host_slabs;      /* of which held in host memory                      */
  double host_bytes;       /* bytes of the factor in host memory               */
  double host_read_bytes;  /* bytes the factor's slab updates read from host
                              memory (over the CPU-GPU link)                   */
  double ms_host_read;     /* device time of those reads (profile = 1)          */
  double deflation_c;      /* c of the deflated small-t solve (0: not used);
                              rel_residual, z_norm_inf and w_norm_inf are then
                              those of Z w = 1, the refinement's counts those
                              of A u = 1                                       */
  int32_t factor_reused;   /* mag_solve_rhs (mag_grad's adjoint solve) refined
                              with the factor the last solve of the same points
                              (pointer, size and contents) and t left in the
                              context, without generating or factoring again */
  int32_t reserved2;
  double ms_update_busy;   /* length of the union of the update launches'
                              intervals (profile = 1): the time during which
                              at least one update launch was in flight; the
                              look-ahead streams overlap, so ms_update, a sum
                              of intervals, counts shared stretches twice    */
  int32_t batch_threads;   /* mag_solve_batch: threads per CTA of the launch   */
  int32_t batch_ctas_per_sm; /* ... the CTAs per SM of its shape              */
  int32_t batch_tensor_cores; /* ... 1: the factor's trailing update on the
                              tensor cores (split TF32), 0: CUDA cores      */
  int32_t residual_evals_ff; /* refinement residuals taken in float-float from
                              the stored tiles (far above the tolerance; the
                              deciding ones are FP64, in residual_evals)     */
  int32_t batch_left_looking; /* mag_solve_batch: 1 left-looking factor      */
  int32_t sweeps_used;     /* triangular sweeps of the last correction: 0 the
                              chain sweeps with FP16 tiles, 1 with FP32 tiles,
                              2 the progress-counter sweeps (FP64 factor, out
                              of core, options.sweep_kind = 2); -1 none     */
  int32_t exact_distances; /* 1: the distances came from the exact integer
                              pass (options.exact_distances)                */
  int32_t reserved6;
} mag_info;

typedef struct mag_ctx mag_ctx;

/* Fill *opt with the defaults listed above. */
int mag_options_default(mag_options* opt);

/* Create a context bound to the current CUDA device and `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  opt == NULL = defaults.
 * The options are copied. */
int mag_ctx_create(mag_ctx** ctx, void* stream, const mag_options* opt);
/* Replace the options of an existing context. */
int mag_ctx_set_options(mag_ctx* ctx, const mag_options* opt);
/* Free the context and its workspace (NULL is a no-op). */
int mag_ctx_destroy(mag_ctx* ctx);
/* Message of the last error on this context ("" if none).  Valid until the
 * next call on the context. */
const char* mag_last_error(const mag_ctx* ctx);
/* Static name of a status code. */
const char* mag_status_string(int status);
/* Device bytes the workspace of a solve of size n needs under ctx's options. */
int mag_workspace_bytes(const mag_ctx* ctx, int64_t n, int32_t m, double* bytes);

/* a1 (Sec. 1): min_{j != k} d_jk and the bound t = log(n-1) / min d, from one
 * pass over all pairs on the device.  points: device, n x m.  Host outputs.
 * MAG_EDUPLICATE if two points coincide (then *dmin = 0, *t_bound = inf). */
int mag_min_distance(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double* dmin,
                     double* t_bound);

/* a2 (Sec. 2): Z = exp[-t d] from the fused generator, unpacked to a dense
 * n x n row-major array Z_out (device; FP64 when precision == MAG_PREC_FP64,
 * else FP32, the values the factor starts from).  For inspection and tests of
 * the generator; the solver itself never forms the dense matrix. */
int mag_similarity_matrix(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                          int32_t precision, void* Z_out);

/* a2+a3 (Sec. 3.2): the lower Cholesky factor L of Z = L L^T computed by the
 * blocked solver in `precision` (MAG_PREC_FP64 -> FP64 output, else FP32),
 * unpacked to a dense n x n row-major array L_out (device; zeros above the
 * diagonal).  MAG_ENOTPD if a pivot is not positive. */
int mag_cholesky_factor(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                        int32_t precision, void* L_out);

/* a2-a7 (Sec. 2, Eq. weighting): solve Zw = 1 for Z = exp[-t d] and return
 * Mag = 1^T w.  points: device n x m FP64; w: device output, n FP64; mag:
 * host output.  The factor precision follows ctx's options (MAG_PREC_AUTO:
 * one scaled-FP16 product when the Gershgorin bound gives lambda_min >= 0.5,
 * else the scaled-FP16 split);
 * FP64 iterative refinement with a residual formed in FP64 runs until the
 * relative residual is <= ir_tol, escalating to GMRES-IR and then to an FP64
 * factor when allow_fallback is set.  MAG_ENOCONV returns the best w found. */
int mag_solve(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t, double* w,
              double* mag, mag_info* info);

/* a2-a7 for several values of t on the same points (Sec. 2: Z = exp[-t d]
 * shares d across t): ts (host, nt values), W (device, nt x n row-major: the
 * weighting of ts[i] in row i), mags (host, nt), infos (host, nt, nullable).
 * A value ts[i] <= 0 stands for the Sec. 1 bound t = log(n-1) / min d, with
 * min d taken from the first solve of the call (the generator finds it while
 * it forms Z): the positive values are solved first, in their order, then the
 * bound entries (a call with only bound entries makes one min-distance pass
 * first); infos[i].t reports the t solved.  The FP64 distances are computed
 * once and kept for the call (see reuse_distances).  Returns the first non-OK
 * status; later t values are still solved. */
int mag_solve_multi(mag_ctx* ctx, const double* points, int64_t n, int32_t m, const double* ts, int32_t nt,
                    double* W, double* mags, mag_info* infos);

/* The same solve for a general right-hand side: Z x = b (b: device, n).  Used
 * for the adjoint solve lambda = Z^{-1} dL/dw of mag_grad.  When the last
 * solve on this context (mag_solve, mag_solve_multi's last t, mag_solve_rhs)
 * had the same points -- pointer, n, m and a checksum of the contents -- and
 * the same t, its factor is still in the workspace and the call only refines
 * with it (info.factor_reused = 1); it factors again if that refinement does
 * not reach the tolerance. */
int mag_solve_rhs(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
                  const double* b, double* x, mag_info* info);

/* a5 (accuracy measure of "numerically exact", Sec. 1): the FP64 residual
 * r = b - Z w with Z = exp[-t d] regenerated from the points on the fly (no
 * n x n storage), row sums compensated.  points: device n x m; w: device n;
 * b: device n, or NULL for the all-ones right-hand side of Eq. weighting;
 * r_out: device n, or NULL if only the norms are wanted.  norms (host, 4
 * doubles): ||r||inf / (||Z||inf ||w||inf), ||r||inf, ||Z||inf (max row
 * sum), ||w||inf. */
int mag_residual(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t, const double* w,
                 const double* b, double* r_out, double* norms);

/* Largest n accepted by mag_residual_noalloc. */
#define MAG_NOALLOC_MAX_N 262144

/* The FP64 residual of mag_residual for callers that must not allocate device
 * memory: code that runs under an external memory manager (a framework's
 * caching allocator or a fixed memory budget) where a hidden cudaMalloc would
 * fragment or exceed the budget, and latency-critical loops where cudaMalloc
 * and cudaFree would synchronize the device.  (The paper has no counterpart;
 * this is an interface convenience.)
 *
 * It needs no context and calls no allocating routine.  Its scratch (3 FP64
 * partial sums per row and the norm maxima) is one static device array of
 * 3 * MAG_NOALLOC_MAX_N + 32 doubles (about 6 MiB), which every GPU that loads
 * this library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the
 * caller's device current; make that first call before any stream capture.
 * All calls share the array: the norm maxima are cleared at the start of
 * each call, and calls that overlap on the GPU (other streams or threads)
 * race on it, so serialize them.
 *
 * points: device n x m; w: device n; b: device n or NULL (all ones);
 * r_out: device n (required); norms: host, 4 doubles as in mag_residual;
 * stream: cudaStream_t (NULL = legacy default stream) of the current device,
 * which must also be the device that holds the arrays.  The call returns
 * after the stream has completed the work.  MAG_EINVAL for bad arguments
 * (including m > MAG_MAX_DIM), MAG_ENOMEM when n > MAG_NOALLOC_MAX_N,
 * MAG_ECUDA if a CUDA call fails. */
int mag_residual_noalloc(const double* points, int64_t n, int32_t m, double t, const double* w,
                         const double* b, double* r_out, double* norms, void* stream);

/* a8 (Sec. 2 and its footnote): the cutoff t_+ on the sign of min_j w_j by
 * bisection (default) or Ridders' method (options.tplus_method = 1, the
 * root-finder Sec. 2 prefers).  feasible(t) <=> min_j w_j(t) >= 0.
 * t_hi <= 0 uses the Sec. 1 bound.  The bracket keeps feasible(hi) and not
 * feasible(lo).  Bisection solves at the FP64 midpoint lo + (hi - lo)/2.
 * Ridders evaluates the midpoint x3, then x4 = x3 + (x3 - lo) sign(f(lo) -
 * f(hi)) f(x3) / sqrt(f(x3)^2 - f(lo) f(hi)) with f = min_j w_j when x4 lies
 * inside the bracket, and once two successive x4 agree to rel_tol hi / 2 one
 * more point x4 -/+ rel_tol hi / 2 toward the other end; every evaluation
 * moves the bracket end of its feasibility class.  Both stop when
 * hi - lo <= rel_tol * hi.  Outputs (host): *t_plus = hi, t_bracket[0..1] =
 * {lo, hi}; w (device, n) and *mag are those at t_plus.  If feasible(t_lo)
 * holds, returns MAG_OK with t_plus = t_lo and info->below_bracket = 1.  If
 * feasible(t_hi) fails, MAG_ENOBRACKET. */
int mag_sweep_tplus(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t_lo,
                    double t_hi, double rel_tol, double* t_plus, double* t_bracket, double* w,
                    double* mag, mag_info* info);

/* The weighting at scale zero (App. C, Eq. scaleZero):
 *   w0 = lim_{t -> 0} Z(t)^{-1} 1 = d^{-1} 1 / (1^T d^{-1} 1).
 * d (zero diagonal) is indefinite; the library solves instead
 * M z = 1 with M = 1 1^T - d / c, positive definite for c large enough and
 * with d^{-1} 1 proportional to M^{-1} 1 (Sherman-Morrison), so that
 * w0 = z / 1^T z and 1^T d^{-1} 1 = 1^T z / (c (1^T z - 1)).  c starts at
 * 4 max_j ||x_j - x_0|| (>= 2 max d) and doubles on a non-positive pivot.
 * M has the structure of Z (unit diagonal, entries in [0, 1]), so the same
 * tensor-core factor, FP64 refinement (to options.ir_tol on M z = 1) and
 * fallbacks apply.  Outputs: w0 (device, n, sums to 1), *s = 1^T d^{-1} 1
 * (host); info as for mag_solve on M (min_w is min_j w0_j).  Errors as
 * mag_solve; MAG_EDUPLICATE if two points coincide. */
int mag_scale_zero(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double* w0, double* s,
                   mag_info* info);

/* a9: gradients by implicit differentiation of Zw = 1 (not in the paper).
 * For a loss L(w) with g = dL/dw (device, n; NULL means L = Mag, g = 1):
 *   lambda = Z^{-1} g (lambda = w when g = 1),
 *   dL/dt   = lambda^T (d o Z) w,
 *   dL/dx_i = t sum_{k != i} Z_ik (x_i - x_k)/d_ik (lambda_i w_k + lambda_k w_i).
 * w (device, n) may be NULL, in which case it is solved first.  Outputs:
 * *dL_dt (host), dL_dx (device, n x m row-major). */
int mag_grad(mag_ctx* ctx, const double* points, int64_t n, int32_t m, double t,
             const double* w, const double* dL_dw, double* dL_dt, double* dL_dx, mag_info* info);

/* One problem of a batch: points of cloud c start at points + point_offset
 * (units of doubles, n x m row-major); its weighting is written at
 * w_out + w_offset (n doubles) and its magnitude at mag_out[index]. */
typedef struct mag_batch_desc {
  int64_t point_offset;
  int64_t w_offset;
  int32_t n;
  int32_t m;
  double t;
} mag_batch_desc;

/* a10: many independent solves (uneven n, any t) in one persistent launch
 * sequence.  desc: HOST array of count descriptors; points, w_out: device;
 * mag_out: device, count doubles.  Each problem is factored in FP32 and
 * refined in FP64 to ctx's ir_tol.  status_out (device, count int32, may be
 * NULL) receives a per-problem mag_status.  Returns MAG_OK when every
 * problem converged, else the first failing status. */
int mag_solve_batch(mag_ctx* ctx, const mag_batch_desc* desc, int32_t count, const double* points,
                    double* w_out, double* mag_out, int32_t* status_out, mag_info* info);

#ifdef __cplusplus
}
#endif

#endif /* MAGNITUDE_H */
