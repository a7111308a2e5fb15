/*
 * rsrs.h -- C ABI of the GB300 (sm_103a) implementation of randomized strong
 * recursive skeletonization (RSRS), Yesypenko & Martinsson, arXiv 2311.01451.
 *
 * The library follows the paper's statement of the problem (Sec. 1 and
 * Algorithm 1): given a matrix A reachable through products with A and A*,
 * points x_i in R^d with a quad/octree over them, a rank k and a sample count s,
 * it draws (or takes) Gaussian test matrices Omega, Psi (N x s), forms the
 * sketches Y = A Omega, Z = A* Psi (eq. rand_sample_setting), and post-processes
 * them level by level into the invertible factorization
 *     A ~ V_1 ... V_M P D P^T W_M ... W_1            (eq. Afact)
 * whose inverse gives a direct solver / preconditioner (eq. Ainvfact).
 *
 * Conventions for every entry point:
 *  - Every function returns rsrs_status; 0 (RSRS_OK) is success.  The library
 *    never aborts, exits or traps.  Invalid arguments are rejected before any
 *    device work (RSRS_E_INVAL); conditions found on the device (a zero or
 *    non-finite pivot) are reported after the call's stream synchronises.
 *  - "stream" is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls synchronise that stream before they return.
 *  - Device pointers ("_dev") are CUDA device memory owned by the caller, read
 *    during the call or overwritten in place where stated.  Host pointers
 *    ("_host") are read during the call only.
 *  - Right-hand-side blocks are column-major N x nrhs with leading dimension
 *    ld >= N, indexed by ORIGINAL point number; the library permutes internally.
 *  - Trees and factors are opaque and library-owned until freed.
 */
#ifndef RSRS_H
#define RSRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSRS_OK = 0,
  RSRS_E_INVAL = 1,         /* bad argument (null pointer, size, layout)           */
  RSRS_E_UNDERSAMPLED = 2,  /* s below the sample bound of Sec. 4.5 (see s_req)     */
  RSRS_E_SINGULAR = 3,      /* zero pivot in the LU of an X_RR block or the root    */
  RSRS_E_NONFINITE = 4,     /* NaN/Inf met in a sketch, a Gram or a pivot           */
  RSRS_E_NOMEM = 5,         /* device allocation failed                             */
  RSRS_E_CUDA = 6,          /* a CUDA runtime call failed                           */
  RSRS_E_CALLBACK = 7,      /* the user matvec callback returned non-zero           */
  RSRS_E_TIMEOUT = 8,       /* a bounded device wait ran out                        */
  RSRS_E_NOT_CONVERGED = 9  /* refinement stopped at maxit above rtol               */
} rsrs_status;

typedef struct rsrs_tree rsrs_tree;
typedef struct rsrs_factor rsrs_factor;

/* Operator kinds.  Built-in kernels are A = diag_shift*I + scale*K with
 * K_ij = log|x_i - x_j| (2D) or 1/|x_i - x_j| (3D) for i != j and K_ii = 0,
 * evaluated on the fly on the device (symmetric, so A* = A). */
enum { RSRS_OP_LOG2D = 1, RSRS_OP_INVR3D = 2, RSRS_OP_CALLBACK = 3 };

/* User matvec: Y = A X (adjoint = 0) or Y = A* X (adjoint = 1), all device
 * memory, column-major n x ncols with leading dimensions ldx, ldy, rows in
 * ORIGINAL point order.  It must enqueue its work on `stream` only and return
 * 0 on success; any other value aborts the call with RSRS_E_CALLBACK. */
typedef int (*rsrs_matvec_fn)(void* ctx, int adjoint, int64_t n, int32_t ncols,
                              const double* X_dev, int64_t ldx, double* Y_dev,
                              int64_t ldy, void* stream);

typedef struct {
  int kind;            /* RSRS_OP_*                                            */
  double diag_shift;   /* built-in kernels: A = diag_shift*I + scale*K           */
  double scale;
  rsrs_matvec_fn fn;   /* RSRS_OP_CALLBACK only                                  */
  void* ctx;
} rsrs_operator;

/* Arithmetic of the build and of the factor. */
enum {
  RSRS_PREC_FP64 = 0,   /* every step in FP64                                               */
  RSRS_PREC_MIXED = 1   /* FP32 arithmetic (FP64 storage) for the sampling product, the      */
                        /* near-field Grams, Cholesky factors, projections, the E/F and     */
                        /* Schur updates, X_RR^-1 (Gauss-Jordan with partial pivoting; from */
                        /* an FP64 LU when r > 224), Lc, Uc and the solve sweeps; FP64 for  */
                        /* the CPQR pivots, extraction, the root and the refinement residual */
};

/* Tile shapes of the tensor-core sampling product: accumulators of 128 rows per CTA x column tile x
 * pipeline stages (of 32 points unless stated).  Every CTA loads its own B tiles; two accumulators
 * share each loaded B stage. */
enum {
  RSRS_SAMPLE_TILE_DEFAULT = 0,  /* the library's choice (2 x 256 x 3 of 16 points)             */
  RSRS_SAMPLE_TILE_256x2 = 1,    /* one accumulator, 256 columns per CTA, two stages             */
  RSRS_SAMPLE_TILE_128x3 = 2,    /* one accumulator, 128 columns, three stages                   */
  RSRS_SAMPLE_TILE_192x2 = 3,    /* one accumulator, 192 columns, two stages                     */
  RSRS_SAMPLE_TILE_256x4_K16 = 4, /* one accumulator, 256 columns, four stages of 16 points      */
  RSRS_SAMPLE_TILE_192x5_K16 = 5, /* one accumulator, 192 columns, five stages of 16 points      */
  RSRS_SAMPLE_TILE_2x256x3_K16 = 6, /* two accumulators (256 rows), 256 columns, three stages of  */
                                    /* 16 points                                                  */
  RSRS_SAMPLE_TILE_2x192x4_K16 = 7  /* two accumulators, 192 columns, four stages of 16 points    */
};

/* Launch shapes of the kernels whose best shape depends on the problem and the device; all zero
 * selects the library's defaults.  Every value computes the same quantities (the shapes change at
 * most the grouping of floating-point sums: the sampling tiles not even that), so a tuned
 * configuration can be reused for any problem of its kind.  rsrs_autotune picks one by timing.
 * Not in the paper (a property of this GPU implementation). */
typedef struct {
  int32_t sample_tile;     /* RSRS_SAMPLE_TILE_*                                            */
  int32_t cpqr_cluster;    /* mixed path's cluster CPQR: CTAs per box, 0 = the fewest whose  */
                           /* distributed shared memory holds the sketch; 2, 4, 8 or 16     */
                           /* (never below that fewest)                                     */
  int32_t cpqr_threads;    /* threads per CTA of that CPQR: 0 = 1024; 256, 512 or 1024      */
  int32_t residual_split;  /* point-range splits of the float-float refinement residual:    */
                           /* 0 = enough CTAs for four per SM; 1..16                        */
  int32_t reserved[4];     /* zero                                                          */
} rsrs_tune_t;

typedef struct {
  int precision;          /* RSRS_PREC_*                                               */
  int p;                  /* oversampling; < 0 selects p = k (Sec. 5)                  */
  int proj_passes;        /* projection passes of the nullification, 1..4; 0 selects 2 */
  uint64_t seed;          /* key of the device Philox4x32-10 draws used when no test   */
                          /* matrices are given: entry (i, c) of Omega (Psi) is member */
                          /* (i*s+c) mod 2 of the Box-Muller pair from counter         */
                          /* ((i*s+c)/2, stream 0 (1)), two 53-bit uniforms per pair   */
  const double* omega_host; /* optional caller test matrices, row-major N x s in        */
  const double* psi_host;   /* ORIGINAL point order (point i's samples contiguous)      */
  const double* omega_dev;  /* same, in device memory (used when the host ones are NULL) */
  const double* psi_dev;
  int keep_sketches;      /* keep the final Y, Z, Omega, Psi on the device (tests)     */
  int profile;            /* record CUDA-event time per kernel class into rsrs_stats    */
  int sample_kernel;      /* mixed precision, built-in kernels: 1 FP32 SIMT, 2 (and the  */
                          /* default 0) 3xTF32 on the tensor cores (tcgen05, TMA);      */
                          /* FP64, one built-in-kernel problem: 3 = FP64-accurate       */
                          /* products by the Ozaki scheme on the bf16 tensor cores (the */
                          /* refinement residual's digit store, made by the build, 20 N^2 */
                          /* bytes; the FP64 SIMT product when it does not fit), 0 =    */
                          /* the FP64 SIMT product                                     */
  int mixed_cpqr;         /* mixed precision: 0 default = FP32 reflectors on the sketch  */
                          /* held in distributed shared memory (thread-block cluster of */
                          /* up to 16 CTAs), pivots chosen on FP64 residual norms, when */
                          /* the box fits; 1 = FP64 CPQR in global memory (FP64 always) */
  int mixed_gemm;         /* mixed precision: 0 default = Grams, their blocked Cholesky   */
                          /* factors and L^-T, least-squares right-hand sides, solves, */
                          /* projection updates, Lc and Uc as 3xTF32 tcgen05 products */
                          /* (X_RR^-1 by FP32 Gauss-Jordan);                           */
                          /* 1 = FP32 SIMT (Cholesky and substitution, FP64 X_RR LU)    */
  int use_graph;          /* 1: capture the build's launch sequence as one CUDA graph    */
                          /* kept with the factors, so rsrs_refactor can replay it;    */
                          /* needs device-drawn test matrices; no per-class timings   */
  int residual_fp64;      /* residual arithmetic of rsrs_refine / rsrs_residual /        */
                          /* rsrs_gmres with a built-in kernel, RSRS_RESIDUAL_*:       */
                          /* 0 default (Ozaki scheme when its slice store fits in     */
                          /* device memory, else float-float), 1 FP64, 2 float-float, */
                          /* 3 Ozaki scheme only (RSRS_E_NOMEM when it does not fit)  */
  rsrs_tune_t tune;       /* launch shapes (zero: defaults); kept with the factor       */
} rsrs_options;

typedef struct {
  int d;                  /* dimension of the points                                  */
  int depth;              /* deepest level L of the tree                              */
  int64_t n;              /* number of points                                         */
  int64_t n_boxes;        /* boxes in the tree                                        */
  int64_t n_leaves;
  int64_t n_compress;     /* boxes compressed by Algorithm 1 for this k               */
  int64_t n_groups;       /* (level, colour) groups = launches per step                */
  int64_t max_l;          /* largest |B_act| + |N_act| at processing time             */
  int64_t root_size;      /* |B_t|                                                    */
  int64_t s_req;          /* smallest admissible s: max(max_l + k + p, |B_t| + p)     */
  int64_t s_req_mixed;    /* smallest s for RSRS_PREC_MIXED: also keeps every box's   */
                          /* near-field Gram W W^T well conditioned in FP32 (mixed  */
                          /* builds with s below it return RSRS_E_UNDERSAMPLED)     */
} rsrs_tree_info_t;

/* Kernel classes of the build, for per-class timings and algorithmic FLOP counts. */
enum {
  RSRS_K_SAMPLE = 0, RSRS_K_LISTS, RSRS_K_GRAM, RSRS_K_CHOL, RSRS_K_GATHER, RSRS_K_PROJ_NT,
  RSRS_K_PROJ_SOLVE, RSRS_K_PROJ_ACC, RSRS_K_CPQR, RSRS_K_ID, RSRS_K_EF, RSRS_K_EXTRACT, RSRS_K_LU,
  RSRS_K_LU_RHS, RSRS_K_SCHUR, RSRS_K_ROOT, RSRS_NCLASS
};

typedef struct {
  int64_t n, s, k;
  int64_t n_boxes;        /* compressed boxes (factor blocks)                         */
  int64_t root_size;
  int64_t factor_bytes;   /* device bytes held by the factor                          */
  int64_t work_bytes;     /* peak device workspace of the build                       */
  double t_sample_ms, t_compress_ms, t_root_ms;  /* stream-event timings of the build */
  int64_t kernel_launches; /* kernels launched by the last build                     */
  double class_ms[RSRS_NCLASS];       /* CUDA-event time per class (opts.profile only)   */
  double class_gflop[RSRS_NCLASS];    /* algorithmic GFLOP per class (always filled)     */
  int64_t class_launches[RSRS_NCLASS];
  int64_t solve_bytes;    /* algorithmic bytes one solve reads from the factor, in the  */
                          /* solve's arithmetic (FP32 copies for a mixed factor): T    */
                          /* twice (both sweeps), Lc and Uc once each, X_RR^-1 and the */
                          /* root inverse once; right-hand-side traffic not counted    */
} rsrs_stats;

/* Name of a kernel class ("gram", "schur", ...). */
const char* rsrs_kernel_class_name(int cls);

/* Arithmetic of the residual product B - A X of iterative refinement (an addition to the paper,
 * which pairs the factor with GMRES, Sec. 5), for the built-in kernels:
 *   FP64        the kernel evaluated and multiplied in FP64 arithmetic;
 *   FLOAT_FLOAT the kernel and the products in float-float (48-bit) arithmetic on the FP32 pipe,
 *               about 1e-14 of sum_j |K_ij x_j|;
 *   OZAKI       the Ozaki scheme (Ozaki, Ogita, Oishi & Rump 2012) on the bf16 tensor cores: the
 *               matrix's rows (float-float values) and the columns of X split into ten base-2^7
 *               digits, every digit product exact, the sums exact in integers, about 2e-15 of
 *               sum_j |K_ij x_j|.  The digits of the matrix are made at the factor's first
 *               residual and kept with it (20 N^2 bytes of device memory; 86 GB at N = 65,536);
 *               rsrs_refactor discards them (they are made again at the next residual).
 * A callback operator's residual is the callback's (FP64). */
enum {
  RSRS_RESIDUAL_AUTO = 0,         /* OZAKI when its store fits next to 2 GiB + 5 % of the device's */
                                  /* memory, else FLOAT_FLOAT                                      */
  RSRS_RESIDUAL_FP64 = 1,
  RSRS_RESIDUAL_FLOAT_FLOAT = 2,
  RSRS_RESIDUAL_OZAKI = 3
};

typedef struct {
  int iterations;         /* corrections applied after the first solve                */
  double rel_residual;    /* final max over columns of ||b - A x|| / ||b||            */
  double history[64];     /* relative residual after each step                        */
  int64_t kernel_launches; /* kernels of this library the call launched (a matvec
                              callback's own launches are not counted)                */
  int32_t residual_kind;  /* RSRS_RESIDUAL_FP64, _FLOAT_FLOAT or _OZAKI: the arithmetic the
                             products with A used (FP64 for a callback)               */
} rsrs_refine_report;

/* ---- tree (Sec. 3: quad/octree, adjacency, 2:1 balance) --------------------
 * pts_host: n x d row-major doubles.  leaf_cap: at most leaf_cap points per
 * leaf.  d must be 2 or 3. */
rsrs_status rsrs_tree_build(const double* pts_host, int64_t n, int d, int leaf_cap,
                            rsrs_tree** out);
/* Sizes of Algorithm 1 on this tree for rank k and oversampling p (p < 0: p = k),
 * including the sample bound of Sec. 4.5 (s_req). */
rsrs_status rsrs_tree_info(const rsrs_tree* tree, int k, int p, rsrs_tree_info_t* out);
/* perm_host[t] = original index of the point at tree position t (n entries). */
rsrs_status rsrs_tree_perm(const rsrs_tree* tree, int64_t* perm_host);
/* Per-level schedule dump for tests: for every compressed box in processing
 * order, 6 int64 values (level, colour, morton key, b, n, first tree position).
 * rows_host must hold 6*n_compress values. */
rsrs_status rsrs_tree_schedule(const rsrs_tree* tree, int k, int p, int64_t* rows_host);
void rsrs_tree_free(rsrs_tree* tree);

/* ---- factorization (Algorithm 1) ----------------------------------------------
 * Draws Omega, Psi (or copies opts->omega_host/psi_host), samples Y, Z with the
 * operator, and runs Algorithm 1 on the device.  Returns RSRS_E_UNDERSAMPLED
 * (before any device work) when s < s_req. */
rsrs_status rsrs_build(const rsrs_tree* tree, const rsrs_operator* op, int k, int s,
                       const rsrs_options* opts, void* stream, rsrs_factor** out);

/* A 7-point variable-coefficient operator on an m x m x m cell grid, usable as the matvec callback
 * of an RSRS_OP_CALLBACK operator (fn = rsrs_stencil7_matvec, ctx = the object).  Cell-centred
 * finite volumes: (A u)_i = sum over the faces (i, j) between neighbouring cells of
 * beta_ij (u_i - u_j), beta_ij = 2 b_i b_j / (b_i + b_j), plus 2 b_i u_i for every boundary face of
 * cell i (Dirichlet wall half a cell away); no h^-2 scaling.  Symmetric positive definite.  Not
 * part of the paper's method: it stands in for the paper's PDE-derived operators (Sec. 5, Exp. 3).
 * coef_host: m^3 positive finite coefficients b, cells ordered x fastest, then y, then z (copied;
 * the face coefficients are formed in FP64).  RSRS_E_INVAL on bad arguments, RSRS_E_NOMEM when the
 * device copy fails.  The matvec returns 0, or non-zero (which rsrs_build reports as
 * RSRS_E_CALLBACK) on a size mismatch or a launch error; it enqueues on `stream` only. */
typedef struct rsrs_stencil7 rsrs_stencil7;
rsrs_status rsrs_stencil7_create(const double* coef_host, int m, rsrs_stencil7** out);
int rsrs_stencil7_matvec(void* ctx, int adjoint, int64_t n, int32_t ncols, const double* X_dev, int64_t ldx,
                         double* Y_dev, int64_t ldy, void* stream);
void rsrs_stencil7_free(rsrs_stencil7* s);

/* Several independent problems in one set of launches (same k, s, options): the boxes of all
 * problems at the same height above their deepest level and of the same colour share each
 * launch, and the roots are extracted together.  out receives nprob factors that share device
 * storage (freed with the last of them); each is used like a factor from rsrs_build.  Test
 * matrices are drawn on the device (problem p uses key opts->seed + p); caller test matrices are
 * refused with RSRS_E_INVAL. */
rsrs_status rsrs_build_batched(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k, int s,
                               const rsrs_options* opts, void* stream, rsrs_factor** out);

typedef struct {
  int candidates;         /* builds (and residual products) timed                      */
  int from_cache;         /* 1: the configuration came from the cache file, nothing timed */
  double default_ms;      /* device time of the tuned kernel classes with all-zero tune */
  double tuned_ms;        /* the same with the configuration returned                  */
} rsrs_tune_report;

/* Autotuner (not in the paper: picks launch shapes of this implementation).  Builds the given
 * problem(s) (arguments as rsrs_build_batched; opts->tune is the starting point) once per
 * candidate value of one rsrs_tune_t field at a time, the others held at the best found so far,
 * and keeps the value with the smallest device time of the kernel class the field governs (best
 * of `reps` builds, CUDA events): sample_tile on the sampling product (mixed precision, built-in
 * kernels), cpqr_cluster and cpqr_threads on the CPQR (mixed precision, cluster CPQR), and
 * residual_split on one float-float refinement residual of 16 columns (built-in kernels).  Fields
 * that do not apply stay 0.  cache_path (optional): a text file with one line per tuned
 * configuration, keyed by the device name, operator kind, number of problems, total N, d, k, s
 * and precision; a matching line is returned without timing (report->from_cache = 1), otherwise
 * the result is appended.  Build errors of a candidate are returned as from rsrs_build; no factor
 * is kept.  out receives the configuration; report (optional) the counts and times. */
rsrs_status rsrs_autotune(int nprob, const rsrs_tree* const* trees, const rsrs_operator* ops, int k, int s,
                          const rsrs_options* opts, int reps, const char* cache_path, void* stream,
                          rsrs_tune_t* out, rsrs_tune_report* report);

/* Rebuilds in place every factor of the build that f belongs to (all problems of a batched
 * build) from new test matrices drawn with key `seed` (problem p: seed + p), by replaying the
 * launch sequence captured when it was built with opts.use_graph = 1: same trees, operators, k,
 * s and options, one graph launch instead of thousands of kernel launches.  A callback operator's
 * work was captured at build time, so its matvec is not called again (its kernels rerun on
 * whatever device data they read).  The factors must not be in use meanwhile.  Per-class timings
 * are not recorded.  RSRS_E_INVAL when the build did not use use_graph; device-detected
 * conditions as for rsrs_build. */
rsrs_status rsrs_refactor(rsrs_factor* f, uint64_t seed, void* stream);

/* F <- A_approx^-1 F (eq. Ainvfact), or its adjoint; F_dev column-major N x nrhs.  A
 * mixed-precision factor (RSRS_PREC_MIXED) sweeps in FP32 arithmetic on FP32 copies of its blocks
 * (made at the end of its build): its solves serve as the approximate inverse of FP64 refinement
 * and GMRES, whose FP64-accurate residuals set the final accuracy; an FP64 factor sweeps in FP64.
 * Each sweep direction runs as one cooperative launch of persistent CTAs over the factor's
 * (level, colour) groups with a bounded grid-wide barrier between dependent steps (the root's
 * dense step in between), or, where a cooperative launch is refused, as one launch per group and
 * product; both compute the same values.  Asynchronous on `stream` (like rsrs_apply): the call's
 * scratch (N x nrhs doubles, as many floats for a mixed factor, four barrier words) comes from
 * CUDA's stream-ordered allocator and is released in stream order, so it neither synchronises the
 * device nor waits for the stream; F_dev holds the result once the stream reaches it.  Concurrent
 * calls on one factor are allowed (the factor is only read). */
rsrs_status rsrs_solve(const rsrs_factor* f, double* F_dev, int64_t ldf, int32_t nrhs,
                       int adjoint, void* stream);
/* rsrs_solve_noalloc: rsrs_solve for callers that must not allocate device memory.  The paper
 * has no counterpart: it is a deployment variant of rsrs_solve, computing the same result with the
 * same kernels.
 *
 * Who needs it: rsrs_solve takes an N x nrhs staging block from CUDA's stream-ordered allocator
 * on every call, whose pool grows from free device memory.  A caller whose device memory is all
 * reserved by another allocator (a caching allocator such as PyTorch's holds freed blocks instead
 * of returning them, so an allocation can fail while memory is nominally free) cannot make that
 * call succeed.  This entry point stages the block in library-wide static device buffers instead
 * (one of RSRS_NOALLOC_MAX_ELEMS doubles, one of as many floats for a mixed-precision factor's FP32
 * sweeps, and four words for the fused sweeps' grid barrier: 12 MiB held on every device that
 * loads the library) and calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Limit: N * nrhs <= RSRS_NOALLOC_MAX_ELEMS (2^20, e.g. N = 65,536 with 16 right-hand sides);
 * larger blocks return RSRS_E_INVAL before any launch.  Nothing in the buffers needs to start at
 * zero: the first kernels write every element the sweeps read.
 *
 * The buffers are shared by all calls on a device: calls whose execution overlaps (on different
 * streams, or from host threads without ordering between them) race on it and give wrong
 * results; order them on one stream.  The call enqueues its kernels on `stream` and returns
 * without synchronising; F holds the solution once the stream has reached that point.  The first
 * call on each device resolves the buffers' addresses (cudaGetSymbolAddress with that device
 * current); make that first call before any stream capture.  Arguments, layout and other errors
 * as rsrs_solve. */
#define RSRS_NOALLOC_MAX_ELEMS (1 << 20)
rsrs_status rsrs_solve_noalloc(const rsrs_factor* f, double* F, int64_t ldf, int32_t nrhs, int adjoint,
                               void* stream);

/* F <- A_approx F (eq. Afact), or its adjoint; asynchronous on `stream`, scratch as for rsrs_solve. */
rsrs_status rsrs_apply(const rsrs_factor* f, double* F_dev, int64_t ldf, int32_t nrhs,
                       int adjoint, void* stream);
/* R = B - A X for the operator the factor was built from, in the refinement's residual
 * arithmetic (RSRS_RESIDUAL_*, opts->residual_fp64; FP64 for a callback); B_dev, X_dev, R_dev
 * column-major N x nrhs with leading dimension ld (R may not alias B or X).  The residual of
 * iterative refinement, which the paper does not use (it pairs the factor with GMRES, Sec. 5);
 * nrhs <= 4096.  RSRS_E_NONFINITE when two points coincide (the kernel is unbounded). */
rsrs_status rsrs_residual(const rsrs_factor* f, const double* B_dev, const double* X_dev, double* R_dev,
                          int64_t ld, int32_t nrhs, void* stream);
/* Iterative refinement to FP64 accuracy (an addition to the paper's method, with the factor as the
 * approximate inverse): X = A_approx^-1 B, then X += A_approx^-1 (B - A X) until
 * max_j ||B_j - A X_j|| / ||B_j|| <= rtol or maxit corrections.  The residual is computed as
 * rsrs_residual computes it (RSRS_RESIDUAL_*; FP64 through the callback for a callback operator).
 * B_dev, X_dev column-major N x nrhs with leading dimension ld, nrhs <= 64; X's input is ignored.
 * out (may be null): corrections, final relative residual, its history, kernels launched, the
 * residual arithmetic used.  RSRS_E_NOT_CONVERGED (out still filled) when rtol is not reached;
 * RSRS_E_NONFINITE for a non-finite residual. */
rsrs_status rsrs_refine(const rsrs_factor* f, const double* B_dev, double* X_dev, int64_t ld,
                        int32_t nrhs, double rtol, int maxit, void* stream,
                        rsrs_refine_report* out);
/* Restarted GMRES(restart) (Saad and Schultz 1986) on A X = B with the factor as right
 * preconditioner, A (A_approx)^-1 Y = B, X = (A_approx)^-1 Y: the Krylov method Sec. 5 pairs
 * with the factorization, against iterative refinement.  Every column is its own GMRES run (its
 * own Arnoldi basis, classical Gram-Schmidt applied twice, Givens rotations); the columns share
 * the launches.  Products with A in the refinement's residual arithmetic (RSRS_RESIDUAL_*, the
 * callback for a callback operator); X starts at 0 (its input
 * is ignored).  Stops when the true residual max_j ||B_j - A X_j|| / ||B_j|| <= rtol (checked
 * when the Arnoldi estimate reaches rtol, at each restart and at the end) or after maxit
 * iterations in total.  out: iterations = Krylov iterations (preconditioner solves),
 * history = the initial relative residual, then each iteration's estimate (max over columns)
 * and each restart's true residual, rel_residual = the last true residual.  restart 1..64,
 * nrhs <= 64; device memory (2 restart + 5) N nrhs doubles.  RSRS_E_NOT_CONVERGED after maxit. */
rsrs_status rsrs_gmres(const rsrs_factor* f, const double* B_dev, double* X_dev, int64_t ld, int32_t nrhs,
                       double rtol, int restart, int maxit, void* stream, rsrs_refine_report* out);
/* Y = A X with the factor's operator in FP64 (the residual product of rsrs_refine). */
rsrs_status rsrs_matvec(const rsrs_factor* f, const double* X_dev, double* Y_dev, int64_t ld,
                        int32_t nrhs, void* stream);

rsrs_status rsrs_factor_stats(const rsrs_factor* f, rsrs_stats* out);

/* Host copy of one compressed box's factor block, for parity tests.  Index
 * lists are ORIGINAL point numbers; matrices are row-major.  Call with NULL
 * buffers to get the sizes (b, n, kp, r) first. */
typedef struct {
  int32_t level, colour;
  int64_t b, n, kp, r;
  int64_t* S;       /* kp  skeletons, pivot order                               */
  int64_t* R;       /* r   redundant, tree order                                */
  int64_t* N;       /* n   active neighbours, tree order                        */
  double* T;        /* kp x r                                                   */
  double* XRR;      /* r x r (as extracted, before factorization)               */
  double* LcS;      /* kp x r   X_SR X_RR^-1                                    */
  double* LcN;      /* n  x r   X_NR X_RR^-1                                    */
  double* UcS;      /* r  x kp  X_RR^-1 X_RS                                    */
  double* UcN;      /* r  x n   X_RR^-1 X_RN                                    */
} rsrs_box_view;
rsrs_status rsrs_factor_box(const rsrs_factor* f, int64_t i, rsrs_box_view* v);
/* Root block: indices (original numbering, tree order) and the dense r x r
 * extracted matrix, row-major.  Either buffer may be NULL. */
rsrs_status rsrs_factor_root(const rsrs_factor* f, int64_t* idx_host, double* A_host,
                             int64_t* size_out);
/* Final sketches (requires keep_sketches): row-major N x s, original order. */
rsrs_status rsrs_factor_sketches(const rsrs_factor* f, double* Y_host, double* Z_host,
                                 double* Om_host, double* Ps_host);

void rsrs_factor_free(rsrs_factor* f);
const char* rsrs_status_string(rsrs_status st);
/* Message of the last failed call on this thread (empty string if none). */
const char* rsrs_last_error(void);

/* Failure-detection self-test (no counterpart in the paper).  Every wait of the tensor-core kernels
 * on an mbarrier is bounded: after a fixed number of polls it records a timeout in the device
 * status word, the kernel releases what it holds and returns, and the call reports
 * RSRS_E_TIMEOUT with the context still usable.  This launches one CTA that initialises an
 * mbarrier expecting one arrival, makes that arrival only when arrive = 1, and waits for it
 * through the same bounded wait with at most `polls` polls (1..2^26).  Returns RSRS_E_TIMEOUT
 * when the wait expired (always, for arrive = 0), RSRS_OK when it completed, RSRS_E_INVAL for
 * arguments out of range.  Synchronises `stream`; allocates and frees one device int. */
rsrs_status rsrs_wait_selftest(int64_t polls, int arrive, void* stream);

/* The same for the grid-wide barrier of the fused solve sweeps (no counterpart in the paper): a
 * cooperative launch of two CTAs meets at the barrier, CTA 1 only when arrive = 1; CTA 0 waits
 * with at most `polls` polls (1..2^26).  RSRS_E_TIMEOUT when the wait expired (always, for
 * arrive = 0), RSRS_OK when both arrived, RSRS_E_CUDA when the cooperative launch was refused,
 * RSRS_E_INVAL for arguments out of range.  Synchronises `stream`; allocates four device words. */
rsrs_status rsrs_grid_wait_selftest(int64_t polls, int arrive, void* stream);

/* Self-test of the FP64 <-> FP32 conversions the mixed path's sketch updates run on the integer
 * pipes (no counterpart in the paper; IEEE 754 binary64/binary32 layouts).  For the n device
 * doubles x: f[i] = x[i] rounded to binary32 (to nearest, ties to even), g[i] = f[i] widened to
 * binary64; both device arrays of n.  They must equal the hardware conversions bit for bit
 * (NaN payloads aside).  Asynchronous on `stream`; RSRS_E_INVAL for a null array with n > 0. */
rsrs_status rsrs_convert_selftest(const double* x, int64_t n, float* f, double* g, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RSRS_H */
