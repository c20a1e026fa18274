/*
 * bbfmm.h -- C ABI of the GB300 black-box FMM library (libbbfmm.so).
 *
 * The library evaluates phi = K sigma, phi_i = sum_j K(x_i, x_j) sigma_j
 * (Sec. 1, Eq. summation / Eq. matvec of arXiv 1903.02153), targets = sources,
 * with the black-box FMM of Sec. 2: a uniform octree (Sec. 2.1, Def. 2.1),
 * Chebyshev interpolation (Sec. 2.2, Def. 2.2, Eq. low-rank-form), the four
 * stages P2M/M2M, M2L, L2L/L2P, P2P (Sec. 2.3), SVD-compressed M2L operators
 * (Sec. 2.5 "Fast M2L translation"), leaf-level operators scaled per level for
 * homogeneous kernels (Sec. 2.5 "Homogeneous kernel"), and several weight
 * vectors at once (Sec. 2.5 "Multiple right-hand-sides").  Every stage of a
 * matvec runs in the library's own CUDA kernels for sm_103a.
 *
 * Conventions shared by all entry points:
 *   - Return value: BBFMM_OK (0) or a negative status below.  No entry point
 *     throws or aborts; bbfmm_last_error() gives a message for the calling
 *     thread's last failure.
 *   - Pointers may be host or device memory where stated; the library asks the
 *     CUDA runtime which one it got.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; an entry point returns before the GPU finishes unless it
 *     says otherwise.
 *   - Arrays of several right-hand sides are column-major with leading
 *     dimension n (column c of sigma starts at sigma + c*n).
 *   - sigma and phi are indexed in the caller's original point order.
 */
#ifndef BBFMM_H
#define BBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BBFMM_OK 0
#define BBFMM_EINVAL -1    /* invalid argument (sizes, NaN coordinates, null pointers) */
#define BBFMM_ENOMEM -2    /* device or host allocation failed; nothing leaked */
#define BBFMM_ECUDA -3     /* a CUDA runtime / driver call failed */
#define BBFMM_ETIMEOUT -4  /* a device-side wait ran out of iterations (status word) */
#define BBFMM_EBUSY -5     /* the plan is in use by another thread */
#define BBFMM_EINTERNAL -6 /* a device-side consistency check failed */

/* kernels K(x, y) = k(|x - y|) (Sec. 1 and Sec. 4 name 1/r and exp(-r)) */
#define BBFMM_K_INV_R 1        /* 1/r, 0 at r = 0; homogeneous of degree -1 */
#define BBFMM_K_INV_R2 2       /* 1/r^2, 0 at r = 0; homogeneous of degree -2 */
#define BBFMM_K_EXP 3          /* exp(-r/ell) (exponential covariance) */
#define BBFMM_K_GAUSS 4        /* exp(-(r/ell)^2) */
#define BBFMM_K_TEST_POLY 100  /* 1 + d1 - 2 d2 d3 + 3 d1^2 d2, d = x - y: exact for p >= 3 */
#define BBFMM_K_TEST_CONST 101 /* 1 */
#define BBFMM_K_USER_FIRST 1000 /* ids of kernels registered by bbfmm_kernel_register */

/* interpolation nodes and the M2L that goes with them (Sec. 2.2 node sets,
 * Sec. 2.5 "Fast M2L translation") */
#define BBFMM_INTERP_CHEBYSHEV 0 /* Chebyshev nodes, SVD-compressed M2L (default) */
#define BBFMM_INTERP_UNIFORM 1   /* equally spaced nodes (end points included); the
                                    block-Toeplitz M2L applied in the Fourier domain:
                                    per box a (2p-1)^3 DFT of its coefficients, per
                                    frequency a 189-term sum over the interaction list,
                                    an inverse DFT per box; FP32; no compression */

/* near-field evaluation order (Sec. 2.5, symmetry of the kernel) */
#define BBFMM_NEAR_AUTO 0      /* where SYMMETRIC applies, the faster order: measured
                                  by the autotuner (opts.autotune), else SYMMETRIC
                                  when the near-field pairs per point / 27 (the
                                  occupancy of the leaves the work meets) is 16 to
                                  48; otherwise ORDERED (default) */
#define BBFMM_NEAR_ORDERED 1   /* every target leaf evaluates all its neighbour pairs */
#define BBFMM_NEAR_SYMMETRIC 2 /* symmetric kernel, targets = sources, one right-hand
                                  side: each pair of neighbour leaves is evaluated once
                                  and used both ways; otherwise as ORDERED */

/* arithmetic of the M2L stage (every other stage computes in FP32) */
#define BBFMM_PREC_FP32 0   /* FP32 FMA on the CUDA cores */
#define BBFMM_PREC_TF32 1   /* tensor cores, one TF32 pass, FP32 accumulation */
#define BBFMM_PREC_TF32X3 2 /* tensor cores, 3-pass split TF32 (hi*hi + hi*lo + lo*hi), ~21 bits */
#define BBFMM_PREC_BF16X3 3 /* tensor cores, 3-pass split BF16 (hi*hi + hi*lo + lo*hi), ~16 bits */
#define BBFMM_PREC_FP16X3 4 /* tensor cores, 3-pass split FP16 with power-of-two scaling per
                               level (hi*hi + hi*lo + lo*hi), ~21 bits */

typedef struct bbfmm_plan_s *bbfmm_plan_t; /* opaque; owned by the library */

typedef struct {
    double ell;        /* kernel length scale for BBFMM_K_EXP / _GAUSS (default 1) */
    double svd_eps;    /* keep singular values >= svd_eps * sigma_max of the M2L
                          operators (Sec. 2.5 "SVD truncation error"); default 1e-7;
                          0 disables compression (rank = p^3) */
    int precision;     /* BBFMM_PREC_* (default BBFMM_PREC_FP32) */
    int domain_given;  /* 1: use lo/side below; 0: bounding cube of the points */
    double lo[3];      /* lower corner of the cubical domain */
    double side;       /* side length of the domain (> 0) */
    int max_nrhs;      /* largest nrhs a matvec on this plan may use (default 1) */
    int split_accumulate; /* 3-pass tensor-core forms: 1 (default) issues each K
                             chunk's correction products hi*lo + lo*hi before its
                             hi*hi products, so only the hi*hi additions round at
                             the scale of the result; 0 issues hi*hi first */
    int use_graph;     /* 1 (default): the first matvec with a given nrhs captures
                          the whole launch sequence into a CUDA graph, later ones
                          replay it; 0: launch the kernels one by one */
    int keep_coefficients; /* 1: every matvec also stores the multipole (M) and
                              local (F) coefficients of every level for
                              bbfmm_get_coefficients; 0 (default): they stay in
                              the passes' on-chip memory and are not allocated */
    int interp;        /* BBFMM_INTERP_* (default CHEBYSHEV); UNIFORM takes
                          precision = BBFMM_PREC_FP32 and ignores svd_eps */
    int near_mode;     /* BBFMM_NEAR_* (default AUTO).  The symmetric form holds 13
                          floats per point more (the two-way column sums); both
                          orders are deterministic, and they differ by FP32 rounding */
    int close_refine;  /* 1 (default): near-field pairs closer than 1/64 of a leaf
                          box side enter the result as if evaluated in FP64 (Sec. 2.3
                          near field; the FP32 leaf-local coordinates round x - y by up
                          to ~1e-7 box sides, which the singular kernels amplify on
                          close pairs).  The plan lists such pairs once with FP64
                          correction coefficients (a few bytes per pair); each matvec
                          adds them in one small launch after the near field.
                          0: the FP32 values only */
    int autotune;      /* 1 (default): the first matvec with a given nrhs measures
                          the launch choices of bbfmm_tuning (bbfmm_autotune) and
                          keeps the fastest; the choice is cached per process for
                          plans of the same shape.  0: the defaults of
                          bbfmm_tuning, and near_mode AUTO by leaf occupancy */
} bbfmm_opts;

typedef struct {
    int64_t n;          /* points (the sources of a bbfmm_plan_targets plan) */
    int depth;          /* tree depth D: 8^D leaves, M2L on levels 2..D */
    int order;          /* Chebyshev nodes per axis p */
    int rank;           /* rank r of the compressed M2L operators */
    int kernel;         /* BBFMM_K_* */
    int precision;      /* BBFMM_PREC_* */
    int max_nrhs;
    double lo[3], side; /* domain actually used */
    int64_t device_bytes; /* device memory held by the plan */
    int64_t nonempty_leaves;  /* leaves holding sources */
    int64_t max_leaf_points;  /* most sources in one leaf */
    int64_t p2p_pairs;  /* near-field kernel evaluations per right-hand side */
    int64_t m2l_pairs;  /* M2L translations per right-hand side (dense grid) */
    int64_t n_targets;  /* targets (= n unless built by bbfmm_plan_targets) */
    int near_symmetric; /* 1: one-RHS matvecs evaluate each neighbour leaf pair once */
    int close_pairs;    /* (target, source) near-field pairs listed for FP64
                           correction (opts.close_refine) */
    int64_t p2p_evals;  /* near-field kernel evaluations of a one-RHS matvec:
                           p2p_pairs, or about half of it with the symmetric form */
    int reserved[2];
} bbfmm_info;

/*
 * Launch choices of a plan, per nrhs (they change how the work is cut into
 * launches, never what is computed; results of different choices differ by
 * FP32 rounding only).  Sec. 2.5 "Multiple right-hand-sides": the work of a
 * launch grows with nrhs, and the fastest choice moves with it.
 */
typedef struct {
    int near_mode;  /* BBFMM_NEAR_ORDERED or BBFMM_NEAR_SYMMETRIC: the near-field
                       order of one-RHS matvecs (several-RHS ones are ordered) */
    int m2l_tile;   /* targets per tile of the tensor-core M2L: 128, or 256 with
                       BBFMM_PREC_FP16X3 / BF16X3 (the default there) */
    int m2l_stages; /* pipeline stages of the tensor-core M2L: 0 = as many as fit
                       in shared memory (default), else 2 up to that */
    int measured;   /* bbfmm_get_tuning: 1 if chosen by a measured sweep (or its
                       cache); ignored by bbfmm_set_tuning */
    int near_box;   /* ORDERED one-RHS near field: 1 = a work item per level-(D-1)
                       box (its 8 leaves' targets against the 4x4x4 leaves around
                       it, staged once), for leaves of a few points; 0 = a work
                       item per leaf (default).  Needs depth >= 1 */
    int leaf_gemm;  /* 1: the leaf level's compression M~ = V^T M runs as a
                       tensor-core GEMM (3 x TF32) after the upward pass (the
                       default where the plan has it: Chebyshev nodes, depth >= 2,
                       V fits in shared memory, e.g. p <= 5); 0: inside the
                       upward pass on the CUDA cores */
    int reserved[2];
} bbfmm_tuning;

/*
 * bbfmm_kernel_register: a kernel function supplied by the caller (the
 * black-box interface: the method needs only evaluations of K, Sec. 1 and
 * Sec. 3).  source is CUDA C that defines
 *     __device__ double bbfmm_kernel_f64(double d0, double d1, double d2);
 *     __device__ float  bbfmm_kernel_f32(float d0, float d1, float d2);
 * K(x, y) = k(d), d = x - y in the caller's units; both must give the value
 * wanted at d = 0 (the self and duplicate-point terms of the near field).
 * The FP64 function fills the operator tables, the FP32 one runs in the near
 * field.  The source is compiled at once with NVRTC for sm_103a.
 *   homogeneity: m with k(a d) = a^m k(d) for all a > 0 (one operator set for
 *                every level, scaled), or 0 (operators per level); -8..8.
 *   symmetric:   1 if k(-d) = k(d): one Gram matrix in the SVD, and the
 *                symmetric near field (BBFMM_NEAR_SYMMETRIC / AUTO) may use
 *                each kernel value for both points of a pair; else 0.  A
 *                kernel registered symmetric that is not gives wrong results.
 *   kernel_id:   receives an id >= BBFMM_K_USER_FIRST, usable as kernel_id
 *                in bbfmm_plan and bbfmm_plan_targets (opts.ell is unused
 *                for it).  Registrations last until the process exits.
 * Errors: EINVAL (NULL, homogeneity; a compile error, with the NVRTC log in
 * bbfmm_last_error), ECUDA (no device, NVRTC not found, load failure).
 */
int bbfmm_kernel_register(const char *source, int homogeneity, int symmetric, int *kernel_id);

/* Fill *opts with the defaults listed above. */
void bbfmm_default_opts(bbfmm_opts *opts);

/*
 * bbfmm_plan: build the tree and the operators for a point set (the
 * H2_3D_Tree constructor + buildFMMTree + FMMDistribute of Sec. 3).
 *   points:     n x 3 row-major FP64 coordinates, host or device; copied.
 *   n:          1 <= n < 2^31.
 *   kernel_id:  BBFMM_K_*.
 *   cheb_order: p, Chebyshev nodes per axis (Sec. 2.2), 2..10.
 *   depth:      D, 0..8; leaves are the 8^D boxes of level D.
 *   opts:       NULL = defaults.
 *   stream:     the plan's device work (tree build, uploads) runs on it; the
 *               call synchronizes the stream before returning.
 *   out:        receives the plan.
 * Errors: EINVAL (bad sizes, NaN/inf coordinates, points outside a given
 * domain by more than rounding), ENOMEM (device memory; partial allocations
 * are released), ECUDA.
 */
int bbfmm_plan(const double *points, int64_t n, int kernel_id, int cheb_order, int depth,
               const bbfmm_opts *opts, void *stream, bbfmm_plan_t *out);

/*
 * bbfmm_plan_targets: a plan whose targets x_i are a point set of their own,
 * apart from the sources y_j (Sec. 1: f(x_i) = sum_j K(x_i, y_j) sigma_j
 * with x and y different sets).  Both sets are binned into the one tree of
 * the domain (given in opts, else the bounding cube of both sets); the upward
 * pass runs over the sources, the downward pass and the near field over the
 * targets, and the M2L visits the target boxes that hold targets.  A target
 * at distance 0 from a source follows the r = 0 convention of the kernel.
 *   sources: ns x 3 row-major FP64, host or device; copied.  1 <= ns < 2^31.
 *   targets: nt x 3 row-major FP64, host or device; copied.  1 <= nt < 2^31.
 *   other arguments and errors as for bbfmm_plan.
 * bbfmm_matvec on such a plan reads sigma as ns x nrhs and writes phi as
 * nt x nrhs; bbfmm_get_leaf_cells reports the sources; bbfmm_rand_eig
 * rejects it (EINVAL).
 */
int bbfmm_plan_targets(const double *sources, int64_t ns, const double *targets, int64_t nt, int kernel_id,
                       int cheb_order, int depth, const bbfmm_opts *opts, void *stream, bbfmm_plan_t *out);

/*
 * bbfmm_matvec: phi = K_hat sigma (Sec. 2.3, all four stages).
 *   sigma: n x nrhs column-major FP32 (n sources), host or device; read only.
 *   phi:   nt x nrhs column-major FP32 (nt targets; nt = n unless the plan
 *          came from bbfmm_plan_targets), host or device; overwritten.
 *   nrhs:  1..opts.max_nrhs of the plan.
 * Device buffers: the call only enqueues work on `stream`.  Host buffers: the
 * call copies sigma in and phi out through the plan's device buffers on
 * `stream` and synchronizes it before returning.
 * A plan runs one matvec at a time: concurrent calls on one plan from several
 * threads return EBUSY; calls on one plan on different streams must be ordered
 * by the caller.  Errors: EINVAL, EBUSY, ECUDA.
 */
int bbfmm_matvec(bbfmm_plan_t plan, const float *sigma, float *phi, int nrhs, void *stream);

/* Release a plan (NULL is a no-op).  Synchronizes the device first. */
int bbfmm_destroy(bbfmm_plan_t plan);

/* Message for the calling thread's last failing call ("" if none). */
const char *bbfmm_last_error(void);

/* Sizes and counts of a plan. */
int bbfmm_plan_info(bbfmm_plan_t plan, bbfmm_info *info);

/*
 * bbfmm_rand_eig: the k largest eigenvalues (and eigenvectors) of the kernel
 * matrix K of a plan (K_ij = K(x_i, x_j), symmetric kernels), by the
 * randomized range finder and Rayleigh-Ritz step of the randomized PCA used
 * in Sec. 4.3 (two batched matvecs with m right-hand sides, plus `power`
 * subspace iterations): Y = K Omega; Q = orth(Y); B = Q^T K Q = V L V^T;
 * evals = the k largest of L, evecs = Q V.  The matvecs are bbfmm_matvec;
 * the tall-skinny products run in the library's kernels (FP32 products,
 * FP64 sums), the m x m eigenproblems on the host in FP64.
 *   omega:  device, n x m column-major FP32, the caller's random test block
 *           (e.g. standard normal), caller's point order; read only.
 *   m:      columns of omega, k <= m <= opts.max_nrhs of the plan.
 *   k:      eigenpairs wanted.
 *   power:  subspace iterations, 0..8 (0 = the plain range finder).
 *   evals:  host, k doubles, decreasing; 0 past the rank of K Omega.
 *   evecs:  device n x k column-major FP32 (caller's point order), or NULL.
 * Allocates 2 n m floats of scratch for the call; synchronizes the stream.
 * Errors: EINVAL (ranges, NULL, host pointers, K Omega = 0), ENOMEM, ECUDA,
 * EBUSY.
 */
int bbfmm_rand_eig(bbfmm_plan_t plan, const float *omega, int m, int k, int power, double *evals,
                   float *evecs, void *stream);

/*
 * bbfmm_get_coefficients: copy the coefficients of the last matvec at one
 * level to host memory, for stage-by-stage checks.
 *   which: 0 = multipole M (Sec. 2.3 upward pass), 1 = local F after the
 *          downward pass at that level (Sec. 2.3 items 2-3).
 *   level: 2..D.
 *   out:   host, 8^level x nrhs x p^3 FP32, boxes in lexicographic order
 *          (a + 2^l (b + 2^l c)), node index i1 + p i2 + p^2 i3.
 * Needs a plan built with opts.keep_coefficients = 1.  Synchronizes the
 * device.  Errors: EINVAL (bad arguments, or coefficients not kept).
 */
int bbfmm_get_coefficients(bbfmm_plan_t plan, int which, int level, int nrhs, float *out);

/*
 * bbfmm_get_leaf_cells: the leaf cell (a, b, c) the plan assigned to each
 * point, in the caller's point order (FMMDistribute, Sec. 3).
 *   out: host, n x 3 int32.  Synchronizes the device.
 */
int bbfmm_get_leaf_cells(bbfmm_plan_t plan, int32_t *out);

/*
 * bbfmm_stage_times: device milliseconds of each stage of the last matvec,
 * measured with CUDA events on the matvec's streams when the plan was built
 * with timing on (see bbfmm_set_timing).  With timing on, the near field
 * starts after the far field instead of beside it, so each stage's time is
 * that stage alone (and the whole matvec is their sum).  out[0..7] = gather, upward (P2M +
 * M2M + compress), M2L, downward (decompress + L2L + L2P, one launch), L2P
 * (0: part of the downward launch), P2P, combine, whole matvec.
 * Synchronizes the device.
 */
int bbfmm_stage_times(bbfmm_plan_t plan, float *out);

/*
 * bbfmm_get_tuning: the launch choices matvecs with nrhs right-hand sides
 * use (or will use: the defaults, before the first such matvec of a plan with
 * opts.autotune).  bbfmm_set_tuning: use these instead (EINVAL when the plan
 * cannot run them: SYMMETRIC without a symmetric kernel and one point set, or
 * with nrhs > 1, or when the plan was built with near_mode ORDERED, or without
 * autotune and AUTO chose ORDERED; a tile size the precision does not have;
 * more stages than fit).  Setting drops the matvec graph of that nrhs; the
 * call synchronizes the device.  Errors: EINVAL, EBUSY.
 */
int bbfmm_get_tuning(bbfmm_plan_t plan, int nrhs, bbfmm_tuning *out);
int bbfmm_set_tuning(bbfmm_plan_t plan, int nrhs, const bbfmm_tuning *tuning);

/*
 * bbfmm_autotune: measure the launch choices for nrhs now and keep the
 * fastest (also refreshing the process-wide cache).  Candidates: both
 * near-field orders (one RHS, near_mode AUTO, symmetric kernel, one point
 * set), every M2L tile size of the precision, every M2L pipeline depth that
 * fits.  Each runs 1 + 3 matvecs with zero weights in the plan's own buffers
 * (allocating 4 (n + nt) max_nrhs bytes of staging on first use); the fastest
 * mean device time wins.  Synchronizes the device and `stream`.
 * Errors: EINVAL, EBUSY, ENOMEM, ECUDA.
 */
int bbfmm_autotune(bbfmm_plan_t plan, int nrhs, void *stream);

/*
 * bbfmm_matvec_launches: the kernels one matvec with nrhs right-hand sides
 * launches, counted as the kernel nodes of the CUDA graph that the plan
 * captured for that nrhs (its first matvec with opts.use_graph and timing
 * off).  The count follows the tuning in force when the graph was captured;
 * bbfmm_set_tuning drops the graph.
 *   launches: receives the count.
 * Errors: EINVAL (NULL plan or launches, nrhs out of range, no graph captured
 * for nrhs yet).
 */
int bbfmm_matvec_launches(bbfmm_plan_t plan, int nrhs, int *launches);

/* Turn per-stage event timing on (1) or off (0) for later matvecs. */
int bbfmm_set_timing(bbfmm_plan_t plan, int on);

/*
 * bbfmm_status: synchronize the device, read and clear the plan's device
 * status word.  Kernels that wait on barriers give up after a bounded number
 * of cycles and record it there instead of hanging.
 *   word: optional; receives the raw bits (1 = bounds check, 2 = wait timeout).
 * Returns BBFMM_OK, BBFMM_ETIMEOUT or BBFMM_EINTERNAL.
 */
int bbfmm_status(bbfmm_plan_t plan, int *word);

/*
 * bbfmm_sort_points_static: the tree build that bbfmm_plan performs (leaf
 * binning, stable sort by the Morton index of the leaf, leaf offsets), written
 * to caller buffers and allocating nothing.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc when they build a tree,
 * e.g. code working inside a device-memory budget that another runtime has
 * already reserved, or on a path where a synchronous allocation would stall
 * other work on the GPU.
 *   points:   device, n x 3 row-major FP64 (host pointers are rejected).
 *   n:        1 <= n <= 1,048,576 (the size of the library's fixed scratch).
 *   depth:    0..8.
 *   lo, side: host, the cubical domain (lo[3], side > 0); cell of a point =
 *             min(floor((x - lo) / h_D), 2^depth - 1) per axis, as in bbfmm_plan.
 *   perm:     device, n int32, overwritten: perm[i] = original index of the
 *             i-th point in sorted order (increasing inside a leaf).
 *   leaf_off: device, 8^depth + 1 int32, overwritten: sorted points of the
 *             leaf with Morton index m are perm[leaf_off[m] .. leaf_off[m+1]).
 * Scratch: one file-scope device array of about 13.6 MB, resident on every GPU
 * that loads the library until the process exits.  Its address is looked up on
 * the first call made on a device (with that device current) and kept; make
 * that first call before any stream capture.  The kept address does not
 * survive cudaDeviceReset: do not call this entry point again after resetting
 * a device.  All calls share the array: calls that overlap on the GPU (other
 * streams, other threads) race and must be ordered by the caller.  The call
 * synchronizes `stream` to read the error flag.
 * Errors: EINVAL (sizes, host pointers, device memory of a GPU other than the
 * current one, NaN or out-of-domain points), ECUDA.
 */
int bbfmm_sort_points_static(const double *points, int64_t n, int depth, const double *lo, double side,
                             int32_t *perm, int32_t *leaf_off, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BBFMM_H */
