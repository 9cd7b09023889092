/*
 * logdet.h -- C ABI of liblogdet: log det Q and its hyperparameter gradient for
 * large sparse SPD precision matrices on one NVIDIA GB300 (sm_103a).
 *
 * Method (Aune & Simpson, "Parameter Estimation in High Dimensional Gaussian
 * Distributions"):
 *   log det Q = tr log Q                                  (Sec. 2.1, Eq. "eq_logdet_ident")
 *   tr log Q ~ sum_c v_c^T log(Q) v_c, v_c = indicator of colour class c of a
 *              distance-d colouring of the graph of Q     (Sec. 2.1, probing vectors)
 *   log(Q) v ~ sum_l alpha_l (Q - sigma_l I)^{-1} v       (Sec. 2.1, Eq. "eq_rat_app",
 *              contour-integral midpoint rule of Hale, Higham & Trefethen)
 *   all shifted systems solved on one Krylov space by multi-shift CG
 *              (CG-M / COCG-M)                            (Sec. 2.1, last two paragraphs)
 *   gradient   d log det Q / d eta = tr(Q^{-1} dQ/d eta), estimated with the
 *              same probing vectors and the seed solutions Q^{-1} v_c.
 *
 * Conventions shared by every entry point:
 *   - Every call returns ld_status.  Outputs are written only on LD_OK (the
 *     ld_info record, when given, is always filled).  Nothing aborts, throws,
 *     exits or traps across this boundary; ld_last_error() describes the most
 *     recent failure on the calling thread.
 *   - Pointers are HOST pointers unless the parameter name ends in _dev.  Host
 *     inputs are borrowed only for the duration of the call: the library
 *     copies what it needs into device memory it owns.
 *   - A context is used by one host thread at a time.  Calls are blocking:
 *     work is queued on the context's stream and the call synchronises that
 *     stream before it returns.
 *   - Vertex order is natural: index = x + nx*(y + ny*z).
 */
#ifndef PAPER_1105_5256_GB300_LOGDET_H
#define PAPER_1105_5256_GB300_LOGDET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LD_ABI_VERSION 6

typedef struct ld_ctx ld_ctx;

typedef enum {
    LD_OK = 0,
    LD_EINVAL = 1,        /* bad argument (null pointer, size, unsupported combination) */
    LD_ENOMEM = 2,        /* device or host allocation failed */
    LD_ECUDA = 3,         /* a CUDA runtime call failed */
    LD_ENOTSPD = 4,       /* p^T Q p <= 0 met in CG: Q is not SPD */
    LD_ENOTCONV = 5,      /* max_iter reached before every shifted system converged */
    LD_ENUMERIC = 6,      /* NaN/Inf in the CG scalars */
    LD_ETIMEOUT = 7,      /* a bounded device wait ran out */
    LD_EUNSUPPORTED = 8,  /* combination not implemented */
    LD_ECALLBACK = 9      /* a caller-supplied matvec callback returned nonzero */
} ld_status;

typedef enum { LD_FP64 = 0, LD_MIXED = 1 } ld_precision;

/* Matrix kinds.  Grid kinds describe the SPDE precisions of Sec. 3 on a
 * regular lattice; "non-periodic" means Dirichlet truncation (out-of-grid
 * neighbours dropped, diagonal kept). */
typedef enum {
    LD_CSR = 0,            /* general symmetric CSR matrix */
    LD_STENCIL_2D5 = 1,    /* scale*(diag(kappa2) - Lap_5pt + tau*diag(mask)) on nx x ny */
    LD_STENCIL_2D13_SQ = 2,/* scale*(kappa2 I - Lap_5pt)^2 (13-point Matern alpha=2) */
    LD_STENCIL_3D7 = 3,    /* scale*(diag(kappa2) - Lap_7pt + tau*diag(mask)) on nx x ny x nz */
    LD_MATFREE = 4         /* kind of an ld_create_matfree context (not valid in ld_matrix) */
} ld_kind;

/* Hyperparameter ids for gradients: dQ/d eta. */
enum {
    LD_P_KAPPA2 = 0,  /* kappa2 (or the multiplier c of a kappa2 field: kappa2(s) = c*field(s)) */
    LD_P_TAU = 1,     /* tau of the observation term tau*diag(mask) */
    LD_P_SCALE = 2    /* prior scale s of Q = s*Q0 */
};

typedef struct {
    int32_t kind;             /* ld_kind */
    int32_t periodic;         /* grid kinds: 1 = torus, 0 = Dirichlet truncation */
    int64_t n;                /* CSR: rows; grid kinds: ignored (product of dims) */
    const int64_t *rowptr;    /* CSR: n+1 row offsets */
    const int32_t *colidx;    /* CSR: column indices, symmetric pattern */
    const double *val;        /* CSR: values */
    int32_t dims[3];          /* grid kinds: nx, ny[, nz]; unused dims = 1 */
    double kappa2;            /* scalar kappa^2, or multiplier c when kappa2_field != NULL */
    const double *kappa2_field; /* grid kinds 2D5/3D7: per-vertex kappa^2 (n), or NULL */
    double tau;               /* observation precision (grid kinds 2D5/3D7) */
    const uint8_t *obs_mask;  /* n bytes, 1 = observed node; NULL = no observation term */
    double scale;             /* prior scale s (> 0); 0 is read as 1 */
} ld_matrix;

typedef struct {
    int32_t precision;        /* ld_precision: FP64 vectors, or FP32 vectors with FP64 scalars */
    int32_t tile_width;       /* probing vectors per tile: 0 = choose automatically */
    int32_t max_iter;         /* CG iteration cap per tile; 0 = 100000 */
    int32_t keep_x0;          /* keep seed solutions Q^{-1} v_c for ld_grad (extra HBM traffic) */
    double lambda_min;        /* > 0 (with lambda_max): user spectral interval; else the library's:
                                 grid kinds exact (Weyl on the lattice eigenvalues), CSR the
                                 Gershgorin upper bound and half the converged smallest
                                 Lanczos Ritz value, as ld_csr_bounds (ld_create fails with
                                 its LD_ENOTCONV / LD_ENOTSPD) */
    double lambda_max;        /* > 0: user upper spectral bound; else library bound */
    void *cuda_stream;        /* cudaStream_t to run on; NULL = a stream the context owns */
    const int32_t *colouring; /* optional host colouring (n ints >= 0); NULL = greedy */
    int32_t engine;           /* 0 auto, 1 multi-CTA grid engine, 2 one-CTA-per-tile engine */
    int32_t chunk_iters;      /* iterations per captured CUDA graph chunk; 0 = auto */
    double reliable_delta;    /* > 0: reliable-update residual replacement (grid engine).  The
                                 seed solution is split into an FP64 part x_hi and a vector-
                                 precision correction x_lo that the pass updates; whenever a
                                 column's recursive residual norm falls below reliable_delta
                                 times its largest norm since the last replacement, x_hi +=
                                 x_lo, x_lo = 0 and every active tile's residual is replaced
                                 by v - Q x_hi formed with FP64 arithmetic.  Keeps x0 on the
                                 device (as keep_x0).  0 = off. */
    int32_t lattice_pass;     /* grid engine, FP32 vectors on a 2D lattice, tiles of 2 or 4
                                 columns: 0 = the lean pass (the solve state is r and p, or r
                                 and Q1 p for the Matern kind; Q p is recomputed each pass: 4
                                 words per vertex and column per pass) wherever it applies
                                 (not for the Matern kind while x0 is kept); 1 = always the
                                 stored-w pass (r, Q p, p: 6 words).  Results agree to
                                 rounding. */
} ld_options;

typedef struct {
    int32_t status;           /* ld_status of the call */
    int32_t n_colours;        /* probing vectors C */
    int32_t n_shifts;         /* quadrature nodes N */
    int32_t iters;            /* CG iterations (maximum over tiles) */
    int32_t tile_width;
    int32_t engine;           /* 1 multi-CTA grid engine, 2 one-CTA-per-tile, 3 matrix-free driver */
    double lambda_min, lambda_max; /* interval enclosing the spectrum used for the nodes */
    double quad_cert;         /* max |f_N(lambda) - log lambda| on [lambda_min, lambda_max] */
    double ms;                /* device time of the solve (CUDA events) */
    double iter_ms;           /* device time spent in CG iterations (events around each
                                 iteration launch on the context stream) */
    int64_t tile_iters;       /* sum over tiles of the iterations each tile ran */
    int64_t gpu_launches;     /* kernels this call launched (graph nodes counted) */
    int32_t bulk_rows;        /* grid engine on a 2D lattice: 1 when lattice rows move by
                                 bulk (TMA) copies, 0 by per-thread copies; -1 otherwise */
    int32_t reliable_updates; /* residual replacements this call made */
    double rel_resid_max;     /* when x0 is kept (keep_x0, a gradient or reliable_delta > 0):
                                 max over the call's columns of ||v_c - Q x_c|| / ||v_c||, the
                                 true seed residual formed in FP64; -1 otherwise */
    int32_t pass_words;       /* grid engine: vector words per vertex and probing vector that
                                 one CG pass reads plus writes for the solve state -- 4 for the
                                 lean lattice pass (FP32 on 2D lattices: r and p, or r and Q1 p
                                 for the Matern kind, with Q p recomputed), 6 for the stored-w
                                 pass (r, Q p, p), 8 for the CSR pass (its step, then its
                                 product re-reads r and p), plus 2 when the pass also updates
                                 the kept seed solution; -1 for the other engines */
    int64_t vertex_tile_iters; /* sum over tiles of vertices x the iterations the tile ran
                                 (a batch: over every instance's tiles; a matrix-free context:
                                 over columns): the CG state a solve streams is 4 words per
                                 vertex and column of a pass, so 4 x word x T x this bytes */
} ld_info;

/* ABI version (LD_ABI_VERSION).  Never fails. */
int ld_abi_version(void);

/* Fill *opt with defaults (FP64, automatic tile width and engine). */
ld_status ld_default_options(ld_options *opt);

/* Create a context for Q (Sec. 2.1 method set-up).
 *   Q                  matrix description (host, borrowed for this call).
 *   colouring_distance d >= 0: probing vectors from a distance-d greedy colouring of
 *                      the graph of Q (Sec. 2.1; natural order, smallest free colour),
 *                      unless opt->colouring supplies one.
 *   n_shifts           N >= 1 quadrature nodes of the rational log (Eq. "eq_rat_app"), or 0:
 *                      the smallest N (4..256) whose measured certificate
 *                      max |f_N - log| on [lambda_min, lambda_max] is at most
 *                      1e-10 |log lambda_max - log lambda_min| (Sec. 2.1 gives the error
 *                      rate of the quadrature), chosen again whenever ld_set_params
 *                      moves the interval; ld_info.n_shifts reports it.
 *   tol                relative residual at which each shifted system is converged
 *                      (|zeta| ||r|| <= tol ||v_c||), 0 < tol < 1.
 *   opt                NULL = defaults.
 *   out                receives the context (owned by the caller; ld_destroy frees it).
 * Copies Q, the colouring and any fields into device memory on the current device.
 * Errors: LD_EINVAL, LD_EUNSUPPORTED, LD_ENOMEM, LD_ECUDA. */
ld_status ld_create(const ld_matrix *Q, int colouring_distance, int n_shifts, double tol,
                    const ld_options *opt, ld_ctx **out);

/* Matrix-free operator (Sec. 1: the method needs Q only through products Q v).
 * Enqueue W = Q P on `stream` (a cudaStream_t; or finish the product before returning).
 * P_dev and W_dev are device arrays of n x ncols doubles owned by the library, row-major (entry
 * (i, c) at i * ncols + c; column c is the probing vector of colour colour_begin + c of
 * the solve, or right-hand side c of ld_logmv / ld_invsqrt_mv); P is read-only, every
 * entry of W must be written.  Called once per CG iteration from the thread that called
 * the solve.  Return 0 on success; anything else stops the solve with LD_ECALLBACK. */
typedef int (*ld_matvec_fn)(void *user, int64_t n, int32_t ncols, const double *P_dev,
                            double *W_dev, void *stream);

/* Derivative product of a matrix-free operator Q(eta): enqueue Y = (dQ/d eta_param) X on
 * `stream` for param in [0, n_params) of ld_matfree_set_derivative; layouts, ownership and
 * the return value as ld_matvec_fn (X_dev read-only, every entry of Y_dev written). */
typedef int (*ld_dmatvec_fn)(void *user, int32_t param, int64_t n, int32_t ncols,
                             const double *X_dev, double *Y_dev, void *stream);

/* Create a context for an SPD operator given only by matvec (Sec. 2.1 method without a
 * matrix):
 *   n              dimension, 1 <= n <= 2^40.
 *   matvec, user   the product callback and its opaque argument (borrowed for the
 *                  context's lifetime).
 *   colouring      n colours in [0, n) (host, copied): the probing vectors are the
 *                  indicators of its classes; a distance-d colouring of the operator's
 *                  graph (ld_colour_csr on its pattern) gives the method's estimate.
 *   lambda_min, lambda_max   0 < lambda_min < lambda_max enclosing the spectrum (the
 *                  library cannot estimate them without the matrix).
 *   n_shifts, tol  as ld_create.
 *   opt            NULL = defaults; cuda_stream, max_iter and keep_x0 are used, precision
 *                  must be LD_FP64 (LD_EUNSUPPORTED otherwise), the rest is ignored.
 * The solve runs CG in its one-reduction form with the projected multi-shift recurrences
 * in the library's kernels (three launches around each product), n x C FP64 vectors
 * r, p, w (and x with keep_x0 or a gradient) on the device; the seed system Q x = v_c is
 * followed to the tolerance like the shifted ones, so ld_column_terms reports its
 * projections.  ld_logdet, ld_logdet_partial, ld_logdet_grad and ld_grad (after
 * ld_matfree_set_derivative), ld_column_terms, ld_logmv, ld_invsqrt_mv, ld_hutchinson,
 * ld_get_colouring, ld_get_nodes and ld_destroy accept the context; the rest return
 * LD_EUNSUPPORTED.
 * Errors: LD_EINVAL (checked before any device call), LD_EUNSUPPORTED, LD_ENOMEM,
 * LD_ECUDA; the solves add LD_ECALLBACK, LD_ENOTSPD, LD_ENOTCONV, LD_ENUMERIC. */
ld_status ld_create_matfree(int64_t n, ld_matvec_fn matvec, void *user, const int32_t *colouring,
                            double lambda_min, double lambda_max, int n_shifts, double tol,
                            const ld_options *opt, ld_ctx **out);

/* Register the derivative products of a matrix-free context (the gradient of Sec. 3's
 * likelihood, d log det Q / d eta_j = tr(Q^{-1} dQ/d eta_j), probed as
 * sum_c v_c^T (dQ/d eta_j) Q^{-1} v_c with the seed solutions of the same solve).  After
 * it, ld_logdet_grad and ld_grad take parameter ids in [0, n_params) instead of LD_P_*.
 *   dmatvec, user  the callback and its argument (borrowed for the context's lifetime);
 *                  dmatvec NULL unregisters.
 *   n_params       1 <= n_params <= 3.
 * Errors: LD_EINVAL (bad arguments or not a matrix-free context).  Host only. */
ld_status ld_matfree_set_derivative(ld_ctx *ctx, ld_dmatvec_fn dmatvec, void *user, int n_params);

/* Replace kappa2 (or its field multiplier), tau and scale, keeping the pattern and
 * colouring (Sec. 3: colourings are computed once and stored).  Spectral bounds and
 * nodes are recomputed unless the user fixed them.  CSR contexts: LD_EUNSUPPORTED. */
ld_status ld_set_params(ld_ctx *ctx, double kappa2, double tau, double scale);

/* log det Q ~ sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c
 * (Sec. 2.1, Eqs. "eq_logdet_ident", "eq_rat_app").  *logdet on LD_OK.
 * Errors: LD_ENOTSPD, LD_ENOTCONV (no output), LD_ENUMERIC, LD_ECUDA. */
ld_status ld_logdet(ld_ctx *ctx, double *logdet, ld_info *info);

/* log det Q and grad[i] = d log det Q / d eta_{ids[i]} ~ sum_c (E v_c)^T Q^{-1} v_c,
 * E = dQ/d eta (tr(Q^{-1} dQ/d eta) probed with the same v_c and the CG seed
 * solutions).  ids from LD_P_* (matrix-free contexts: indices of the parameters of
 * ld_matfree_set_derivative, LD_EINVAL when none is registered); n_params in [1, 3]. */
ld_status ld_logdet_grad(ld_ctx *ctx, int n_params, const int *param_ids, double *logdet,
                         double *grad, ld_info *info);

/* Backward pass on the seed solutions saved by the last ld_logdet of a context
 * created with keep_x0 = 1: grad[i] = sum_c (E_{ids[i]} v_c)^T x0_c.
 * Errors: LD_EINVAL when no solve with keep_x0 precedes it. */
ld_status ld_grad(ld_ctx *ctx, int n_params, const int *param_ids, double *grad);

/* The same estimate restricted to colours [colour_begin, colour_end): the unit of
 * work the paper hands to one node (Sec. 2.1, "Each node gets one probing vector").
 * Partials over a split of [0, C) sum to ld_logdet's value. */
ld_status ld_logdet_partial(ld_ctx *ctx, int colour_begin, int colour_end, double *partial,
                            ld_info *info);

/* Per-colour terms of the last solve: terms[c] = Re sum_l alpha_l v_c^T x^{sigma_l}_c
 * (n_colours doubles) and, if seed != NULL, seed[c] = v_c^T Q^{-1} v_c.
 * LD_EINVAL before the first completed solve. */
ld_status ld_column_terms(const ld_ctx *ctx, double *terms, double *seed);

/* Colouring used by the context: colour (n int32), *n_colours. */
ld_status ld_get_colouring(const ld_ctx *ctx, int32_t *colour, int32_t *n_colours);

/* Quadrature nodes in use: sigma, alpha as interleaved (re, im) pairs, N each. */
ld_status ld_get_nodes(const ld_ctx *ctx, double *sigma, double *alpha, int32_t *n_shifts);

/* y = Q x for ncols columns with the library's own SpMM (operator check).
 * x, y host arrays, row-major n x ncols, in FP64; the operator runs in the
 * context's precision. */
ld_status ld_apply(ld_ctx *ctx, int ncols, const double *x, double *y);

/* y_j ~ log(Q) v_j = Re sum_l alpha_l (Q - sigma_l I)^{-1} v_j for arbitrary right-hand
 * sides (Sec. 2.1, Eq. "eq_rat_app"), by the vector form of CG-M: the seed CG on Q x = v_j
 * plus one complex search direction per shift, accumulating y directly.  V, Y host arrays,
 * row-major n x ncols, FP64 (the vectors run in the context's precision).  Uses the
 * context's operator, nodes and tolerance; needs about (6 w + 16 N + 8) n ncols bytes of
 * device memory for the call (a matrix-free context: the caller's product, FP64 vectors,
 * (16 N + 40) n ncols bytes).  Errors as ld_logdet. */
ld_status ld_logmv(ld_ctx *ctx, int ncols, const double *V, double *Y, ld_info *info);

/* Q^{-1/2} V for the columns of V (n x ncols, row-major, FP64), by the same contour,
 * nodes and shifted solves as ld_logmv with the weights of z^{-1/2} (the paper has no
 * sampler; this draws x = Q^{-1/2} z ~ N(0, Q^{-1}) for standard normal z, the synthetic
 * fields a likelihood fit of Sec. 3 needs).  Errors as ld_logmv. */
ld_status ld_invsqrt_mv(ld_ctx *ctx, int ncols, const double *V, double *Y, ld_info *info);

/* Colouring distance by decay (Sec. 2.1, the heuristic for the power p of Q^p): forms
 * y = log(Q) e_j with the context's method (as ld_logmv: the context's operator, nodes,
 * tolerance and precision) and returns *distance = min { d(l, j) : |y_l| < eps |y_j| },
 * d the graph distance in the graph of Q (lattice distance for grid kinds, breadth-first
 * search for CSR), or -1 when no vertex within max_d qualifies.  eps is relative to
 * |y_j|.  profile: NULL or max_d + 1 doubles, profile[d] = max over vertices at graph
 * distance d of |y_l| / |y_j|.  0 <= j < n, eps > 0, 0 <= max_d <= 4096; errors as
 * ld_logmv. */
ld_status ld_select_distance(ld_ctx *ctx, int64_t j, double eps, int max_d, int32_t *distance,
                             double *profile, ld_info *info);

/* Hutchinson estimator (Sec. 2.1, Eq. "eq_est_eq"), the stochastic alternative the
 * probing method is compared with: tr log Q ~ (1/s) sum_k z_k^T log(Q) z_k for the s
 * columns of Z (n x s, row-major, FP64; the caller draws them, normally +-1 with
 * probability 1/2 each).  log(Q) Z is formed as by ld_logmv.  *estimate = the mean,
 * *std_error = sample standard deviation / sqrt(s) (0 when s = 1), samples: NULL or s
 * doubles z_k^T log(Q) z_k.  Errors as ld_logmv. */
ld_status ld_hutchinson(ld_ctx *ctx, int s, const double *Z, double *estimate, double *std_error,
                        double *samples, ld_info *info);

/* Failure-path self-test of the library's bounded device waits (the paper has no
 * counterpart): one CTA on the current device waits on a barrier that nothing
 * completes, gives up after limit_ns nanoseconds (1e3 .. 1e10) and the call returns
 * LD_ETIMEOUT, as a pass whose bulk copies never arrived would; LD_OK would mean the
 * wait was not bounded as documented.  Allocates 4 bytes of device memory. */
ld_status ld_wait_selftest(int64_t limit_ns);

/* Host utilities (no device work; usable without a GPU). */

/* Greedy distance-d colouring of the CSR pattern in natural order (Sec. 2.1).
 * colour: n int32 out.  *n_colours out. */
ld_status ld_colour_csr(int64_t n, const int64_t *rowptr, const int32_t *colidx, int d,
                        int32_t *colour, int32_t *n_colours);

/* Nodes of ld_invsqrt_mv's rational z^{-1/2} on [lmin, lmax]: the log nodes' poles sigma
 * and weights beta_j = -(2 i h / pi) w'(t_j), interleaved (re, im), N each (2N doubles per
 * array).  LD_EINVAL unless 0 < lmin < lmax and 1 <= N <= 256. */
ld_status ld_hht_invsqrt_nodes(double lmin, double lmax, int N, double *sigma, double *beta);

/* P1 finite-element SPDE precision on a triangulation (general-mesh input for LD_CSR; the
 * SPDE model of Sec. 3, tau (kappa - Laplacian) u = W with kappa^2 for kappa, on a mesh):
 *   xy         n vertex coordinates (x, y), n x 2 row-major; 3 <= n < 2^31.
 *   tri        m triangles as vertex indices, m x 3 row-major, either orientation.
 *   alpha      1: Q = tau (kappa^2 C + G);  2: Q = tau K C^{-1} K with K = kappa^2 C + G,
 *              C the lumped mass (a third of each incident triangle's area on the diagonal),
 *              G the stiffness (integrals of grad phi_i . grad phi_j, Neumann boundary).
 *   kappa2, tau > 0.
 * Output: sorted CSR of Q (exact zeros dropped) in rowptr (n + 1), colidx and val (*nnz
 * each), written only when capacity >= *nnz and all three are non-NULL; otherwise only
 * *nnz is set (call once to size the arrays, then again to fill them).
 * LD_EINVAL for bad sizes or parameters, an index outside [0, n), a zero-area triangle or
 * a vertex in no triangle.  Host only. */
ld_status ld_spde_fem_csr(int64_t n, const double *xy, int64_t m, const int64_t *tri, double kappa2,
                          int alpha, double tau, int64_t capacity, int64_t *rowptr, int32_t *colidx,
                          double *val, int64_t *nnz);

/* Spectral interval a CSR context uses without user bounds: *lmax = Gershgorin bound of
 * scale * val, *lmin = half the smallest Ritz value of a Lanczos run from a fixed +-1 start
 * vector, run until that Ritz value has stagnated (less than 1e-3 relative change over the
 * second half of the steps; about sqrt(condition number) steps, more than n allowed) within
 * a host budget of about 4e9 flop (at least 300 steps).  LD_ENOTCONV when it has not
 * converged by then (pass lambda_min / lambda_max instead), LD_ENOTSPD when the estimate
 * is not positive.  Host only. */
ld_status ld_csr_bounds(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *val,
                        double scale, double *lmin, double *lmax);

/* Same colouring for a grid kind (lattice-ball search, no CSR needed). */
ld_status ld_colour_grid(int kind, const int32_t dims[3], int periodic, int d, int32_t *colour,
                         int32_t *n_colours);

/* The node count ld_create uses for n_shifts = 0: the smallest N in 4..256 whose
 * certificate max |f_N - log| on [lambda_min, lambda_max] (2001 log-spaced samples) is at
 * most 1e-10 |log lambda_max - log lambda_min| (256 when none is; Sec. 2.1's error rate).
 * Host only.  Errors: LD_EINVAL (NULL output, bad interval). */
ld_status ld_auto_shifts(double lambda_min, double lambda_max, int32_t *n_shifts);

/* Nodes/weights of the rational log on [lmin, lmax] (Eq. "eq_rat_app"):
 * sigma, alpha interleaved (re, im), N each; *cert = max |f_N - log| on the interval. */
ld_status ld_hht_nodes(double lmin, double lmax, int N, double *sigma, double *alpha,
                       double *cert);

/* Spectral interval the library uses for a grid kind (Weyl bounds). */
ld_status ld_grid_bounds(const ld_matrix *Q, double *lmin, double *lmax);

/* Batched evaluation of many independent grid GMRFs of uneven size in one persistent
 * launch (each (instance, tile) a work item).  Qs[count] (grid kinds), distances[count]
 * as in ld_create; every instance gets its own colouring, spectral bounds and nodes.
 * opt: precision, max_iter, tile_width (0 = chosen by timing short runs of the persistent
 * launch per candidate, cached per batch shape), cuda_stream.  An instance whose one-CTA
 * solve would outlast the batch (estimated from its size, its condition number and the
 * measured time of a CTA step) runs on the multi-CTA grid engine instead, several at once
 * on their own streams from host threads; for those to overlap, the process should set
 * CUDA_DEVICE_MAX_CONNECTIONS=32 (or more) before it creates its CUDA context (the Python
 * binding does so on import).  Errors: as ld_create, reported with the failing instance's
 * index. */
ld_status ld_batch_create(int count, const ld_matrix *Qs, const int *distances, int n_shifts,
                          double tol, const ld_options *opt, ld_ctx **out);

/* Evaluate every instance: logdets[count]; grads[count] = d log det / d kappa2 for
 * scalar-kappa2 5/7-point instances (tr Q^{-1} probed, from the projected seed sums),
 * NaN for the others; grads and info may be NULL.  One CUDA-graph launch: a queue
 * reset, a per-instance prep kernel, the persistent solve (CTAs pull (instance, tile)
 * items, longest first, and run each tile's whole CG-M in one CTA) and a per-instance
 * sum; beside it the grid-engine instances.  info: ms is the host wall time of the whole
 * batch, tile_iters and vertex_tile_iters the exact passes every tile ran.  Errors: the
 * first failing instance's status (no outputs written). */
ld_status ld_batch_logdet(ld_ctx *ctx, double *logdets, double *grads, ld_info *info);

/* ---------------------------------------------------------------------------
 * Evaluation without device allocation (no counterpart in the paper).
 *
 * For callers that may not call cudaMalloc/cudaFree when they need a log det,
 * e.g. code running under a framework allocator or memory arena that owns all
 * device memory, or a latency-critical callback where an allocation would
 * synchronise the device.  Every work buffer lives in one static device array
 * of LD_STATIC_SCRATCH_BYTES that each GPU loading the library keeps until the
 * process exits; the call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine) and copies its inputs into that array.
 *
 *   Q          grid kinds 2D5, 2D13_SQ, 3D7 with scalar kappa2, no field, no mask.
 *   colour     host, n ints in [0, n_colours): the probing colouring (e.g. from
 *              ld_colour_grid); n_colours <= LD_STATIC_MAX_COLOURS.
 *   n_shifts   quadrature nodes (1..256); tol, max_iter as in ld_create/ld_options.
 *   cuda_stream stream to run on (NULL = default stream); the call synchronises it.
 *   logdet     host output, written on LD_OK.
 * Runs the same probed rational-log multi-shift CG as ld_logdet in FP64 with one
 * CTA per probing vector (small problems).  Needs 48*n*n_colours bytes plus small
 * tables inside the array; larger problems return LD_EINVAL ("needs more than
 * LD_STATIC_SCRATCH_BYTES").  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress): make that first call outside any stream
 * capture.  Every call shares the one array and leaves its contents behind (the
 * call clears what must start at zero): calls that overlap on the GPU, from two
 * threads or two streams, race and corrupt each other. */
#define LD_STATIC_SCRATCH_BYTES (8u << 20)
#define LD_STATIC_MAX_COLOURS 1024
ld_status ld_logdet_static(const ld_matrix *Q, const int32_t *colour, int n_colours, int n_shifts,
                           double tol, int max_iter, void *cuda_stream, double *logdet);

/* Message for the last failure on this thread; never NULL. */
const char *ld_last_error(void);

/* Free a context (NULL-safe). */
void ld_destroy(ld_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif
