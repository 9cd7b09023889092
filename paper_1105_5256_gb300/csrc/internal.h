// Internal declarations shared by the host runtime (api.cpp, colouring.cpp,
// hht.cpp) and the CUDA engine (engine.cu).  Not part of the public ABI.
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace ld {

enum { KIND_CSR = 0, KIND_2D5 = 1, KIND_2D13_SQ = 2, KIND_3D7 = 3 };

// ---------------------------------------------------------------- host helpers
void set_last_error(const char *msg);   // message returned by ld_last_error() on this thread
int colour_csr(int64_t n, const int64_t *rowptr, const int32_t *colidx, int d, int32_t *colour);
int colour_grid(int kind, const int32_t dims[3], int periodic, int d, int32_t *colour);
double ellip_k(double m);
void jacobi_real(double u, double m, double *sn, double *cn, double *dn);
int hht_log_nodes(double lmin, double lmax, int N, std::complex<double> *sigma,
                  std::complex<double> *alpha);
int hht_invsqrt_nodes(double lmin, double lmax, int N, std::complex<double> *sigma,
                      std::complex<double> *beta);
double hht_certificate(double lmin, double lmax, int N, const std::complex<double> *sigma,
                       const std::complex<double> *alpha);

// ---------------------------------------------------------------- device problem
// Operator description read by the kernels (device pointers).  Q is
//   grid 2D5/3D7:  scale * (kappa2_i + 2*dim + tau*mask_i) on the diagonal, -scale off it
//                  (kappa2_i = kappa2 * field_i when field != nullptr)
//   grid 2D13_SQ:  scale * (kappa2 I - Lap)^2, expanded as a 13-point stencil
//   CSR:           scale * val
struct Operator {
    int kind;
    int periodic;
    int nx, ny, nz;
    int64_t n;
    double kappa2;
    double tau;
    double scale;
    float kappa2_f, tau_f, scale_f;   // FP32 copies (set_f32_coefs), read by FP32 kernels
    const double *field_d;   // kappa2 field base values, FP64 copy
    const float *field_f;    // FP32 copy
    const uint8_t *mask;     // observation mask (or nullptr)
    // 2D5/3D7 with a field or a mask: the diagonal term kappa2*field_i + tau*mask_i per
    // vertex (FP64, and rounded once to FP32), so that passes read one word per vertex
    const double *diag_d;
    const float *diag_f;
    const int64_t *rowptr;   // CSR
    const int32_t *colidx;
    const double *val_d;
    const float *val_f;
};

// FP32 copies of the operator's coefficients, so that FP32 kernels convert nothing
inline void set_f32_coefs(Operator &op) {
    op.kappa2_f = (float)op.kappa2;
    op.tau_f = (float)op.tau;
    op.scale_f = (float)op.scale;
}

// Status codes written by kernels into the device status word.
enum { DEV_OK = 0, DEV_NOTSPD = 4, DEV_NUMERIC = 6, DEV_TIMEOUT = 7 };

// Everything one solve's kernels need (passed by value).
struct Solve {
    Operator op;
    int T;                 // columns per tile
    int ntiles;
    int ncols;             // padded columns = ntiles * T
    int nshift;            // N
    int bpt;               // CTAs per tile (grid engine)
    int strips, seg;       // 2D kinds: lattice strips per tile, rows per CTA segment
    int bulk;              // 2D kinds: rows arrive by bulk (TMA) copies (alignment permits)
    int share;             // solves running on the device at once (a batch's grid-engine
                           // instances): the plan sizes a launch for 1/share of it (<= 1: all)
    int lean;              // FP32: 0 the stored-w pass (state r, w, p); 2D kinds X = 1, 2 the
                           // lean pass (state r and p, or r and u = Q1 p for the Matern
                           // kind; w recomputed), X lattice columns per thread; 3 the lean
                           // 3D pass
    const uint8_t *lane;   // lean pass: per-tile lane codes in strip layout (or null)
    int lane_mask;         // lean pass, 5-point, scalar kappa^2 with a mask: the codes' high
                           // bit is the mask bit (diagonal kappa^2 + tau mask_i formed in the pass)
    int tile0, tstride;    // grid engine: a launch covers tiles tile0, tile0 + tstride, ...
                           // (grid.y of them; tstride 0 reads as 1)
    int precision;         // 0 fp64, 1 mixed
    int keep_x0;
    double tol;
    const int32_t *colour; // n
    // CG state, two sets read/written alternately by consecutive passes:
    // set[k & 1] -> set[(k & 1) ^ 1]; each [ntiles][n][T] in the vector precision
    void *rbuf[2], *wbuf[2], *pbuf[2];
    void *x;               // seed solution (gradient mode); with reliable updates, the
                           // correction x_lo since the last residual replacement
    double *xhi;           // reliable updates: FP64 part x_hi of the seed solution (or null)
    // per-column scalars (ncols)
    double *rho, *alpha, *beta, *alpha_prev, *beta_prev, *vnorm2, *pi0, *phi0;
    int32_t *col_active, *col_iters;
    // per (column, shift): [ncols][nshift]
    double2 *zeta, *zeta_prev, *pi, *phi;
    uint8_t *sh_active;
    double2 *asig, *bsig;  // shifted-vector mode: alpha^sigma, beta^sigma of the last pass (or null)
    const double2 *shift;  // s_l = -sigma_l
    const double2 *weight; // alpha_l
    // per tile
    int32_t *tile_done, *tile_ctr, *tile_par;
    double *partial;       // [ntiles][bpt][NDOT*T]
    int32_t *remaining;    // tiles not yet converged
    int32_t *status;       // first error code
    double *terms;         // per column Re sum alpha_l pi_l
    const double *class_size; // |colour class| per column (0 for padding)
    double *result;        // [0] = sum of terms, [1] = sum of seed projections
};

// dot products per column reduced each pass: r.r, p.w, r.w, w.w, v.r, v.w
constexpr int NDOT = 6;

// Engine entry points (engine.cu); all asynchronous on `stream`.
int engine_init(const Solve &s, int col_begin, int col_end, void *stream, bool vectors = true);
int engine_iteration(const Solve &s, int parity, void *stream);      // one fused CG pass
int engine_cta_solve(const Solve &s, int max_iter, void *stream);    // whole solve, one CTA per tile
int engine_flush_x(const Solve &s, void *stream);                    // last seed-solution update
// shifted-vector mode: which = 0 init (p^sigma = v, y = 0), 1 update after a pass that
// wrote set `nxt`
int engine_modev(const Solve &s, int which, int nxt, double2 *psig, double *y, void *stream);
// batched engine: all instances' tiles in one persistent launch (plus prep/finish)
int engine_batch_occupancy(int precision, int T);
int engine_batch(const Solve *solves_dev, const int *ncolours_dev, int count, const int2 *items_dev,
                 int nitems, int *queue_dev, int max_iter, int precision, int T, int grid,
                 double *logdet_dev, double *seed_dev, int *flag_dev, int *iters_dev, int *tile_passes_dev,
                 void *stream);
int engine_finish(const Solve &s, int col_begin, int col_end, void *stream);
int engine_apply(const Operator &op, int precision, int T, int ntiles, const void *x, void *y,
                 void *stream);
int engine_grad_params(const Solve &s, int nparam, const int *ids, double *out_dev, void *stream);
// one CTA waits on an mbarrier nothing arrives at, giving up after limit_ns: writes
// DEV_TIMEOUT (or DEV_OK) to *status_dev
int engine_wait_selftest(uint64_t limit_ns, int32_t *status_dev, void *stream);
// diag_d[i] = kappa2 * (field ? field[i] : 1) + tau * (mask ? mask[i] : 0), diag_f its FP32 copy
int engine_fill_diag(const Operator &op, double *diag_d, float *diag_f, void *stream);
// reliable updates: x_hi += x_lo, x_lo = 0 (all tiles); then with replace != 0 the active
// tiles' residuals in set `set` become v - Q x_hi.  norm2_dev[ncols] (zeroed here) receives
// ||v_c - Q x_c||^2 in FP64 for c in [col_begin, col_end), x = x_hi when present, else x.
int engine_true_residual(const Solve &s, int set, int col_begin, int col_end, int replace,
                         double *norm2_dev, void *stream);
int engine_plan(Solve &s);   // sets bpt (and strips/seg) for s.lean's pass; returns bpt
// lean pass: lattice columns per thread it uses for this solve's kind, precision, tile
// width and grid (0: not available; the stored-w pass runs)
int engine_lean_x(const Solve &s, bool keep_x0);
// bytes of the lane codes for the current plan (s.lean > 0), and their construction
size_t engine_lean_code_bytes(const Solve &s);
int engine_lean_codes(const Solve &s, uint8_t *out, void *stream);
const char *engine_error_string(int cuda_err);

// host: graph distances from vertex j (colouring.cpp)
void graph_distances(int kind, const int32_t dims[3], int periodic, int64_t n, const int64_t *rowptr,
                     const int32_t *colidx, int64_t j, int max_d, int32_t *dist);

// ---------------------------------------------------------------- matrix-free operator
// (matfree.cu) the caller supplies W = Q P; state and buffers of one context
struct Matfree;
struct MatfreeStats {
    int iters;             // iterations run (maximum over columns)
    int64_t column_iters;  // sum over columns of their iterations
    int64_t launches;      // kernels launched (callback work not counted)
    int callback_rc;       // nonzero return of the callback, if it stopped the solve
    float ms;              // device time of the solve, callback included
};
// fn is an ld_matvec_fn; colour (host, n entries in [0, C)) is copied; 0 or a CUDA error
int matfree_create(Matfree **out, int64_t n, const int32_t *colour, int C, int N, void *fn, void *user);
void matfree_destroy(Matfree *m);
// one solve: the probing vectors of colours [cb, ce), or (rhs != nullptr) ncols given
// right-hand sides with the vector form y = Re sum_l yweight_l (Q - sigma_l I)^{-1} v
struct MatfreeJob {
    int cb = 0, ce = 0;
    const double *rhs = nullptr;                     // host, n x ncols row-major
    int ncols = 0;
    const std::complex<double> *yweight = nullptr;   // host, n_shifts (nullptr: the log weights)
    double *y_out = nullptr;                         // host, n x ncols
    int n_shifts = 0;
    bool keep_x = false;                             // keep the seed solutions for matfree_grad
};
// terms_out[c] = Re sum_l weight_l v_c^T (Q - sigma_l I)^{-1} v_c, seeds_out[c] = v_c^T
// Q^{-1} v_c (nullable); returns an ld_status (message through set_last_error)
int matfree_solve(Matfree *m, const MatfreeJob &job, const std::complex<double> *sigma,
                  const std::complex<double> *weight, double tol, int max_iter, cudaStream_t stream,
                  double *terms_out, double *seeds_out, MatfreeStats *st);
// grad[k] = sum_c v_c^T (dQ/d eta_{ids[k]}) x_c over the seed solutions kept by the last
// probing solve (dfn an ld_dmatvec_fn); LD_EINVAL when none are kept
int matfree_grad(Matfree *m, int n_params, const int *ids, void *dfn, void *duser, cudaStream_t stream,
                 double *grad, int *callback_rc);

// host: P1 finite-element SPDE precision of a triangulation as sorted CSR (fem.cpp);
// 0, or -1 vertex index out of range, -2 degenerate triangle, -3 vertex in no triangle
int fem_spde(int64_t n, const double *xy, int64_t m, const int64_t *tri, double kappa2, int alpha,
             double tau, std::vector<int64_t> &rowptr, std::vector<int32_t> &colidx,
             std::vector<double> &val);

// host: spectral interval of a CSR matrix (Gershgorin / half the converged smallest
// Lanczos Ritz value; bounds.cpp); 0 on success, -1 when the estimate is not positive,
// -2 when the Ritz value did not converge within the step cap; *steps = Lanczos steps run
int csr_bounds(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *val, double scale,
               double *lmin, double *lmax, int *steps = nullptr);

}  // namespace ld
