// C ABI of liblogdet (declarations and contracts in include/logdet.h).
//
// Host runtime around the CUDA engine: argument checking, the probing
// colouring (Sec. 2.1), spectral bounds and quadrature nodes (Eq.
// "eq_rat_app"), device buffers, the CG iteration driver (CUDA-graph chunks
// with an on-device convergence counter) and the gradient pass.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/logdet.h"
#include "internal.h"

#include <nvtx3/nvToolsExt.h>

using ld::Operator;
using ld::Solve;

namespace {

// NVTX range for profilers (a no-op unless a tool is attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

thread_local std::string g_err = "no error";

ld_status fail(ld_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? LD_ENOMEM : LD_ECUDA, "%s: %s", #expr, \
                        cudaGetErrorString(e_));                                              \
    } while (0)

#define ENGINE_TRY(expr)                                                                      \
    do {                                                                                      \
        int e_ = (expr);                                                                      \
        if (e_ != 0) return fail(LD_ECUDA, "%s: %s", #expr, ld::engine_error_string(e_));     \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t b) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = b;
        if (b == 0) return cudaSuccess;
        return cudaMalloc(&p, b);
    }
    template <class X>
    X *as() const { return static_cast<X *>(p); }
};

}  // namespace

void ld::set_last_error(const char *msg) { g_err = msg; }

struct ld_ctx {
    // problem
    int kind = 0, periodic = 0;
    int32_t dims[3] = {1, 1, 1};
    int64_t n = 0;
    double kappa2 = 0, tau = 0, scale = 1;
    bool has_field = false, has_mask = false, mask_any = false;
    int distance = 0, nshift = 0;
    bool auto_shift = false;   // n_shifts = 0: N chosen from the quadrature certificate
    int nshift_cap = 0;        // shift-state capacity of d_shift / d_nodes (columns x nodes)
    double tol = 0;
    ld_options opt{};
    bool user_bounds = false;
    double csr_lmin = 0.0, csr_lmax = 0.0;   // library estimate for CSR without user bounds
    // colouring
    std::vector<int32_t> colour;
    int ncolours = 0;
    // tiling
    int T = 4, ntiles = 0, ncols = 0, engine = 1, chunk = 16;
    // nodes
    double lmin = 0, lmax = 0, cert = 0;
    std::vector<std::complex<double>> sigma, alpha;
    // device
    DevBuf d_colour, d_field_d, d_field_f, d_mask, d_rowptr, d_colidx, d_val_d, d_val_f;
    DevBuf d_r[2], d_w[2], d_p[2], d_x;
    DevBuf d_xhi, d_norm2;   // reliable updates: FP64 seed solution part; residual norms
    DevBuf d_diag_d, d_diag_f;   // per-vertex diagonal term (field and/or mask models)
    DevBuf d_lane;     // lane codes of the lean lattice pass (built on first use)
    bool lane_built = false;   // d_lane holds the lane codes of this context's colouring
    int lean_plan_x0 = -1;     // keep_x0 the current lean plan was made for
    DevBuf d_colscal;  // 8 double arrays [ncols]
    DevBuf d_colint;   // 2 int arrays [ncols]
    DevBuf d_shift;    // 4 double2 arrays [ncols*N] + uint8 [ncols*N]
    DevBuf d_nodes;    // shift[N], weight[N] (double2)
    DevBuf d_tile;     // tile_done, tile_ctr, tile_par [ntiles]; remaining, status
    DevBuf d_partial;
    DevBuf d_terms;    // terms[ncols], class_size[ncols], result[2], grad[3]
    std::vector<double> class_size;
    Solve s{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    cudaEvent_t evc[2] = {nullptr, nullptr};   // ends of the chunks in flight (two slots)
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    // grid engine: tile groups iterate on their own streams inside the captured graph
    static constexpr int kMaxGroups = 16;
    int ngroups = 0;
    cudaStream_t gstream[kMaxGroups] = {};
    cudaEvent_t gfork = nullptr, gjoin[kMaxGroups] = {};
    int32_t *h_pinned = nullptr;  // remaining, status
    bool have_x0 = false;
    int last_cb = 0, last_ce = 0;
    bool solved = false;
    // batch mode: independent problems solved by one persistent launch
    bool is_batch = false;
    std::vector<ld_ctx *> subs;
    DevBuf d_solves, d_items, d_queue, d_bout, d_bint;
    int nitems = 0, bgrid = 0;
    // batch: instances in the persistent launch (small) and on the multi-CTA engine (large)
    std::vector<int> small_idx, large_idx;
    cudaGraphExec_t bgraph = nullptr;
    // matrix-free operator (ld_create_matfree): the caller's W = Q P drives the solve
    ld::Matfree *mf = nullptr;
    std::vector<double> mf_terms, mf_seeds;
    void *mf_dfn = nullptr, *mf_duser = nullptr;   // ld_dmatvec_fn and its argument
    int mf_nparams = 0;
    bool l2_persist = false;   // captured kernels mark the colours persisting in L2

    ~ld_ctx() {
        if (l2_persist) cudaCtxResetPersistingL2Cache();   // return those lines to normal
        if (mf) ld::matfree_destroy(mf);
        if (bgraph) cudaGraphExecDestroy(bgraph);
        for (ld_ctx *c : subs) delete c;
        if (graph) cudaGraphExecDestroy(graph);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (ev2) cudaEventDestroy(ev2);
        if (ev3) cudaEventDestroy(ev3);
        for (cudaEvent_t e : evc)
            if (e) cudaEventDestroy(e);
        if (h_pinned) cudaFreeHost(h_pinned);
        for (int g = 0; g < kMaxGroups; ++g) {
            if (gstream[g]) cudaStreamDestroy(gstream[g]);
            if (gjoin[g]) cudaEventDestroy(gjoin[g]);
        }
        if (gfork) cudaEventDestroy(gfork);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

int64_t grid_n(const int32_t dims[3]) { return (int64_t)dims[0] * dims[1] * dims[2]; }

// Weyl bounds with the exact extreme eigenvalues of the truncated / periodic
// second difference per dimension (matches ld_grid_bounds' contract).
void lap_extremes(int N, int periodic, double *lo, double *hi) {
    if (periodic) {
        double best = 0.0;
        for (int k = 0; k < N; ++k) best = std::max(best, 2.0 - 2.0 * std::cos(2.0 * M_PI * k / N));
        *lo = 0.0;
        *hi = best;
    } else {
        *lo = 2.0 - 2.0 * std::cos(M_PI / (N + 1));
        *hi = 2.0 + 2.0 * std::cos(M_PI / (N + 1));
    }
}

void grid_bounds(int kind, const int32_t dims[3], int periodic, double k2min, double k2max,
                 double tau_max, double scale, double *lmin, double *lmax) {
    const int nd = (kind == ld::KIND_3D7) ? 3 : 2;
    double mlo = 0.0, mhi = 0.0;
    for (int d = 0; d < nd; ++d) {
        double a, b;
        lap_extremes(dims[d], periodic, &a, &b);
        mlo += a;
        mhi += b;
    }
    double lo = k2min + mlo, hi = k2max + tau_max + mhi;
    if (kind == ld::KIND_2D13_SQ) {
        lo *= lo;
        hi *= hi;
    }
    lo *= scale;
    hi *= scale;
    hi = std::max(hi, 1.01 * lo);
    *lmin = lo;
    *lmax = hi;
}

ld_status validate_matrix(const ld_matrix *Q) {
    if (!Q) return fail(LD_EINVAL, "Q is NULL");
    if (Q->kind < LD_CSR || Q->kind > LD_STENCIL_3D7) return fail(LD_EINVAL, "unknown kind %d", Q->kind);
    const double scale = Q->scale == 0.0 ? 1.0 : Q->scale;
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(LD_EINVAL, "scale must be > 0");
    if (Q->kind == LD_CSR) {
        if (Q->n <= 0 || !Q->rowptr || !Q->colidx || !Q->val) return fail(LD_EINVAL, "CSR needs n > 0, rowptr, colidx, val");
        if (Q->rowptr[0] != 0) return fail(LD_EINVAL, "rowptr[0] must be 0");
        for (int64_t i = 0; i < Q->n; ++i)
            if (Q->rowptr[i + 1] < Q->rowptr[i]) return fail(LD_EINVAL, "rowptr not monotone at %lld", (long long)i);
        const int64_t nnz = Q->rowptr[Q->n];
        for (int64_t e = 0; e < nnz; ++e) {
            if (Q->colidx[e] < 0 || Q->colidx[e] >= Q->n) return fail(LD_EINVAL, "colidx out of range at %lld", (long long)e);
            if (!std::isfinite(Q->val[e])) return fail(LD_EINVAL, "non-finite value at %lld", (long long)e);
        }
        return LD_OK;
    }
    const int nd = (Q->kind == LD_STENCIL_3D7) ? 3 : 2;
    for (int d = 0; d < 3; ++d) {
        if (d < nd && Q->dims[d] < 1) return fail(LD_EINVAL, "dims[%d] must be >= 1", d);
        if (d >= nd && Q->dims[d] != 1 && Q->dims[d] != 0) return fail(LD_EINVAL, "dims[%d] must be 1 for this kind", d);
    }
    if ((double)Q->dims[0] * (double)Q->dims[1] * (double)(nd == 3 ? Q->dims[2] : 1) > 4.0e12)
        return fail(LD_EINVAL, "grid has more than 4e12 vertices");
    if (!std::isfinite(Q->kappa2) || Q->kappa2 < 0.0) return fail(LD_EINVAL, "kappa2 must be finite and >= 0");
    if (Q->kind == LD_STENCIL_2D13_SQ && (Q->kappa2_field || (Q->obs_mask && Q->tau != 0.0)))
        return fail(LD_EUNSUPPORTED, "13-point Matern kind takes a scalar kappa2 and no observation term");
    if (!std::isfinite(Q->tau) || Q->tau < 0.0) return fail(LD_EINVAL, "tau must be finite and >= 0");
    return LD_OK;
}

// tile width: fewest padded columns; ties go to the narrower tile (8-byte packs
// keep the streaming pass's registers low and its occupancy high, measured fastest)
int choose_tile(int precision, int C, int requested) {
    const int *opts;
    static const int f64[4] = {1, 2, 3, 4};
    static const int f32[4] = {2, 4, 6, 8};
    opts = precision == LD_FP64 ? f64 : f32;
    if (requested > 0) {
        for (int k = 0; k < 4; ++k)
            if (opts[k] == requested) return requested;
        return -1;
    }
    int best = opts[0];
    int64_t best_cols = INT64_MAX;
    for (int k = 0; k < 4; ++k) {
        const int t = opts[k];
        const int64_t cols = (int64_t)((C + t - 1) / t) * t;
        if (cols < best_cols) {
            best_cols = cols;
            best = t;
        }
    }
    return best;
}

void invalidate_graph(ld_ctx *c);

// Shift state (per column and node) and the node table sized for `cap` nodes; the solve
// uses the first nshift of them.  Rebinds the Solve's pointers.
ld_status bind_shift_state(ld_ctx *c, int cap) {
    const int C = c->ncols;
    CUDA_TRY(c->d_shift.alloc((size_t)4 * C * cap * sizeof(double2) + (size_t)C * cap));
    CUDA_TRY(c->d_nodes.alloc((size_t)2 * cap * sizeof(double2)));
    c->nshift_cap = cap;
    Solve &s = c->s;
    double2 *sh = c->d_shift.as<double2>();
    s.zeta = sh;
    s.zeta_prev = sh + (size_t)C * cap;
    s.pi = sh + (size_t)2 * C * cap;
    s.phi = sh + (size_t)3 * C * cap;
    s.sh_active = reinterpret_cast<uint8_t *>(sh + (size_t)4 * C * cap);
    s.shift = c->d_nodes.as<double2>();
    s.weight = c->d_nodes.as<double2>() + cap;
    invalidate_graph(c);
    return LD_OK;
}

// Automatic node count: the smallest N in [4, 256] whose measured certificate
// max |f_N - log| on [m, M] is at most 1e-10 |log M - log m|.  The search starts from the
// square-root method's rate exp(-2 pi^2 N / (log(M/m) + 6)) and steps by one.
int auto_shift_count(double lmin, double lmax) {
    const double target = 1e-10 * std::fabs(std::log(lmax) - std::log(lmin));
    const double rate = 2.0 * M_PI * M_PI / (std::log(lmax / lmin) + 6.0);
    int N = (int)std::ceil(std::log(1.0 / target) / rate);
    N = std::min(256, std::max(4, N));
    std::vector<std::complex<double>> sg(256), al(256);
    auto cert = [&](int k) -> double {
        if (ld::hht_log_nodes(lmin, lmax, k, sg.data(), al.data()) != 0) return INFINITY;
        return ld::hht_certificate(lmin, lmax, k, sg.data(), al.data());
    };
    if (cert(N) > target) {
        while (N < 256 && cert(N) > target) ++N;
    } else {
        while (N > 4 && cert(N - 1) <= target) --N;
    }
    return N;
}

ld_status set_nodes(ld_ctx *c) {
    if (c->auto_shift) {
        const int N = auto_shift_count(c->lmin, c->lmax);
        if (N != c->nshift) {
            c->nshift = N;
            c->s.nshift = N;
            invalidate_graph(c);
        }
        if (N > c->nshift_cap)
            if (ld_status st = bind_shift_state(c, std::max(N, 2 * c->nshift_cap))) return st;
    }
    c->sigma.assign(c->nshift, 0.0);
    c->alpha.assign(c->nshift, 0.0);
    if (ld::hht_log_nodes(c->lmin, c->lmax, c->nshift, c->sigma.data(), c->alpha.data()) != 0)
        return fail(LD_EINVAL, "bad spectral interval [%g, %g]", c->lmin, c->lmax);
    c->cert = ld::hht_certificate(c->lmin, c->lmax, c->nshift, c->sigma.data(), c->alpha.data());
    std::vector<double2> h(2 * c->nshift_cap, make_double2(0.0, 0.0));
    for (int l = 0; l < c->nshift; ++l) {
        h[l] = make_double2(-c->sigma[l].real(), -c->sigma[l].imag());    // s_l = -sigma_l
        h[c->nshift_cap + l] = make_double2(c->alpha[l].real(), c->alpha[l].imag());
    }
    CUDA_TRY(cudaMemcpy(c->d_nodes.p, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
    return LD_OK;
}

ld_status compute_bounds(ld_ctx *c, const double *field) {
    if (c->user_bounds) {
        c->lmin = c->opt.lambda_min;
        c->lmax = std::max(c->opt.lambda_max, 1.01 * c->opt.lambda_min);
        return LD_OK;
    }
    if (c->kind == LD_CSR) {
        c->lmin = c->csr_lmin;
        c->lmax = c->csr_lmax;
        return LD_OK;
    }
    double k2min = c->kappa2, k2max = c->kappa2;
    if (c->has_field) {
        k2min = INFINITY;
        k2max = -INFINITY;
        for (int64_t i = 0; i < c->n; ++i) {
            k2min = std::min(k2min, c->kappa2 * field[i]);
            k2max = std::max(k2max, c->kappa2 * field[i]);
        }
    }
    grid_bounds(c->kind, c->dims, c->periodic, k2min, k2max, c->mask_any ? c->tau : 0.0, c->scale,
                &c->lmin, &c->lmax);
    if (!(c->lmin > 0.0)) return fail(LD_EINVAL, "spectral lower bound %g is not positive (kappa2 = 0 on a torus?)", c->lmin);
    return LD_OK;
}

void fill_operator(ld_ctx *c) {
    Operator &op = c->s.op;
    op.kind = c->kind;
    op.periodic = c->periodic;
    op.nx = c->dims[0];
    op.ny = c->dims[1];
    op.nz = c->dims[2];
    op.n = c->n;
    op.kappa2 = c->kappa2;
    op.tau = c->tau;
    op.scale = c->kind == LD_CSR ? 1.0 : c->scale;
    ld::set_f32_coefs(op);
    op.field_d = c->d_field_d.as<double>();
    op.field_f = c->d_field_f.as<float>();
    op.mask = c->d_mask.as<uint8_t>();
    op.rowptr = c->d_rowptr.as<int64_t>();
    op.colidx = c->d_colidx.as<int32_t>();
    op.val_d = c->d_val_d.as<double>();
    op.val_f = c->d_val_f.as<float>();
}

// per-vertex diagonal coefficients of field / mask models (see Operator::diag_d)
ld_status fill_diag(ld_ctx *c) {
    Operator &op = c->s.op;
    op.diag_d = nullptr;
    op.diag_f = nullptr;
    const bool grid = c->kind == LD_STENCIL_2D5 || c->kind == LD_STENCIL_3D7;
    if (!grid || (!op.field_d && !op.mask)) return LD_OK;
    if (!c->d_diag_d.p) {
        CUDA_TRY(c->d_diag_d.alloc((size_t)c->n * sizeof(double)));
        CUDA_TRY(c->d_diag_f.alloc((size_t)c->n * sizeof(float)));
    }
    op.diag_d = c->d_diag_d.as<double>();
    op.diag_f = c->d_diag_f.as<float>();
    ENGINE_TRY(ld::engine_fill_diag(op, c->d_diag_d.as<double>(), c->d_diag_f.as<float>(), c->stream));
    return LD_OK;
}

void invalidate_graph(ld_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
}

// Tile groups of the grid engine: tiles are independent solves, so each group
// (tiles g, g + G, ...) iterates on its own stream and one group's end-of-pass
// reduction and last CTAs overlap the other groups' sweeps.
ld_status ensure_groups(ld_ctx *c) {
    // CSR: one group, so that the CTAs of every tile walk the same rows together and the
    // matrix rows each of them reads come from L2 after the first
    const int want = c->kind == LD_CSR ? 1 : std::min(c->ntiles, (int)ld_ctx::kMaxGroups);
    if (c->ngroups == want) return LD_OK;
    if (!c->gfork) CUDA_TRY(cudaEventCreateWithFlags(&c->gfork, cudaEventDisableTiming));
    for (int g = 0; g < want; ++g) {
        if (!c->gstream[g]) CUDA_TRY(cudaStreamCreateWithFlags(&c->gstream[g], cudaStreamNonBlocking));
        if (!c->gjoin[g]) CUDA_TRY(cudaEventCreateWithFlags(&c->gjoin[g], cudaEventDisableTiming));
    }
    c->ngroups = want;
    return LD_OK;
}

// The colour array is read by every tile's pass.  With several tiles per pass its lines are
// evicted by the streamed vectors between one tile's read and the next (on the 1024^2 Matern
// the colours reached DRAM once per tile, 7 % of the pass traffic), so the captured kernels
// mark it persisting in L2 (best effort: skipped where the device offers no persisting L2).
void colour_persistence(ld_ctx *c, cudaGraph_t g) {
    if (c->ntiles < 2 || !c->d_colour.p) return;
    int dev = 0, maxp = 0, maxw = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess ||
        maxp <= 0 || maxw <= 0) {
        cudaGetLastError();
        return;
    }
    const size_t bytes = std::min(c->d_colour.bytes, (size_t)maxw);
    size_t lim = 0;
    if (cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize) != cudaSuccess) lim = 0;
    const size_t want = std::min(bytes, (size_t)maxp);
    if (lim < want) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess ||
            cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    if (lim == 0) return;
    cudaLaunchAttributeValue v{};
    v.accessPolicyWindow.base_ptr = c->d_colour.p;
    v.accessPolicyWindow.num_bytes = bytes;
    v.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)lim / (double)bytes);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess) {
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributeAccessPolicyWindow, &v);
        }
    }
    cudaGetLastError();
    c->l2_persist = true;
}

ld_status ensure_graph(ld_ctx *c) {
    if (c->graph && c->graph_chunk == c->chunk) return LD_OK;
    invalidate_graph(c);
    if (ld_status st = ensure_groups(c)) return st;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int err = 0;
    const int G = c->ngroups;
    if (G <= 1) {
        for (int j = 0; j < c->chunk && !err; ++j) err = ld::engine_iteration(c->s, j & 1, c->stream);
    } else {
        err = (int)cudaEventRecord(c->gfork, c->stream);
        for (int gi = 0; gi < G && !err; ++gi) {
            err = (int)cudaStreamWaitEvent(c->gstream[gi], c->gfork, 0);
            Solve sg = c->s;
            sg.tile0 = gi;
            sg.tstride = G;
            for (int j = 0; j < c->chunk && !err; ++j) err = ld::engine_iteration(sg, j & 1, c->gstream[gi]);
            if (!err) err = (int)cudaEventRecord(c->gjoin[gi], c->gstream[gi]);
            if (!err) err = (int)cudaStreamWaitEvent(c->stream, c->gjoin[gi], 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (err) {
        if (g) cudaGraphDestroy(g);
        return fail(LD_ECUDA, "capture: %s", ld::engine_error_string(err));
    }
    if (e2 != cudaSuccess) return fail(LD_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
    colour_persistence(c, g);
    cudaError_t e3 = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        c->graph = nullptr;
        return fail(LD_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));
    }
    c->graph_chunk = c->chunk;
    return LD_OK;
}

void fill_info(const ld_ctx *c, ld_info *info, ld_status st, int iters, float ms, int64_t launches,
               double iter_ms = 0.0, int64_t tile_iters = 0) {
    if (!info) return;
    info->iter_ms = iter_ms;
    info->tile_iters = tile_iters;
    info->vertex_tile_iters = c->n * tile_iters;
    info->status = st;
    info->n_colours = c->ncolours;
    info->n_shifts = c->nshift;
    info->iters = iters;
    info->tile_width = c->T;
    info->engine = c->engine;
    info->lambda_min = c->lmin;
    info->lambda_max = c->lmax;
    info->quad_cert = c->cert;
    info->ms = ms;
    info->gpu_launches = launches;
    const bool lattice2d = c->s.op.kind == ld::KIND_2D5 || c->s.op.kind == ld::KIND_2D13_SQ;
    info->bulk_rows = c->engine == 1 && lattice2d && !c->mf ? c->s.bulk : -1;
    info->reliable_updates = 0;
    info->rel_resid_max = -1.0;
    info->pass_words = -1;
    if (c->engine == 1 && !c->mf && !c->is_batch)
        info->pass_words = (c->s.lean ? 4 : c->kind == LD_CSR ? 8 : 6) + (c->s.keep_x0 ? 2 : 0);
}

// entry points a matrix-free context does not support (they need the matrix itself)
#define REJECT_MATFREE(c)                                                                     \
    do {                                                                                      \
        if ((c)->mf) return fail(LD_EUNSUPPORTED, "matrix-free context: no matrix to apply, " \
                                                  "re-parametrise or select a distance on");  \
    } while (0)

// matrix-free solve over colours [cb, ce); out[0] = sum of the terms, out[1] = sum of the
// seed projections v^T Q^{-1} v; keep_x keeps the seed solutions for ld_grad
ld_status run_matfree(ld_ctx *c, int cb, int ce, bool keep_x, double out[2], ld_info *info) {
    Range range("ld matrix-free solve");
    ld::MatfreeStats ms{};
    std::vector<double> terms(std::max(ce - cb, 0)), seeds(terms.size());
    const int max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 100000;
    ld::MatfreeJob job;
    job.cb = cb;
    job.ce = ce;
    job.n_shifts = c->nshift;
    job.keep_x = keep_x;
    c->have_x0 = false;
    const ld_status st = (ld_status)ld::matfree_solve(c->mf, job, c->sigma.data(), c->alpha.data(), c->tol,
                                                      max_iter, c->stream, terms.data(), seeds.data(), &ms);
    fill_info(c, info, st, ms.iters, ms.ms, ms.launches, ms.ms, ms.column_iters);
    if (st != LD_OK) return st;
    double sum = 0.0, ssum = 0.0;
    for (int k = 0; k < ce - cb; ++k) {
        c->mf_terms[cb + k] = terms[k];
        c->mf_seeds[cb + k] = seeds[k];
        sum += terms[k];
        ssum += seeds[k];
    }
    if (!std::isfinite(sum)) return fail(LD_ENUMERIC, "non-finite log det");
    out[0] = sum;
    out[1] = ssum;
    c->solved = true;
    c->have_x0 = keep_x;
    c->last_cb = cb;
    c->last_ce = ce;
    return LD_OK;
}

// f(Q) V on a matrix-free context: the vector form with the caller's product; yweight
// pairs with the context's shifts (log: the context's weights)
ld_status matfree_funmv(ld_ctx *c, int ncols, const double *V, double *Y, ld_info *info,
                        const std::complex<double> *yweight) {
    Range range("ld matrix-free vector form");
    ld::MatfreeStats ms{};
    std::vector<double> terms(ncols), seeds(ncols);
    const int max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 100000;
    ld::MatfreeJob job;
    job.rhs = V;
    job.ncols = ncols;
    job.yweight = yweight;
    job.y_out = Y;
    job.n_shifts = c->nshift;
    c->have_x0 = false;   // the vector form overwrites the kept seed solutions' buffers
    const ld_status st = (ld_status)ld::matfree_solve(c->mf, job, c->sigma.data(), c->alpha.data(), c->tol,
                                                      max_iter, c->stream, terms.data(), seeds.data(), &ms);
    fill_info(c, info, st, ms.iters, ms.ms, ms.launches, ms.ms, ms.column_iters);
    return st;
}

// grad[k] = d log det / d eta_{ids[k]} over the seed solutions kept by the last solve
ld_status matfree_grad(ld_ctx *c, int n_params, const int *ids, double *grad) {
    if (!c->have_x0) return fail(LD_EINVAL, "no seed solutions saved: run ld_logdet on a keep_x0 context first");
    std::vector<double> g(n_params);
    int rc = 0;
    const ld_status st = (ld_status)ld::matfree_grad(c->mf, n_params, ids, c->mf_dfn, c->mf_duser, c->stream,
                                                     g.data(), &rc);
    if (st != LD_OK) return st;
    for (int k = 0; k < n_params; ++k) {
        if (!std::isfinite(g[k])) return fail(LD_ENUMERIC, "non-finite gradient");
        grad[k] = g[k];
    }
    return LD_OK;
}

// One probed solve over colours [cb, ce).  On LD_OK, result[0..1] hold
// sum of terms and sum of seed projections on the device and in *out.
ld_status run_solve(ld_ctx *c, int cb, int ce, bool keep_x0, double out[2], ld_info *info) {
    Range range("ld solve");
    int64_t launches = 0;
    int iters = 0;
    float ms = 0.f;
    // reliable updates (grid engine): x kept as x_hi (FP64) + x_lo, residual replaced
    // by v - Q x_hi whenever a column's residual norm fell by reliable_delta
    const bool ru = c->opt.reliable_delta > 0.0 && c->engine == 1;
    if (ru) keep_x0 = true;
    if (ru && !c->d_xhi.p) CUDA_TRY(c->d_xhi.alloc((size_t)c->ntiles * c->n * c->T * sizeof(double)));
    if (keep_x0 && !c->d_norm2.p) CUDA_TRY(c->d_norm2.alloc((size_t)c->ncols * sizeof(double)));
    double *want_xhi = ru ? c->d_xhi.as<double>() : nullptr;
    if (c->s.xhi != want_xhi) {
        c->s.xhi = want_xhi;
        invalidate_graph(c);
    }
    if (ru) CUDA_TRY(cudaMemsetAsync(c->d_xhi.p, 0, c->d_xhi.bytes, c->stream));
    int updates = 0;
    std::vector<double> rmax, h_rho(c->ncols), h_norm2(c->ncols);
    std::vector<int32_t> h_act(c->ncols);
    if (ru) {
        rmax.assign(c->ncols, 0.0);
        for (int col = cb; col < ce; ++col) rmax[col] = std::sqrt(c->class_size[col]);
    }
    if (keep_x0 && !c->d_x.p) {
        const size_t vb = (size_t)c->ntiles * c->n * c->T * (c->opt.precision == LD_FP64 ? 8 : 4);
        CUDA_TRY(c->d_x.alloc(vb));
        c->s.x = c->d_x.p;
        invalidate_graph(c);
    }
    const int want_x0 = keep_x0 ? 1 : 0;
    if (c->s.keep_x0 != want_x0) {
        c->s.keep_x0 = want_x0;
        invalidate_graph(c);
    }
    // the lean lattice pass (four state words per vertex and column) wherever it applies;
    // the stored-w pass otherwise (FP64, other kinds, the Matern kind with a kept x0)
    const int want_lean = c->engine == 1 && c->opt.lattice_pass == 0 ? ld::engine_lean_x(c->s, keep_x0) : 0;
    if (c->s.lean != want_lean || (want_lean && c->lean_plan_x0 != want_x0)) {
        c->s.lean = want_lean;
        ld::engine_plan(c->s);           // the lean plan's occupancy depends on keep_x0
        c->lean_plan_x0 = want_x0;
        const bool codes = want_lean && c->kind != LD_STENCIL_3D7;   // the 3D pass reads colours
        if (codes && !c->lane_built) {
            CUDA_TRY(c->d_lane.alloc(ld::engine_lean_code_bytes(c->s)));
            ENGINE_TRY(ld::engine_lean_codes(c->s, c->d_lane.as<uint8_t>(), c->stream));
            c->lane_built = true;
        }
        c->s.lane = codes ? c->d_lane.as<uint8_t>() : nullptr;
        invalidate_graph(c);
    }
    c->have_x0 = false;
    c->solved = false;
    const int max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 100000;
    CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    ENGINE_TRY(ld::engine_init(c->s, cb, ce, c->stream));
    launches += 3;
    ld_status st = LD_OK;
    double iter_ms = 0.0;
    if (c->engine == 2) {
        CUDA_TRY(cudaEventRecord(c->ev2, c->stream));
        ENGINE_TRY(ld::engine_cta_solve(c->s, max_iter, c->stream));
        CUDA_TRY(cudaEventRecord(c->ev3, c->stream));
        launches += 1;
        CUDA_TRY(cudaMemcpyAsync(c->h_pinned, c->s.remaining, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->h_pinned + 1, c->s.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, c->ev2, c->ev3));
        iter_ms += e;
    } else if (!ru) {
        if (ld_status g = ensure_graph(c)) return g;
        // One chunk queued ahead of the host: chunk k + 1 is launched before the host waits
        // for chunk k's convergence count (pinned slot k mod 2), so the stream never drains
        // between chunks.  A chunk launched after the solve converged finds every tile done
        // and its kernels return at once.
        int done_iters = 0, last = 0;
        auto launch_chunk = [&](int slot) -> ld_status {
            CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
            CUDA_TRY(cudaMemcpyAsync(c->h_pinned + 2 * slot, c->s.remaining, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     c->stream));
            CUDA_TRY(cudaMemcpyAsync(c->h_pinned + 2 * slot + 1, c->s.status, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaEventRecord(c->evc[slot], c->stream));
            // one launch per tile group and pass (two on CSR: the step and the product)
            launches += (int64_t)c->chunk * std::max(c->ngroups, 1) * (c->kind == LD_CSR ? 2 : 1);
            done_iters += c->chunk;
            return LD_OK;
        };
        CUDA_TRY(cudaEventRecord(c->ev2, c->stream));
        if (ld_status g = launch_chunk(0)) return g;
        for (int k = 0;; ++k) {
            const int slot = k & 1;
            const bool more = done_iters < max_iter;
            if (more)
                if (ld_status g = launch_chunk(slot ^ 1)) return g;
            CUDA_TRY(cudaEventSynchronize(c->evc[slot]));
            last = slot;
            if (c->h_pinned[2 * slot] <= 0 || c->h_pinned[2 * slot + 1] != 0 || !more) break;
        }
        // passes' time: from the first chunk to the end of the one that finished the solve
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, c->ev2, c->evc[last]));
        iter_ms += e;
        c->h_pinned[0] = c->h_pinned[2 * last];
        c->h_pinned[1] = c->h_pinned[2 * last + 1];
    } else {
        if (ld_status g = ensure_graph(c)) return g;
        int done_iters = 0;
        for (;;) {
            CUDA_TRY(cudaEventRecord(c->ev2, c->stream));
            CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
            CUDA_TRY(cudaEventRecord(c->ev3, c->stream));
            // one launch per tile group and pass (two on CSR: the step and the product)
            launches += (int64_t)c->chunk * std::max(c->ngroups, 1) * (c->kind == LD_CSR ? 2 : 1);
            done_iters += c->chunk;
            CUDA_TRY(cudaMemcpyAsync(c->h_pinned, c->s.remaining, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(c->h_pinned + 1, c->s.status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            if (ru) {
                CUDA_TRY(cudaMemcpyAsync(h_rho.data(), c->s.rho, c->ncols * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                CUDA_TRY(cudaMemcpyAsync(h_act.data(), c->s.col_active, c->ncols * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            }
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            float e = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&e, c->ev2, c->ev3));
            iter_ms += e;
            if (c->h_pinned[0] <= 0 || c->h_pinned[1] != 0 || done_iters >= max_iter) break;
            if (ru) {
                // chunks hold an even number of passes: the next pass reads set 0, which
                // holds r_k beside x_k = x_hi + x_lo
                bool fire = false;
                for (int col = cb; col < ce && !fire; ++col)
                    fire = h_act[col] && std::sqrt(h_rho[col]) < c->opt.reliable_delta * rmax[col];
                if (fire) {
                    ENGINE_TRY(ld::engine_true_residual(c->s, 0, cb, ce, 1, c->d_norm2.as<double>(), c->stream));
                    launches += 3;
                    ++updates;
                    CUDA_TRY(cudaMemcpyAsync(h_norm2.data(), c->d_norm2.p, c->ncols * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                    CUDA_TRY(cudaStreamSynchronize(c->stream));
                    for (int col = cb; col < ce; ++col) rmax[col] = std::sqrt(h_norm2[col]);
                }
            }
        }
    }
    const int dev_status = c->h_pinned[1];
    const int remaining = c->h_pinned[0];
    double rel_resid = -1.0;
    if (c->s.keep_x0) {
        ENGINE_TRY(ld::engine_flush_x(c->s, c->stream));
        launches += 1;
        // true seed residuals (folding x_lo into x_hi first under reliable updates)
        ENGINE_TRY(ld::engine_true_residual(c->s, 0, cb, ce, 0, c->d_norm2.as<double>(), c->stream));
        launches += ru ? 3 : 2;
        CUDA_TRY(cudaMemcpyAsync(h_norm2.data(), c->d_norm2.p, c->ncols * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    ENGINE_TRY(ld::engine_finish(c->s, cb, ce, c->stream));
    launches += 1;
    CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    CUDA_TRY(cudaMemcpyAsync(out, c->s.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    std::vector<int32_t> it(c->ncols);
    CUDA_TRY(cudaMemcpyAsync(it.data(), c->s.col_iters, c->ncols * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    for (int v : it) iters = std::max(iters, v);
    int64_t tile_iters = 0;
    for (int t = 0; t < c->ntiles; ++t) {
        int m = 0;
        for (int k = 0; k < c->T; ++k) m = std::max(m, it[t * c->T + k]);
        tile_iters += m;
    }
    if (dev_status == ld::DEV_NOTSPD) st = fail(LD_ENOTSPD, "p^T Q p <= 0: Q is not SPD");
    else if (dev_status == ld::DEV_NUMERIC) st = fail(LD_ENUMERIC, "non-finite CG scalar");
    else if (dev_status == ld::DEV_TIMEOUT) st = fail(LD_ETIMEOUT, "device wait timed out");
    else if (dev_status != 0) st = fail(LD_ECUDA, "device status %d", dev_status);
    else if (remaining > 0) st = fail(LD_ENOTCONV, "%d tiles not converged after %d iterations", remaining, iters);
    else if (!std::isfinite(out[0])) st = fail(LD_ENUMERIC, "non-finite log det");
    if (c->s.keep_x0) {
        rel_resid = 0.0;
        for (int col = cb; col < ce; ++col)
            if (c->class_size[col] > 0)
                rel_resid = std::max(rel_resid, std::sqrt(h_norm2[col] / c->class_size[col]));
    }
    fill_info(c, info, st, iters, ms, launches, iter_ms, tile_iters);
    if (info) {
        info->reliable_updates = updates;
        info->rel_resid_max = rel_resid;
    }
    if (st == LD_OK) {
        c->have_x0 = keep_x0;
        c->solved = true;
        c->last_cb = cb;
        c->last_ce = ce;
    }
    return st;
}

// ---------------------------------------------------------------- tile-width autotuner
// For large grid-engine problems created with tile_width = 0, a few CG passes are
// timed for every candidate tile width (trial contexts sharing the colouring) and
// the fastest is kept, per (kind, precision, boundary, dims, colours).  Results are
// cached for the process and, when LD_AUTOTUNE_CACHE names a file, in that JSON
// file ({"key": tile_width, ...}).
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const ld_matrix *Q, int precision, int lattice_pass, int ncolours) {
    std::ostringstream k;
    k << Q->kind << ":" << precision << (lattice_pass ? "w" : "") << ":" << (Q->periodic ? 1 : 0) << ":" << Q->dims[0] << "x"
      << Q->dims[1] << "x" << (Q->kind == LD_STENCIL_3D7 ? Q->dims[2] : 1) << ":" << ncolours
      << (Q->kappa2_field ? ":field" : "") << (Q->obs_mask ? ":mask" : "");
    if (Q->kind == LD_CSR) {
        // a CSR pattern: its size and an FNV-1a hash of 64 sampled row starts and indices
        const int64_t n = Q->n, nnz = Q->rowptr[n];
        uint64_t h = 1469598103934665603ull;
        auto mix = [&h](int64_t v) {
            for (int b = 0; b < 8; ++b) {
                h ^= (uint64_t)((v >> (8 * b)) & 0xff);
                h *= 1099511628211ull;
            }
        };
        for (int q = 0; q < 64; ++q) {
            const int64_t i = n * q / 64;
            mix(Q->rowptr[i]);
            if (nnz > 0) mix(Q->colidx[std::min<int64_t>(nnz - 1, Q->rowptr[i])]);
        }
        k << ":csr" << n << "/" << nnz << "/" << std::hex << h;
    }
    return k.str();
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("LD_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        const size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = s.substr(pos + 1, end - pos - 1);
        const size_t colon = s.find(':', end);
        if (colon == std::string::npos) break;
        const int t = std::atoi(s.c_str() + colon + 1);
        if (t > 0) g_tune[key] = t;
        pos = s.find_first_of(",}", colon);
        if (pos == std::string::npos) break;
    }
}

void tune_save_locked() {
    const char *path = std::getenv("LD_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(path);
    f << "{";
    bool first = true;
    for (const auto &kv : g_tune) {
        f << (first ? "" : ", ") << "\"" << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "}\n";
}

int autotune_tile(const ld_matrix *Q, int d, int N, double tol, const ld_options &opt,
                  const std::vector<int32_t> &colour, int ncolours, double csr_lmin, double csr_lmax) {
    const std::string key = tune_key(Q, opt.precision, opt.lattice_pass, ncolours);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    static const int f64[4] = {1, 2, 3, 4};
    static const int f32[4] = {2, 4, 6, 8};
    const int *cand = opt.precision == LD_FP64 ? f64 : f32;
    int best = -1;
    double best_ms = 1e300;
    for (int k = 0; k < 4; ++k) {
        const int T = cand[k];
        const int cols = (ncolours + T - 1) / T * T;
        if (8 * (cols - ncolours) > ncolours) continue;   // more than 1/8 padding
        // each candidate is timed without and with the seed solution kept (log det alone,
        // and the gradient evaluations, which run the passes that also update x): the
        // widths' order differs between the two, and a context serves both
        double per_pass = 0.0;
        bool ok = true;
        for (int kx = 0; kx < 2 && ok; ++kx) {
            ld_options sub = opt;
            sub.tile_width = T;
            sub.colouring = colour.data();
            sub.max_iter = 16;
            sub.chunk_iters = 8;
            sub.engine = 1;
            sub.keep_x0 = kx;
            if (Q->kind == LD_CSR && !(sub.lambda_min > 0.0 && sub.lambda_max > 0.0)) {
                sub.lambda_min = csr_lmin;   // the interval the context computed once
                sub.lambda_max = csr_lmax;
            }
            ld_ctx *t = nullptr;
            if (ld_create(Q, d, N, tol, &sub, &t) != LD_OK) {
                ok = false;
                break;
            }
            double v;
            ld_info info{};
            // usually LD_ENOTCONV after 16 passes: only the timing matters; the second run's
            // (the first pays the graph's upload and the kernels' first launches)
            ld_logdet(t, &v, &info);
            ld_logdet(t, &v, &info);
            ld_destroy(t);
            if (info.iters < 1 || !(info.iter_ms > 0.0)) ok = false;
            else per_pass += info.iter_ms / info.iters;
        }
        if (!ok) continue;
        if (per_pass < best_ms) {
            best_ms = per_pass;
            best = T;
        }
    }
    g_err = "no error";
    if (best > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = best;
        tune_save_locked();
    }
    return best;
}

ld_status check_params(const ld_ctx *c, int n_params, const int *ids) {
    if (n_params < 1 || n_params > 3 || !ids) return fail(LD_EINVAL, "n_params must be 1..3 with ids");
    if (c->mf) {   // the caller's parameters of ld_matfree_set_derivative
        if (!c->mf_dfn) return fail(LD_EINVAL, "matrix-free context without ld_matfree_set_derivative");
        for (int k = 0; k < n_params; ++k)
            if (ids[k] < 0 || ids[k] >= c->mf_nparams)
                return fail(LD_EINVAL, "parameter id %d outside [0, %d)", ids[k], c->mf_nparams);
        return LD_OK;
    }
    for (int k = 0; k < n_params; ++k) {
        const int p = ids[k];
        if (p < LD_P_KAPPA2 || p > LD_P_SCALE) return fail(LD_EINVAL, "unknown parameter id %d", p);
        if (c->kind == LD_CSR && p != LD_P_SCALE) return fail(LD_EUNSUPPORTED, "CSR matrices only have the scale parameter");
        if (c->kind == LD_STENCIL_2D13_SQ && p == LD_P_TAU) return fail(LD_EUNSUPPORTED, "no tau in the Matern kind");
    }
    return LD_OK;
}

}  // namespace

extern "C" {

int ld_abi_version(void) { return LD_ABI_VERSION; }

const char *ld_last_error(void) { return g_err.c_str(); }

ld_status ld_default_options(ld_options *opt) {
    if (!opt) return fail(LD_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof *opt);
    opt->precision = LD_FP64;
    return LD_OK;
}

ld_status ld_create(const ld_matrix *Q, int colouring_distance, int n_shifts, double tol,
                    const ld_options *opt_in, ld_ctx **out) {
    if (!out) return fail(LD_EINVAL, "out is NULL");
    *out = nullptr;
    if (ld_status v = validate_matrix(Q)) return v;
    if (colouring_distance < 0) return fail(LD_EINVAL, "colouring_distance must be >= 0");
    if (n_shifts < 0 || n_shifts > 256) return fail(LD_EINVAL, "n_shifts must be in [0, 256] (0 = automatic)");
    if (!(tol > 0.0 && tol < 1.0)) return fail(LD_EINVAL, "tol must be in (0, 1)");
    ld_options opt;
    ld_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.precision != LD_FP64 && opt.precision != LD_MIXED) return fail(LD_EINVAL, "bad precision");
    if (opt.max_iter < 0) return fail(LD_EINVAL, "max_iter must be >= 0");
    if (opt.engine < 0 || opt.engine > 2) return fail(LD_EINVAL, "engine must be 0, 1 or 2");
    if (opt.chunk_iters < 0 || opt.chunk_iters > 4096) return fail(LD_EINVAL, "chunk_iters out of range");
    if (!(opt.reliable_delta >= 0.0 && opt.reliable_delta < 1.0))
        return fail(LD_EINVAL, "reliable_delta must be in [0, 1)");
    if (opt.lattice_pass < 0 || opt.lattice_pass > 1) return fail(LD_EINVAL, "lattice_pass must be 0 or 1");

    ld_ctx *c = new (std::nothrow) ld_ctx();
    if (!c) return fail(LD_ENOMEM, "host allocation");
    std::unique_ptr<ld_ctx> guard(c);
    c->kind = Q->kind;
    c->periodic = Q->periodic ? 1 : 0;
    c->opt = opt;
    c->distance = colouring_distance;
    c->auto_shift = n_shifts == 0;
    c->nshift = c->auto_shift ? 20 : n_shifts;       // automatic N: set with the nodes
    c->tol = tol;
    c->scale = Q->scale == 0.0 ? 1.0 : Q->scale;
    c->kappa2 = Q->kappa2;
    c->tau = Q->tau;
    c->user_bounds = opt.lambda_min > 0.0 && opt.lambda_max > 0.0;
    if (c->kind == LD_CSR) {
        c->n = Q->n;
    } else {
        c->dims[0] = Q->dims[0];
        c->dims[1] = Q->dims[1];
        c->dims[2] = (Q->kind == LD_STENCIL_3D7) ? Q->dims[2] : 1;
        c->n = grid_n(c->dims);
        if (c->n > ((int64_t)1 << 31) - 1) return fail(LD_EINVAL, "grid too large");
        c->has_field = Q->kappa2_field != nullptr;
        c->has_mask = Q->obs_mask != nullptr;
        if (c->has_mask)
            for (int64_t i = 0; i < c->n && !c->mask_any; ++i) c->mask_any = Q->obs_mask[i] != 0;
    }
    if (c->kind == LD_CSR && !c->user_bounds) {
        int steps = 0;
        const int rc = ld::csr_bounds(c->n, Q->rowptr, Q->colidx, Q->val, c->scale, &c->csr_lmin,
                                      &c->csr_lmax, &steps);
        if (rc == -2)
            return fail(LD_ENOTCONV, "CSR matrix: smallest Lanczos Ritz value not converged after %d "
                                     "steps; pass lambda_min and lambda_max", steps);
        if (rc != 0) return fail(LD_ENOTSPD, "CSR matrix: no positive spectral lower bound (not SPD?)");
    }

    // colouring (Sec. 2.1)
    Range create_range("ld create (colouring, tiling, uploads)");
    c->colour.resize(c->n);
    if (opt.colouring) {
        int mx = -1;
        for (int64_t i = 0; i < c->n; ++i) {
            if (opt.colouring[i] < 0) return fail(LD_EINVAL, "negative colour at %lld", (long long)i);
            mx = std::max(mx, (int)opt.colouring[i]);
            c->colour[i] = opt.colouring[i];
        }
        c->ncolours = mx + 1;
    } else if (c->kind == LD_CSR) {
        c->ncolours = ld::colour_csr(c->n, Q->rowptr, Q->colidx, colouring_distance, c->colour.data());
    } else {
        c->ncolours = ld::colour_grid(c->kind, c->dims, c->periodic, colouring_distance, c->colour.data());
    }
    // tiling: explicit, autotuned (large multi-CTA problems), or the padding rule
    c->T = -1;
    if (opt.tile_width == 0 && opt.engine != 2 && c->n >= 65536)
        c->T = autotune_tile(Q, colouring_distance, n_shifts, tol, opt, c->colour, c->ncolours, c->csr_lmin,
                             c->csr_lmax);
    if (c->T < 0) c->T = choose_tile(opt.precision, c->ncolours, opt.tile_width);
    if (c->T < 0) return fail(LD_EINVAL, "tile_width %d not available for this precision", opt.tile_width);
    c->ntiles = (c->ncolours + c->T - 1) / c->T;
    c->ncols = c->ntiles * c->T;
    c->class_size.assign(c->ncols, 0.0);
    for (int64_t i = 0; i < c->n; ++i) c->class_size[c->colour[i]] += 1.0;
    if (opt.engine) {
        c->engine = opt.engine;
    } else {
        c->engine = (c->n <= 32768 || (c->ntiles >= 152 && c->n <= 262144)) ? 2 : 1;
    }
    c->chunk = opt.chunk_iters > 0 ? opt.chunk_iters + (opt.chunk_iters & 1) : 16;

    // stream, events
    if (opt.cuda_stream) {
        c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CUDA_TRY(cudaEventCreate(&c->ev0));
    CUDA_TRY(cudaEventCreate(&c->ev1));
    CUDA_TRY(cudaEventCreate(&c->ev2));
    CUDA_TRY(cudaEventCreate(&c->ev3));
    CUDA_TRY(cudaEventCreate(&c->evc[0]));
    CUDA_TRY(cudaEventCreate(&c->evc[1]));
    CUDA_TRY(cudaMallocHost((void **)&c->h_pinned, 4 * sizeof(int32_t)));

    // device copies of the problem
    const bool f32 = opt.precision == LD_MIXED;
    CUDA_TRY(c->d_colour.alloc(c->n * sizeof(int32_t)));
    CUDA_TRY(cudaMemcpy(c->d_colour.p, c->colour.data(), c->n * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (c->has_field) {
        std::vector<float> ff(c->n);
        for (int64_t i = 0; i < c->n; ++i) ff[i] = (float)Q->kappa2_field[i];
        CUDA_TRY(c->d_field_d.alloc(c->n * sizeof(double)));
        CUDA_TRY(cudaMemcpy(c->d_field_d.p, Q->kappa2_field, c->n * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(c->d_field_f.alloc(c->n * sizeof(float)));
        CUDA_TRY(cudaMemcpy(c->d_field_f.p, ff.data(), c->n * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (c->has_mask) {
        CUDA_TRY(c->d_mask.alloc(c->n));
        CUDA_TRY(cudaMemcpy(c->d_mask.p, Q->obs_mask, c->n, cudaMemcpyHostToDevice));
    }
    if (c->kind == LD_CSR) {
        const int64_t nnz = Q->rowptr[c->n];
        std::vector<double> vd(nnz);
        std::vector<float> vf(nnz);
        for (int64_t e = 0; e < nnz; ++e) {
            vd[e] = c->scale * Q->val[e];
            vf[e] = (float)vd[e];
        }
        CUDA_TRY(c->d_rowptr.alloc((c->n + 1) * sizeof(int64_t)));
        CUDA_TRY(cudaMemcpy(c->d_rowptr.p, Q->rowptr, (c->n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        CUDA_TRY(c->d_colidx.alloc(std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
        CUDA_TRY(cudaMemcpy(c->d_colidx.p, Q->colidx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
        CUDA_TRY(c->d_val_d.alloc(std::max<int64_t>(nnz, 1) * sizeof(double)));
        CUDA_TRY(cudaMemcpy(c->d_val_d.p, vd.data(), nnz * sizeof(double), cudaMemcpyHostToDevice));
        if (f32) {
            CUDA_TRY(c->d_val_f.alloc(std::max<int64_t>(nnz, 1) * sizeof(float)));
            CUDA_TRY(cudaMemcpy(c->d_val_f.p, vf.data(), nnz * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    // work buffers
    const size_t w = f32 ? 4 : 8;
    const size_t vb = (size_t)c->ntiles * c->n * c->T * w;
    for (int k = 0; k < 2; ++k) {
        CUDA_TRY(c->d_r[k].alloc(vb));
        CUDA_TRY(c->d_w[k].alloc(vb));
        CUDA_TRY(c->d_p[k].alloc(vb));
    }
    const int N = c->nshift, C = c->ncols;
    CUDA_TRY(c->d_colscal.alloc((size_t)8 * C * sizeof(double)));
    CUDA_TRY(c->d_colint.alloc((size_t)2 * C * sizeof(int32_t)));
    CUDA_TRY(c->d_tile.alloc((size_t)(3 * c->ntiles + 2) * sizeof(int32_t)));
    CUDA_TRY(c->d_terms.alloc((size_t)(2 * C + 8) * sizeof(double)));
    CUDA_TRY(cudaMemcpy(c->d_terms.as<double>() + C, c->class_size.data(), C * sizeof(double), cudaMemcpyHostToDevice));

    Solve &s = c->s;
    fill_operator(c);
    if (ld_status st = fill_diag(c)) return st;
    s.T = c->T;
    s.ntiles = c->ntiles;
    s.ncols = C;
    s.nshift = N;
    s.precision = f32 ? 1 : 0;
    s.keep_x0 = 0;
    s.tol = tol;
    s.colour = c->d_colour.as<int32_t>();
    for (int k = 0; k < 2; ++k) {
        s.rbuf[k] = c->d_r[k].p;
        s.wbuf[k] = c->d_w[k].p;
        s.pbuf[k] = c->d_p[k].p;
    }
    s.x = nullptr;
    double *cs = c->d_colscal.as<double>();
    s.rho = cs;
    s.alpha = cs + C;
    s.beta = cs + 2 * C;
    s.alpha_prev = cs + 3 * C;
    s.beta_prev = cs + 4 * C;
    s.vnorm2 = cs + 5 * C;
    s.pi0 = cs + 6 * C;
    s.phi0 = cs + 7 * C;
    s.col_active = c->d_colint.as<int32_t>();
    s.col_iters = s.col_active + C;
    if (ld_status st = bind_shift_state(c, c->auto_shift ? 64 : N)) return st;
    s.tile_done = c->d_tile.as<int32_t>();
    s.tile_ctr = s.tile_done + c->ntiles;
    s.tile_par = s.tile_ctr + c->ntiles;
    s.remaining = s.tile_par + c->ntiles;
    s.status = s.remaining + 1;
    s.terms = c->d_terms.as<double>();
    s.class_size = s.terms + C;
    s.result = s.terms + 2 * C;
    s.lean = 0;
    s.lane = nullptr;
    // the lean 5-point pass forms kappa^2 + tau mask_i from a mask bit in its lane codes
    s.lane_mask = (c->kind == LD_STENCIL_2D5 && c->has_mask && !c->has_field) ? 1 : 0;
    int bpt_max = 0;
    for (int kx = 0; kx < 2; ++kx) {   // the lean lattice pass plans its own strips
        Solve t = s;
        t.keep_x0 = kx;
        t.lean = ld::engine_lean_x(s, kx != 0);
        if (t.lean && c->engine == 1 && opt.lattice_pass == 0) bpt_max = std::max(bpt_max, ld::engine_plan(t));
    }
    bpt_max = std::max(bpt_max, ld::engine_plan(s));
    const size_t part = std::max<size_t>((size_t)c->ntiles * bpt_max * ld::NDOT * c->T, (size_t)152 * 4 * 3);
    CUDA_TRY(c->d_partial.alloc(part * sizeof(double)));
    s.partial = c->d_partial.as<double>();
    CUDA_TRY(cudaMemset(c->d_tile.p, 0, c->d_tile.bytes));

    if (ld_status b = compute_bounds(c, Q->kappa2_field)) return b;
    if (ld_status nd = set_nodes(c)) return nd;
    *out = guard.release();
    return LD_OK;
}

ld_status ld_create_matfree(int64_t n, ld_matvec_fn matvec, void *user, const int32_t *colouring,
                            double lambda_min, double lambda_max, int n_shifts, double tol,
                            const ld_options *opt_in, ld_ctx **out) {
    Range range("ld create matrix-free");
    if (!out) return fail(LD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!matvec || !colouring) return fail(LD_EINVAL, "matvec and colouring must be non-NULL");
    if (n <= 0 || n > ((int64_t)1 << 40)) return fail(LD_EINVAL, "n must be in [1, 2^40]");
    if (n_shifts < 1 || n_shifts > 256) return fail(LD_EINVAL, "n_shifts must be in [1, 256]");
    if (!(tol > 0.0 && tol < 1.0)) return fail(LD_EINVAL, "tol must be in (0, 1)");
    if (!(lambda_min > 0.0) || !(lambda_max > lambda_min) || !std::isfinite(lambda_max))
        return fail(LD_EINVAL, "need 0 < lambda_min < lambda_max (finite)");
    ld_options opt;
    ld_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.precision != LD_FP64) return fail(LD_EUNSUPPORTED, "matrix-free contexts run in FP64");
    if (opt.max_iter < 0) return fail(LD_EINVAL, "max_iter must be >= 0");
    int mx = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (colouring[i] < 0 || colouring[i] >= n) return fail(LD_EINVAL, "colour at %lld outside [0, n)", (long long)i);
        mx = std::max(mx, (int)colouring[i]);
    }
    ld_ctx *c = new (std::nothrow) ld_ctx();
    if (!c) return fail(LD_ENOMEM, "host allocation");
    std::unique_ptr<ld_ctx> guard(c);
    c->kind = LD_MATFREE;
    c->n = n;
    c->dims[0] = (int32_t)std::min<int64_t>(n, INT32_MAX);
    c->opt = opt;
    c->nshift = n_shifts;
    c->tol = tol;
    c->user_bounds = true;
    c->colour.assign(colouring, colouring + n);
    c->ncolours = mx + 1;
    c->ncols = c->ncolours;
    c->T = 0;
    c->engine = 3;
    c->mf_terms.assign(c->ncolours, 0.0);
    c->mf_seeds.assign(c->ncolours, 0.0);
    c->lmin = lambda_min;
    c->lmax = lambda_max;
    c->sigma.assign(n_shifts, 0.0);
    c->alpha.assign(n_shifts, 0.0);
    if (ld::hht_log_nodes(c->lmin, c->lmax, n_shifts, c->sigma.data(), c->alpha.data()) != 0)
        return fail(LD_EINVAL, "bad spectral interval [%g, %g]", c->lmin, c->lmax);
    c->cert = ld::hht_certificate(c->lmin, c->lmax, n_shifts, c->sigma.data(), c->alpha.data());
    if (opt.cuda_stream) {
        c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const int e = ld::matfree_create(&c->mf, n, c->colour.data(), c->ncolours, n_shifts,
                                     reinterpret_cast<void *>(matvec), user);
    if (e != 0)
        return fail(e == (int)cudaErrorMemoryAllocation ? LD_ENOMEM : LD_ECUDA, "matrix-free buffers: %s",
                    cudaGetErrorString((cudaError_t)e));
    *out = guard.release();
    return LD_OK;
}

ld_status ld_matfree_set_derivative(ld_ctx *c, ld_dmatvec_fn dmatvec, void *user, int n_params) {
    if (!c) return fail(LD_EINVAL, "ctx is NULL");
    if (!c->mf) return fail(LD_EINVAL, "not a matrix-free context");
    if (!dmatvec) {
        c->mf_dfn = nullptr;
        c->mf_duser = nullptr;
        c->mf_nparams = 0;
        return LD_OK;
    }
    if (n_params < 1 || n_params > 3) return fail(LD_EINVAL, "n_params must be in [1, 3]");
    c->mf_dfn = reinterpret_cast<void *>(dmatvec);
    c->mf_duser = user;
    c->mf_nparams = n_params;
    return LD_OK;
}

ld_status ld_set_params(ld_ctx *c, double kappa2, double tau, double scale) {
    if (!c) return fail(LD_EINVAL, "ctx is NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    REJECT_MATFREE(c);
    if (c->kind == LD_CSR) return fail(LD_EUNSUPPORTED, "CSR contexts have fixed values");
    if (!std::isfinite(kappa2) || kappa2 < 0.0) return fail(LD_EINVAL, "kappa2 must be finite and >= 0");
    if (!std::isfinite(tau) || tau < 0.0) return fail(LD_EINVAL, "tau must be finite and >= 0");
    if (scale == 0.0) scale = 1.0;
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(LD_EINVAL, "scale must be > 0");
    c->kappa2 = kappa2;
    c->tau = tau;
    c->scale = scale;
    fill_operator(c);
    if (ld_status st = fill_diag(c)) return st;
    invalidate_graph(c);
    c->solved = false;
    c->have_x0 = false;
    if (!c->user_bounds) {
        std::vector<double> field;
        if (c->has_field) {
            field.resize(c->n);
            CUDA_TRY(cudaMemcpy(field.data(), c->d_field_d.p, c->n * sizeof(double), cudaMemcpyDeviceToHost));
        }
        if (ld_status b = compute_bounds(c, field.empty() ? nullptr : field.data())) return b;
    }
    return set_nodes(c);
}

ld_status ld_logdet(ld_ctx *c, double *logdet, ld_info *info) {
    if (!c || !logdet) return fail(LD_EINVAL, "ctx and logdet must be non-NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    double out[2];
    ld_status st = c->mf ? run_matfree(c, 0, c->ncolours, c->opt.keep_x0 != 0, out, info)
                         : run_solve(c, 0, c->ncolours, c->opt.keep_x0 != 0, out, info);
    if (st == LD_OK) *logdet = out[0];
    return st;
}

ld_status ld_grad(ld_ctx *c, int n_params, const int *ids, double *grad) {
    if (!c || !grad) return fail(LD_EINVAL, "ctx and grad must be non-NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    if (ld_status v = check_params(c, n_params, ids)) return v;
    if (c->mf) return matfree_grad(c, n_params, ids, grad);
    if (!c->have_x0) return fail(LD_EINVAL, "no seed solutions saved: run ld_logdet on a keep_x0 context first");
    double *d_out = c->s.result + 2;
    ENGINE_TRY(ld::engine_grad_params(c->s, n_params, ids, d_out, c->stream));
    double h[3];
    CUDA_TRY(cudaMemcpyAsync(h, d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n_params; ++k) {
        if (!std::isfinite(h[k])) return fail(LD_ENUMERIC, "non-finite gradient");
        // a CSR matrix holds s Q0: its kernel summed (Q v)^T x, d/ds takes Q0 = Q / s
        grad[k] = c->kind == LD_CSR ? h[k] / c->scale : h[k];
    }
    return LD_OK;
}

ld_status ld_logdet_grad(ld_ctx *c, int n_params, const int *ids, double *logdet, double *grad,
                         ld_info *info) {
    if (!c || !logdet || !grad) return fail(LD_EINVAL, "ctx, logdet and grad must be non-NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    if (ld_status v = check_params(c, n_params, ids)) return v;
    if (c->mf) {
        double out[2];
        ld_status st = run_matfree(c, 0, c->ncolours, true, out, info);
        if (st != LD_OK) return st;
        if (ld_status g = matfree_grad(c, n_params, ids, grad)) return g;
        if (info) info->gpu_launches += 2 * n_params;
        *logdet = out[0];
        return LD_OK;
    }
    // d/d kappa2 of a scalar-kappa2 5/7-point grid is tr(Q^{-1}) * scale: the projected
    // seed sum v^T Q^{-1} v needs no stored seed vectors.
    bool projected = (c->kind == LD_STENCIL_2D5 || c->kind == LD_STENCIL_3D7) && !c->has_field;
    for (int k = 0; k < n_params; ++k) projected = projected && ids[k] == LD_P_KAPPA2;
    double out[2];
    ld_status st = run_solve(c, 0, c->ncolours, !projected || c->opt.keep_x0, out, info);
    if (st != LD_OK) return st;
    if (projected) {
        for (int k = 0; k < n_params; ++k) grad[k] = c->scale * out[1];
    } else {
        ld_status g = ld_grad(c, n_params, ids, grad);
        if (info) info->gpu_launches += 2;
        if (g != LD_OK) return g;
    }
    *logdet = out[0];
    return LD_OK;
}

ld_status ld_logdet_partial(ld_ctx *c, int cb, int ce, double *partial, ld_info *info) {
    if (!c || !partial) return fail(LD_EINVAL, "ctx and partial must be non-NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    if (cb < 0 || ce < cb || ce > c->ncolours) return fail(LD_EINVAL, "colour range [%d, %d) outside [0, %d)", cb, ce, c->ncolours);
    double out[2];
    ld_status st = c->mf ? run_matfree(c, cb, ce, c->opt.keep_x0 != 0, out, info)
                         : run_solve(c, cb, ce, c->opt.keep_x0 != 0, out, info);
    if (st == LD_OK) *partial = out[0];
    return st;
}

ld_status ld_column_terms(const ld_ctx *c, double *terms, double *seed) {
    if (!c || !terms) return fail(LD_EINVAL, "ctx and terms must be non-NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    if (!c->solved) return fail(LD_EINVAL, "no completed solve on this context");
    if (c->mf) {
        for (int k = 0; k < c->ncolours; ++k) {
            terms[k] = c->mf_terms[k];
            if (seed) seed[k] = c->mf_seeds[k];
        }
        return LD_OK;
    }
    CUDA_TRY(cudaMemcpy(terms, c->s.terms, c->ncolours * sizeof(double), cudaMemcpyDeviceToHost));
    if (seed) CUDA_TRY(cudaMemcpy(seed, c->s.pi0, c->ncolours * sizeof(double), cudaMemcpyDeviceToHost));
    return LD_OK;
}

ld_status ld_get_colouring(const ld_ctx *c, int32_t *colour, int32_t *n_colours) {
    if (!c) return fail(LD_EINVAL, "ctx is NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    if (colour) std::memcpy(colour, c->colour.data(), c->n * sizeof(int32_t));
    if (n_colours) *n_colours = c->ncolours;
    return LD_OK;
}

ld_status ld_get_nodes(const ld_ctx *c, double *sigma, double *alpha, int32_t *n_shifts) {
    if (!c) return fail(LD_EINVAL, "ctx is NULL");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    for (int l = 0; l < c->nshift; ++l) {
        if (sigma) { sigma[2 * l] = c->sigma[l].real(); sigma[2 * l + 1] = c->sigma[l].imag(); }
        if (alpha) { alpha[2 * l] = c->alpha[l].real(); alpha[2 * l + 1] = c->alpha[l].imag(); }
    }
    if (n_shifts) *n_shifts = c->nshift;
    return LD_OK;
}

ld_status ld_apply(ld_ctx *c, int ncols, const double *x, double *y) {
    if (!c || !x || !y || ncols < 1) return fail(LD_EINVAL, "bad arguments");
    if (c->is_batch) return fail(LD_EINVAL, "batched context: use ld_batch_logdet");
    REJECT_MATFREE(c);
    const int T = c->T;
    const int nt = (ncols + T - 1) / T;
    const int64_t n = c->n;
    const bool f32 = c->opt.precision == LD_MIXED;
    const size_t w = f32 ? 4 : 8;
    const size_t elems = (size_t)nt * n * T;
    std::vector<unsigned char> hx(elems * w, 0), hy(elems * w);
    for (int t = 0; t < nt; ++t)
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < T; ++k) {
                const int col = t * T + k;
                const double v = col < ncols ? x[i * ncols + col] : 0.0;
                const size_t q = ((size_t)t * n + i) * T + k;
                if (f32) reinterpret_cast<float *>(hx.data())[q] = (float)v;
                else reinterpret_cast<double *>(hx.data())[q] = v;
            }
    DevBuf dx, dy;
    CUDA_TRY(dx.alloc(elems * w));
    CUDA_TRY(dy.alloc(elems * w));
    CUDA_TRY(cudaMemcpyAsync(dx.p, hx.data(), elems * w, cudaMemcpyHostToDevice, c->stream));
    ENGINE_TRY(ld::engine_apply(c->s.op, f32 ? 1 : 0, T, nt, dx.p, dy.p, c->stream));
    CUDA_TRY(cudaMemcpyAsync(hy.data(), dy.p, elems * w, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int t = 0; t < nt; ++t)
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < T; ++k) {
                const int col = t * T + k;
                if (col >= ncols) continue;
                const size_t q = ((size_t)t * n + i) * T + k;
                y[i * ncols + col] = f32 ? (double)reinterpret_cast<float *>(hy.data())[q]
                                         : reinterpret_cast<double *>(hy.data())[q];
            }
    return LD_OK;
}

// f(Q) V by the vector form of CG-M, for the rational f whose weights (N double2, on the
// device) pair with the context's shifts: log (the context's weights) or z^{-1/2}
static ld_status funmv(ld_ctx *c, int ncols, const double *V, double *Y, ld_info *info,
                       const double2 *weight_dev) {
    Range range("ld vector form");
    if (!c || !V || !Y || ncols < 1) return fail(LD_EINVAL, "bad arguments");
    if (c->is_batch) return fail(LD_EINVAL, "batched context");
    REJECT_MATFREE(c);
    const int T = c->T, N = c->nshift;
    const int nt = (ncols + T - 1) / T, C = nt * T;
    const int64_t n = c->n;
    const bool f32 = c->opt.precision == LD_MIXED;
    const size_t w = f32 ? 4 : 8;
    const size_t elems = (size_t)nt * n * T;
    // host: right-hand sides in the tiled layout, their squared norms
    std::vector<unsigned char> hv(elems * w, 0);
    std::vector<double> norm2(C, 0.0);
    for (int t = 0; t < nt; ++t)
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < T; ++k) {
                const int col = t * T + k;
                const double v = col < ncols ? V[i * ncols + col] : 0.0;
                const size_t q = ((size_t)t * n + i) * T + k;
                if (f32) reinterpret_cast<float *>(hv.data())[q] = (float)v;
                else reinterpret_cast<double *>(hv.data())[q] = v;
                norm2[col] += v * v;
            }
    DevBuf vec[6], cs, ci, sh, sig, tl, part, tm, psig, y;
    for (auto &b : vec) CUDA_TRY(b.alloc(elems * w));
    CUDA_TRY(cs.alloc((size_t)8 * C * sizeof(double)));
    CUDA_TRY(ci.alloc((size_t)2 * C * sizeof(int32_t)));
    CUDA_TRY(sh.alloc((size_t)4 * C * N * sizeof(double2) + (size_t)C * N));
    CUDA_TRY(sig.alloc((size_t)2 * C * N * sizeof(double2)));
    CUDA_TRY(tl.alloc((size_t)(3 * nt + 2) * sizeof(int32_t)));
    CUDA_TRY(tm.alloc((size_t)(2 * C + 8) * sizeof(double)));
    CUDA_TRY(psig.alloc((size_t)C * N * n * sizeof(double2)));
    CUDA_TRY(y.alloc(elems * sizeof(double)));
    Solve s = c->s;
    s.T = T;
    s.ntiles = nt;
    s.ncols = C;
    s.keep_x0 = 0;
    s.x = nullptr;
    s.xhi = nullptr;
    s.weight = weight_dev;
    s.tile0 = 0;
    s.tstride = 1;
    for (int k = 0; k < 2; ++k) {
        s.rbuf[k] = vec[k].p;
        s.wbuf[k] = vec[2 + k].p;
        s.pbuf[k] = vec[4 + k].p;
    }
    double *d = cs.as<double>();
    s.rho = d; s.alpha = d + C; s.beta = d + 2 * C; s.alpha_prev = d + 3 * C;
    s.beta_prev = d + 4 * C; s.vnorm2 = d + 5 * C; s.pi0 = d + 6 * C; s.phi0 = d + 7 * C;
    s.col_active = ci.as<int32_t>();
    s.col_iters = s.col_active + C;
    double2 *z = sh.as<double2>();
    s.zeta = z; s.zeta_prev = z + (size_t)C * N; s.pi = z + (size_t)2 * C * N; s.phi = z + (size_t)3 * C * N;
    s.sh_active = reinterpret_cast<uint8_t *>(z + (size_t)4 * C * N);
    s.asig = sig.as<double2>();
    s.bsig = s.asig + (size_t)C * N;
    s.tile_done = tl.as<int32_t>(); s.tile_ctr = s.tile_done + nt; s.tile_par = s.tile_ctr + nt;
    s.remaining = s.tile_par + nt; s.status = s.remaining + 1;
    s.terms = tm.as<double>(); s.class_size = s.terms + C; s.result = s.terms + 2 * C;
    ld::engine_plan(s);
    CUDA_TRY(part.alloc(std::max<size_t>((size_t)nt * s.bpt * ld::NDOT * T, 1824) * sizeof(double)));
    s.partial = part.as<double>();
    CUDA_TRY(cudaMemsetAsync(tl.p, 0, tl.bytes, c->stream));
    CUDA_TRY(cudaMemsetAsync(sig.p, 0, sig.bytes, c->stream));
    CUDA_TRY(cudaMemcpyAsync(vec[0].p, hv.data(), elems * w, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(vec[2].p, 0, elems * w, c->stream));
    CUDA_TRY(cudaMemsetAsync(vec[4].p, 0, elems * w, c->stream));
    CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(s.class_size), norm2.data(), C * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    ENGINE_TRY(ld::engine_init(s, 0, ncols, c->stream, false));
    ENGINE_TRY(ld::engine_modev(s, 0, 0, psig.as<double2>(), y.as<double>(), c->stream));
    const int max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 100000;
    int it = 0, remaining = 1, status = 0;
    int64_t launches = 5;
    while (it < max_iter && remaining > 0 && status == 0) {
        for (int k = 0; k < 16 && it < max_iter; ++k, ++it) {
            ENGINE_TRY(ld::engine_iteration(s, it & 1, c->stream));
            ENGINE_TRY(ld::engine_modev(s, 1, (it & 1) ^ 1, psig.as<double2>(), y.as<double>(), c->stream));
            launches += 3;
        }
        CUDA_TRY(cudaMemcpyAsync(c->h_pinned, s.remaining, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        remaining = c->h_pinned[0];
        status = c->h_pinned[1];
    }
    CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    std::vector<double> hy(elems);
    CUDA_TRY(cudaMemcpyAsync(hy.data(), y.p, elems * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    ld_status st = LD_OK;
    if (status == ld::DEV_NOTSPD) st = fail(LD_ENOTSPD, "p^T Q p <= 0: Q is not SPD");
    else if (status != 0) st = fail(LD_ENUMERIC, "non-finite CG scalar");
    else if (remaining > 0) st = fail(LD_ENOTCONV, "max_iter reached");
    fill_info(c, info, st, it, ms, launches, ms, 0);
    if (st != LD_OK) return st;
    for (int t = 0; t < nt; ++t)
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < T; ++k) {
                const int col = t * T + k;
                if (col < ncols) Y[i * ncols + col] = hy[((size_t)t * n + i) * T + k];
            }
    return LD_OK;
}

ld_status ld_logmv(ld_ctx *c, int ncols, const double *V, double *Y, ld_info *info) {
    if (!c) return fail(LD_EINVAL, "bad arguments");
    if (c->mf) {
        if (!V || !Y || ncols < 1) return fail(LD_EINVAL, "bad arguments");
        return matfree_funmv(c, ncols, V, Y, info, c->alpha.data());
    }
    return funmv(c, ncols, V, Y, info, c->s.weight);
}

ld_status ld_invsqrt_mv(ld_ctx *c, int ncols, const double *V, double *Y, ld_info *info) {
    if (!c) return fail(LD_EINVAL, "bad arguments");
    if (c->is_batch) return fail(LD_EINVAL, "batched context");
    std::vector<std::complex<double>> sg(c->nshift), be(c->nshift);
    if (ld::hht_invsqrt_nodes(c->lmin, c->lmax, c->nshift, sg.data(), be.data()) != 0)
        return fail(LD_EINVAL, "bad spectral interval [%g, %g]", c->lmin, c->lmax);
    if (c->mf) {   // the same poles as the log nodes, so the context's shifts serve
        if (!V || !Y || ncols < 1) return fail(LD_EINVAL, "bad arguments");
        return matfree_funmv(c, ncols, V, Y, info, be.data());
    }
    std::vector<double2> hw(c->nshift);
    for (int l = 0; l < c->nshift; ++l) hw[l] = make_double2(be[l].real(), be[l].imag());
    DevBuf wd;
    CUDA_TRY(wd.alloc(hw.size() * sizeof(double2)));
    CUDA_TRY(cudaMemcpy(wd.p, hw.data(), hw.size() * sizeof(double2), cudaMemcpyHostToDevice));
    return funmv(c, ncols, V, Y, info, wd.as<double2>());
}

ld_status ld_wait_selftest(int64_t limit_ns) {
    if (limit_ns < 1000 || limit_ns > 10000000000LL) return fail(LD_EINVAL, "limit_ns out of range");
    DevBuf st;
    CUDA_TRY(st.alloc(sizeof(int32_t)));
    CUDA_TRY(cudaMemset(st.p, 0xff, sizeof(int32_t)));
    ENGINE_TRY(ld::engine_wait_selftest((uint64_t)limit_ns, st.as<int32_t>(), nullptr));
    int32_t h = -1;
    CUDA_TRY(cudaMemcpy(&h, st.p, sizeof h, cudaMemcpyDeviceToHost));
    if (h == ld::DEV_TIMEOUT) return fail(LD_ETIMEOUT, "device wait gave up after %lld ns", (long long)limit_ns);
    if (h == ld::DEV_OK) return LD_OK;
    return fail(LD_ECUDA, "self-test kernel did not report (status %d)", h);
}

ld_status ld_hutchinson(ld_ctx *c, int s, const double *Z, double *estimate, double *std_error,
                        double *samples, ld_info *info) {
    if (!c || !Z || !estimate || s < 1) return fail(LD_EINVAL, "bad arguments");
    if (c->is_batch) return fail(LD_EINVAL, "batched context");
    std::vector<double> Y((size_t)c->n * s);
    if (ld_status st = ld_logmv(c, s, Z, Y.data(), info)) return st;
    std::vector<double> q((size_t)s, 0.0);
    for (int64_t i = 0; i < c->n; ++i)
        for (int k = 0; k < s; ++k) q[(size_t)k] += Z[(size_t)i * s + k] * Y[(size_t)i * s + k];
    double mean = 0.0;
    for (double v : q) mean += v;
    mean /= s;
    double var = 0.0;
    for (double v : q) var += (v - mean) * (v - mean);
    *estimate = mean;
    if (std_error) *std_error = s > 1 ? std::sqrt(var / (s - 1) / s) : 0.0;
    if (samples) std::copy(q.begin(), q.end(), samples);
    return LD_OK;
}

ld_status ld_select_distance(ld_ctx *c, int64_t j, double eps, int max_d, int32_t *distance,
                             double *profile, ld_info *info) {
    if (!c || !distance) return fail(LD_EINVAL, "bad arguments");
    if (c->is_batch) return fail(LD_EINVAL, "batched context");
    REJECT_MATFREE(c);   // graph distances need the operator's pattern
    if (j < 0 || j >= c->n) return fail(LD_EINVAL, "vertex %lld out of range", (long long)j);
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(LD_EINVAL, "eps must be > 0");
    if (max_d < 0 || max_d > 4096) return fail(LD_EINVAL, "max_d must be in [0, 4096]");
    std::vector<double> e((size_t)c->n, 0.0), y((size_t)c->n, 0.0);
    e[(size_t)j] = 1.0;
    if (ld_status st = ld_logmv(c, 1, e.data(), y.data(), info)) return st;
    std::vector<int32_t> dist((size_t)c->n);
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colidx;
    if (c->kind == LD_CSR) {   // the pattern lives on the device only
        rowptr.resize((size_t)c->n + 1);
        CUDA_TRY(cudaMemcpy(rowptr.data(), c->d_rowptr.p, rowptr.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
        colidx.resize((size_t)std::max<int64_t>(rowptr.back(), 1));
        CUDA_TRY(cudaMemcpy(colidx.data(), c->d_colidx.p, (size_t)rowptr.back() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    ld::graph_distances(c->kind, c->dims, c->periodic, c->n, rowptr.data(), colidx.data(), j, max_d,
                        dist.data());
    const double yj = std::fabs(y[(size_t)j]);
    if (!(yj > 0.0)) return fail(LD_ENUMERIC, "log(Q) e_j has a zero diagonal entry");
    std::vector<double> prof((size_t)max_d + 1, 0.0);
    int best = -1;
    for (int64_t l = 0; l < c->n; ++l) {
        const int d = dist[(size_t)l];
        if (d < 0) continue;
        const double r = std::fabs(y[(size_t)l]) / yj;
        prof[(size_t)d] = std::max(prof[(size_t)d], r);
        if (r < eps && (best < 0 || d < best)) best = d;
    }
    *distance = best;
    if (profile) std::copy(prof.begin(), prof.end(), profile);
    return LD_OK;
}

ld_status ld_colour_csr(int64_t n, const int64_t *rowptr, const int32_t *colidx, int d,
                        int32_t *colour, int32_t *n_colours) {
    if (n < 1 || !rowptr || !colidx || !colour || d < 0) return fail(LD_EINVAL, "bad arguments");
    const int nc = ld::colour_csr(n, rowptr, colidx, d, colour);
    if (n_colours) *n_colours = nc;
    return LD_OK;
}

ld_status ld_colour_grid(int kind, const int32_t dims[3], int periodic, int d, int32_t *colour,
                         int32_t *n_colours) {
    if (!dims || !colour || d < 0 || kind < LD_STENCIL_2D5 || kind > LD_STENCIL_3D7)
        return fail(LD_EINVAL, "bad arguments");
    int32_t dd[3] = {dims[0], dims[1], kind == LD_STENCIL_3D7 ? dims[2] : 1};
    if (dd[0] < 1 || dd[1] < 1 || dd[2] < 1) return fail(LD_EINVAL, "dims must be >= 1");
    const int nc = ld::colour_grid(kind, dd, periodic ? 1 : 0, d, colour);
    if (n_colours) *n_colours = nc;
    return LD_OK;
}

ld_status ld_auto_shifts(double lambda_min, double lambda_max, int32_t *n_shifts) {
    if (!n_shifts) return fail(LD_EINVAL, "n_shifts is NULL");
    if (!(lambda_min > 0.0) || !(lambda_max > lambda_min) || !std::isfinite(lambda_max))
        return fail(LD_EINVAL, "need 0 < lambda_min < lambda_max (finite)");
    *n_shifts = auto_shift_count(lambda_min, lambda_max);
    return LD_OK;
}

ld_status ld_hht_nodes(double lmin, double lmax, int N, double *sigma, double *alpha, double *cert) {
    if (N < 1 || N > 256 || !sigma || !alpha) return fail(LD_EINVAL, "bad arguments");
    std::vector<std::complex<double>> s(N), a(N);
    if (ld::hht_log_nodes(lmin, lmax, N, s.data(), a.data()) != 0)
        return fail(LD_EINVAL, "need 0 < lmin < lmax");
    for (int l = 0; l < N; ++l) {
        sigma[2 * l] = s[l].real();
        sigma[2 * l + 1] = s[l].imag();
        alpha[2 * l] = a[l].real();
        alpha[2 * l + 1] = a[l].imag();
    }
    if (cert) *cert = ld::hht_certificate(lmin, lmax, N, s.data(), a.data());
    return LD_OK;
}

ld_status ld_hht_invsqrt_nodes(double lmin, double lmax, int N, double *sigma, double *beta) {
    if (N < 1 || N > 256 || !sigma || !beta) return fail(LD_EINVAL, "bad arguments");
    std::vector<std::complex<double>> s(N), b(N);
    if (ld::hht_invsqrt_nodes(lmin, lmax, N, s.data(), b.data()) != 0)
        return fail(LD_EINVAL, "need 0 < lmin < lmax");
    for (int l = 0; l < N; ++l) {
        sigma[2 * l] = s[l].real();
        sigma[2 * l + 1] = s[l].imag();
        beta[2 * l] = b[l].real();
        beta[2 * l + 1] = b[l].imag();
    }
    return LD_OK;
}

ld_status ld_spde_fem_csr(int64_t n, const double *xy, int64_t m, const int64_t *tri, double kappa2,
                          int alpha, double tau, int64_t capacity, int64_t *rowptr, int32_t *colidx,
                          double *val, int64_t *nnz) {
    if (n < 3 || n > INT32_MAX || m < 1 || !xy || !tri || !nnz)
        return fail(LD_EINVAL, "need 3 <= n < 2^31 vertices, m >= 1 triangles, xy, tri and nnz");
    if (alpha != 1 && alpha != 2) return fail(LD_EINVAL, "alpha must be 1 or 2");
    if (!(kappa2 > 0.0) || !std::isfinite(kappa2) || !(tau > 0.0) || !std::isfinite(tau))
        return fail(LD_EINVAL, "kappa2 and tau must be positive and finite");
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(xy[i])) return fail(LD_EINVAL, "non-finite coordinate at %lld", (long long)(i / 2));
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> vv;
    const int rc = ld::fem_spde(n, xy, m, tri, kappa2, alpha, tau, rp, ci, vv);
    if (rc == -1) return fail(LD_EINVAL, "triangle vertex index outside [0, n)");
    if (rc == -2) return fail(LD_EINVAL, "degenerate triangle (zero area)");
    if (rc == -3) return fail(LD_EINVAL, "a vertex belongs to no triangle");
    *nnz = (int64_t)ci.size();
    if (capacity >= *nnz && rowptr && colidx && val) {
        std::copy(rp.begin(), rp.end(), rowptr);
        std::copy(ci.begin(), ci.end(), colidx);
        std::copy(vv.begin(), vv.end(), val);
    }
    return LD_OK;
}

ld_status ld_csr_bounds(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *val,
                        double scale, double *lmin, double *lmax) {
    if (n <= 0 || !rowptr || !colidx || !val || !lmin || !lmax) return fail(LD_EINVAL, "bad arguments");
    if (!(scale > 0.0)) return fail(LD_EINVAL, "scale must be > 0");
    int steps = 0;
    const int rc = ld::csr_bounds(n, rowptr, colidx, val, scale, lmin, lmax, &steps);
    if (rc == -2)
        return fail(LD_ENOTCONV, "smallest Lanczos Ritz value not converged after %d steps", steps);
    if (rc != 0) return fail(LD_ENOTSPD, "no positive spectral lower bound (not SPD?)");
    return LD_OK;
}

ld_status ld_grid_bounds(const ld_matrix *Q, double *lmin, double *lmax) {
    if (!lmin || !lmax) return fail(LD_EINVAL, "bad arguments");
    if (ld_status v = validate_matrix(Q)) return v;
    if (Q->kind == LD_CSR) return fail(LD_EINVAL, "grid kinds only");
    int32_t dd[3] = {Q->dims[0], Q->dims[1], Q->kind == LD_STENCIL_3D7 ? Q->dims[2] : 1};
    const int64_t n = grid_n(dd);
    double k2min = Q->kappa2, k2max = Q->kappa2;
    if (Q->kappa2_field) {
        k2min = INFINITY;
        k2max = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            k2min = std::min(k2min, Q->kappa2 * Q->kappa2_field[i]);
            k2max = std::max(k2max, Q->kappa2 * Q->kappa2_field[i]);
        }
    }
    bool mask = false;
    if (Q->obs_mask)
        for (int64_t i = 0; i < n && !mask; ++i) mask = Q->obs_mask[i] != 0;
    grid_bounds(Q->kind, dd, Q->periodic ? 1 : 0, k2min, k2max, mask ? Q->tau : 0.0,
                Q->scale == 0.0 ? 1.0 : Q->scale, lmin, lmax);
    return LD_OK;
}

// Build a batch context with tile width T.  step_s: seconds of one CTA step (one lattice
// row of 128 vertices) of the persistent engine, from the tuner's measurement; an instance
// whose one-CTA solve would outlast the batch runs on the grid engine (step_s <= 0: none).
// host threads driving a batch's grid-engine instances at once
constexpr int kBatchLargeThreads = 8;

ld_status batch_build(int count, const ld_matrix *Qs, const int *distances, int n_shifts, double tol,
                      const ld_options &opt, int T, double step_s, ld_ctx **out) {
    ld_ctx *c = new (std::nothrow) ld_ctx();
    if (!c) return fail(LD_ENOMEM, "host allocation");
    std::unique_ptr<ld_ctx> guard(c);
    c->is_batch = true;
    c->opt = opt;
    c->nshift = n_shifts;
    c->tol = tol;
    if (opt.cuda_stream) {
        c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CUDA_TRY(cudaEventCreate(&c->ev0));
    CUDA_TRY(cudaEventCreate(&c->ev1));
    // Every instance gets a context with a common tile width.  A tile in the persistent
    // launch is one CTA's whole solve, so an instance whose solve would outlast the rest
    // of the batch (CG iterations ~ 8 sqrt(cond), a lattice row of 128 vertices per CTA
    // step of step_s: more than 0.8 s) runs on the multi-CTA grid engine instead, on its
    // own stream beside the persistent launch.
    ld_options sub = opt;
    sub.keep_x0 = 0;
    sub.colouring = nullptr;
    sub.tile_width = T;
    c->T = T;
    c->subs.reserve(count);
    for (int i = 0; i < count; ++i) {
        if (Qs[i].kind == LD_CSR) return fail(LD_EUNSUPPORTED, "batched instances are grid kinds");
        double lo = 0.0, hi = 0.0;
        if (ld_status st = ld_grid_bounds(&Qs[i], &lo, &hi)) return st;
        int32_t dd[3] = {Qs[i].dims[0], Qs[i].dims[1], Qs[i].kind == LD_STENCIL_3D7 ? Qs[i].dims[2] : 1};
        const double est_s = 8.0 * std::sqrt(hi / lo) * ((double)grid_n(dd) / 128.0) * step_s;
        const bool large = step_s > 0.0 && est_s > 0.8 && grid_n(dd) >= 32768;
        ld_options o = sub;
        o.engine = large ? 1 : 2;
        o.cuda_stream = large ? nullptr : c->stream;
        ld_ctx *sc = nullptr;
        ld_status st = ld_create(&Qs[i], distances[i], n_shifts, tol, &o, &sc);
        if (st != LD_OK) {
            std::string msg = g_err;
            return fail(st, "instance %d: %s", i, msg.c_str());
        }
        c->subs.push_back(sc);
        (large ? c->large_idx : c->small_idx).push_back(i);
    }
    // the grid-engine instances run kBatchLargeThreads at a time: each plans for its share
    const int share = std::min((int)c->large_idx.size(), kBatchLargeThreads);
    for (int i : c->large_idx) {
        ld_ctx *sc = c->subs[i];
        sc->s.share = share;
        ld::engine_plan(sc->s);
        invalidate_graph(sc);
    }
    // device table of the small instances' solves and their work items, longest first
    const int nsmall = (int)c->small_idx.size();
    std::vector<Solve> solves(std::max(nsmall, 1));
    std::vector<int> ncol(std::max(nsmall, 1));
    struct Item { double cost; int inst, tile; };
    std::vector<Item> items;
    for (int k = 0; k < nsmall; ++k) {
        const ld_ctx *sc = c->subs[c->small_idx[k]];
        solves[k] = sc->s;
        ncol[k] = sc->ncolours;
        const double cost = (double)sc->n * std::sqrt(sc->lmax / sc->lmin);
        for (int t = 0; t < sc->ntiles; ++t) items.push_back({cost, k, t});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
    if (nsmall > 0) {
        std::vector<int2> hitems(items.size());
        for (size_t k = 0; k < items.size(); ++k) hitems[k] = make_int2(items[k].inst, items[k].tile);
        c->nitems = (int)items.size();
        CUDA_TRY(c->d_solves.alloc(sizeof(Solve) * nsmall));
        CUDA_TRY(cudaMemcpy(c->d_solves.p, solves.data(), sizeof(Solve) * nsmall, cudaMemcpyHostToDevice));
        CUDA_TRY(c->d_items.alloc(sizeof(int2) * hitems.size()));
        CUDA_TRY(cudaMemcpy(c->d_items.p, hitems.data(), sizeof(int2) * hitems.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c->d_queue.alloc(sizeof(int)));
        CUDA_TRY(c->d_bout.alloc(sizeof(double) * 2 * nsmall));
        CUDA_TRY(c->d_bint.alloc(sizeof(int) * 4 * nsmall));   // flags, iters, colours, tile passes
        CUDA_TRY(cudaMemcpy(c->d_bint.as<int>() + 2 * nsmall, ncol.data(), sizeof(int) * nsmall, cudaMemcpyHostToDevice));
        int dev = 0, sms = 152;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int occ = ld::engine_batch_occupancy(opt.precision == LD_MIXED ? 1 : 0, c->T);
        c->bgrid = std::max(1, std::min(c->nitems, occ * sms));
        // one CUDA graph: queue reset, per-instance prep, the persistent solve, per-instance sums
        const int max_iter = opt.max_iter > 0 ? opt.max_iter : 100000;
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int err = ld::engine_batch(c->d_solves.as<Solve>(), c->d_bint.as<int>() + 2 * nsmall, nsmall,
                                         c->d_items.as<int2>(), c->nitems, c->d_queue.as<int>(), max_iter,
                                         opt.precision == LD_MIXED ? 1 : 0, c->T, c->bgrid,
                                         c->d_bout.as<double>(), c->d_bout.as<double>() + nsmall,
                                         c->d_bint.as<int>(), c->d_bint.as<int>() + nsmall,
                                         c->d_bint.as<int>() + 3 * nsmall, c->stream);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (err) {
            if (g) cudaGraphDestroy(g);
            return fail(LD_ECUDA, "batch capture: %s", ld::engine_error_string(err));
        }
        if (e2 != cudaSuccess) return fail(LD_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
        cudaError_t e3 = cudaGraphInstantiate(&c->bgraph, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            c->bgraph = nullptr;
            return fail(LD_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));
        }
    }
    *out = guard.release();
    return LD_OK;
}


// Tile width and step cost of a batch, tuned once per batch shape and process: for every
// candidate tile width the persistent launch runs 16 iterations of every instance (all in
// the persistent engine); the fastest width wins, and its time gives the cost of one CTA
// step (total lattice-row steps over the resident CTAs) for the engine split.
std::map<std::string, std::pair<int, double>> g_batch_tune;

std::string batch_key(int count, const ld_matrix *Qs, const int *distances, int n_shifts, int precision) {
    std::ostringstream k;
    k << "batch:" << precision << ":" << n_shifts << ":" << count;
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < count; ++i) {
        const int64_t v[5] = {Qs[i].kind, Qs[i].dims[0], Qs[i].dims[1], Qs[i].kind == LD_STENCIL_3D7 ? Qs[i].dims[2] : 1,
                              distances[i]};
        for (int64_t x : v) h = (h ^ (uint64_t)x) * 1099511628211ull;
    }
    k << ":" << std::hex << h;
    return k.str();
}

ld_status ld_batch_create(int count, const ld_matrix *Qs, const int *distances, int n_shifts,
                          double tol, const ld_options *opt_in, ld_ctx **out) {
    if (!out) return fail(LD_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !Qs || !distances) return fail(LD_EINVAL, "count >= 1 with Qs and distances");
    ld_options opt;
    ld_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.precision != LD_FP64 && opt.precision != LD_MIXED) return fail(LD_EINVAL, "bad precision");
    if (n_shifts < 1 || n_shifts > 256) return fail(LD_EINVAL, "n_shifts must be in [1, 256]");
    if (!(tol > 0.0 && tol < 1.0)) return fail(LD_EINVAL, "tol must be in (0, 1)");
    if (opt.max_iter < 0) return fail(LD_EINVAL, "max_iter must be >= 0");
    if (opt.tile_width != 0 && choose_tile(opt.precision, 1, opt.tile_width) < 0)
        return fail(LD_EINVAL, "tile_width %d not available for this precision", opt.tile_width);
    // every instance is checked on the host before any device work
    for (int i = 0; i < count; ++i) {
        if (ld_status v = validate_matrix(&Qs[i])) {
            std::string msg = g_err;
            return fail(v, "instance %d: %s", i, msg.c_str());
        }
        if (Qs[i].kind == LD_CSR) return fail(LD_EUNSUPPORTED, "batched instances are grid kinds");
        if (distances[i] < 0) return fail(LD_EINVAL, "instance %d: colouring_distance must be >= 0", i);
    }
    const double default_step = 1.2e-6;   // one CTA step before any measurement
    int T = opt.tile_width;
    double step_s = default_step;
    const std::string key = batch_key(count, Qs, distances, n_shifts, opt.precision);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_batch_tune.find(key);
        if (it != g_batch_tune.end()) {
            if (T == 0) T = it->second.first;
            step_s = it->second.second;
        }
    }
    if (T == 0) {
        static const int f64[2] = {1, 2}, f32[2] = {2, 4};
        const int *cand = opt.precision == LD_FP64 ? f64 : f32;
        double best_ms = 1e300;
        double steps_per_cta = 0.0;
        for (int k = 0; k < 2; ++k) {
            ld_options o = opt;
            o.max_iter = 16;
            ld_ctx *t = nullptr;
            if (batch_build(count, Qs, distances, n_shifts, tol, o, cand[k], 0.0, &t) != LD_OK) continue;
            std::vector<double> v(count);
            ld_info info{};
            ld_batch_logdet(t, v.data(), nullptr, &info);      // warm (usually LD_ENOTCONV)
            ld_batch_logdet(t, v.data(), nullptr, &info);
            // lattice-row steps of the trial (16 iterations of every tile) per resident CTA
            double rows = 0.0;
            for (ld_ctx *sc : t->subs) rows += 16.0 * sc->ntiles * ((double)sc->n / 128.0);
            const double per_cta = rows / std::max(1, t->bgrid);
            ld_destroy(t);
            if (!(info.ms > 0.0)) continue;
            if (info.ms < best_ms) {
                best_ms = info.ms;
                T = cand[k];
                steps_per_cta = per_cta;
            }
        }
        g_err = "no error";
        if (T == 0) T = opt.precision == LD_MIXED ? 2 : 1;
        else if (steps_per_cta > 0.0) step_s = best_ms * 1e-3 / steps_per_cta;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_batch_tune[key] = {T, step_s};
    }
    return batch_build(count, Qs, distances, n_shifts, tol, opt, T, step_s, out);
}

ld_status ld_batch_logdet(ld_ctx *c, double *logdets, double *grads, ld_info *info) {
    Range range("ld batch");
    if (!c || !logdets) return fail(LD_EINVAL, "ctx and logdets must be non-NULL");
    if (!c->is_batch) return fail(LD_EINVAL, "not a batched context");
    const int count = (int)c->subs.size();
    const int nsmall = (int)c->small_idx.size();
    std::vector<double> out(2 * std::max(nsmall, 1));
    std::vector<int> flags(4 * std::max(nsmall, 1));
    const auto t0 = std::chrono::steady_clock::now();
    // the persistent launch for the small instances first (asynchronous) ...
    if (nsmall > 0) CUDA_TRY(cudaGraphLaunch(c->bgraph, c->stream));
    // ... then the large ones, each across the GPU on its own stream; up to kLargeThreads
    // host threads drive them at once (a solve waits on its own stream between chunks of
    // passes, so one host thread per instance keeps several instances' passes in flight)
    const size_t nl = c->large_idx.size();
    std::vector<double> lval(nl), lseed(nl);
    std::vector<ld_info> linfo(nl);
    std::vector<ld_status> lst(nl, LD_OK);
    std::vector<std::string> lmsg(nl);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        for (size_t k = next++; k < nl; k = next++) {
            ld_ctx *sc = c->subs[c->large_idx[k]];
            double o[2] = {0.0, 0.0};
            std::memset(&linfo[k], 0, sizeof linfo[k]);
            lst[k] = run_solve(sc, 0, sc->ncolours, false, o, &linfo[k]);
            if (lst[k] != LD_OK) lmsg[k] = g_err;   // this thread's message
            lval[k] = o[0];
            lseed[k] = o[1];
        }
    };
    const size_t nth = std::min(nl, (size_t)kBatchLargeThreads);
    if (nth <= 1) {
        worker();
    } else {
        std::vector<std::thread> pool;
        for (size_t k = 0; k < nth; ++k) pool.emplace_back(worker);
        for (std::thread &th : pool) th.join();
    }
    int iters = 0;
    int64_t tile_iters = 0, vertex_tile_iters = 0, launches = nsmall > 0 ? 3 : 0;
    ld_status st = LD_OK;
    for (size_t k = 0; k < nl; ++k) {
        if (lst[k] != LD_OK) {
            if (st == LD_OK) st = fail(lst[k], "instance %d: %s", c->large_idx[k], lmsg[k].c_str());
            continue;
        }
        iters = std::max(iters, (int)linfo[k].iters);
        tile_iters += linfo[k].tile_iters;
        vertex_tile_iters += linfo[k].vertex_tile_iters;
        launches += linfo[k].gpu_launches;
    }
    if (nsmall > 0) {
        CUDA_TRY(cudaMemcpyAsync(out.data(), c->d_bout.p, sizeof(double) * 2 * nsmall, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(flags.data(), c->d_bint.p, sizeof(int) * 4 * nsmall, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nsmall && st == LD_OK; ++k) {
        iters = std::max(iters, flags[nsmall + k]);
        tile_iters += flags[3 * nsmall + k];
        vertex_tile_iters += c->subs[c->small_idx[k]]->n * flags[3 * nsmall + k];
        const int f = flags[k];
        if (f == 0) continue;
        const int i = c->small_idx[k];
        if (f == ld::DEV_NOTSPD) st = fail(LD_ENOTSPD, "instance %d: Q is not SPD", i);
        else if (f == -1) st = fail(LD_ENOTCONV, "instance %d: max_iter reached", i);
        else st = fail(LD_ENUMERIC, "instance %d: non-finite CG scalar", i);
    }
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->status = st;
        info->n_shifts = c->nshift;
        info->iters = iters;
        info->tile_width = c->T;
        info->engine = 2;
        info->ms = ms;          // host wall time of the whole batch (both engines)
        info->iter_ms = ms;
        info->gpu_launches = launches;
        info->bulk_rows = -1;
        info->rel_resid_max = -1.0;
        info->tile_iters = tile_iters;
        info->vertex_tile_iters = vertex_tile_iters;
        info->n_colours = 0;
        for (ld_ctx *sc : c->subs) info->n_colours += sc->ncolours;
    }
    if (st != LD_OK) return st;
    auto put = [&](int i, double v, double seed) {
        logdets[i] = v;
        if (grads) {
            const ld_ctx *sc = c->subs[i];
            const bool projected = (sc->kind == LD_STENCIL_2D5 || sc->kind == LD_STENCIL_3D7) && !sc->has_field;
            grads[i] = projected ? sc->scale * seed : std::nan("");
        }
    };
    for (int k = 0; k < nsmall; ++k) put(c->small_idx[k], out[k], out[nsmall + k]);
    for (size_t k = 0; k < c->large_idx.size(); ++k) put(c->large_idx[k], lval[k], lseed[k]);
    (void)count;
    return LD_OK;
}

void ld_destroy(ld_ctx *c) { delete c; }

}  // extern "C"
