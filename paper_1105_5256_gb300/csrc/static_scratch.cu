// ld_logdet_static: a log det evaluation that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// log det: code running inside a custom memory pool or arena that forbids
// cudaMalloc/cudaFree (a framework allocator that owns all device memory), or
// a callback in a latency-critical loop where an allocation would synchronise
// the device.  This entry point serves them for small grid models: every
// work buffer of the solve (CG vectors, scalars, shift state, colouring,
// quadrature nodes) lives in one fixed static device array, `g_scratch`, which
// every GPU that loads the library holds until the process exits.
//
// The solve is the same probed rational-log multi-shift CG as ld_logdet, run
// by the one-CTA-per-probing-vector engine in FP64 (tile width 1).
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/logdet.h"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)LD_STATIC_SCRATCH_BYTES;

// The scratch array.  In host code `g_scratch` names a host-side stand-in, not
// device memory: its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_scratch[LD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

ld_status fail(ld_status st, const char *msg) {
    ld::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" ld_status ld_logdet_static(const ld_matrix *Q, const int32_t *colour, int n_colours,
                                      int n_shifts, double tol, int max_iter, void *cuda_stream,
                                      double *logdet) {
    using ld::Solve;
    if (!Q || !colour || !logdet) return fail(LD_EINVAL, "Q, colour and logdet must be non-NULL");
    if (Q->kind != LD_STENCIL_2D5 && Q->kind != LD_STENCIL_2D13_SQ && Q->kind != LD_STENCIL_3D7)
        return fail(LD_EINVAL, "grid kinds only");
    if (Q->kappa2_field || Q->obs_mask)
        return fail(LD_EUNSUPPORTED, "scalar kappa2 without observation term only");
    const int nd = Q->kind == LD_STENCIL_3D7 ? 3 : 2;
    int64_t n = 1;
    for (int d = 0; d < nd; ++d) {
        if (Q->dims[d] < 1) return fail(LD_EINVAL, "dims must be >= 1");
        n *= Q->dims[d];
        // every vertex needs at least one FP64 word of scratch: stop before n can overflow
        if (n > (int64_t)(kScratchBytes / sizeof(double)))
            return fail(LD_EINVAL, "problem needs more than LD_STATIC_SCRATCH_BYTES of scratch");
    }
    if (!(Q->kappa2 >= 0.0) || !(tol > 0.0 && tol < 1.0) || n_shifts < 1 || n_shifts > 256 ||
        n_colours < 1 || n_colours > LD_STATIC_MAX_COLOURS || max_iter < 1)
        return fail(LD_EINVAL, "bad kappa2, tol, n_shifts, n_colours or max_iter");
    const double scale = Q->scale == 0.0 ? 1.0 : Q->scale;
    if (!(scale > 0.0)) return fail(LD_EINVAL, "scale must be > 0");
    // ---- carve the scratch: FP64, tile width 1 (one CTA per probing vector)
    const int C = n_colours, N = n_shifts, T = 1;
    const size_t vec = align256((size_t)n * C * sizeof(double));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_vec = take(6 * vec);
    const size_t o_col = take((size_t)n * sizeof(int32_t));
    const size_t o_cs = take((size_t)8 * C * sizeof(double));
    const size_t o_ci = take((size_t)2 * C * sizeof(int32_t));
    const size_t o_sh = take((size_t)4 * C * N * sizeof(double2) + (size_t)C * N);
    const size_t o_nd = take((size_t)2 * N * sizeof(double2));
    const size_t o_tl = take((size_t)(3 * C + 2) * sizeof(int32_t));
    const size_t o_tm = take((size_t)(2 * C + 8) * sizeof(double));
    if (off > kScratchBytes)
        return fail(LD_EINVAL, "problem needs more than LD_STATIC_SCRATCH_BYTES of scratch");
    // the colouring is scanned only once the problem is known to fit
    for (int64_t i = 0; i < n; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return fail(LD_EINVAL, "colour out of range");

    void *base = nullptr;
    if (cudaError_t e = scratch_address(&base); e != cudaSuccess)
        return fail(LD_ECUDA, cudaGetErrorString(e));
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // ---- host-side set-up in fixed-size arrays (no heap)
    double lmin, lmax;
    {
        ld_matrix q = *Q;
        q.scale = scale;
        ld_status s = ld_grid_bounds(&q, &lmin, &lmax);
        if (s != LD_OK) return fail(s, "bounds");
    }
    std::complex<double> sigma[256], alpha[256];
    if (ld::hht_log_nodes(lmin, lmax, N, sigma, alpha) != 0) return fail(LD_EINVAL, "nodes");
    double2 nodes[512];
    for (int l = 0; l < N; ++l) {
        nodes[l] = make_double2(-sigma[l].real(), -sigma[l].imag());
        nodes[N + l] = make_double2(alpha[l].real(), alpha[l].imag());
    }
    double cls[LD_STATIC_MAX_COLOURS];
    for (int c = 0; c < C; ++c) cls[c] = 0.0;
    for (int64_t i = 0; i < n; ++i) cls[colour[i]] += 1.0;

    cudaError_t e = cudaMemsetAsync(b, 0, off, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_col, colour, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_nd, nodes, (size_t)2 * N * sizeof(double2), cudaMemcpyHostToDevice, st);
    double *terms = reinterpret_cast<double *>(b + o_tm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(terms + C, cls, (size_t)C * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(LD_ECUDA, cudaGetErrorString(e));

    Solve s{};
    s.op.kind = Q->kind;
    s.op.periodic = Q->periodic ? 1 : 0;
    s.op.nx = Q->dims[0];
    s.op.ny = Q->dims[1];
    s.op.nz = nd == 3 ? Q->dims[2] : 1;
    s.op.n = n;
    s.op.kappa2 = Q->kappa2;
    s.op.tau = 0.0;
    s.op.scale = scale;
    set_f32_coefs(s.op);
    s.T = T;
    s.ntiles = C;
    s.ncols = C;
    s.nshift = N;
    s.bpt = 1;
    s.strips = 1;
    s.seg = 1;
    s.precision = 0;
    s.keep_x0 = 0;
    s.tol = tol;
    s.colour = reinterpret_cast<const int32_t *>(b + o_col);
    for (int k = 0; k < 2; ++k) {
        s.rbuf[k] = b + o_vec + (size_t)k * vec;
        s.wbuf[k] = b + o_vec + (size_t)(2 + k) * vec;
        s.pbuf[k] = b + o_vec + (size_t)(4 + k) * vec;
    }
    double *cs = reinterpret_cast<double *>(b + o_cs);
    s.rho = cs;
    s.alpha = cs + C;
    s.beta = cs + 2 * C;
    s.alpha_prev = cs + 3 * C;
    s.beta_prev = cs + 4 * C;
    s.vnorm2 = cs + 5 * C;
    s.pi0 = cs + 6 * C;
    s.phi0 = cs + 7 * C;
    s.col_active = reinterpret_cast<int32_t *>(b + o_ci);
    s.col_iters = s.col_active + C;
    double2 *sh = reinterpret_cast<double2 *>(b + o_sh);
    s.zeta = sh;
    s.zeta_prev = sh + (size_t)C * N;
    s.pi = sh + (size_t)2 * C * N;
    s.phi = sh + (size_t)3 * C * N;
    s.sh_active = reinterpret_cast<uint8_t *>(sh + (size_t)4 * C * N);
    s.shift = reinterpret_cast<const double2 *>(b + o_nd);
    s.weight = s.shift + N;
    int32_t *tl = reinterpret_cast<int32_t *>(b + o_tl);
    s.tile_done = tl;
    s.tile_ctr = tl + C;
    s.tile_par = tl + 2 * C;
    s.remaining = tl + 3 * C;
    s.status = s.remaining + 1;
    s.partial = nullptr;
    s.terms = terms;
    s.class_size = terms + C;
    s.result = terms + 2 * C;

    int err = ld::engine_init(s, 0, C, st);
    if (!err) err = ld::engine_cta_solve(s, max_iter, st);
    if (!err) err = ld::engine_finish(s, 0, C, st);
    if (err) return fail(LD_ECUDA, ld::engine_error_string(err));
    double res[2];
    int32_t flags[2];
    e = cudaMemcpyAsync(res, s.result, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flags, s.remaining, sizeof flags, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LD_ECUDA, cudaGetErrorString(e));
    if (flags[1] == ld::DEV_NOTSPD) return fail(LD_ENOTSPD, "Q is not SPD");
    if (flags[1] != 0) return fail(LD_ENUMERIC, "non-finite CG scalar");
    if (flags[0] > 0) return fail(LD_ENOTCONV, "max_iter reached");
    *logdet = res[0];
    return LD_OK;
}
