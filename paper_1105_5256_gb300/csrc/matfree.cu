// Matrix-free operator: the probed rational log det of Sec. 2.1 when Q is available
// only as a product W = Q P computed by the caller (Sec. 1: the method touches Q only
// through matrix-vector products).
//
// The pass kernels of the stencil and CSR paths fuse the product into the CG update;
// here the product is the caller's, so one iteration is the caller's product and three
// launches around it, in the one-reduction form of CG the fused passes use:
//
//   W = Q P_k                 caller (ld_matvec_fn, on the context stream)
//   k_mf_dots     per-block partials of the six dots of column c:
//                 r.r, p.w, r.w, w.w, v.r, v.w   (r = r_k, p = p_k, w = Q p_k)
//   k_mf_tail     one warp per column: alpha = rr / pw, ||r_{k+1}||^2 = rr - 2 alpha rw
//                 + alpha^2 ww, beta = ||r_{k+1}||^2 / rr, v.r_{k+1} = vr - alpha vw; the
//                 seed projections and the CG-M shift recurrences; convergence
//   k_mf_update   r_{k+1} = r_k - alpha w, p_{k+1} = r_{k+1} + beta p_k, x += alpha p_k
//                 (kept seed solution), and the shifted vectors of the vector form
//
// Outside the caller's product an iteration reads r, p, w twice and writes r and p
// (8 words per vertex and column; 3 more with the kept x).
//
// Vectors are n x C row-major (the C entries of a vertex adjacent), the layout the
// caller's product sees.  Every kernel walks that array column-stationary: the launch's
// G threads are cut into R = floor(G / C) replicas of C consecutive threads, thread g
// keeps column g mod C and rows g / C, g / C + R, ...; consecutive threads touch
// consecutive addresses whatever C is, and each thread accumulates one column.
// Reductions are two-stage with a fixed order (per block in thread order, then one warp
// per column over the blocks), so results are bitwise repeatable.
//
// Shifted systems (Q + s I) x = v, s = -sigma_l, keep only the projections
// pi = v^T x^sigma and phi = v^T p^sigma (scalar recurrences of CG-M / COCG-M):
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} / (a_{k-1} zeta_{k-1} (1 + s a_k)
//                                             + a_k b_{k-1} (zeta_{k-1} - zeta_k))
//   a^s_k = a_k zeta_{k+1} / zeta_k,   b^s_k = b_k (zeta_{k+1} / zeta_k)^2
//   pi += a^s_k phi,                   phi = zeta_{k+1} (v^T r_{k+1}) + b^s_k phi
// with zeta_{-1} = zeta_0 = 1, a_{-1} = 1, b_{-1} = 0, phi_0 = v^T v.  The vector form
// keeps p^s itself (x^s += a^s_k p^s, p^s = zeta_{k+1} r_{k+1} + b^s_k p^s) and adds the
// increments straight into y = Re sum_l w_l x^{s_l}.  A shift stops when |zeta_{k+1}|
// ||r_{k+1}|| <= tol ||v||, the seed (s = 0) when ||r_{k+1}|| <= tol ||v||; a column stops
// when its seed and all its shifts have.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/logdet.h"
#include "internal.h"

namespace {

constexpr int kThreads = 256;          // every streaming kernel: 8 warps
constexpr int kMaxBlocks = 152 * 8;    // a multiple of the SM count
constexpr int kDots = 6;               // rr, pw, rw, ww, vr, vw

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a / b by Smith's algorithm (R. L. Smith, CACM 1962): scales by the larger component of
// b so that |b|^2 is never formed
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    const double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }

// column-stationary walk of a row-major n x C array (C <= threads of the launch)
struct ColMap {
    int64_t R;     // replicas: threads per column
    int64_t rho;   // first row of this thread
    int c;         // column of this thread
    bool on;       // g < R * C
    __device__ __forceinline__ explicit ColMap(int C) {
        const int64_t G = (int64_t)gridDim.x * blockDim.x;
        const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        R = G / C;
        on = g < R * C;
        c = (int)(g % C);
        rho = g / C;
    }
};

// Per-block column sums of K per-thread values, in thread order:
// part[(k * gridDim.x + block) * C + c] for every column c (0 where the block has no
// thread of column c).  sm: K * kThreads doubles.
template <int K>
__device__ __forceinline__ void block_column_partials(const double (&acc)[K], int C, double *sm,
                                                      double *__restrict__ part) {
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k * kThreads + t] = acc[k];
    __syncthreads();
    const int64_t G = (int64_t)gridDim.x * kThreads, S = (G / C) * C;
    const int64_t base = (int64_t)blockIdx.x * kThreads;
    const int lim = (int)max((int64_t)0, min((int64_t)kThreads, S - base));
    const int b0 = (int)(base % C);
    for (int j = t; j < K * C; j += kThreads) {
        const int k = j / C, c = j - k * C;
        int u = c - b0;
        if (u < 0) u += C;
        double s = 0.0;
        for (; u < lim; u += C) s += sm[k * kThreads + u];
        part[((int64_t)k * gridDim.x + blockIdx.x) * C + c] = s;
    }
}

// sum over blocks of one column's partials: lanes take blocks lane, lane + 32, ... in
// order, then a fixed butterfly (every lane gets the sum)
__device__ __forceinline__ double warp_column_sum(const double *partial, int nblk, int C, int c) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[(size_t)b * C + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct ColState {        // per column, device
    double alpha;        // a_k (this iteration, applied by k_mf_update)
    double beta;         // b_k (0 once the column has stopped)
    double alpha_prev;   // a_{k-1}
    double beta_prev;    // b_{k-1}
    double vnorm;        // ||v_c||
    double pi0, phi0;    // seed system: v^T x, v^T p
    int active;          // 1 while the seed or some shift of the column is unconverged
    int was;             // 1 when this iteration's tail advanced the column
    int iters;           // iterations the column ran
    int pad;
};

struct ShiftState {      // per (column, shift), device
    double2 zeta_prev, zeta, pi, phi;
    double2 as, bs;      // this iteration's a^s, b^s (vector form)
    int done;
    int upd;             // 1 when this iteration's tail advanced the shift
};

__global__ void k_mf_init(int64_t n, int C, int cb, const int32_t *__restrict__ colour,
                          const double *__restrict__ v, double *__restrict__ r, double *__restrict__ p,
                          double *__restrict__ x) {
    const ColMap m(C);
    if (!m.on) return;
    for (int64_t i = m.rho; i < n; i += m.R) {
        const int64_t e = i * C + m.c;
        const double val = v ? v[e] : (colour[i] == cb + m.c ? 1.0 : 0.0);
        r[e] = val;
        p[e] = val;
        if (x) x[e] = 0.0;
    }
}

// shifted vectors p^s_0 = v (layout [shift][n][C]) and y = 0
__global__ void k_mf_init_vec(int64_t n, int C, int N, const double *__restrict__ v, double2 *__restrict__ psig,
                              double *__restrict__ y) {
    const ColMap m(C);
    if (!m.on) return;
    const int64_t nc = n * C;
    for (int64_t i = m.rho; i < n; i += m.R) {
        const int64_t e = i * C + m.c;
        const double2 val = make_double2(v[e], 0.0);
        for (int l = 0; l < N; ++l) psig[l * nc + e] = val;
        y[e] = 0.0;
    }
}

__global__ void k_mf_init_scalars(int C, int N, const double *__restrict__ norm2,
                                  ColState *__restrict__ cs, ShiftState *__restrict__ ss) {
    const int c = blockIdx.x;
    if (c >= C) return;
    const double m = norm2[c];
    if (threadIdx.x == 0) {
        ColState s;
        s.alpha = 0.0;
        s.beta = 0.0;
        s.alpha_prev = 1.0;
        s.beta_prev = 0.0;
        s.vnorm = sqrt(m);
        s.pi0 = 0.0;
        s.phi0 = m;
        s.active = m > 0.0 ? 1 : 0;   // an empty colour class (v = 0) contributes nothing
        s.was = 0;
        s.iters = 0;
        s.pad = 0;
        cs[c] = s;
    }
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
        ShiftState t;
        t.zeta_prev = make_double2(1.0, 0.0);
        t.zeta = make_double2(1.0, 0.0);
        t.pi = make_double2(0.0, 0.0);
        t.phi = make_double2(m, 0.0);
        t.as = make_double2(0.0, 0.0);
        t.bs = make_double2(0.0, 0.0);
        t.done = m > 0.0 ? 0 : 1;
        t.upd = 0;
        ss[(size_t)c * N + l] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_mf_dots(int64_t n, int C, int cb, const int32_t *__restrict__ colour,
                                                      const double *__restrict__ v, const double *__restrict__ r,
                                                      const double *__restrict__ p, const double *__restrict__ w,
                                                      const ColState *__restrict__ cs, double *__restrict__ part) {
    __shared__ double sm[kDots * kThreads];
    const ColMap m(C);
    double acc[kDots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (m.on && cs[m.c].active) {
        for (int64_t i = m.rho; i < n; i += m.R) {
            const int64_t e = i * C + m.c;
            const double re = r[e], pe = p[e], we = w[e];
            const double ve = v ? v[e] : (colour[i] == cb + m.c ? 1.0 : 0.0);
            acc[0] = fma(re, re, acc[0]);
            acc[1] = fma(pe, we, acc[1]);
            acc[2] = fma(re, we, acc[2]);
            acc[3] = fma(we, we, acc[3]);
            acc[4] = fma(ve, re, acc[4]);
            acc[5] = fma(ve, we, acc[5]);
        }
    }
    block_column_partials<kDots>(acc, C, sm, part);
}

__global__ void k_mf_tail(int nblk, int C, int N, const double *__restrict__ part,
                          const double2 *__restrict__ shift, double tol, ColState *__restrict__ cs,
                          ShiftState *__restrict__ ss, int *__restrict__ status) {
    const int c = blockIdx.x, lane = threadIdx.x;
    ColState col = cs[c];
    if (!col.active) {
        if (col.was) {   // stopped in the last iteration: no vector update from now on
            for (int l = lane; l < N; l += 32) ss[(size_t)c * N + l].upd = 0;
            if (lane == 0) cs[c].was = 0;
        }
        return;
    }
    double d[kDots];
#pragma unroll
    for (int k = 0; k < kDots; ++k) d[k] = warp_column_sum(part + (size_t)k * nblk * C, nblk, C, c);
    const double rr = d[0], pw = d[1], rw = d[2], ww = d[3], vr = d[4], vw = d[5];
    if (!(pw > 0.0)) {                       // p^T Q p <= 0: Q is not SPD
        if (lane == 0) {
            atomicCAS(status, 0, isfinite(pw) ? (int)LD_ENOTSPD : (int)LD_ENUMERIC);
            cs[c].active = 0;
            cs[c].was = 0;
        }
        for (int l = lane; l < N; l += 32) ss[(size_t)c * N + l].upd = 0;
        return;
    }
    const double a = rr / pw;
    const double rhon = fmax(rr - 2.0 * a * rw + a * a * ww, 0.0);   // ||r_{k+1}||^2
    const double b = rr > 0.0 ? rhon / rr : 0.0;
    const double vrn = vr - a * vw;                                    // v^T r_{k+1}
    if (!isfinite(a) || !isfinite(b) || !isfinite(vrn)) {
        if (lane == 0) {
            atomicCAS(status, 0, (int)LD_ENUMERIC);
            cs[c].active = 0;
            cs[c].was = 0;
        }
        for (int l = lane; l < N; l += 32) ss[(size_t)c * N + l].upd = 0;
        return;
    }
    const double ap = col.alpha_prev, bp = col.beta_prev;
    const double rnorm = sqrt(rhon), lim = tol * col.vnorm;
    bool live = rnorm > lim;                 // the seed system
    for (int l = lane; l < N; l += 32) {
        ShiftState t = ss[(size_t)c * N + l];
        if (t.done) {
            if (t.upd) ss[(size_t)c * N + l].upd = 0;
            continue;
        }
        const double2 s = shift[l];
        // den = a_{k-1} zeta_{k-1} (1 + s a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)
        const double2 one_sa = make_double2(1.0 + s.x * a, s.y * a);
        const double2 den = cadd(cmul(cscale(t.zeta_prev, ap), one_sa), cscale(csub(t.zeta_prev, t.zeta), a * bp));
        const double2 znew = cdiv(cscale(cmul(t.zeta, t.zeta_prev), ap), den);
        const double2 ratio = cdiv(znew, t.zeta);
        t.as = cscale(ratio, a);
        t.bs = cscale(cmul(ratio, ratio), b);
        t.pi = cadd(t.pi, cmul(t.as, t.phi));
        t.phi = cadd(cscale(znew, vrn), cmul(t.bs, t.phi));
        t.zeta_prev = t.zeta;
        t.zeta = znew;
        t.upd = 1;
        if (cabs_(znew) * rnorm <= lim) t.done = 1;
        if (!isfinite(t.pi.x) || !isfinite(t.pi.y)) {
            atomicCAS(status, 0, (int)LD_ENUMERIC);
            t.done = 1;
        }
        live = live || !t.done;
        ss[(size_t)c * N + l] = t;
    }
    live = __any_sync(0xffffffffu, live);
    if (lane == 0) {
        col.pi0 += a * col.phi0;             // seed: v^T x_{k+1}
        col.phi0 = vrn + b * col.phi0;       // v^T p_{k+1}
        col.alpha = a;
        col.beta = live ? b : 0.0;
        col.alpha_prev = a;
        col.beta_prev = b;
        col.iters += 1;
        col.active = live ? 1 : 0;
        col.was = 1;
        cs[c] = col;
    }
}

// r_{k+1} = r_k - a w, p_{k+1} = r_{k+1} + b p_k, x += a p_k; vector form: y += Re sum_l
// w_l a^s_l p^s_l, p^s_l = zeta_{k+1} r_{k+1} + b^s_l p^s_l
__global__ void __launch_bounds__(kThreads) k_mf_update(int64_t n, int C, int N, double *__restrict__ r,
                                                        double *__restrict__ p, const double *__restrict__ w,
                                                        double *__restrict__ x, const ColState *__restrict__ cs,
                                                        const ShiftState *__restrict__ ss,
                                                        const double2 *__restrict__ yweight,
                                                        double2 *__restrict__ psig, double *__restrict__ y) {
    const ColMap m(C);
    if (!m.on) return;
    const ColState col = cs[m.c];
    if (!col.was) return;
    const double a = col.alpha, b = col.beta;
    const bool go = col.active != 0;
    const int64_t nc = n * C;
    const ShiftState *st = ss + (size_t)m.c * N;
    for (int64_t i = m.rho; i < n; i += m.R) {
        const int64_t e = i * C + m.c;
        const double pe = p[e];
        const double r1 = fma(-a, w[e], r[e]);
        if (x) x[e] = fma(a, pe, x[e]);
        if (psig) {
            double acc = 0.0;
            for (int l = 0; l < N; ++l) {
                if (!st[l].upd) continue;
                double2 *pp = psig + l * nc + e;
                const double2 ps = *pp;
                const double2 g = cmul(yweight[l], st[l].as);        // w_l a^s_l
                acc += g.x * ps.x - g.y * ps.y;                        // Re(w_l x^s increment)
                *pp = cadd(cscale(st[l].zeta, r1), cmul(st[l].bs, ps));
            }
            y[e] += acc;
        }
        if (go) {
            r[e] = r1;
            p[e] = fma(b, pe, r1);
        }
    }
}

// per-block partials of sum_i v_c(i) X[i, c] (v_c the colour indicator or a given vector)
__global__ void __launch_bounds__(kThreads) k_mf_vdot(int64_t n, int C, int cb, const int32_t *__restrict__ colour,
                                                      const double *__restrict__ v, const double *__restrict__ X,
                                                      double *__restrict__ part) {
    __shared__ double sm[kThreads];
    const ColMap m(C);
    double acc[1] = {0.0};
    if (m.on)
        for (int64_t i = m.rho; i < n; i += m.R) {
            const int64_t e = i * C + m.c;
            if (v) acc[0] = fma(v[e], X[e], acc[0]);
            else if (colour[i] == cb + m.c) acc[0] += X[e];
        }
    block_column_partials<1>(acc, C, sm, part);
}

__global__ void k_mf_colsum(int nblk, int C, const double *__restrict__ part, double *__restrict__ out) {
    const int c = blockIdx.x;
    const double s = warp_column_sum(part, nblk, C, c);
    if (threadIdx.x == 0) out[c] = s;
}

// active-column count and the error status
__global__ void k_mf_count(int C, const ColState *__restrict__ cs, const int *__restrict__ status,
                           int *__restrict__ out) {
    int a = 0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) a += cs[c].active;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    __shared__ int sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
        out[0] = s;
        out[1] = *status;
    }
}

// term_c = Re sum_l weight_l pi_{c,l}, lanes over shifts in order, then a fixed butterfly;
// seed_c = v_c^T x_c
__global__ void k_mf_finish(int C, int N, const double2 *__restrict__ weight, const ShiftState *__restrict__ ss,
                            const ColState *__restrict__ cs, double *__restrict__ terms,
                            double *__restrict__ seeds, int *__restrict__ iters) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double s = 0.0;
    for (int l = lane; l < N; l += 32) {
        const double2 w = weight[l], pi = ss[(size_t)c * N + l].pi;
        s += w.x * pi.x - w.y * pi.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        terms[c] = s;
        seeds[c] = cs[c].pi0;
        iters[c] = cs[c].iters;
    }
}

// device buffer that frees itself
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { cudaFree(p); }
    template <typename U>
    U *as() const { return static_cast<U *>(p); }
    // at least `want` bytes (contents not kept)
    cudaError_t reserve(size_t want) {
        if (want <= bytes && p) return cudaSuccess;
        cudaFree(p);
        p = nullptr;
        bytes = 0;
        const cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 16));
        if (e == cudaSuccess) bytes = std::max<size_t>(want, 16);
        return e;
    }
};

}  // namespace

namespace ld {

constexpr int kPollEvery = 4;   // iterations between convergence polls
constexpr int kRing = 4;        // poll slots
constexpr int kLag = 2;         // poll groups in flight before the host waits for the oldest

struct Matfree {
    int64_t n = 0;
    int C = 0;                        // colours
    ld_matvec_fn fn = nullptr;
    void *user = nullptr;
    Buf colour;                       // int32, n
    Buf r, p, w, x, v;                // n x (columns of the solve), FP64
    Buf part;                         // kDots x nblk x columns
    Buf norm2, nodes, cs, ss, terms, seeds, iters, status, count, psig, y;
    int *h_count = nullptr;           // pinned, 2 per poll slot
    std::vector<double> h_class;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evp[kRing] = {};
    // the kept seed solutions of the last solve over colours [x_cb, x_cb + x_cols)
    bool have_x = false;
    int x_cb = 0, x_cols = 0;

    ~Matfree() {
        if (h_count) cudaFreeHost(h_count);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : evp)
            if (e) cudaEventDestroy(e);
    }
};

void matfree_destroy(Matfree *m) { delete m; }

int matfree_create(Matfree **out, int64_t n, const int32_t *colour, int C, int N, void *fn, void *user) {
    (void)N;
    *out = nullptr;
    Matfree *m = new (std::nothrow) Matfree();
    if (!m) return (int)cudaErrorMemoryAllocation;
    m->n = n;
    m->C = C;
    m->fn = reinterpret_cast<ld_matvec_fn>(fn);
    m->user = user;
    m->h_class.assign(C, 0.0);
    for (int64_t i = 0; i < n; ++i) m->h_class[colour[i]] += 1.0;
    cudaError_t e = m->colour.reserve((size_t)n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&m->h_count, 2 * kRing * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev1);
    for (int k = 0; k < kRing && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&m->evp[k], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->colour.p, colour, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete m;
        return (int)e;
    }
    *out = m;
    return 0;
}

namespace {

// blocks of the streaming kernels for n x C: about four elements a thread, at most
// kMaxBlocks, at least one thread a column; with many columns fewer blocks so that the
// per-block column partials stay small
int stream_blocks(int64_t n, int C) {
    int64_t want = std::min<int64_t>((int64_t)kMaxBlocks * kThreads, std::max<int64_t>(n * C / 4, kThreads));
    int64_t nb = (want + kThreads - 1) / kThreads;
    const int64_t need = ((int64_t)C + kThreads - 1) / kThreads;
    if ((int64_t)C > kThreads) nb = std::min<int64_t>(nb, std::max<int64_t>(need, ((int64_t)1 << 18) / C));
    return (int)std::max<int64_t>(nb, need);
}

}  // namespace

int matfree_solve(Matfree *m, const MatfreeJob &job, const std::complex<double> *sigma,
                  const std::complex<double> *weight, double tol, int max_iter, cudaStream_t stream,
                  double *terms_out, double *seeds_out, MatfreeStats *st) {
    const bool vec = job.rhs != nullptr;
    const int C = vec ? job.ncols : job.ce - job.cb;
    const int cb = vec ? 0 : job.cb;
    const int N = job.n_shifts;
    const int64_t n = m->n;
    st->iters = 0;
    st->launches = 0;
    st->callback_rc = 0;
    st->column_iters = 0;
    st->ms = 0.0f;
    m->have_x = false;
    if (C <= 0) return LD_OK;
    const bool keep_x = job.keep_x;
    const int nblk = stream_blocks(n, C);
    const size_t vec_bytes = (size_t)n * C * sizeof(double);
    cudaError_t e;
#define MF_TRY(expr)                                                        \
    do {                                                                    \
        e = (expr);                                                         \
        if (e != cudaSuccess) {                                             \
            ld::set_last_error(cudaGetErrorString(e));                      \
            return e == cudaErrorMemoryAllocation ? LD_ENOMEM : LD_ECUDA;   \
        }                                                                   \
    } while (0)
    MF_TRY(m->r.reserve(vec_bytes));
    MF_TRY(m->p.reserve(vec_bytes));
    MF_TRY(m->w.reserve(vec_bytes));
    if (keep_x) MF_TRY(m->x.reserve(vec_bytes));
    if (vec) {
        MF_TRY(m->v.reserve(vec_bytes));
        MF_TRY(m->psig.reserve((size_t)N * n * C * sizeof(double2)));
        MF_TRY(m->y.reserve(vec_bytes));
    }
    MF_TRY(m->part.reserve((size_t)kDots * nblk * C * sizeof(double)));
    MF_TRY(m->norm2.reserve((size_t)C * sizeof(double)));
    MF_TRY(m->nodes.reserve((size_t)3 * N * sizeof(double2)));
    MF_TRY(m->cs.reserve((size_t)C * sizeof(ColState)));
    MF_TRY(m->ss.reserve((size_t)C * N * sizeof(ShiftState)));
    MF_TRY(m->terms.reserve((size_t)C * sizeof(double)));
    MF_TRY(m->seeds.reserve((size_t)C * sizeof(double)));
    MF_TRY(m->iters.reserve((size_t)C * sizeof(int)));
    MF_TRY(m->status.reserve(sizeof(int)));
    MF_TRY(m->count.reserve((size_t)2 * kRing * sizeof(int)));
    // host: shifts s_l = -sigma_l, the log weights, the vector form's weights; ||v_c||^2
    std::vector<double2> h_nodes(3 * N);
    for (int l = 0; l < N; ++l) {
        h_nodes[l] = make_double2(-sigma[l].real(), -sigma[l].imag());
        h_nodes[N + l] = make_double2(weight[l].real(), weight[l].imag());
        const std::complex<double> yw = vec && job.yweight ? job.yweight[l] : weight[l];
        h_nodes[2 * N + l] = make_double2(yw.real(), yw.imag());
    }
    std::vector<double> norm2(C, 0.0);
    if (vec) {
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < C; ++c) norm2[c] += job.rhs[i * C + c] * job.rhs[i * C + c];
    } else {
        for (int c = 0; c < C; ++c) norm2[c] = m->h_class[cb + c];
    }
    double2 *shift = m->nodes.as<double2>(), *wts = shift + N, *ywts = shift + 2 * N;
    double *r = m->r.as<double>(), *p = m->p.as<double>(), *w = m->w.as<double>();
    double *x = keep_x ? m->x.as<double>() : nullptr;
    const double *v = vec ? m->v.as<double>() : nullptr;
    double2 *psig = vec ? m->psig.as<double2>() : nullptr;
    double *y = vec ? m->y.as<double>() : nullptr;
    ColState *cs = m->cs.as<ColState>();
    ShiftState *ss = m->ss.as<ShiftState>();
    const int32_t *colour = m->colour.as<int32_t>();
    int *status_d = m->status.as<int>(), *count_d = m->count.as<int>();
    double *part = m->part.as<double>();
    MF_TRY(cudaMemcpyAsync(shift, h_nodes.data(), h_nodes.size() * sizeof(double2), cudaMemcpyHostToDevice, stream));
    MF_TRY(cudaMemcpyAsync(m->norm2.p, norm2.data(), C * sizeof(double), cudaMemcpyHostToDevice, stream));
    if (vec) MF_TRY(cudaMemcpyAsync(m->v.p, job.rhs, vec_bytes, cudaMemcpyHostToDevice, stream));
    MF_TRY(cudaMemsetAsync(status_d, 0, sizeof(int), stream));
    MF_TRY(cudaEventRecord(m->ev0, stream));
    k_mf_init<<<nblk, kThreads, 0, stream>>>(n, C, cb, colour, v, r, p, x);
    k_mf_init_scalars<<<C, 32, 0, stream>>>(C, N, m->norm2.as<double>(), cs, ss);
    int64_t launches = 2;
    if (vec) {
        k_mf_init_vec<<<nblk, kThreads, 0, stream>>>(n, C, N, v, psig, y);
        ++launches;
    }
    MF_TRY(cudaGetLastError());
    int status = LD_OK, k = 0;
    bool converged = false, stop = false;
    int64_t groups = 0, read = 0;
    auto consume = [&](int slot) {
        const int active = m->h_count[2 * slot], stat = m->h_count[2 * slot + 1];
        if (stat != 0) {
            status = stat;
            stop = true;
        } else if (active == 0) {
            converged = true;
            stop = true;
        }
    };
    for (k = 0; k < max_iter && !stop; ++k) {
        const int rc = m->fn(m->user, n, C, p, w, (void *)stream);
        if (rc != 0) {
            st->callback_rc = rc;
            cudaStreamSynchronize(stream);
            ld::set_last_error("matvec callback returned nonzero");
            status = LD_ECALLBACK;
            break;
        }
        k_mf_dots<<<nblk, kThreads, 0, stream>>>(n, C, cb, colour, v, r, p, w, cs, part);
        k_mf_tail<<<C, 32, 0, stream>>>(nblk, C, N, part, shift, tol, cs, ss, status_d);
        k_mf_update<<<nblk, kThreads, 0, stream>>>(n, C, N, r, p, w, x, cs, ss, ywts, psig, y);
        launches += 3;
        MF_TRY(cudaGetLastError());
        if ((k + 1) % kPollEvery == 0) {
            const int slot = (int)(groups % kRing);
            k_mf_count<<<1, 256, 0, stream>>>(C, cs, status_d, count_d + 2 * slot);
            ++launches;
            MF_TRY(cudaGetLastError());
            MF_TRY(cudaMemcpyAsync(m->h_count + 2 * slot, count_d + 2 * slot, 2 * sizeof(int),
                                   cudaMemcpyDeviceToHost, stream));
            MF_TRY(cudaEventRecord(m->evp[slot], stream));
            ++groups;
        }
        // read the polls that have landed; wait only when more than kLag are in flight, so
        // that the stream never drains while the host waits
        while (read < groups && !stop) {
            const int slot = (int)(read % kRing);
            if (groups - read > kLag) {
                MF_TRY(cudaEventSynchronize(m->evp[slot]));
            } else {
                const cudaError_t q = cudaEventQuery(m->evp[slot]);
                if (q == cudaErrorNotReady) {
                    (void)cudaGetLastError();
                    break;
                }
                MF_TRY(q);
            }
            consume(slot);
            ++read;
        }
    }
    if (status == LD_OK && !stop) {   // max_iter reached between polls: one final count
        k_mf_count<<<1, 256, 0, stream>>>(C, cs, status_d, count_d);
        ++launches;
        MF_TRY(cudaGetLastError());
        MF_TRY(cudaMemcpyAsync(m->h_count, count_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
        MF_TRY(cudaStreamSynchronize(stream));
        consume(0);
    }
    if (status != LD_OK && status != LD_ECALLBACK)
        ld::set_last_error(status == LD_ENOTSPD ? "p^T Q p <= 0: the operator is not SPD"
                                                : "non-finite value in the iteration");
    if (status == LD_OK && !converged) {
        ld::set_last_error("max_iter reached before every shifted system converged");
        status = LD_ENOTCONV;
    }
    k_mf_finish<<<C, 32, 0, stream>>>(C, N, wts, ss, cs, m->terms.as<double>(), m->seeds.as<double>(),
                                      m->iters.as<int>());
    launches += 1;
    MF_TRY(cudaGetLastError());
    MF_TRY(cudaEventRecord(m->ev1, stream));
    std::vector<int> it(C);
    MF_TRY(cudaMemcpyAsync(terms_out, m->terms.p, C * sizeof(double), cudaMemcpyDeviceToHost, stream));
    if (seeds_out) MF_TRY(cudaMemcpyAsync(seeds_out, m->seeds.p, C * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MF_TRY(cudaMemcpyAsync(it.data(), m->iters.p, C * sizeof(int), cudaMemcpyDeviceToHost, stream));
    if (vec && status == LD_OK && job.y_out)
        MF_TRY(cudaMemcpyAsync(job.y_out, y, vec_bytes, cudaMemcpyDeviceToHost, stream));
    MF_TRY(cudaStreamSynchronize(stream));
#undef MF_TRY
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, m->ev0, m->ev1);
    st->ms = ms;
    st->launches = launches;
    int kmax = 0;
    for (int c = 0; c < C; ++c) {
        st->column_iters += it[c];
        kmax = std::max(kmax, it[c]);
    }
    st->iters = kmax;
    if (status == LD_OK && keep_x && !vec) {
        m->have_x = true;
        m->x_cb = cb;
        m->x_cols = C;
    }
    return status;
}

int matfree_grad(Matfree *m, int n_params, const int *ids, void *dfn, void *duser, cudaStream_t stream,
                 double *grad, int *callback_rc) {
    *callback_rc = 0;
    if (!m->have_x) return LD_EINVAL;
    const int C = m->x_cols, cb = m->x_cb;
    const int64_t n = m->n;
    const int nblk = stream_blocks(n, C);
    auto fn = reinterpret_cast<ld_dmatvec_fn>(dfn);
    cudaError_t e;
#define MF_TRY(expr)                                                        \
    do {                                                                    \
        e = (expr);                                                         \
        if (e != cudaSuccess) {                                             \
            ld::set_last_error(cudaGetErrorString(e));                      \
            return LD_ECUDA;                                                \
        }                                                                   \
    } while (0)
    std::vector<double> cols(C);
    for (int k = 0; k < n_params; ++k) {
        // Y = (dQ / d eta) X into w (scratch after the solve), then sum_c v_c^T Y_c
        const int rc = fn(duser, ids[k], n, C, m->x.as<double>(), m->w.as<double>(), (void *)stream);
        if (rc != 0) {
            *callback_rc = rc;
            cudaStreamSynchronize(stream);
            ld::set_last_error("derivative callback returned nonzero");
            return LD_ECALLBACK;
        }
        k_mf_vdot<<<nblk, kThreads, 0, stream>>>(n, C, cb, m->colour.as<int32_t>(), nullptr, m->w.as<double>(),
                                                 m->part.as<double>());
        k_mf_colsum<<<C, 32, 0, stream>>>(nblk, C, m->part.as<double>(), m->terms.as<double>());
        MF_TRY(cudaGetLastError());
        MF_TRY(cudaMemcpyAsync(cols.data(), m->terms.p, C * sizeof(double), cudaMemcpyDeviceToHost, stream));
        MF_TRY(cudaStreamSynchronize(stream));
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += cols[c];
        grad[k] = s;
    }
#undef MF_TRY
    return LD_OK;
}

}  // namespace ld
