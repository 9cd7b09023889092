// Matrix-free operator: the probed rational log det of Sec. 2.1 when Q is available
// only as a product W = Q P computed by the caller (Sec. 1: the method touches Q only
// through matrix-vector products).
//
// The pass kernels of the stencil and CSR paths fuse the product into the CG update;
// here the product is the caller's, so the iteration is split around it:
//
//   W = Q P                         caller (ld_matvec_fn, on the context stream)
//   k_mf_dot       partials of p.w per column
//   k_mf_alpha     alpha_c = r.r / p.w                       (one warp per column)
//   k_mf_update_r  r -= alpha w; partials of r.r and v.r
//   k_mf_tail      beta_c, the CG-M shift recurrences, convergence (one warp per column)
//   k_mf_update_p  p = r + beta p
//
// Vectors are n x C row-major (the C probing-vector entries of a vertex adjacent), the
// layout the caller's product sees.  Every reduction is two-stage with a fixed order
// (per-block partials, then one warp per column), so results are bitwise repeatable.
//
// Shifted systems (Q + s I) x = v, s = -sigma_l, keep only the projections
// pi = v^T x^sigma and phi = v^T p^sigma (scalar recurrences of CG-M / COCG-M):
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} / (a_{k-1} zeta_{k-1} (1 + s a_k)
//                                             + a_k b_{k-1} (zeta_{k-1} - zeta_k))
//   a^s_k = a_k zeta_{k+1} / zeta_k,   b^s_k = b_k (zeta_{k+1} / zeta_k)^2
//   pi += a^s_k phi,                   phi = zeta_{k+1} (v^T r_{k+1}) + b^s_k phi
// with zeta_{-1} = zeta_0 = 1, a_{-1} = 1, b_{-1} = 0, phi_0 = v^T v.  A shift stops when
// |zeta_{k+1}| ||r_{k+1}|| <= tol ||v||; a column stops when all its shifts have.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/logdet.h"
#include "internal.h"

namespace {

constexpr int kThreads = 256;          // reduction / update blocks: 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kMaxBlocks = 152 * 4;    // partial-sum blocks (a multiple of the SM count)

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

// rows [r0, r1) of block b
__device__ __forceinline__ void block_rows(int64_t n, int64_t *r0, int64_t *r1) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    *r0 = (int64_t)blockIdx.x * per;
    *r1 = min(n, *r0 + per);
}

// Column-chunked block reduction helper: warp w of the block accumulated `acc` for column
// (chunk + lane) over rows r0 + w, r0 + w + 8, ...; combine the 8 warps in order.
__device__ __forceinline__ void block_partial(double acc, double *sm, double *out, int col, int C) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sm[w * 32 + lane] = acc;
    __syncthreads();
    if (w == 0 && col < C) {
        double s = 0.0;
        for (int k = 0; k < kWarps; ++k) s += sm[k * 32 + lane];
        out[(size_t)blockIdx.x * C + col] = s;
    }
    __syncthreads();
}

// sum over blocks of one column's partials: lanes take blocks lane, lane + 32, ... in
// order, then a fixed butterfly
__device__ __forceinline__ double warp_column_sum(const double *partial, int nblk, int C, int c) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[(size_t)b * C + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct ColState {        // per column, device
    double rr;           // r_k . r_k
    double alpha_prev;   // a_{k-1}
    double beta_prev;    // b_{k-1}
    double alpha;        // a_k (this iteration)
    double beta;         // b_k (for the p update)
    double vnorm;        // ||v_c||
    int active;          // 1 while some shift of the column is unconverged
    int iters;           // iterations the column ran
};

struct ShiftState {      // per (column, shift), device
    double2 zeta_prev, zeta, pi, phi;
    int done;
    int pad;
};

__global__ void k_mf_init(int64_t n, int C, int cb, const int32_t *__restrict__ colour,
                          double *__restrict__ r, double *__restrict__ p) {
    const int64_t total = n * C;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / C;
        const int c = (int)(e - i * C);
        const double v = colour[i] == cb + c ? 1.0 : 0.0;
        r[e] = v;
        p[e] = v;
    }
}

__global__ void k_mf_init_scalars(int C, int N, const double *__restrict__ class_size,
                                  ColState *__restrict__ cs, ShiftState *__restrict__ ss) {
    const int c = blockIdx.x;
    if (c >= C) return;
    const double m = class_size[c];
    if (threadIdx.x == 0) {
        ColState s;
        s.rr = m;
        s.alpha_prev = 1.0;
        s.beta_prev = 0.0;
        s.alpha = 0.0;
        s.beta = 0.0;
        s.vnorm = sqrt(m);
        s.active = m > 0.0 ? 1 : 0;   // an empty colour class contributes nothing
        s.iters = 0;
        cs[c] = s;
    }
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
        ShiftState t;
        t.zeta_prev = make_double2(1.0, 0.0);
        t.zeta = make_double2(1.0, 0.0);
        t.pi = make_double2(0.0, 0.0);
        t.phi = make_double2(m, 0.0);
        t.done = m > 0.0 ? 0 : 1;
        t.pad = 0;
        ss[(size_t)c * N + l] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_mf_dot(int64_t n, int C, const double *__restrict__ p,
                                                     const double *__restrict__ w,
                                                     const ColState *__restrict__ cs,
                                                     double *__restrict__ partial) {
    __shared__ double sm[kThreads];
    int64_t r0, r1;
    block_rows(n, &r0, &r1);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int chunk = 0; chunk < C; chunk += 32) {
        const int c = chunk + lane;
        double acc = 0.0;
        if (c < C && cs[c].active)
            for (int64_t i = r0 + wp; i < r1; i += kWarps) acc += p[i * C + c] * w[i * C + c];
        block_partial(acc, sm, partial, c, C);
    }
}

__global__ void k_mf_alpha(int nblk, int C, const double *__restrict__ partial, ColState *__restrict__ cs,
                           int *__restrict__ status) {
    const int c = blockIdx.x;
    const double pw = warp_column_sum(partial, nblk, C, c);
    if (threadIdx.x != 0 || !cs[c].active) return;
    if (!(pw > 0.0) || !isfinite(pw)) {           // p^T Q p <= 0: Q is not SPD
        atomicCAS(status, 0, (int)LD_ENOTSPD);
        cs[c].active = 0;
        cs[c].alpha = 0.0;
        return;
    }
    cs[c].alpha = cs[c].rr / pw;
}

__global__ void __launch_bounds__(kThreads) k_mf_update_r(int64_t n, int C, int cb,
                                                          const int32_t *__restrict__ colour,
                                                          double *__restrict__ r,
                                                          const double *__restrict__ w,
                                                          const ColState *__restrict__ cs,
                                                          double *__restrict__ part_rr,
                                                          double *__restrict__ part_vr) {
    __shared__ double sm[kThreads];
    int64_t r0, r1;
    block_rows(n, &r0, &r1);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int chunk = 0; chunk < C; chunk += 32) {
        const int c = chunk + lane;
        double rr = 0.0, vr = 0.0;
        if (c < C && cs[c].active) {
            const double a = cs[c].alpha;
            for (int64_t i = r0 + wp; i < r1; i += kWarps) {
                const double x = r[i * C + c] - a * w[i * C + c];
                r[i * C + c] = x;
                rr += x * x;
                if (colour[i] == cb + c) vr += x;
            }
        }
        block_partial(rr, sm, part_rr, c, C);
        block_partial(vr, sm, part_vr, c, C);
    }
}

__global__ void k_mf_tail(int nblk, int C, int N, const double *__restrict__ part_rr,
                          const double *__restrict__ part_vr, const double2 *__restrict__ shift,
                          double tol, ColState *__restrict__ cs, ShiftState *__restrict__ ss,
                          int *__restrict__ status) {
    const int c = blockIdx.x, lane = threadIdx.x;
    const double rr_new = warp_column_sum(part_rr, nblk, C, c);
    const double vr = warp_column_sum(part_vr, nblk, C, c);
    ColState col = cs[c];
    if (!col.active) return;
    if (!isfinite(rr_new) || !isfinite(vr)) {
        if (lane == 0) {
            atomicCAS(status, 0, (int)LD_ENUMERIC);
            cs[c].active = 0;
        }
        return;
    }
    const double a = col.alpha, ap = col.alpha_prev, bp = col.beta_prev;
    const double b = rr_new / col.rr;
    const double rnorm = sqrt(rr_new);
    bool all_done = true;
    for (int l = lane; l < N; l += 32) {
        ShiftState t = ss[(size_t)c * N + l];
        if (!t.done) {
            const double2 s = shift[l];
            // den = a_{k-1} zeta_{k-1} (1 + s a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)
            const double2 one_sa = make_double2(1.0 + s.x * a, s.y * a);
            const double2 den = cadd(cmul(cscale(t.zeta_prev, ap), one_sa),
                                     cscale(csub(t.zeta_prev, t.zeta), a * bp));
            const double2 znew = cdiv(cscale(cmul(t.zeta, t.zeta_prev), ap), den);
            const double2 ratio = cdiv(znew, t.zeta);
            const double2 as = cscale(ratio, a);
            t.pi = cadd(t.pi, cmul(as, t.phi));
            const double2 bs = cscale(cmul(ratio, ratio), b);
            t.phi = cadd(cscale(znew, vr), cmul(bs, t.phi));
            t.zeta_prev = t.zeta;
            t.zeta = znew;
            if (cabs_(znew) * rnorm <= tol * col.vnorm) t.done = 1;
            if (!isfinite(t.pi.x) || !isfinite(t.pi.y)) {
                atomicCAS(status, 0, (int)LD_ENUMERIC);
                t.done = 1;
            }
            ss[(size_t)c * N + l] = t;
        }
        all_done = all_done && t.done;
    }
    all_done = __all_sync(0xffffffffu, all_done);
    if (lane == 0) {
        col.rr = rr_new;
        col.alpha_prev = a;
        col.beta_prev = b;
        col.beta = b;
        col.iters += 1;
        col.active = all_done ? 0 : 1;
        cs[c] = col;
    }
}

__global__ void k_mf_update_p(int64_t n, int C, const double *__restrict__ r, double *__restrict__ p,
                              const ColState *__restrict__ cs) {
    const int64_t total = n * C;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        if (cs[c].active) p[e] = r[e] + cs[c].beta * p[e];
    }
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

// term_c = Re sum_l weight_l pi_{c,l}, lanes over shifts in order, then a fixed butterfly
__global__ void k_mf_finish(int C, int N, const double2 *__restrict__ weight, const ShiftState *__restrict__ ss,
                            const ColState *__restrict__ cs, double *__restrict__ terms,
                            int *__restrict__ iters) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double s = 0.0;
    for (int l = lane; l < N; l += 32) {
        const double2 w = weight[l], pi = ss[(size_t)c * N + l].pi;
        s += w.x * pi.x - w.y * pi.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        terms[c] = s;
        iters[c] = cs[c].iters;
    }
}

}  // namespace

namespace ld {

struct Matfree {
    int64_t n = 0;
    int C = 0, N = 0;
    ld_matvec_fn fn = nullptr;
    void *user = nullptr;
    int32_t *colour = nullptr;       // device, n
    double *r = nullptr, *p = nullptr, *w = nullptr;   // device, n x C
    double *part = nullptr;          // device, 3 x nblk x C
    double *class_size = nullptr;    // device, C
    double2 *nodes = nullptr;        // device, shift[N], weight[N]
    ColState *cs = nullptr;
    ShiftState *ss = nullptr;
    int *status = nullptr;           // device
    double *terms = nullptr;         // device, C
    int *iters = nullptr;            // device, C
    int *count = nullptr;            // device: active count, status
    int *h_count = nullptr;          // pinned host copy
    std::vector<double> h_class;
    int nblk = 1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    ~Matfree() {
        cudaFree(colour);
        cudaFree(r);
        cudaFree(p);
        cudaFree(w);
        cudaFree(part);
        cudaFree(class_size);
        cudaFree(nodes);
        cudaFree(cs);
        cudaFree(ss);
        cudaFree(status);
        cudaFree(terms);
        cudaFree(iters);
        cudaFree(count);
        if (h_count) cudaFreeHost(h_count);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

void matfree_destroy(Matfree *m) { delete m; }

int matfree_create(Matfree **out, int64_t n, const int32_t *colour, int C, int N, void *fn, void *user) {
    *out = nullptr;
    Matfree *m = new (std::nothrow) Matfree();
    if (!m) return (int)cudaErrorMemoryAllocation;
    m->n = n;
    m->C = C;
    m->N = N;
    m->fn = reinterpret_cast<ld_matvec_fn>(fn);
    m->user = user;
    m->nblk = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxBlocks, (n + 31) / 32));
    m->h_class.assign(C, 0.0);
    for (int64_t i = 0; i < n; ++i) m->h_class[colour[i]] += 1.0;
    const size_t vec = (size_t)n * C * sizeof(double);
    cudaError_t e = cudaSuccess;
#define MF_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
    MF_ALLOC(m->colour, (size_t)n * sizeof(int32_t));
    MF_ALLOC(m->r, vec);
    MF_ALLOC(m->p, vec);
    MF_ALLOC(m->w, vec);
    MF_ALLOC(m->part, (size_t)3 * m->nblk * C * sizeof(double));
    MF_ALLOC(m->class_size, (size_t)C * sizeof(double));
    MF_ALLOC(m->nodes, (size_t)2 * N * sizeof(double2));
    MF_ALLOC(m->cs, (size_t)C * sizeof(ColState));
    MF_ALLOC(m->ss, (size_t)C * N * sizeof(ShiftState));
    MF_ALLOC(m->status, sizeof(int));
    MF_ALLOC(m->terms, (size_t)C * sizeof(double));
    MF_ALLOC(m->iters, (size_t)C * sizeof(int));
    MF_ALLOC(m->count, 2 * sizeof(int));
#undef MF_ALLOC
    if (e == cudaSuccess) e = cudaMallocHost((void **)&m->h_count, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev1);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->colour, colour, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete m;
        return (int)e;
    }
    *out = m;
    return 0;
}

int matfree_solve(Matfree *m, int cb, int ce, const std::complex<double> *sigma,
                  const std::complex<double> *weight, double tol, int max_iter, cudaStream_t stream,
                  double *terms_out, MatfreeStats *st) {
    const int C = ce - cb, N = m->N;
    const int64_t n = m->n;
    st->iters = 0;
    st->launches = 0;
    st->callback_rc = 0;
    st->ms = 0.0f;
    if (C <= 0) return LD_OK;
    std::vector<double2> h_nodes(2 * N);
    for (int l = 0; l < N; ++l) {
        h_nodes[l] = make_double2(-sigma[l].real(), -sigma[l].imag());   // s_l = -sigma_l
        h_nodes[N + l] = make_double2(weight[l].real(), weight[l].imag());
    }
    cudaError_t e;
#define MF_TRY(expr)                                                        \
    do {                                                                    \
        e = (expr);                                                         \
        if (e != cudaSuccess) {                                             \
            ld::set_last_error(cudaGetErrorString(e));                      \
            return LD_ECUDA;                                                \
        }                                                                   \
    } while (0)
    MF_TRY(cudaMemcpyAsync(m->nodes, h_nodes.data(), h_nodes.size() * sizeof(double2),
                           cudaMemcpyHostToDevice, stream));
    MF_TRY(cudaMemcpyAsync(m->class_size, m->h_class.data() + cb, C * sizeof(double),
                           cudaMemcpyHostToDevice, stream));
    MF_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), stream));
    const int egrid = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (n * C + kThreads - 1) / kThreads));
    const int nblk = m->nblk;
    double *part_pw = m->part, *part_rr = m->part + (size_t)nblk * C, *part_vr = m->part + (size_t)2 * nblk * C;
    MF_TRY(cudaEventRecord(m->ev0, stream));
    k_mf_init<<<egrid, kThreads, 0, stream>>>(n, C, cb, m->colour, m->r, m->p);
    k_mf_init_scalars<<<C, 32, 0, stream>>>(C, N, m->class_size, m->cs, m->ss);
    MF_TRY(cudaGetLastError());
    int64_t launches = 2;
    constexpr int kCheckEvery = 8;
    int status = LD_OK, k = 0;
    bool converged = false;
    for (k = 0; k < max_iter; ++k) {
        const int rc = m->fn(m->user, n, C, m->p, m->w, (void *)stream);
        if (rc != 0) {
            st->callback_rc = rc;
            cudaStreamSynchronize(stream);
            ld::set_last_error("matvec callback returned nonzero");
            status = LD_ECALLBACK;
            break;
        }
        k_mf_dot<<<nblk, kThreads, 0, stream>>>(n, C, m->p, m->w, m->cs, part_pw);
        k_mf_alpha<<<C, 32, 0, stream>>>(nblk, C, part_pw, m->cs, m->status);
        k_mf_update_r<<<nblk, kThreads, 0, stream>>>(n, C, cb, m->colour, m->r, m->w, m->cs, part_rr, part_vr);
        k_mf_tail<<<C, 32, 0, stream>>>(nblk, C, N, part_rr, part_vr, m->nodes, tol, m->cs, m->ss, m->status);
        k_mf_update_p<<<egrid, kThreads, 0, stream>>>(n, C, m->r, m->p, m->cs);
        launches += 5;
        MF_TRY(cudaGetLastError());
        if ((k + 1) % kCheckEvery == 0 || k + 1 == max_iter) {
            k_mf_count<<<1, 256, 0, stream>>>(C, m->cs, m->status, m->count);
            launches += 1;
            MF_TRY(cudaGetLastError());
            MF_TRY(cudaMemcpyAsync(m->h_count, m->count, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
            MF_TRY(cudaStreamSynchronize(stream));
            const int active = m->h_count[0];
            const int stat = m->h_count[1];
            if (stat != 0) {
                status = stat;
                ld::set_last_error(stat == LD_ENOTSPD ? "p^T Q p <= 0: the operator is not SPD"
                                                      : "non-finite value in the iteration");
                ++k;
                break;
            }
            if (active == 0) {
                converged = true;
                ++k;
                break;
            }
        }
    }
    if (status == LD_OK && !converged) {
        ld::set_last_error("max_iter reached before every shifted system converged");
        status = LD_ENOTCONV;
    }
    k_mf_finish<<<C, 32, 0, stream>>>(C, N, m->nodes + N, m->ss, m->cs, m->terms, m->iters);
    launches += 1;
    MF_TRY(cudaGetLastError());
    MF_TRY(cudaEventRecord(m->ev1, stream));
    std::vector<int> it(C);
    MF_TRY(cudaMemcpyAsync(terms_out, m->terms, C * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MF_TRY(cudaMemcpyAsync(it.data(), m->iters, C * sizeof(int), cudaMemcpyDeviceToHost, stream));
    MF_TRY(cudaStreamSynchronize(stream));
#undef MF_TRY
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, m->ev0, m->ev1);
    st->ms = ms;
    st->iters = k;
    st->launches = launches;
    st->column_iters = 0;
    for (int c = 0; c < C; ++c) st->column_iters += it[c];
    return status;
}

}  // namespace ld
