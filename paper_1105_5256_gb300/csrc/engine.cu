// CUDA engine entry points and the kernels outside the per-iteration pass:
// vector initialisation, the one-CTA and batched persistent engines, the
// vector form (log(Q) V), operator application, gradients (sm_103a).
#include "engine_device.cuh"
#include "engine_lean.cuh"
#include "engine_lean3d.cuh"

namespace ld {

// ------------------------------------------------------------------ CTA engine
// One CTA runs a tile's whole solve (small problems): the same fused pass,
// block barriers only, sets alternating inside the kernel (coherent loads).
template <typename V, int T, int KIND>
__global__ void __launch_bounds__(256) k_cta_solve(Solve s, int max_iter) {
    constexpr int K = NDOT * T;
    const int tile = blockIdx.x;
    __shared__ double red[8 * K];
    __shared__ double sums[K];
    __shared__ int done;
    if (threadIdx.x == 0) done = s.tile_done[tile];
    __syncthreads();
    for (int it = 0; it < max_iter && !done; ++it) {
        const int cur = it & 1;
        Dots<V, T> d;
        d.zero();
        pass_points<V, T, KIND, false>(s, tile, cur, threadIdx.x, blockDim.x, d);
        V flat[K];
        d.flat(flat);
        block_sum_to<V, K>(flat, red, sums);
        fused_tail(s, tile, cur, sums);
        __syncthreads();
        if (threadIdx.x == 0) done = s.tile_done[tile] || (*s.status != 0);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ batched engine
// Many independent problems (one Solve each, in device memory) in one
// persistent launch: CTAs pull (instance, tile) items from an atomic queue
// (the host sorts items longest first), initialise the tile's state and run
// its whole solve with block barriers, exactly as the one-CTA engine does.

// tile state as the init kernels set it (all colours of the instance active)
template <typename V, int T>
__device__ void tile_init(const Solve &s, int tile) {
    const int64_t n = s.op.n;
    const int64_t off = (int64_t)tile * n * T;
    V *r = static_cast<V *>(s.rbuf[0]) + off;
    V *w = static_cast<V *>(s.wbuf[0]) + off;
    V *p = static_cast<V *>(s.pbuf[0]) + off;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int lc = s.colour[i] - tile * T;
        V a[T], z[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            a[t] = (lc == t && s.class_size[tile * T + t] > 0.0) ? (V)1 : (V)0;
            z[t] = (V)0;
        }
        stpack<V, T>(r, i, a);
        stpack<V, T>(w, i, z);
        stpack<V, T>(p, i, z);
    }
    const int N = s.nshift;
    for (int q = threadIdx.x; q < T * N; q += blockDim.x) {
        const int c = tile * T + q / N;
        const double vv = s.class_size[c];
        const int idx = c * N + (q % N);
        s.zeta[idx] = make_double2(1.0, 0.0);
        s.zeta_prev[idx] = make_double2(1.0, 0.0);
        s.pi[idx] = make_double2(0.0, 0.0);
        s.phi[idx] = make_double2(vv, 0.0);
        s.sh_active[idx] = (uint8_t)(vv > 0.0);
    }
    if (threadIdx.x < T) {
        const int c = tile * T + threadIdx.x;
        const double vv = s.class_size[c];
        s.rho[c] = vv;
        s.vnorm2[c] = vv;
        s.alpha[c] = 0.0;
        s.beta[c] = 0.0;
        s.alpha_prev[c] = 1.0;
        s.beta_prev[c] = 0.0;
        s.pi0[c] = 0.0;
        s.phi0[c] = vv;
        s.col_active[c] = vv > 0.0;
        s.col_iters[c] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int t = 0; t < T; ++t) any |= s.col_active[tile * T + t];
        s.tile_done[tile] = !any;
        s.tile_ctr[tile] = 0;
        s.tile_par[tile] = 0;
    }
    __syncthreads();
}

// A tile's whole solve in the calling CTA (block barriers only).
template <typename V, int T, int KIND>
__device__ void tile_solve(const Solve &s, int tile, int max_iter, double *red, double *sums,
                           int *done) {
    constexpr int K = NDOT * T;
    if (threadIdx.x == 0) *done = s.tile_done[tile];
    __syncthreads();
    for (int it = 0; it < max_iter && !*done; ++it) {
        const int cur = it & 1;
        Dots<V, T> d;
        d.zero();
        pass_points<V, T, KIND, false>(s, tile, cur, threadIdx.x, blockDim.x, d);
        V flat[K];
        d.flat(flat);
        block_sum_to<V, K>(flat, red, sums);
        fused_tail(s, tile, cur, sums);
        __syncthreads();
        if (threadIdx.x == 0) *done = s.tile_done[tile] || (*s.status != 0);
        __syncthreads();
    }
}

// The persistent batch kernel: 2D lattice instances run the streaming sweep (the
// CTA walks every strip of its tile, all rows, per pass), the other kinds the
// gather pass; either way one CTA owns the tile's whole solve.
template <typename V, int T>
__global__ void __launch_bounds__(SW * stream_groups<V, T>(), stream_min_blocks_t<V, T>())
    k_batch_solve(const Solve *solves, const int2 *items, int nitems, int *queue, int max_iter) {
    constexpr int K = NDOT * T, G = stream_groups<V, T>(), NW = SW * G / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[NW * K];
    __shared__ double sums[K];
    __shared__ int done, item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(queue, 1);
        __syncthreads();
        const int my = item;
        if (my >= nitems) break;
        const int2 it = items[my];
        const Solve &s = solves[it.x];
        const int tile = it.y;
        tile_init<V, T>(s, tile);
        const int kind = s.op.kind;
        if (kind == KIND_2D5 || kind == KIND_2D13_SQ) {
            const int W = kind == KIND_2D13_SQ ? Strip<KIND_2D13_SQ>::W : Strip<KIND_2D5>::W;
            const int strips = (s.op.nx + W - 1) / W;
            if (threadIdx.x == 0) done = s.tile_done[tile];
            __syncthreads();
            for (int pass = 0; pass < max_iter && !done; ++pass) {
                const int cur = pass & 1;
                StreamAcc<V, T / G> acc;
                acc.zero();
                for (int st = 0; st < strips; ++st) {
                    if (kind == KIND_2D13_SQ)
                        stream_sweep<V, T, G, KIND_2D13_SQ, false>(s, tile, cur, st, 0, s.op.ny, smem, acc);
                    else
                        stream_sweep<V, T, G, KIND_2D5, false>(s, tile, cur, st, 0, s.op.ny, smem, acc);
                }
                stream_cta_sums<V, T, G>(acc, smem, sums);
                fused_tail(s, tile, cur, sums);
                __syncthreads();
                if (threadIdx.x == 0) done = s.tile_done[tile] || (*s.status != 0);
                __syncthreads();
            }
        } else if (kind == KIND_3D7) {
            tile_solve<V, T, KIND_3D7>(s, tile, max_iter, red, sums, &done);
        } else {
            tile_solve<V, T, KIND_CSR>(s, tile, max_iter, red, sums, &done);
        }
        // per-column terms Re sum_l alpha_l pi_{c,l}
        if (threadIdx.x < T) {
            const int c = tile * T + threadIdx.x;
            double acc = 0.0;
            for (int l = 0; l < s.nshift; ++l) {
                const double2 w = s.weight[l], p = s.pi[c * s.nshift + l];
                acc += w.x * p.x - w.y * p.y;
            }
            s.terms[c] = acc;
        }
        __syncthreads();
    }
}

// per instance: remaining tiles and status before the solve
__global__ void k_batch_prep(const Solve *solves, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        *solves[i].remaining = solves[i].ntiles;
        *solves[i].status = 0;
    }
}

// per instance (fixed column order): log det, the projected seed sum, convergence flag
__global__ void k_batch_finish(const Solve *solves, const int *ncolours, int count, double *logdet,
                               double *seed, int *flag, int *iters, int *tile_passes) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const Solve &s = solves[i];
        double a = 0.0, b = 0.0;
        int it = 0;
        for (int c = 0; c < ncolours[i]; ++c) {
            a += s.terms[c];
            b += s.pi0[c];
            it = max(it, s.col_iters[c]);
        }
        logdet[i] = a;
        seed[i] = b;
        iters[i] = it;
        // passes the instance's tiles ran: a tile runs until its last column stops
        int tp = 0;
        for (int t = 0; t < s.ntiles; ++t) {
            int m = 0;
            for (int k = 0; k < s.T; ++k) m = max(m, s.col_iters[t * s.T + k]);
            tp += m;
        }
        tile_passes[i] = tp;
        flag[i] = *s.status != 0 ? *s.status : (*s.remaining > 0 ? -1 : 0);
    }
}

template <typename V, int T, int KIND>
struct BatchLauncher {
    static int run(const Solve *solves, const int2 *items, int nitems, int *queue, int max_iter,
                   int grid, cudaStream_t st) {
        constexpr int G = stream_groups<V, T>();
        k_batch_solve<V, T><<<grid, SW * G, stream_smem_bytes<V, T, G>(), st>>>(solves, items, nitems,
                                                                              queue, max_iter);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct BatchOcc {
    static int run(int *out) {
        constexpr int G = stream_groups<V, T>();
        constexpr size_t sm = stream_smem_bytes<V, T, G>();
        cudaError_t e = cudaFuncSetAttribute(k_batch_solve<V, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return (int)e;
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_batch_solve<V, T>, SW * G, sm);
    }
};

// ------------------------------------------------------------------ shifted vectors (mode V)
// Optional vector form of CG-M: besides the projections, keep every shifted search
// direction p^sigma (complex) and accumulate y = Re sum_l alpha_l x^{sigma_l} directly,
//   x^sigma += alpha^sigma_k p^sigma_k,  p^sigma = zeta_{k+1} r_{k+1} + beta^sigma_k p^sigma,
// with r_{k+1} = r_k - alpha_k w_k from the set the pass just wrote.  Gives log(Q) v for
// arbitrary right-hand sides and cross-checks the projected recurrences.
// psig: [ncols][N][n] complex; y: [ntiles][n][T] in FP64.
template <typename V, int T>
__global__ void k_modev(Solve s, int nxt, double2 *psig, double *y) {
    const int64_t n = s.op.n;
    const int N = s.nshift;
    const int64_t total = (int64_t)s.ntiles * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(q / n);
        const int64_t i = q - (int64_t)tile * n;
        const Pack<V, T> rk = ldpack<V, T, false>(static_cast<const V *>(nxt ? s.rbuf[1] : s.rbuf[0]), q);
        const Pack<V, T> wk = ldpack<V, T, false>(static_cast<const V *>(nxt ? s.wbuf[1] : s.wbuf[0]), q);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int c = tile * T + t;
            const double r1 = (double)rk.v[t] - s.alpha[c] * (double)wk.v[t];   // r_{k+1}
            double acc = 0.0;
            for (int l = 0; l < N; ++l) {
                const int idx = c * N + l;
                const double2 as = s.asig[idx];
                if (as.x == 0.0 && as.y == 0.0) continue;
                double2 *pp = psig + (int64_t)idx * n + i;
                const double2 p = *pp;
                const double2 wgt = cmul(s.weight[l], as);          // alpha_l alpha^sigma
                acc += wgt.x * p.x - wgt.y * p.y;                    // Re(alpha_l x^sigma increment)
                const double2 zn = s.zeta[idx];
                *pp = cadd(cscale(r1, zn), cmul(s.bsig[idx], p));
            }
            y[q * T + t] += acc;
        }
    }
}

__global__ void k_modev_clear(Solve s) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < s.ncols * s.nshift; q += gridDim.x * blockDim.x)
        s.asig[q] = make_double2(0.0, 0.0);
}

// p^sigma_0 = v for every shift (v read from the initial residual set 0), y = 0
template <typename V, int T>
__global__ void k_modev_init(Solve s, double2 *psig, double *y) {
    const int64_t n = s.op.n;
    const int N = s.nshift;
    const int64_t total = (int64_t)s.ntiles * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(q / n);
        const int64_t i = q - (int64_t)tile * n;
        const Pack<V, T> r0 = ldpack<V, T, false>(static_cast<const V *>(s.rbuf[0]), q);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int c = tile * T + t;
            for (int l = 0; l < N; ++l) psig[((int64_t)c * N + l) * n + i] = make_double2((double)r0.v[t], 0.0);
            y[q * T + t] = 0.0;
        }
    }
}

template <typename V, int T, int KIND>
struct ModeVLauncher {
    static int run(const Solve &s, int which, int nxt, double2 *psig, double *y, cudaStream_t st) {
        const int64_t total = (int64_t)s.ntiles * s.op.n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks < 1) blocks = 1;
        if (which == 0)
            k_modev_init<V, T><<<blocks, 256, 0, st>>>(s, psig, y);
        else {
            k_modev<V, T><<<blocks, 256, 0, st>>>(s, nxt, psig, y);
            k_modev_clear<<<64, 256, 0, st>>>(s);
        }
        return (int)cudaGetLastError();
    }
};

// ------------------------------------------------------------------ init / flush / finish
template <typename V, int T>
__global__ void k_init_vectors(Solve s) {
    const int64_t n = s.op.n;
    const int64_t total = (int64_t)s.ntiles * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(q / n);
        const int64_t i = q - (int64_t)tile * n;
        const int lc = s.colour[i] - tile * T;
        V a[T], z[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int c = tile * T + t;
            a[t] = (lc == t && s.col_active[c]) ? (V)1 : (V)0;
            z[t] = (V)0;
        }
        stpack<V, T>(static_cast<V *>(s.rbuf[0]), q, a);
        stpack<V, T>(static_cast<V *>(s.wbuf[0]), q, z);
        stpack<V, T>(static_cast<V *>(s.pbuf[0]), q, z);
        if (s.keep_x0) stpack<V, T>(static_cast<V *>(s.x), q, z);
    }
}

// the final x += alpha_J p_J of each tile (its last pass J wrote p_J to set tile_par)
template <typename V, int T>
__global__ void k_flush_x(Solve s) {
    const int64_t n = s.op.n;
    const int64_t total = (int64_t)s.ntiles * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(q / n);
        if (!s.tile_done[tile]) continue;
        const V *p = static_cast<const V *>(s.pbuf[s.tile_par[tile]]);
        V *x = static_cast<V *>(s.x);
        const Pack<V, T> pp = ldpack<V, T, false>(p, q);
        Pack<V, T> xo = ldpack<V, T, false>(x, q);
#pragma unroll
        for (int t = 0; t < T; ++t) xo.v[t] = fma((V)s.alpha[tile * T + t], pp.v[t], xo.v[t]);
        *reinterpret_cast<Pack<V, T> *>(x + q * T) = xo;
    }
}

__global__ void k_init_scalars(Solve s, int col_begin, int col_end, const double *class_size) {
    const int N = s.nshift;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < s.ncols * N; q += gridDim.x * blockDim.x) {
        const int c = q / N;
        const double vv = class_size[c];
        const int act = (c >= col_begin && c < col_end && vv > 0.0);
        s.zeta[q] = make_double2(1.0, 0.0);
        s.zeta_prev[q] = make_double2(1.0, 0.0);
        s.pi[q] = make_double2(0.0, 0.0);
        s.phi[q] = make_double2(vv, 0.0);
        s.sh_active[q] = (uint8_t)act;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < s.ncols; c += gridDim.x * blockDim.x) {
        const double vv = class_size[c];
        const int act = (c >= col_begin && c < col_end && vv > 0.0);
        s.rho[c] = vv;
        s.vnorm2[c] = vv;
        s.alpha[c] = 0.0;
        s.beta[c] = 0.0;
        s.alpha_prev[c] = 1.0;
        s.beta_prev[c] = 0.0;
        s.pi0[c] = 0.0;
        s.phi0[c] = vv;
        s.col_active[c] = act;
        s.col_iters[c] = 0;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.ntiles; t += gridDim.x * blockDim.x) {
        s.tile_ctr[t] = 0;
        s.tile_par[t] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.status = 0;
}

// tile_done / remaining from the column flags (one block)
__global__ void k_init_tiles(Solve s) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < s.ntiles; t += blockDim.x) {
        int any = 0;
        for (int k = 0; k < s.T; ++k) any |= s.col_active[t * s.T + k];
        s.tile_done[t] = !any;
        if (any) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *s.remaining = cnt;
}

// terms[c] = Re sum_l alpha_l pi_{c,l}; result = sums over [cb, ce) in column order.
__global__ void k_finish(Solve s, int cb, int ce) {
    const int N = s.nshift;
    for (int c = threadIdx.x; c < s.ncols; c += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < N; ++l) {
            const double2 w = s.weight[l], p = s.pi[c * N + l];
            acc += w.x * p.x - w.y * p.y;
        }
        s.terms[c] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0, seed = 0.0;
        for (int c = cb; c < ce; ++c) { sum += s.terms[c]; seed += s.pi0[c]; }
        s.result[0] = sum;
        s.result[1] = seed;
    }
}

// ------------------------------------------------------------------ operator apply
template <typename V, int T, int KIND>
__global__ void k_apply(Operator op, int ntiles, const V *x, V *y) {
    const int64_t n = op.n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)ntiles * n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(q / n);
        const int64_t i = q - (int64_t)tile * n;
        LoadP<V, T, true> ld;
        ld.p = x + (int64_t)tile * n * T;
        V w[T], self[T];
        apply_row<V, T, KIND>(op, i, ld, w, self);
        stpack<V, T>(y + (int64_t)tile * n * T, i, w);
    }
}

// ------------------------------------------------------------------ bounded-wait self-test
// One CTA waits on an mbarrier that nothing arrives at: the bounded wait must give up
// after limit_ns and report DEV_TIMEOUT through the status word, leaving the context
// usable (the failure path of the bulk-copy waits, exercised without a fault).
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) *status = ok ? DEV_OK : DEV_TIMEOUT;
}

// ------------------------------------------------------------------ diagonal coefficients
__global__ void k_fill_diag(Operator op, double *dd, float *df) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < op.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double d = op.field_d ? op.kappa2 * op.field_d[i] : op.kappa2;
        if (op.mask) d += op.tau * (double)op.mask[i];
        dd[i] = d;
        df[i] = (float)d;
    }
}

// ------------------------------------------------------------------ reliable updates
// Residual replacement for mixed precision: the seed solution is x_hi (FP64) + x_lo
// (vector precision, the pass's running correction).  Folding moves x_lo into x_hi;
// the true residual v - Q x is then formed with FP64 arithmetic throughout.
template <typename V, int T>
__global__ void k_fold_x(Solve s) {
    const int64_t total = (int64_t)s.ntiles * s.op.n * T;
    V *xl = static_cast<V *>(s.x);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        s.xhi[e] += (double)xl[e];
        xl[e] = (V)0;
    }
}

template <typename V, int T>
struct LoadWiden {   // an FP64 view of a vector-precision block (or of x_hi itself)
    const V *p;
    const double *d;
    __device__ __forceinline__ void operator()(int64_t j, double (&o)[T]) const {
#pragma unroll
        for (int t = 0; t < T; ++t) o[t] = d ? d[j * T + t] : (double)p[j * T + t];
    }
};

// grid (blocks, ntiles): one tile per blockIdx.y; per-column sums by block reduction
template <typename V, int T, int KIND>
__global__ void __launch_bounds__(256) k_true_residual(Solve s, int set, int cb, int ce, int replace,
                                                        double *norm2) {
    const int tile = blockIdx.y;
    const int64_t n = s.op.n;
    const int64_t off = (int64_t)tile * n * T;
    LoadWiden<V, T> ld;
    ld.p = static_cast<const V *>(s.x) + off;
    ld.d = s.xhi ? s.xhi + off : nullptr;
    V *r = static_cast<V *>(set ? s.rbuf[1] : s.rbuf[0]) + off;
    const bool write = replace && !s.tile_done[tile];
    double acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double w[T], self[T];
        apply_row<double, T, KIND>(s.op, i, ld, w, self);
        const int col = s.colour[i];
        V out[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int c = tile * T + t;
            const double v = (col == c && c >= cb && c < ce) ? 1.0 : 0.0;
            const double res = (c >= cb && c < ce) ? v - w[t] : 0.0;
            acc[t] = fma(res, res, acc[t]);
            out[t] = (V)res;
        }
        if (write) stpack<V, T>(r, i, out);
    }
    __shared__ double red[8 * T];
    __shared__ double tot[T];
    block_sum_to<double, T>(acc, red, tot);
    if (threadIdx.x < T) atomicAdd(&norm2[tile * T + threadIdx.x], tot[threadIdx.x]);
}

// ------------------------------------------------------------------ gradient (backward)
// g_eta = sum_c (E_eta v_c)^T x0_c = sum_i sum_j E_ij x0[i, colour(j)], E = dQ/d eta.
// E per parameter id: kappa2 -> scale*diag(field or 1) (grid 5/7-pt), 2*scale*Q1 (13-pt);
// tau -> scale*diag(mask); scale -> Q/scale.
template <typename V>
__device__ __forceinline__ double x0_at(const Solve &s, int64_t i, int c) {
    const int tile = c / s.T, lane = c - tile * s.T;
    const int64_t e = ((int64_t)tile * s.op.n + i) * s.T + lane;
    if (s.xhi) return s.xhi[e];
    return (double)static_cast<const V *>(s.x)[e];
}

template <typename V>
__device__ double grad_row(const Solve &s, int pid, int64_t i) {
    const Operator &op = s.op;
    const int ci = s.colour[i];
    if (op.kind == KIND_CSR) {
        // scale: E = Q0 = Q / s; the values on the device are Q's (scaled), so this sums
        // (Q v)^T x and the caller divides by s
        if (pid != 2) return 0.0;
        double g = 0.0;
        for (int64_t e = op.rowptr[i]; e < op.rowptr[i + 1]; ++e)
            g += op.val_d[e] * x0_at<V>(s, i, s.colour[op.colidx[e]]);
        return g;
    }
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int64_t yz = i / nx;
    const int x = (int)(i - yz * nx);
    const int z = (int)(yz / ny), y = (int)(yz - (int64_t)z * ny);
    const bool per = op.periodic;
    // neighbour index with wrap/truncation; -1 when absent
    auto nbr = [&](int dx, int dy, int dz) -> int64_t {
        int xx = x + dx, yy = y + dy, zz = z + dz;
        if (per) {
            xx = ((xx % nx) + nx) % nx;
            yy = ((yy % ny) + ny) % ny;
            zz = ((zz % nz) + nz) % nz;
        } else if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) {
            return -1;
        }
        return (int64_t)xx + (int64_t)nx * ((int64_t)yy + (int64_t)ny * zz);
    };
    if (op.kind == KIND_2D5 || op.kind == KIND_3D7) {
        const bool is3 = op.kind == KIND_3D7;
        if (pid == 0) {
            const double f = op.field_d ? op.field_d[i] : 1.0;
            return op.scale * f * x0_at<V>(s, i, ci);
        }
        if (pid == 1) {
            return op.mask ? op.scale * (double)op.mask[i] * x0_at<V>(s, i, ci) : 0.0;
        }
        // scale: E = Q / scale
        const double k2 = op.field_d ? op.kappa2 * op.field_d[i] : op.kappa2;
        double dg = k2 + (is3 ? 6.0 : 4.0) + (op.mask ? op.tau * (double)op.mask[i] : 0.0);
        double g = dg * x0_at<V>(s, i, ci);
        const int D[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        for (int q = 0; q < (is3 ? 6 : 4); ++q) {
            const int64_t j = nbr(D[q][0], D[q][1], D[q][2]);
            if (j >= 0) g -= x0_at<V>(s, i, s.colour[j]);
        }
        return g;
    }
    // 13-point Matern: kappa2 -> 2*scale*Q1; scale -> Q/scale = Q1^2
    const double a = op.kappa2 + 4.0;
    if (pid == 0) {
        double g = 2.0 * op.scale * a * x0_at<V>(s, i, ci);
        const int D[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        for (int q = 0; q < 4; ++q) {
            const int64_t j = nbr(D[q][0], D[q][1], 0);
            if (j >= 0) g -= 2.0 * op.scale * x0_at<V>(s, i, s.colour[j]);
        }
        return g;
    }
    if (pid == 1) return 0.0;
    int nbx, nby;
    if (per) { nbx = 2; nby = 2; } else { nbx = (x > 0) + (x < nx - 1); nby = (y > 0) + (y < ny - 1); }
    double g = (a * a + nbx + nby) * x0_at<V>(s, i, ci);
    const int DX[12] = {-1, 1, 0, 0, -2, 2, 0, 0, -1, 1, -1, 1};
    const int DY[12] = {0, 0, -1, 1, 0, 0, -2, 2, -1, -1, 1, 1};
    for (int q = 0; q < 12; ++q) {
        const int64_t j = nbr(DX[q], DY[q], 0);
        if (j < 0) continue;
        const double cf = q < 4 ? -2.0 * a : (q < 8 ? 1.0 : 2.0);
        g += cf * x0_at<V>(s, i, s.colour[j]);
    }
    return g;
}

template <typename V>
__global__ void k_grad(Solve s, int nparam, int p0, int p1, int p2, double *part) {
    const int pid[3] = {p0, p1, p2};
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.op.n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < nparam; ++k) acc[k] += grad_row<V>(s, pid[k], i);
    __shared__ double red[32 * 3];
    __shared__ double tot[3];
    block_sum_to<double, 3>(acc, red, tot);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = tot[k];
}

__global__ void k_grad_finish(int nblocks, const double *part, double *out) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[b * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <typename V, int T, int KIND>
struct CtaLauncher {
    static int run(const Solve &s, int max_iter, cudaStream_t st) {
        k_cta_solve<V, T, KIND><<<s.ntiles, 256, 0, st>>>(s, max_iter);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct FlushLauncher {
    static int run(const Solve &s, cudaStream_t st) {
        const int64_t total = (int64_t)s.ntiles * s.op.n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks < 1) blocks = 1;
        k_flush_x<V, T><<<blocks, 256, 0, st>>>(s);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct InitLauncher {
    static int run(const Solve &s, cudaStream_t st) {
        const int64_t total = (int64_t)s.ntiles * s.op.n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks < 1) blocks = 1;
        k_init_vectors<V, T><<<blocks, 256, 0, st>>>(s);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct ResidualLauncher {
    static int run(const Solve &s, int set, int cb, int ce, int replace, double *norm2, cudaStream_t st) {
        int e = (int)cudaMemsetAsync(norm2, 0, (size_t)s.ncols * sizeof(double), st);
        if (e) return e;
        if (s.xhi) {
            const int64_t total = (int64_t)s.ntiles * s.op.n * T;
            int blocks = (int)((total + 255) / 256);
            if (blocks > 152 * 16) blocks = 152 * 16;
            if (blocks < 1) blocks = 1;
            k_fold_x<V, T><<<blocks, 256, 0, st>>>(s);
            e = (int)cudaGetLastError();
            if (e) return e;
        }
        int bx = (int)((s.op.n + 255) / 256);
        if (bx > 152 * 8) bx = 152 * 8;
        if (bx < 1) bx = 1;
        k_true_residual<V, T, KIND><<<dim3(bx, s.ntiles), 256, 0, st>>>(s, set, cb, ce, replace, norm2);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct ApplyLauncher {
    static int run(const Operator &op, int ntiles, const void *x, void *y, cudaStream_t st) {
        const int64_t total = (int64_t)ntiles * op.n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks < 1) blocks = 1;
        k_apply<V, T, KIND><<<blocks, 256, 0, st>>>(op, ntiles, static_cast<const V *>(x),
                                                     static_cast<V *>(y));
        return (int)cudaGetLastError();
    }
};

int engine_lean_x(const Solve &s, bool keep_x0) {
    const int k = s.op.kind;
    if (s.precision != 1 || (k != KIND_2D5 && k != KIND_2D13_SQ && k != KIND_3D7) || (s.T != 2 && s.T != 4))
        return 0;
    if (s.asig) return 0;                               // shifted-vector mode reads w
    if (k == KIND_3D7) return LEAN_3D;
    if (k == KIND_2D13_SQ && keep_x0) return 0;         // the Matern state holds no p
    // two columns a thread at T = 2 on even widths (16-byte aligned pairs), else one
    return s.T == 2 && s.op.nx % 2 == 0 ? 2 : 1;
}

namespace {
void lean_geom(const Solve &s, int &swl, int &xh, int &w) {
    const int X = s.lean;
    if (s.op.kind == KIND_2D13_SQ) {
        swl = LEAN_NT * X;
        xh = LeanGeom<KIND_2D13_SQ>::XH;
    } else {
        swl = LEAN_NT * X;
        xh = LeanGeom<KIND_2D5>::XH;
    }
    w = swl - 2 * xh;
}
}  // namespace

size_t engine_lean_code_bytes(const Solve &s) {
    if (s.lean <= 0) return 0;
    int swl, xh, w;
    lean_geom(s, swl, xh, w);
    return (size_t)s.ntiles * s.strips * s.op.ny * swl;
}

// Lane codes of the lean pass in strip layout, [tile][strip][row][SWL]: in the low seven
// bits colour - tile*T when that is a column of the tile and the vertex is owned by the
// strip, else LEAN_NONE; in the high bit (when the pass takes its diagonal from the codes)
// the mask bit of the column's vertex, for every in-grid or wrapped column of the strip.
__global__ void k_lean_codes(const int32_t *colour, const uint8_t *mask, int nx, int ny, int periodic, int T,
                             int ntiles, int strips, int SWL, int XH, int W, uint8_t *out) {
    const int64_t total = (int64_t)ntiles * strips * ny * SWL;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int xl = (int)(q % SWL);
        int64_t r = q / SWL;
        const int y = (int)(r % ny);
        r /= ny;
        const int strip = (int)(r % strips);
        const int tile = (int)(r / strips);
        const int gx = strip * W - XH + xl;
        uint8_t c = LEAN_NONE;
        if (xl >= XH && xl < XH + W && gx < nx) {
            const int lc = colour[(int64_t)y * nx + gx] - tile * T;
            if (lc >= 0 && lc < T) c = (uint8_t)lc;
        }
        if (mask) {
            int g = gx;
            if (periodic) g = ((g % nx) + nx) % nx;
            if (g >= 0 && g < nx && mask[(int64_t)y * nx + g]) c |= LEAN_MASK_BIT;
        }
        out[q] = c;
    }
}

int engine_lean_codes(const Solve &s, uint8_t *out, void *stream) {
    int swl, xh, w;
    lean_geom(s, swl, xh, w);
    const int64_t total = (int64_t)s.ntiles * s.strips * s.op.ny * swl;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (blocks < 1) blocks = 1;
    k_lean_codes<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        s.colour, s.lane_mask ? s.op.mask : nullptr, s.op.nx, s.op.ny, s.op.periodic, s.T, s.ntiles, s.strips,
        swl, xh, w, out);
    return (int)cudaGetLastError();
}

int engine_plan(Solve &s) {
    int dev = 0, sms = 152, occ = 8;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool lattice2d = s.op.kind == KIND_2D5 || s.op.kind == KIND_2D13_SQ;
    const bool lean3d = s.op.kind == KIND_3D7 && s.lean == LEAN_3D && s.precision == 1 && !s.asig &&
                        (s.T == 2 || s.T == 4);
    if ((!lattice2d && !lean3d) || s.precision != 1 || s.asig) s.lean = 0;   // shifted-vector mode reads w
    // bulk row copies measured faster for packs of 24 bytes and more; per-thread
    // copies win for 8- and 16-byte packs (fewer instructions on the critical path)
    const int pack_bytes = s.T * (s.precision == 0 ? (int)sizeof(double) : (int)sizeof(float));
    s.bulk = lattice2d && !s.lean && pack_bytes >= 24 && stream_bulk_ok(s.op.nx, pack_bytes);
    const int oe = s.precision == 0
                       ? iteration_occupancy<double>(s.T, s.op.kind, s.bulk != 0, 0, s.keep_x0 != 0, &occ)
                       : iteration_occupancy<float>(s.T, s.op.kind, s.bulk != 0, s.lean, s.keep_x0 != 0, &occ);
    if (oe != 0 || occ < 1) occ = 1;
    // one resident wave; with several tiles (tile groups run concurrently on their own
    // streams) 1.5 waves, so that CTAs of one group fill the gaps of another
    int64_t target = (int64_t)sms * occ;
    if (s.ntiles >= 2 && s.op.kind != KIND_CSR) target = target * 3 / 2;
    // several solves at once (a batch's grid-engine instances): each takes its share, in
    // longer row segments rather than more CTAs of a few rows each
    if (s.share > 1) target = std::max<int64_t>(1, target / s.share);
    s.strips = 1;
    s.seg = 1;
    if (lattice2d) {
        int W = s.op.kind == KIND_2D13_SQ ? Strip<KIND_2D13_SQ>::W : Strip<KIND_2D5>::W;
        if (s.lean) {
            int swl, xh;
            lean_geom(s, swl, xh, W);
        }
        s.strips = (s.op.nx + W - 1) / W;
        int64_t nsegs = target / ((int64_t)s.strips * s.ntiles);
        if (nsegs < 1) nsegs = 1;
        if (nsegs > s.op.ny) nsegs = s.op.ny;
        s.seg = (int)((s.op.ny + nsegs - 1) / nsegs);
        nsegs = (s.op.ny + s.seg - 1) / s.seg;
        s.bpt = (int)(s.strips * nsegs);
        return s.bpt;
    }
    if (s.op.kind == KIND_3D7) {
        // one CTA per (x-y tile, z segment); segments only when the x-y tiles are too few
        const int tx = lean3d ? (s.op.nx + L3_OWNX - 1) / L3_OWNX : (s.op.nx + P3X - 3) / (P3X - 2);
        const int ty = lean3d ? (s.op.ny + L3_OWNY - 1) / L3_OWNY : (s.op.ny + P3Y - 3) / (P3Y - 2);
        s.strips = tx * ty;
        int64_t nsegs = target / ((int64_t)s.strips * s.ntiles);
        if (nsegs < 1) nsegs = 1;
        if (nsegs > s.op.nz) nsegs = s.op.nz;
        s.seg = (int)((s.op.nz + nsegs - 1) / nsegs);
        nsegs = (s.op.nz + s.seg - 1) / s.seg;
        s.bpt = (int)(s.strips * nsegs);
        return s.bpt;
    }
    // CSR: one resident wave over all tiles (one tile group), CTA x of every tile on the
    // same rows at the same time
    int64_t bpt = target / s.ntiles;
    const int64_t need = (s.op.n + 255) / 256;
    if (bpt > need) bpt = need;
    if (bpt < 1) bpt = 1;
    s.bpt = (int)bpt;
    return s.bpt;
}

int engine_init(const Solve &s, int col_begin, int col_end, void *stream, bool vectors) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_init_scalars<<<64, 256, 0, st>>>(s, col_begin, col_end, s.class_size);
    int e = (int)cudaGetLastError();
    if (e) return e;
    k_init_tiles<<<1, 256, 0, st>>>(s);
    e = (int)cudaGetLastError();
    if (e) return e;
    if (!vectors) return 0;
    return dispatch<InitLauncher>(s.precision, s.T, s.op.kind, s, st);
}

int engine_iteration(const Solve &s, int parity, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return s.precision == 0 ? iteration_launch<double>(s, parity, st)
                            : iteration_launch<float>(s, parity, st);
}

int engine_cta_solve(const Solve &s, int max_iter, void *stream) {
    return dispatch<CtaLauncher>(s.precision, s.T, s.op.kind, s, max_iter,
                                 static_cast<cudaStream_t>(stream));
}

int engine_batch_occupancy(int precision, int T) {
    int occ = 0;
    if (dispatch<BatchOcc>(precision, T, KIND_2D5, &occ) != 0 || occ < 1) return 1;
    return occ;
}

int engine_batch(const Solve *solves_dev, const int *ncolours_dev, int count, const int2 *items_dev,
                 int nitems, int *queue_dev, int max_iter, int precision, int T, int grid,
                 double *logdet_dev, double *seed_dev, int *flag_dev, int *iters_dev, int *tile_passes_dev,
                 void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int e = (int)cudaMemsetAsync(queue_dev, 0, sizeof(int), st);
    if (e) return e;
    k_batch_prep<<<(count + 255) / 256, 256, 0, st>>>(solves_dev, count);
    if ((e = (int)cudaGetLastError())) return e;
    e = dispatch<BatchLauncher>(precision, T, KIND_2D5, solves_dev, items_dev, nitems, queue_dev,
                                max_iter, grid, st);
    if (e) return e;
    k_batch_finish<<<(count + 127) / 128, 128, 0, st>>>(solves_dev, ncolours_dev, count, logdet_dev,
                                                       seed_dev, flag_dev, iters_dev, tile_passes_dev);
    return (int)cudaGetLastError();
}

int engine_modev(const Solve &s, int which, int nxt, double2 *psig, double *y, void *stream) {
    return dispatch<ModeVLauncher>(s.precision, s.T, s.op.kind, s, which, nxt, psig, y,
                                   static_cast<cudaStream_t>(stream));
}

int engine_flush_x(const Solve &s, void *stream) {
    return dispatch<FlushLauncher>(s.precision, s.T, s.op.kind, s, static_cast<cudaStream_t>(stream));
}

int engine_finish(const Solve &s, int col_begin, int col_end, void *stream) {
    k_finish<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(s, col_begin, col_end);
    return (int)cudaGetLastError();
}

int engine_apply(const Operator &op, int precision, int T, int ntiles, const void *x, void *y,
                 void *stream) {
    return dispatch<ApplyLauncher>(precision, T, op.kind, op, ntiles, x, y,
                                   static_cast<cudaStream_t>(stream));
}

int engine_wait_selftest(uint64_t limit_ns, int32_t *status_dev, void *stream) {
    k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, status_dev);
    return (int)cudaGetLastError();
}

int engine_fill_diag(const Operator &op, double *diag_d, float *diag_f, void *stream) {
    int blocks = (int)((op.n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_fill_diag<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(op, diag_d, diag_f);
    return (int)cudaGetLastError();
}

int engine_true_residual(const Solve &s, int set, int col_begin, int col_end, int replace,
                         double *norm2_dev, void *stream) {
    return dispatch<ResidualLauncher>(s.precision, s.T, s.op.kind, s, set, col_begin, col_end, replace,
                                      norm2_dev, static_cast<cudaStream_t>(stream));
}

int engine_grad_params(const Solve &s, int nparam, const int *ids, double *out_dev, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = 152 * 4;
    double *part = s.partial;   // reuse: needs nb*3 doubles (host sizes it)
    int p[3] = {0, 0, 0};
    for (int k = 0; k < nparam; ++k) p[k] = ids[k];
    if (s.precision == 0)
        k_grad<double><<<nb, 256, 0, st>>>(s, nparam, p[0], p[1], p[2], part);
    else
        k_grad<float><<<nb, 256, 0, st>>>(s, nparam, p[0], p[1], p[2], part);
    int e = (int)cudaGetLastError();
    if (e) return e;
    k_grad_finish<<<1, 32, 0, st>>>(nb, part, out_dev);
    return (int)cudaGetLastError();
}

const char *engine_error_string(int e) { return cudaGetErrorString((cudaError_t)e); }

}  // namespace ld

