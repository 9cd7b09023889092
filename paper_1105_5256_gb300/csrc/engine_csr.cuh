// CSR pass of the grid engine: the one-reduction CG step of Sec. 2.1's seed system for a
// general sparse Q (FEM meshes, any pattern), in two launches per tile and pass.
//
//   k_csr_step   r_k = r - alpha w,  p_k = r_k + beta p,  x += alpha p       (streaming)
//   k_csr_spmv   w_k = Q p_k by rows; dots r.r, p.w, r.w, w.w, v.r, v.w of r_k, p_k, w_k;
//                the tile's last CTA reduces the partials and runs the multi-shift tail
//
// Forming p_k inside the product (as the stencil passes do) would gather r, w and p at
// every matrix entry; splitting the step off gathers only p_k, written by the step just
// before, so a matrix row costs one T-wide gather per entry.  Bytes a pass: the step reads
// r, w, p and writes r, p; the product reads r_k and p_k and writes w (8 words a vertex and
// column, 2 more with x), plus the matrix (index and value a stored entry, a row pointer
// a vertex) and the colour (4 bytes a vertex).
//
// Thread layout of the product: T consecutive lanes own one matrix row, lane t column t
// of the tile, so the row's T-wide pack of p_k at a neighbour is one contiguous T-word
// load of the group; a warp holds floor(32 / T) rows (T = 6: five rows, two lanes idle).
// The warp's rows are consecutive, so their column indices and values are one contiguous
// run of the matrix: the warp stages it in shared memory with coalesced loads, and each
// group then issues its row's gathers up to CSR_U at a time from there.
#pragma once
#include "engine_device.cuh"

namespace ld {

constexpr int CSR_NT = 256;
constexpr int CSR_EW = 256;   // matrix entries a warp stages per batch of rows
constexpr int CSR_U = 8;      // gathers a lane issues before it waits

template <typename V, int T>
__global__ void __launch_bounds__(CSR_NT) k_csr_step(Solve s, int cur) {
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    const int64_t n = s.op.n;
    const int64_t off = (int64_t)tile * n * T;
    const V *r = static_cast<const V *>(s.rbuf[cur]) + off;
    const V *w = static_cast<const V *>(s.wbuf[cur]) + off;
    const V *p = static_cast<const V *>(s.pbuf[cur]) + off;
    V *rn = static_cast<V *>(s.rbuf[cur ^ 1]) + off;
    V *pn = static_cast<V *>(s.pbuf[cur ^ 1]) + off;
    V *x = s.keep_x0 ? static_cast<V *>(s.x) + off : nullptr;
    V a[T], b[T];
    load_coefs<V, T>(s, tile, a, b);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const Pack<V, T> ri = ldpack<V, T, true>(r, i), wi = ldpack<V, T, true>(w, i),
                         pi = ldpack<V, T, true>(p, i);
        V rv[T], pv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            rv[t] = fma(-a[t], wi.v[t], ri.v[t]);
            pv[t] = fma(b[t], pi.v[t], rv[t]);
        }
        stpack<V, T>(rn, i, rv);
        stpack<V, T>(pn, i, pv);
        if (x) {
            Pack<V, T> xo = ldpack<V, T, false>(x, i);
            V xv[T];
#pragma unroll
            for (int t = 0; t < T; ++t) xv[t] = fma(a[t], pi.v[t], xo.v[t]);
            stpack<V, T>(x, i, xv);
        }
    }
}

template <typename V, int T>
__global__ void __launch_bounds__(CSR_NT) k_csr_spmv(Solve s, int cur) {
    constexpr int RW = 32 / T;              // rows a warp
    constexpr int NW = CSR_NT / 32;
    __shared__ double red[CSR_NT * NDOT];   // per-thread dots, then the tail's scratch
    __shared__ double cta[NDOT * T];
    __shared__ int32_t s_idx[NW][CSR_EW];   // a warp's staged column indices
    __shared__ __align__(8) unsigned char s_val[NW * CSR_EW * sizeof(V)];   // and values
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / T, t = lane - grp * T;
    const bool lane_on = grp < RW;
    const int64_t n = s.op.n;
    const int64_t off = (int64_t)tile * n * T;
    const V *pk = static_cast<const V *>(s.pbuf[cur ^ 1]) + off;
    const V *rk = static_cast<const V *>(s.rbuf[cur ^ 1]) + off;
    V *wn = static_cast<V *>(s.wbuf[cur ^ 1]) + off;
    const int64_t *rowptr = s.op.rowptr;
    const int32_t *colidx = s.op.colidx;
    const V *val;
    if constexpr (sizeof(V) == 8) val = s.op.val_d; else val = s.op.val_f;
    const int cbase = tile * T;
    V acc[NDOT];
#pragma unroll
    for (int k = 0; k < NDOT; ++k) acc[k] = (V)0;
    const int64_t wstride = (int64_t)gridDim.x * NW * RW;
    int32_t *sj = s_idx[warp];
    V *sv = reinterpret_cast<V *>(s_val) + warp * CSR_EW;
    for (int64_t row0 = ((int64_t)blockIdx.x * NW + warp) * RW; row0 < n; row0 += wstride) {
        // the warp's rows are consecutive, so their entries are one contiguous run: stage it
        // in shared memory with coalesced loads when it fits
        const int64_t rlast = min(row0 + RW, n);
        const int64_t b0 = __ldg(rowptr + row0), b1 = __ldg(rowptr + rlast);
        const bool staged = b1 - b0 <= CSR_EW;
        if (staged) {
            for (int q = lane; q < (int)(b1 - b0); q += 32) {
                sj[q] = __ldg(colidx + b0 + q);
                sv[q] = __ldg(val + b0 + q);
            }
        }
        __syncwarp();
        const int64_t i = row0 + grp;
        if (lane_on && i < n) {
            const int64_t e0 = __ldg(rowptr + i), e1 = __ldg(rowptr + i + 1);
            V w = (V)0;
            if (staged) {
                // up to CSR_U independent T-wide gathers of p_k in flight, then their sum in
                // entry order
                for (int q = (int)(e0 - b0), q1 = (int)(e1 - b0); q < q1; q += CSR_U) {
                    V g[CSR_U];
#pragma unroll
                    for (int k = 0; k < CSR_U; ++k)
                        g[k] = q + k < q1 ? __ldg(pk + (int64_t)sj[q + k] * T + t) : (V)0;
#pragma unroll
                    for (int k = 0; k < CSR_U; ++k)
                        if (q + k < q1) w = fma(sv[q + k], g[k], w);
                }
            } else {   // a run longer than the buffer: read the row directly
                for (int64_t e = e0; e < e1; ++e)
                    w = fma(__ldg(val + e), __ldg(pk + (int64_t)__ldg(colidx + e) * T + t), w);
            }
            const V r = rk[i * T + t], p = pk[i * T + t];
            wn[i * T + t] = w;
            acc[0] = fma(r, r, acc[0]);
            acc[1] = fma(p, w, acc[1]);
            acc[2] = fma(r, w, acc[2]);
            acc[3] = fma(w, w, acc[3]);
            if (s.colour[i] == cbase + t) {
                acc[4] += r;
                acc[5] += w;
            }
        }
        __syncwarp();   // the buffer is refilled by the next batch
    }
    // column sums over the block in a fixed order (warp, then row slot), widened to FP64
#pragma unroll
    for (int k = 0; k < NDOT; ++k) red[threadIdx.x * NDOT + k] = (double)acc[k];
    __syncthreads();
    for (int j = threadIdx.x; j < NDOT * T; j += CSR_NT) {
        const int k = j / T, tc = j - k * T;
        double sum = 0.0;
        for (int wv = 0; wv < NW; ++wv)
            for (int g = 0; g < RW; ++g) sum += red[(wv * 32 + g * T + tc) * NDOT + k];
        cta[j] = sum;
    }
    __syncthreads();
    publish_and_tail<NDOT * T>(s, tile, cur, cta, red);
}

}  // namespace ld
