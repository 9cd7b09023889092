// CUDA engine for probed log det via rational log and multi-shift CG (sm_103a).
//
// Method (Sec. 2.1): log det Q = tr log Q ~ sum_c v_c^T f_N(Q) v_c with
// f_N(Q) v = sum_l alpha_l (Q - sigma_l I)^{-1} v (Eq. "eq_rat_app"); every
// shifted system shares the Krylov space of the real seed CG on Q x = v_c,
// so only the seed vectors are iterated and the shifted solutions enter
// through scalar recurrences (CG-M; complex shifts with the bilinear form,
// COCG-M).  Only the projections v_c^T x^sigma are kept:
//   pi  += alpha^s phi,   phi = zeta_{k+1} v^T r_{k+1} + beta^s phi.
//
// Data layout in HBM: the C probing vectors are padded to ncols = ntiles*T and
// stored tile-interleaved, [tile][vertex][T]: one vertex's T columns are one
// 16/32-byte vector, a warp touches 32 consecutive vertices (fully coalesced),
// and per-vertex data (stencil coefficients, colour, kappa^2 field, mask) is
// read once per tile.  The SpMM is HBM-bound: no tensor cores (not a dense
// contraction).
//
// Per CG iteration k (all columns of a tile in lockstep, each its own CG):
//   phase A  p_k = r_k + beta_{k-1} p_{k-1} (formed on the fly, also at the
//            stencil neighbours), w = Q p_k, store p_k, partial p_k^T w;
//            the last block of the tile reduces the partials in a fixed order
//            and sets alpha_k = rho_k / p_k^T Q p_k.
//   phase B  w = Q p_k recomputed from the stored p_k, r_{k+1} = r_k - alpha_k w,
//            (x += alpha_k p_k when the seed solution is kept), partials
//            r^T r and v^T r; the last block runs the scalar tail: beta_k, the
//            shift recurrences, projections and convergence flags.
// Traffic per iteration: read r, p_{k-1}, p_k, r; write p_k, r  (6 n T words
// per tile) plus x in gradient mode.
//
// Two engines share these device functions:
//   grid engine  phases as separate launches, many CTAs per tile, partial
//                sums reduced by the tile's last CTA; launched in CUDA-graph
//                chunks by the host.
//   CTA engine   one CTA runs a tile's whole solve (small problems, batches);
//                block barriers only.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace ld {

// ------------------------------------------------------------------ packs
template <typename V, int T>
struct alignas((sizeof(V) * T) >= 16 ? 16 : (sizeof(V) * T)) Pack {
    V v[T];
};

// read-only (non-coherent) vector load of one pack
template <typename V, int T>
__device__ __forceinline__ Pack<V, T> ldg_raw(const Pack<V, T> *p) {
    Pack<V, T> out;
    constexpr int BYTES = sizeof(V) * T;
    if constexpr (BYTES % 16 == 0) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        float4 *o = reinterpret_cast<float4 *>(&out);
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k) o[k] = __ldg(q + k);
    } else if constexpr (BYTES == 8) {
        *reinterpret_cast<float2 *>(&out) = __ldg(reinterpret_cast<const float2 *>(p));
    } else {
        *reinterpret_cast<float *>(&out) = __ldg(reinterpret_cast<const float *>(p));
    }
    return out;
}

template <typename V, int T, bool NC>
__device__ __forceinline__ Pack<V, T> ldpack(const V *base, int64_t j) {
    const Pack<V, T> *p = reinterpret_cast<const Pack<V, T> *>(base + j * T);
    if constexpr (NC) {
        return ldg_raw<V, T>(p);
    } else {
        return *p;
    }
}

template <typename V, int T>
__device__ __forceinline__ void stpack(V *base, int64_t j, const V (&a)[T]) {
    Pack<V, T> q;
#pragma unroll
    for (int t = 0; t < T; ++t) q.v[t] = a[t];
    *reinterpret_cast<Pack<V, T> *>(base + j * T) = q;
}

}  // namespace ld

namespace ld {

// ------------------------------------------------------------------ loaders
// p_k at vertex j formed on the fly from r_k and p_{k-1}.
template <typename V, int T, bool NC>
struct LoadRP {
    const V *r;
    const V *p;
    V beta[T];
    __device__ __forceinline__ void operator()(int64_t j, V (&o)[T]) const {
        Pack<V, T> a = ldpack<V, T, NC>(r, j);
        Pack<V, T> b = ldpack<V, T, NC>(p, j);
#pragma unroll
        for (int t = 0; t < T; ++t) o[t] = fma(beta[t], b.v[t], a.v[t]);
    }
};

template <typename V, int T, bool NC>
struct LoadP {
    const V *p;
    __device__ __forceinline__ void operator()(int64_t j, V (&o)[T]) const {
        Pack<V, T> b = ldpack<V, T, NC>(p, j);
#pragma unroll
        for (int t = 0; t < T; ++t) o[t] = b.v[t];
    }
};

template <typename V, int T>
__device__ __forceinline__ void axpy(V (&w)[T], V c, const V (&a)[T]) {
#pragma unroll
    for (int t = 0; t < T; ++t) w[t] = fma(c, a[t], w[t]);
}

template <typename V>
__device__ __forceinline__ V field_at(const Operator &op, int64_t i);
template <>
__device__ __forceinline__ double field_at<double>(const Operator &op, int64_t i) {
    return op.field_d ? op.kappa2 * op.field_d[i] : op.kappa2;
}
template <>
__device__ __forceinline__ float field_at<float>(const Operator &op, int64_t i) {
    return op.field_f ? (float)op.kappa2 * op.field_f[i] : (float)op.kappa2;
}

// Lattice neighbour of (x, y, z) shifted by (dx, dy, dz): wrapped on a torus,
// -1 outside a Dirichlet-truncated grid.
__device__ __forceinline__ int64_t lattice_nbr(const Operator &op, int x, int y, int z, int dx,
                                               int dy, int dz) {
    int xx = x + dx, yy = y + dy, zz = z + dz;
    if (op.periodic) {
        if (xx < 0) xx += op.nx; else if (xx >= op.nx) xx -= op.nx;
        if (yy < 0) yy += op.ny; else if (yy >= op.ny) yy -= op.ny;
        if (zz < 0) zz += op.nz; else if (zz >= op.nz) zz -= op.nz;
        // offsets of 2 on sides of 1 wrap twice
        if (xx < 0) xx += op.nx; else if (xx >= op.nx) xx -= op.nx;
        if (yy < 0) yy += op.ny; else if (yy >= op.ny) yy -= op.ny;
    } else if (xx < 0 || xx >= op.nx || yy < 0 || yy >= op.ny || zz < 0 || zz >= op.nz) {
        return -1;
    }
    return (int64_t)xx + (int64_t)op.nx * ((int64_t)yy + (int64_t)op.ny * zz);
}

// Shifted Laplacian in difference form, the FP32-safe way to apply it:
//   ((kappa2 + tau m) I - Lap) p at i = (kappa2 + tau m + 2*dim - nb) p_i + sum_j (p_i - p_j)
// with nb the number of in-grid neighbours j (all 2*dim on a torus).  Smooth
// vectors give small differences, so rounding error scales with (kappa2 + mu)|p|
// rather than with the diagonal.
template <typename V, int T>
__device__ __forceinline__ void diff_accum(V (&w)[T], const V (&pc)[T], const V (&pj)[T]) {
#pragma unroll
    for (int t = 0; t < T; ++t) w[t] += pc[t] - pj[t];
}

// w = (Q p)(i) and self = p(i) for one vertex; `load(j, out)` yields p(j).
template <typename V, int T, int KIND, class L>
__device__ __forceinline__ void apply_row(const Operator &op, int64_t i, const L &load,
                                          V (&w)[T], V (&self)[T]) {
    load(i, self);
    if constexpr (KIND == KIND_2D5 || KIND == KIND_3D7) {
        constexpr int NB = (KIND == KIND_3D7) ? 6 : 4;
        const int nx = op.nx, ny = op.ny;
        const int64_t yz = i / nx;
        const int x = (int)(i - yz * nx);
        int y, z;
        if constexpr (KIND == KIND_3D7) {
            z = (int)(yz / ny);
            y = (int)(yz - (int64_t)z * ny);
        } else {
            y = (int)yz;
            z = 0;
        }
        const int DX[6] = {-1, 1, 0, 0, 0, 0}, DY[6] = {0, 0, -1, 1, 0, 0}, DZ[6] = {0, 0, 0, 0, -1, 1};
        V acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = (V)0;
        int nb = 0;
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int64_t j = lattice_nbr(op, x, y, z, DX[q], DY[q], DZ[q]);
            if (j >= 0) {
                V pj[T];
                load(j, pj);
                diff_accum(acc, self, pj);
                ++nb;
            }
        }
        V dg = field_at<V>(op, i) + (V)(NB - nb);
        if (op.mask) dg += (V)op.tau * (V)op.mask[i];
        const V sc = (V)op.scale;
#pragma unroll
        for (int t = 0; t < T; ++t) w[t] = sc * fma(dg, self[t], acc[t]);
    } else if constexpr (KIND == KIND_2D13_SQ) {
        // Q = scale * Q1 (Q1 p), Q1 = kappa2 I - Lap (5-point, difference form):
        // u_j = (Q1 p)_j at the centre and its four neighbours, then w = (Q1 u)_i.
        const int nx = op.nx;
        const int y = (int)(i / nx);
        const int x = (int)(i - (int64_t)y * nx);
        const V k2 = (V)op.kappa2;
        const int DX[4] = {-1, 1, 0, 0}, DY[4] = {0, 0, -1, 1};
        V uc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) uc[t] = (V)0;
        V u[4][T];
        int has[4];
        int nbc = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = lattice_nbr(op, x, y, 0, DX[q], DY[q], 0);
            has[q] = j >= 0;
            if (j >= 0) {
                ++nbc;
                V pj[T];
                load(j, pj);
                diff_accum(uc, self, pj);
                // (Q1 p)_j: neighbours of j are i and three more lattice points
                V aj[T];
#pragma unroll
                for (int t = 0; t < T; ++t) aj[t] = pj[t] - self[t];
                int nbj = 1;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (DX[r] == -DX[q] && DY[r] == -DY[q]) continue;   // back to i
                    const int64_t k = lattice_nbr(op, x, y, 0, DX[q] + DX[r], DY[q] + DY[r], 0);
                    if (k >= 0) {
                        V pk[T];
                        load(k, pk);
                        diff_accum(aj, pj, pk);
                        ++nbj;
                    }
                }
                const V dj = k2 + (V)(4 - nbj);
#pragma unroll
                for (int t = 0; t < T; ++t) u[q][t] = fma(dj, pj[t], aj[t]);
            } else {
#pragma unroll
                for (int t = 0; t < T; ++t) u[q][t] = (V)0;
            }
        }
        const V dc = k2 + (V)(4 - nbc);
#pragma unroll
        for (int t = 0; t < T; ++t) uc[t] = fma(dc, self[t], uc[t]);
        V acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = (V)0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (has[q]) diff_accum(acc, uc, u[q]);
        const V sc = (V)op.scale;
#pragma unroll
        for (int t = 0; t < T; ++t) w[t] = sc * fma(dc, uc[t], acc[t]);
    } else {  // CSR (values pre-scaled)
#pragma unroll
        for (int t = 0; t < T; ++t) w[t] = (V)0;
        const int64_t e0 = op.rowptr[i], e1 = op.rowptr[i + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = op.colidx[e];
            V c;
            if constexpr (sizeof(V) == 8) c = op.val_d[e]; else c = op.val_f[e];
            V pj[T];
            load(j, pj);
            axpy(w, c, pj);
        }
    }
}

// ------------------------------------------------------------------ reductions
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *smem /* >= 32*K */) {
    // warp shuffle tree, then one value per warp through shared memory;
    // on return thread 0 holds the block sums (fixed order: deterministic).
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) smem[wid * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += smem[w * K + k];
            v[k] = s;
        }
    }
}

__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// Scalar tail of one CG-M iteration for the T columns of `tile`, given the new
// residual norms rho_{k+1} = r^T r and projections v^T r_{k+1} (sums in
// sh_rr[t], sh_vr[t]).  Whole block calls it.  Updates beta_k, the seed and
// shifted projections and the convergence flags; sets tile_done.
__device__ void scalar_tail(const Solve &s, int tile, const double *sh_rr, const double *sh_vr,
                            int *sh_any) {
    const int T = s.T, N = s.nshift;
    __shared__ double sh_beta[32];
    __shared__ int sh_was_active[32];
    if (threadIdx.x < T) {
        const int t = threadIdx.x, c = tile * T + t;
        sh_any[t] = 0;
        const int act = s.col_active[c];
        sh_was_active[t] = act;
        double beta = 0.0;
        if (act) {
            const double rho_new = sh_rr[t];
            const double vr = sh_vr[t];
            beta = rho_new / s.rho[c];
            if (!isfinite(beta) || !isfinite(vr)) set_status(s.status, DEV_NUMERIC);
            const double alpha = s.alpha[c];
            // seed system (sigma = 0): pi0 = v^T x0, phi0 = v^T p
            s.pi0[c] += alpha * s.phi0[c];
            s.phi0[c] = vr + beta * s.phi0[c];
            const double thr = s.tol * sqrt(s.vnorm2[c]);
            if (sqrt(rho_new) > thr) sh_any[t] = 1;
        }
        sh_beta[t] = beta;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < T * N; q += blockDim.x) {
        const int t = q / N, l = q - t * N, c = tile * T + t;
        if (!sh_was_active[t]) continue;
        const int idx = c * N + l;
        if (!s.sh_active[idx]) continue;
        const double alpha = s.alpha[c], beta = sh_beta[t];
        const double ap = s.alpha_prev[c], bp = s.beta_prev[c];
        const double2 sl = s.shift[l];
        const double2 z = s.zeta[idx], zp = s.zeta_prev[idx];
        // zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
        //              (a_{k-1} zeta_{k-1} (1 + s a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k))
        const double2 num = cscale(ap, cmul(z, zp));
        const double2 one_sa = make_double2(1.0 + sl.x * alpha, sl.y * alpha);
        const double2 den = cadd(cscale(ap, cmul(zp, one_sa)), cscale(alpha * bp, csub(zp, z)));
        const double2 zn = cdiv(num, den);
        const double2 ratio = cdiv(zn, z);
        const double2 as = cscale(alpha, ratio);
        const double2 bs = cscale(beta, cmul(ratio, ratio));
        const double2 phi = s.phi[idx];
        s.pi[idx] = cadd(s.pi[idx], cmul(as, phi));
        s.phi[idx] = cadd(cscale(sh_vr[t], zn), cmul(bs, phi));
        s.zeta_prev[idx] = z;
        s.zeta[idx] = zn;
        const double res = cabs2(zn) * sqrt(sh_rr[t]);
        if (!isfinite(res)) set_status(s.status, DEV_NUMERIC);
        if (res > s.tol * sqrt(s.vnorm2[c])) {
            atomicOr(&sh_any[t], 1);
        } else {
            s.sh_active[idx] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x < T) {
        const int t = threadIdx.x, c = tile * T + t;
        if (sh_was_active[t]) {
            s.alpha_prev[c] = s.alpha[c];
            s.beta_prev[c] = sh_beta[t];
            s.rho[c] = sh_rr[t];
            s.col_iters[c] += 1;
            const int still = sh_any[t];
            s.col_active[c] = still;
            s.beta[c] = still ? sh_beta[t] : 0.0;
            if (!still) s.alpha[c] = 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int t = 0; t < T; ++t) any |= s.col_active[tile * T + t];
        if (!any) {
            s.tile_done[tile] = 1;
            atomicSub(s.remaining, 1);
        }
    }
}

// after phase A sums: alpha_k = rho_k / p^T Q p per active column
__device__ __forceinline__ void set_alpha(const Solve &s, int tile, int t, double pw) {
    const int c = tile * s.T + t;
    if (s.col_active[c]) {
        if (!(pw > 0.0)) {
            set_status(s.status, isfinite(pw) ? DEV_NOTSPD : DEV_NUMERIC);
            s.alpha[c] = 0.0;
        } else {
            s.alpha[c] = s.rho[c] / pw;
        }
    } else {
        s.alpha[c] = 0.0;
    }
}

// accumulator type: FP64 vectors accumulate in FP64; FP32 vectors accumulate each
// thread's share in FP32 and every cross-thread sum in FP64.
template <typename V>
struct AccT { using type = V; };

// ------------------------------------------------------------------ phase bodies
template <typename V, int T, int KIND, bool NC>
__device__ __forceinline__ void phaseA_points(const Solve &s, int tile, int64_t i0, int64_t stride,
                                              const V *pold, V *pnew, double (&out)[T]) {
    const int64_t n = s.op.n;
    const V *r = static_cast<const V *>(s.r) + (int64_t)tile * n * T;
    LoadRP<V, T, NC> ld;
    ld.r = r;
    ld.p = pold;
#pragma unroll
    for (int t = 0; t < T; ++t) ld.beta[t] = (V)s.beta[tile * T + t];
    typename AccT<V>::type acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = 0;
    for (int64_t i = i0; i < n; i += stride) {
        V w[T], self[T];
        apply_row<V, T, KIND>(s.op, i, ld, w, self);
        stpack<V, T>(pnew, i, self);
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = fma(self[t], w[t], acc[t]);
    }
#pragma unroll
    for (int t = 0; t < T; ++t) out[t] = (double)acc[t];
}

template <typename V, int T, int KIND, bool NC>
__device__ __forceinline__ void phaseB_points(const Solve &s, int tile, int64_t i0, int64_t stride,
                                              const V *pcur, double (&out)[2 * T]) {
    const int64_t n = s.op.n;
    V *r = static_cast<V *>(s.r) + (int64_t)tile * n * T;
    V *x = s.keep_x0 ? static_cast<V *>(s.x) + (int64_t)tile * n * T : nullptr;
    V alpha[T];
#pragma unroll
    for (int t = 0; t < T; ++t) alpha[t] = (V)s.alpha[tile * T + t];
    LoadP<V, T, NC> ld;
    ld.p = pcur;
    typename AccT<V>::type rr[T], vr[T];
#pragma unroll
    for (int t = 0; t < T; ++t) { rr[t] = 0; vr[t] = 0; }
    const int cbase = tile * T;
    for (int64_t i = i0; i < n; i += stride) {
        V w[T], pv[T];
        apply_row<V, T, KIND>(s.op, i, ld, w, pv);
        Pack<V, T> rp = ldpack<V, T, false>(r, i);
        V rn[T];
#pragma unroll
        for (int t = 0; t < T; ++t) rn[t] = fma(-alpha[t], w[t], rp.v[t]);
        stpack<V, T>(r, i, rn);
        if (x) {
            Pack<V, T> xp = ldpack<V, T, false>(x, i);
            V xn[T];
#pragma unroll
            for (int t = 0; t < T; ++t) xn[t] = fma(alpha[t], pv[t], xp.v[t]);
            stpack<V, T>(x, i, xn);
        }
        const int lc = s.colour[i] - cbase;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            rr[t] = fma(rn[t], rn[t], rr[t]);
            if (lc == t) vr[t] += rn[t];
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) { out[t] = (double)rr[t]; out[T + t] = (double)vr[t]; }
}

// ------------------------------------------------------------------ grid engine
template <int K>
__device__ __forceinline__ bool tile_last_block(const Solve &s, int tile, const double (&v)[K],
                                                double *part_base) {
    // thread 0 holds the block sums: publish them, count the block in.
    __shared__ int is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part_base[k] = v[k];
        __threadfence();
        const int prev = atomicAdd(&s.tile_ctr[tile], 1);
        is_last = (prev == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

template <typename V, int T, int KIND>
__global__ void __launch_bounds__(256) k_phaseA(Solve s, int parity) {
    const int tile = blockIdx.y;
    if (s.tile_done[tile]) return;
    const int64_t off = (int64_t)tile * s.op.n * T;
    const V *pold = static_cast<const V *>(parity ? s.p1 : s.p0) + off;
    V *pnew = static_cast<V *>(parity ? s.p0 : s.p1) + off;
    double v[T];
    phaseA_points<V, T, KIND, true>(s, tile, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                    (int64_t)gridDim.x * blockDim.x, pold, pnew, v);
    __shared__ double red[32 * T];
    block_sum<T>(v, red);
    double *part = s.partial + ((int64_t)tile * s.bpt + blockIdx.x) * T * 2;
    if (tile_last_block<T>(s, tile, v, part)) {
        if (threadIdx.x < T) {
            double pw = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b)
                pw += s.partial[((int64_t)tile * s.bpt + b) * T * 2 + threadIdx.x];
            set_alpha(s, tile, threadIdx.x, pw);
        }
        if (threadIdx.x == 0) s.tile_ctr[tile] = 0;
    }
}

template <typename V, int T, int KIND>
__global__ void __launch_bounds__(256) k_phaseB(Solve s, int parity) {
    const int tile = blockIdx.y;
    if (s.tile_done[tile]) return;
    const int64_t off = (int64_t)tile * s.op.n * T;
    const V *pcur = static_cast<const V *>(parity ? s.p0 : s.p1) + off;
    double v[2 * T];
    phaseB_points<V, T, KIND, true>(s, tile, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                    (int64_t)gridDim.x * blockDim.x, pcur, v);
    __shared__ double red[32 * 2 * T];
    block_sum<2 * T>(v, red);
    double *part = s.partial + ((int64_t)tile * s.bpt + blockIdx.x) * T * 2;
    if (tile_last_block<2 * T>(s, tile, v, part)) {
        __shared__ double sh_rr[T], sh_vr[T];
        __shared__ int sh_any[T];
        if (threadIdx.x < T) {
            double a = 0.0, b = 0.0;
            for (int bl = 0; bl < (int)gridDim.x; ++bl) {
                const double *q = s.partial + ((int64_t)tile * s.bpt + bl) * T * 2;
                a += q[threadIdx.x];
                b += q[T + threadIdx.x];
            }
            sh_rr[threadIdx.x] = a;
            sh_vr[threadIdx.x] = b;
        }
        __syncthreads();
        scalar_tail(s, tile, sh_rr, sh_vr, sh_any);
        if (threadIdx.x == 0) s.tile_ctr[tile] = 0;
    }
}

// ------------------------------------------------------------------ CTA engine
template <typename V, int T, int KIND>
__global__ void __launch_bounds__(512) k_cta_solve(Solve s, int max_iter) {
    const int tile = blockIdx.x;
    const int64_t off = (int64_t)tile * s.op.n * T;
    __shared__ double red[32 * 2 * T];
    __shared__ double sh_rr[T], sh_vr[T];
    __shared__ int sh_any[T];
    __shared__ int done;
    if (threadIdx.x == 0) done = s.tile_done[tile];
    __syncthreads();
    for (int it = 0; it < max_iter && !done; ++it) {
        const int parity = it & 1;
        const V *pold = static_cast<const V *>(parity ? s.p1 : s.p0) + off;
        V *pnew = static_cast<V *>(parity ? s.p0 : s.p1) + off;
        double va[T];
        phaseA_points<V, T, KIND, false>(s, tile, threadIdx.x, blockDim.x, pold, pnew, va);
        block_sum<T>(va, red);
        if (threadIdx.x == 0) {
            for (int t = 0; t < T; ++t) red[t] = va[t];
        }
        __syncthreads();
        if (threadIdx.x < T) set_alpha(s, tile, threadIdx.x, red[threadIdx.x]);
        __syncthreads();
        double vb[2 * T];
        phaseB_points<V, T, KIND, false>(s, tile, threadIdx.x, blockDim.x, pnew, vb);
        block_sum<2 * T>(vb, red);
        if (threadIdx.x == 0) {
            for (int t = 0; t < T; ++t) { sh_rr[t] = vb[t]; sh_vr[t] = vb[T + t]; }
        }
        __syncthreads();
        scalar_tail(s, tile, sh_rr, sh_vr, sh_any);
        __syncthreads();
        if (threadIdx.x == 0) done = s.tile_done[tile] || (*s.status != 0);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ init / finish
template <typename V, int T>
__global__ void k_init_vectors(Solve s) {
    const int64_t n = s.op.n;
    const int64_t total = (int64_t)s.ntiles * n;
    V *r = static_cast<V *>(s.r), *p0 = static_cast<V *>(s.p0), *p1 = static_cast<V *>(s.p1);
    V *x = s.keep_x0 ? static_cast<V *>(s.x) : nullptr;
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
        stpack<V, T>(r, q, a);
        stpack<V, T>(p0, q, z);
        stpack<V, T>(p1, q, z);
        if (x) stpack<V, T>(x, q, z);
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
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s.ntiles; t += gridDim.x * blockDim.x)
        s.tile_ctr[t] = 0;
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

// terms[c] = Re sum_l alpha_l pi_{c,l}; result = sum over [cb, ce) in column order.
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

// ------------------------------------------------------------------ gradient (backward)
// g_eta = sum_c (E_eta v_c)^T x0_c = sum_i sum_j E_ij x0[i, colour(j)], E = dQ/d eta.
// E per parameter id: kappa2 -> scale*diag(field or 1) (grid 5/7-pt), 2*scale*Q1 (13-pt);
// tau -> scale*diag(mask); scale -> Q/scale.
template <typename V>
__device__ __forceinline__ double x0_at(const Solve &s, int64_t i, int c) {
    const int tile = c / s.T, lane = c - tile * s.T;
    const V *x = static_cast<const V *>(s.x);
    return (double)x[((int64_t)tile * s.op.n + i) * s.T + lane];
}

template <typename V>
__device__ double grad_row(const Solve &s, int pid, int64_t i) {
    const Operator &op = s.op;
    const int ci = s.colour[i];
    if (op.kind == KIND_CSR) {
        if (pid != 2) return 0.0;
        double g = 0.0;
        for (int64_t e = op.rowptr[i]; e < op.rowptr[i + 1]; ++e)
            g += op.val_d[e] / op.scale * x0_at<V>(s, i, s.colour[op.colidx[e]]);
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
    block_sum<3>(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = acc[k];
}

__global__ void k_grad_finish(int nblocks, const double *part, double *out) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[b * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// ------------------------------------------------------------------ dispatch
template <typename V, int T, template <typename, int, int> class Launcher, class... A>
static int dispatch_kind(int kind, A &&...args) {
    switch (kind) {
        case KIND_2D5: return Launcher<V, T, KIND_2D5>::run(args...);
        case KIND_2D13_SQ: return Launcher<V, T, KIND_2D13_SQ>::run(args...);
        case KIND_3D7: return Launcher<V, T, KIND_3D7>::run(args...);
        case KIND_CSR: return Launcher<V, T, KIND_CSR>::run(args...);
    }
    return (int)cudaErrorInvalidValue;
}

template <template <typename, int, int> class Launcher, class... A>
static int dispatch(int precision, int T, int kind, A &&...args) {
    if (precision == 0) {
        switch (T) {
            case 1: return dispatch_kind<double, 1, Launcher>(kind, args...);
            case 2: return dispatch_kind<double, 2, Launcher>(kind, args...);
            case 4: return dispatch_kind<double, 4, Launcher>(kind, args...);
        }
    } else {
        switch (T) {
            case 2: return dispatch_kind<float, 2, Launcher>(kind, args...);
            case 4: return dispatch_kind<float, 4, Launcher>(kind, args...);
            case 8: return dispatch_kind<float, 8, Launcher>(kind, args...);
        }
    }
    return (int)cudaErrorInvalidValue;
}

template <typename V, int T, int KIND>
struct IterLauncher {
    static int run(const Solve &s, int parity, cudaStream_t st) {
        dim3 grid(s.bpt, s.ntiles);
        k_phaseA<V, T, KIND><<<grid, 256, 0, st>>>(s, parity);
        k_phaseB<V, T, KIND><<<grid, 256, 0, st>>>(s, parity);
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct CtaLauncher {
    static int run(const Solve &s, int max_iter, cudaStream_t st) {
        k_cta_solve<V, T, KIND><<<s.ntiles, 512, 0, st>>>(s, max_iter);
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

int engine_blocks_per_tile(const Solve &s) {
    const int64_t target = 152 * 8;   // one resident wave of 256-thread CTAs
    int64_t bpt = (target + s.ntiles - 1) / s.ntiles;
    const int64_t need = (s.op.n + 255) / 256;
    if (bpt > need) bpt = need;
    if (bpt < 1) bpt = 1;
    return (int)bpt;
}

int engine_init(const Solve &s, int col_begin, int col_end, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_init_scalars<<<64, 256, 0, st>>>(s, col_begin, col_end, s.class_size);
    int e = (int)cudaGetLastError();
    if (e) return e;
    k_init_tiles<<<1, 256, 0, st>>>(s);
    e = (int)cudaGetLastError();
    if (e) return e;
    return dispatch<InitLauncher>(s.precision, s.T, s.op.kind, s, st);
}

int engine_iteration(const Solve &s, int parity, void *stream) {
    return dispatch<IterLauncher>(s.precision, s.T, s.op.kind, s, parity,
                                  static_cast<cudaStream_t>(stream));
}

int engine_cta_solve(const Solve &s, int max_iter, void *stream) {
    return dispatch<CtaLauncher>(s.precision, s.T, s.op.kind, s, max_iter,
                                 static_cast<cudaStream_t>(stream));
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
