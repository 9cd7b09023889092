// Device code shared by the engine's translation units (sm_103a).
#pragma once
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
// 8..32-byte vector, a warp touches 32 consecutive vertices (fully coalesced),
// and per-vertex data (colour, kappa^2 field, mask) is read once per tile.
// Columns of a tile iterate in lockstep (each its own CG) until all converge.
// The SpMM is HBM-bound: no tensor cores (not a dense contraction).
//
// Engines sharing the device functions below:
//   grid engine   one fused pass per CG iteration (see "fused CG-M pass"),
//                 many CTAs per tile, partial sums reduced by the tile's last
//                 CTA, launched by the host in CUDA-graph chunks; the 2D
//                 lattice kinds use a shared-memory tiled, cp.async-pipelined
//                 pass kernel, the other kinds a gather kernel.
//   CTA engine    one CTA runs a tile's whole solve (small problems).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace ld {

// ------------------------------------------------------------------ packs
// alignment: largest power of two dividing the pack size, at most 16 bytes
constexpr int pack_align(int bytes) {
    return (bytes % 16 == 0) ? 16 : (bytes % 8 == 0) ? 8 : (bytes % 4 == 0) ? 4 : bytes;
}

template <typename V, int T>
struct alignas(pack_align(sizeof(V) * T)) Pack {
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
    } else if constexpr (BYTES % 8 == 0) {
        const float2 *q = reinterpret_cast<const float2 *>(p);
        float2 *o = reinterpret_cast<float2 *>(&out);
#pragma unroll
        for (int k = 0; k < BYTES / 8; ++k) o[k] = __ldg(q + k);
    } else {
        const float *q = reinterpret_cast<const float *>(p);
        float *o = reinterpret_cast<float *>(&out);
#pragma unroll
        for (int k = 0; k < BYTES / 4; ++k) o[k] = __ldg(q + k);
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

// operator coefficients in the vector precision (no conversion in FP32 kernels)
template <typename V>
__device__ __forceinline__ V op_kappa2(const Operator &op) {
    if constexpr (sizeof(V) == 8) return op.kappa2;
    else return op.kappa2_f;
}
template <typename V>
__device__ __forceinline__ V op_tau(const Operator &op) {
    if constexpr (sizeof(V) == 8) return op.tau;
    else return op.tau_f;
}
template <typename V>
__device__ __forceinline__ V op_scale(const Operator &op) {
    if constexpr (sizeof(V) == 8) return op.scale;
    else return op.scale_f;
}

template <typename V>
__device__ __forceinline__ V field_at(const Operator &op, int64_t i);
template <>
__device__ __forceinline__ double field_at<double>(const Operator &op, int64_t i) {
    return op.field_d ? op.kappa2 * op.field_d[i] : op.kappa2;
}
template <>
__device__ __forceinline__ float field_at<float>(const Operator &op, int64_t i) {
    return op.field_f ? op.kappa2_f * op.field_f[i] : op.kappa2_f;
}

// the 2D5/3D7 diagonal term kappa2_i + tau mask_i (without the Laplacian's degree)
template <typename V>
__device__ __forceinline__ V diag_at(const Operator &op, int64_t i) {
    if constexpr (sizeof(V) == 8) {
        if (op.diag_d) return op.diag_d[i];
    } else {
        if (op.diag_f) return op.diag_f[i];
    }
    V dg = field_at<V>(op, i);
    if (op.mask) dg += op_tau<V>(op) * (V)op.mask[i];
    return dg;
}
template <typename V>
__device__ __forceinline__ const V *diag_ptr(const Operator &op) {
    if constexpr (sizeof(V) == 8) return op.diag_d;
    else return op.diag_f;
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
        const V dg = diag_at<V>(op, i) + (V)(NB - nb);
        const V sc = op_scale<V>(op);
#pragma unroll
        for (int t = 0; t < T; ++t) w[t] = sc * fma(dg, self[t], acc[t]);
    } else if constexpr (KIND == KIND_2D13_SQ) {
        // Q = scale * Q1 (Q1 p), Q1 = kappa2 I - Lap (5-point, difference form):
        // u_j = (Q1 p)_j at the centre and its four neighbours, then w = (Q1 u)_i.
        const int nx = op.nx;
        const int y = (int)(i / nx);
        const int x = (int)(i - (int64_t)y * nx);
        const V k2 = op_kappa2<V>(op);
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
        const V sc = op_scale<V>(op);
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
__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

// tile of this CTA in a grid-engine pass launch (grid.y = tiles of the launch)
__device__ __forceinline__ int launch_tile(const Solve &s) {
    return s.tile0 + (int)blockIdx.y * (s.tstride > 0 ? s.tstride : 1);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// ------------------------------------------------------------------ fused CG-M pass
// One pass per CG iteration k, for every column of a tile (Sec. 2.1: the real
// seed CG on Q x = v_c drives every shifted system):
//   r_k = r_{k-1} - alpha_{k-1} w_{k-1}       (alpha, beta from the previous pass)
//   p_k = r_k + beta_{k-1} p_{k-1}
//   w_k = Q p_k
//   dots r.r, p.w, r.w, w.w, v.r, v.w  ->  one reduction
// and the tail of the pass (last CTA of the tile, FP64):
//   alpha_k = r.r / p.w
//   rho_{k+1} = |r_k - alpha_k w_k|^2 = r.r - 2 alpha_k r.w + alpha_k^2 w.w
//   beta_k = rho_{k+1} / r.r,    v^T r_{k+1} = v.r - alpha_k v.w
// then the CG-M shift recurrences with (alpha_k, beta_k, v^T r_{k+1}).  The
// seed solution (gradient mode) gets x += alpha_{k-1} p_{k-1} in the next pass.
// A pass reads set k&1 of (r, w, p) and writes set (k&1)^1: 3 vector reads and
// 3 vector writes per iteration, one stencil application, one reduction.
// The difference-form operator keeps FP32 vectors accurate for ill-conditioned
// Q; scalars, dot sums across threads and the recurrences are FP64.

// p_k at vertex j from set `cur`: (r - alpha w) + beta p
template <typename V, int T, bool NC>
struct LoadFused {
    const V *r, *w, *p;
    V a[T], b[T];
    __device__ __forceinline__ void operator()(int64_t j, V (&o)[T]) const {
        const Pack<V, T> rr = ldpack<V, T, NC>(r, j), ww = ldpack<V, T, NC>(w, j),
                         pp = ldpack<V, T, NC>(p, j);
#pragma unroll
        for (int t = 0; t < T; ++t) o[t] = fma(b[t], pp.v[t], fma(-a[t], ww.v[t], rr.v[t]));
    }
};

// Tail of one pass for the T columns of `tile`; whole block calls it.
// sums[k*T + t] = dot k of column t (order: rr, pw, rw, ww, vr, vw).
static __device__ void fused_tail(const Solve &s, int tile, int cur, const double *sums) {
    const int T = s.T, N = s.nshift;
    __shared__ double sh_a[32], sh_b[32], sh_vrn[32], sh_res[32], sh_lim[32];
    __shared__ int sh_was[32], sh_any[32];
    if (threadIdx.x < T) {
        const int t = threadIdx.x, c = tile * T + t;
        const int act = s.col_active[c];
        sh_was[t] = act;
        sh_any[t] = 0;
        double a = 0.0, b = 0.0, vrn = 0.0, rhon = 0.0;
        const double lim = s.tol * sqrt(s.vnorm2[c]);
        if (act) {
            const double rr = sums[0 * T + t], pw = sums[1 * T + t], rw = sums[2 * T + t];
            const double ww = sums[3 * T + t], vr = sums[4 * T + t], vw = sums[5 * T + t];
            if (!(pw > 0.0)) {
                set_status(s.status, isfinite(pw) ? DEV_NOTSPD : DEV_NUMERIC);
            } else {
                a = rr / pw;
                rhon = fmax(rr - 2.0 * a * rw + a * a * ww, 0.0);
                b = rr > 0.0 ? rhon / rr : 0.0;
                vrn = vr - a * vw;
                if (!isfinite(a) || !isfinite(b) || !isfinite(vrn)) set_status(s.status, DEV_NUMERIC);
            }
            // seed system (sigma = 0): pi0 = v^T x0, phi0 = v^T p
            s.pi0[c] += a * s.phi0[c];
            s.phi0[c] = vrn + b * s.phi0[c];
            s.rho[c] = rhon;
            if (sqrt(rhon) > lim) sh_any[t] = 1;
        }
        sh_a[t] = a;
        sh_b[t] = b;
        sh_vrn[t] = vrn;
        sh_res[t] = sqrt(rhon);     // ||r_{k+1}||: shifted residual = |zeta_{k+1}| ||r_{k+1}||
        sh_lim[t] = lim;
    }
    __syncthreads();
    // one (column, shift) item per thread, spread over the warps (FP64 work on every
    // scheduler): item q = lane * warps + warp
    const int nw = blockDim.x >> 5;
    for (int q = (threadIdx.x & 31) * nw + (threadIdx.x >> 5); q < T * N; q += blockDim.x) {
        const int t = q / N, l = q - t * N, c = tile * T + t;
        const int idx = c * N + l;
        if (!sh_was[t] || !s.sh_active[idx]) {
            if (s.asig) s.asig[idx] = make_double2(0.0, 0.0);   // no shifted-vector update
            continue;
        }
        const double alpha = sh_a[t], beta = sh_b[t];
        const double ap = s.alpha_prev[c], bp = s.beta_prev[c];
        const double2 sl = s.shift[l];
        const double2 z = s.zeta[idx], zp = s.zeta_prev[idx];
        // zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
        //              (a_{k-1} zeta_{k-1} (1 + s a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)),
        // formed as ratio = zeta_{k+1} / zeta_k = a_{k-1} zeta_{k-1} / den (one division)
        const double2 one_sa = make_double2(1.0 + sl.x * alpha, sl.y * alpha);
        const double2 den = cadd(cscale(ap, cmul(zp, one_sa)), cscale(alpha * bp, csub(zp, z)));
        const double inv = 1.0 / (den.x * den.x + den.y * den.y);
        const double2 ratio = cscale(ap * inv, cmul(zp, make_double2(den.x, -den.y)));
        const double2 zn = cmul(ratio, z);
        const double2 as = cscale(alpha, ratio);
        const double2 bs = cscale(beta, cmul(ratio, ratio));
        const double2 phi = s.phi[idx];
        s.pi[idx] = cadd(s.pi[idx], cmul(as, phi));
        if (s.asig) {   // shifted-vector mode: this iteration's coefficients
            s.asig[idx] = as;
            s.bsig[idx] = bs;
        }
        s.phi[idx] = cadd(cscale(sh_vrn[t], zn), cmul(bs, phi));
        s.zeta_prev[idx] = z;
        s.zeta[idx] = zn;
        const double res = sqrt(zn.x * zn.x + zn.y * zn.y) * sh_res[t];
        if (!isfinite(res)) set_status(s.status, DEV_NUMERIC);
        if (res > sh_lim[t]) {
            atomicOr(&sh_any[t], 1);
        } else {
            s.sh_active[idx] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x < T) {
        const int t = threadIdx.x, c = tile * T + t;
        if (sh_was[t]) {
            s.alpha_prev[c] = sh_a[t];
            s.beta_prev[c] = sh_b[t];
            s.col_iters[c] += 1;
            const int still = sh_any[t];
            s.col_active[c] = still;
            s.alpha[c] = sh_a[t];           // applied to r and x by the next pass
            s.beta[c] = still ? sh_b[t] : 0.0;
        } else {
            s.alpha[c] = 0.0;
            s.beta[c] = 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int t = 0; t < T; ++t) any |= s.col_active[tile * T + t];
        if (!any) {
            s.tile_par[tile] = cur ^ 1;     // set holding the final p for the x flush
            s.tile_done[tile] = 1;
            atomicSub(s.remaining, 1);
        }
    }
}

// Per-thread dot accumulators of one pass.
template <typename V, int T>
struct Dots {
    V rr[T], pw[T], rw[T], ww[T], vr[T], vw[T];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int t = 0; t < T; ++t) rr[t] = pw[t] = rw[t] = ww[t] = vr[t] = vw[t] = (V)0;
    }
    // r, p, w of one vertex; lc = colour - tile base (own column if 0 <= lc < T)
    __device__ __forceinline__ void add(const V (&r)[T], const V (&p)[T], const V (&w)[T], int lc) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            rr[t] = fma(r[t], r[t], rr[t]);
            pw[t] = fma(p[t], w[t], pw[t]);
            rw[t] = fma(r[t], w[t], rw[t]);
            ww[t] = fma(w[t], w[t], ww[t]);
            if (lc == t) {
                vr[t] += r[t];
                vw[t] += w[t];
            }
        }
    }
    __device__ __forceinline__ void flat(V (&o)[NDOT * T]) const {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            o[0 * T + t] = rr[t];
            o[1 * T + t] = pw[t];
            o[2 * T + t] = rw[t];
            o[3 * T + t] = ww[t];
            o[4 * T + t] = vr[t];
            o[5 * T + t] = vw[t];
        }
    }
};

template <typename V, int T>
__device__ __forceinline__ void load_coefs(const Solve &s, int tile, V (&a)[T], V (&b)[T]) {
#pragma unroll
    for (int t = 0; t < T; ++t) {
        a[t] = (V)s.alpha[tile * T + t];
        b[t] = (V)s.beta[tile * T + t];
    }
}

// Generic pass body over vertices i0, i0+stride, ... (any kind; stencil taps
// gathered through the loader).  NC: read-only cache path allowed.
template <typename V, int T, int KIND, bool NC>
__device__ __forceinline__ void pass_points(const Solve &s, int tile, int cur, int64_t i0,
                                            int64_t stride, Dots<V, T> &d) {
    const int64_t n = s.op.n;
    const int64_t off = (int64_t)tile * n * T;
    const V *r = static_cast<const V *>(s.rbuf[cur]) + off;
    const V *w = static_cast<const V *>(s.wbuf[cur]) + off;
    const V *p = static_cast<const V *>(s.pbuf[cur]) + off;
    V *rn = static_cast<V *>(s.rbuf[cur ^ 1]) + off;
    V *wn = static_cast<V *>(s.wbuf[cur ^ 1]) + off;
    V *pn = static_cast<V *>(s.pbuf[cur ^ 1]) + off;
    V *x = s.keep_x0 ? static_cast<V *>(s.x) + off : nullptr;
    LoadFused<V, T, NC> ld;
    ld.r = r;
    ld.w = w;
    ld.p = p;
    load_coefs<V, T>(s, tile, ld.a, ld.b);
    const int cbase = tile * T;
    for (int64_t i = i0; i < n; i += stride) {
        V wv[T], pv[T];
        apply_row<V, T, KIND>(s.op, i, ld, wv, pv);
        const Pack<V, T> ri = ldpack<V, T, NC>(r, i), wi = ldpack<V, T, NC>(w, i);
        V rv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) rv[t] = fma(-ld.a[t], wi.v[t], ri.v[t]);
        stpack<V, T>(rn, i, rv);
        stpack<V, T>(pn, i, pv);
        stpack<V, T>(wn, i, wv);
        if (x) {
            const Pack<V, T> po = ldpack<V, T, NC>(p, i);
            Pack<V, T> xo = ldpack<V, T, false>(x, i);
            V xv[T];
#pragma unroll
            for (int t = 0; t < T; ++t) xv[t] = fma(ld.a[t], po.v[t], xo.v[t]);
            stpack<V, T>(x, i, xv);
        }
        d.add(rv, pv, wv, s.colour[i] - cbase);
    }
}

// ------------------------------------------------------------------ grid engine (generic)
// The last CTA of a tile to finish reduces the tile's partials (fixed order)
// and runs the tail.  Returns true in that CTA.
__device__ __forceinline__ bool tile_last_block(const Solve &s, int tile) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(&s.tile_ctr[tile], 1);
        is_last = (prev == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Block sum of K per-thread values into out[K] (shared memory): warp shuffle
// trees, then threads k < K add the per-warp sums in a fixed order.  red needs
// (blockDim/32)*K doubles.  Deterministic for a fixed launch shape.
template <typename A, int K>
__device__ __forceinline__ void block_sum_to(const A (&v)[K], double *red, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // warp trees in the accumulators' own precision (FP64 is a narrow pipe), warp
    // totals widened to FP64 and added in a fixed order
#pragma unroll
    for (int k = 0; k < K; ++k) {
        A x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid * K + k] = (double)x;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[w * K + k];
        out[k] = acc;
    }
    __syncthreads();
}

// Publish this CTA's K sums (cta[], shared memory) as its partial; in the tile's
// last CTA add all partials in a fixed order (chunks of CTAs per thread group,
// then the chunk sums) and run the tail.  scratch: >= blockDim.x doubles.
// Called by every thread of every (non-skipped) CTA of the grid engine.
template <int K>
__device__ __forceinline__ void publish_and_tail(const Solve &s, int tile, int cur,
                                                 const double *cta, double *scratch) {
    __shared__ double sums[K];
    double *part = s.partial + ((int64_t)tile * s.bpt + blockIdx.x) * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) part[k] = cta[k];
    if (!tile_last_block(s, tile)) return;
    const int chunks = blockDim.x / K;          // >= 1 (K <= 48 < blockDim.x)
    const int nb = (int)gridDim.x;
    const int per = (nb + chunks - 1) / chunks;
    if (threadIdx.x < chunks * K) {
        const int k = threadIdx.x % K, ch = threadIdx.x / K;
        const double *src = s.partial + (int64_t)tile * s.bpt * K + k;
        double acc = 0.0;
        const int b1 = min(nb, (ch + 1) * per);
        int b = ch * per;
        // eight independent loads in flight, added in block order
        for (; b + 8 <= b1; b += 8) {
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = src[(int64_t)(b + j) * K];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += v[j];
        }
        for (; b < b1; ++b) acc += src[(int64_t)b * K];
        scratch[ch * K + k] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double acc = 0.0;
        for (int ch = 0; ch < chunks; ++ch) acc += scratch[ch * K + k];
        sums[k] = acc;
    }
    __syncthreads();
    fused_tail(s, tile, cur, sums);
    if (threadIdx.x == 0) s.tile_ctr[tile] = 0;
}

template <typename V, int T>
__device__ __forceinline__ void finish_pass(const Solve &s, int tile, int cur, const Dots<V, T> &d) {
    constexpr int K = NDOT * T;
    __shared__ double red[32 * K];
    __shared__ double cta[K];
    V flat[K];
    d.flat(flat);
    block_sum_to<V, K>(flat, red, cta);
    publish_and_tail<K>(s, tile, cur, cta, red);
}

template <typename V, int T, int KIND>
__global__ void __launch_bounds__(256) k_pass(Solve s, int cur) {
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    Dots<V, T> d;
    d.zero();
    pass_points<V, T, KIND, true>(s, tile, cur, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                  (int64_t)gridDim.x * blockDim.x, d);
    finish_pass<V, T>(s, tile, cur, d);
}

// ------------------------------------------------------------------ streaming 2D grid engine
// For the 2D lattice kinds a CTA owns a strip of SW = 128 lattice columns
// (an H-wide halo on each side, H = 1 for the 5-point Q and 2 for the
// 13-point square) and a segment of rows, and marches down the rows.  G
// threads share one lattice column, each holding TS = T/G probing columns.
// Per row step a thread
//   forms p_k and r_k at (x, y) from r, w, p of the previous set (loads issued
//     two rows ahead into registers),
//   [13-point] forms u = Q1 p at (x, y-1),
//   forms w = Q p at (x, y-H) and writes r_k, p_k, w_k there,
// where vertical neighbours come from the thread's own register window and
// horizontal neighbours from two double-buffered shared-memory rows: one
// barrier per row, about six shared-memory accesses per vertex and column
// pack.  Out-of-grid rows and columns are zero, the Dirichlet ghost values of
// the difference form
//   (kappa2 I - Lap) p at i = kappa2 p_i + sum_{4 neighbours j} (p_i - p_j);
// a torus wraps its indices.  The 13-point square applies that form twice.
constexpr int SW = 128;

// H: stencil reach in rows; XH: halo columns on each side of a strip (2 for both
// kinds, so that strip starts stay 16-byte aligned for bulk row copies)
template <int KIND>
struct Strip {
    static constexpr int H = KIND == KIND_2D13_SQ ? 2 : 1;
    static constexpr int XH = 2;
    static constexpr int W = SW - 2 * XH;   // output columns per strip
};

// threads per lattice column: one thread holds all T columns of its lattice
// column, so per-row address, loop and barrier work is shared by T columns
template <typename V, int T>
__host__ __device__ constexpr int stream_groups() {
    return 1;
}

__device__ __forceinline__ int wrap_coord(int g, int n, bool per, bool &in) {
    if (g >= 0 && g < n) {
        in = true;
        return g;
    }
    if (!per) {
        in = false;
        return 0;
    }
    in = true;
    g %= n;
    return g < 0 ? g + n : g;
}

// asynchronous global -> shared copy of one pack (16- or 8-byte pieces); src-size 0
// zero-fills
template <typename V, int TS>
__device__ __forceinline__ void cp_async_pack(Pack<V, TS> *dst, const V *src, bool valid) {
    constexpr int BYTES = sizeof(V) * TS;
    static_assert(BYTES % 8 == 0, "packs are a multiple of 8 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
    if constexpr (BYTES % 16 == 0) {
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d + 16 * k),
                         "l"(g + 16 * k), "r"(valid ? 16 : 0));
    } else {
#pragma unroll
        for (int k = 0; k < BYTES / 8; ++k)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d + 8 * k),
                         "l"(g + 8 * k), "r"(valid ? 8 : 0));
    }
}
// one 4- or 8-byte word (src-size 0 zero-fills)
template <typename V>
__device__ __forceinline__ void cp_async_word(V *dst, const V *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(V) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename V, int TS>
__device__ __forceinline__ Pack<V, TS> zero_pack() {
    Pack<V, TS> z;
#pragma unroll
    for (int t = 0; t < TS; ++t) z.v[t] = (V)0;
    return z;
}

// ---- elementwise pack arithmetic; FP32 pairs issue as one packed f32x2 instruction
template <typename V, int TS>
struct PackMath {
    using P = Pack<V, TS>;
    static constexpr bool kPaired = std::is_same<V, float>::value && TS % 2 == 0;
    __device__ static __forceinline__ unsigned long long &u(P &a, int j) {
        return reinterpret_cast<unsigned long long *>(a.v)[j];
    }
    __device__ static __forceinline__ unsigned long long cu(const P &a, int j) {
        return reinterpret_cast<const unsigned long long *>(a.v)[j];
    }
    __device__ static __forceinline__ P fma(const P &a, const P &b, const P &c) {
        P o;
        if constexpr (kPaired) {
#pragma unroll
            for (int j = 0; j < TS / 2; ++j)
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(u(o, j)) : "l"(cu(a, j)), "l"(cu(b, j)), "l"(cu(c, j)));
        } else {
#pragma unroll
            for (int t = 0; t < TS; ++t) o.v[t] = ::fma(a.v[t], b.v[t], c.v[t]);
        }
        return o;
    }
    __device__ static __forceinline__ P add(const P &a, const P &b) {
        P o;
        if constexpr (kPaired) {
#pragma unroll
            for (int j = 0; j < TS / 2; ++j)
                asm("add.rn.f32x2 %0, %1, %2;" : "=l"(u(o, j)) : "l"(cu(a, j)), "l"(cu(b, j)));
        } else {
#pragma unroll
            for (int t = 0; t < TS; ++t) o.v[t] = a.v[t] + b.v[t];
        }
        return o;
    }
    __device__ static __forceinline__ P sub(const P &a, const P &b) {
        P o;
        if constexpr (kPaired) {
#pragma unroll
            for (int j = 0; j < TS / 2; ++j)
                asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(u(o, j)) : "l"(cu(a, j)), "l"(cu(b, j)));
        } else {
#pragma unroll
            for (int t = 0; t < TS; ++t) o.v[t] = a.v[t] - b.v[t];
        }
        return o;
    }
    __device__ static __forceinline__ P mul(const P &a, const P &b) {
        P o;
        if constexpr (kPaired) {
#pragma unroll
            for (int j = 0; j < TS / 2; ++j)
                asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(u(o, j)) : "l"(cu(a, j)), "l"(cu(b, j)));
        } else {
#pragma unroll
            for (int t = 0; t < TS; ++t) o.v[t] = a.v[t] * b.v[t];
        }
        return o;
    }
    __device__ static __forceinline__ P splat(V x) {
        P o;
#pragma unroll
        for (int t = 0; t < TS; ++t) o.v[t] = x;
        return o;
    }
    __device__ static __forceinline__ P neg(const P &a) {
        P o;
#pragma unroll
        for (int t = 0; t < TS; ++t) o.v[t] = -a.v[t];
        return o;
    }
};

// c p + ((p - l) + (p - r)) + ((p - d) + (p - u)): one level of the difference-form stencil,
// c a pack (per-vertex diagonal or kappa2 splat)
template <typename V, int TS>
__device__ __forceinline__ Pack<V, TS> diff5p(const Pack<V, TS> &c, const Pack<V, TS> &pc,
                                              const Pack<V, TS> &pl, const Pack<V, TS> &pr,
                                              const Pack<V, TS> &pd, const Pack<V, TS> &pu) {
    using M = PackMath<V, TS>;
    if constexpr (sizeof(V) == 8) {
        // FP64: the direct form (c + 4) p_i - sum_j p_j, half the instructions on the
        // narrow FP64 pipe; its cancellation costs about 3 of FP64's 16 digits
        Pack<V, TS> o;
#pragma unroll
        for (int t = 0; t < TS; ++t)
            o.v[t] = fma(c.v[t] + (V)4, pc.v[t], -((pl.v[t] + pr.v[t]) + (pd.v[t] + pu.v[t])));
        return o;
    } else {
        // FP32: the difference form keeps the cancellation inside each p_i - p_j
        const Pack<V, TS> h = M::add(M::sub(pc, pl), M::sub(pc, pr));
        const Pack<V, TS> v = M::add(M::sub(pc, pd), M::sub(pc, pu));
        return M::fma(c, pc, M::add(h, v));
    }
}

// (c p + sum of the four differences), the difference-form stencil of one level
// resident CTAs per SM the register budget is sized for
template <typename V, int T>
__host__ __device__ constexpr int stream_min_blocks_t() { return sizeof(V) * T <= 8 ? 6 : (sizeof(V) * T <= 16 ? 5 : 3); }

constexpr int STREAM_PD = 6;   // ring depth: rows held per thread (cp.async)

// dynamic shared memory of a streaming sweep; the ring of diagonal terms only for the
// 5-point kind (KIND_2D5; the batched kernel, which runs both kinds, passes it too)
template <typename V, int T, int G, int KIND = KIND_2D5>
constexpr size_t stream_smem_bytes() {
    constexpr int TS = T / G;
    constexpr size_t pk = sizeof(Pack<V, TS>);
    constexpr size_t dg = KIND == KIND_2D5 ? sizeof(V) : 0;
    constexpr size_t rows = (4 + 3 * STREAM_PD) * SW * G * pk + STREAM_PD * SW * G * (sizeof(int) + dg);
    constexpr size_t part = (size_t)SW * G * NDOT * TS * sizeof(V);
    constexpr size_t red = (size_t)SW * G * sizeof(double);
    return rows > part ? (rows > red ? rows : red) : (part > red ? part : red);
}

// per-thread dot accumulators of a streaming sweep (TS columns of the thread)
template <typename V, int TS>
struct StreamAcc {
    Pack<V, TS> rr, pw, rw, ww;
    V vr[TS], vw[TS];
    __device__ __forceinline__ void zero() {
        rr = pw = rw = ww = zero_pack<V, TS>();
#pragma unroll
        for (int t = 0; t < TS; ++t) vr[t] = vw[t] = (V)0;
    }
};

// One CTA sweeps lattice strip `strip`, rows [ys, ye), of one tile: the fused pass
// for those vertices, dot products accumulated into acc.  smem: stream_smem_bytes.
// Returns with no copy in flight and shared memory free (after a barrier).
template <typename V, int T, int G, int KIND, bool KEEPX>
__device__ __forceinline__ void stream_sweep(const Solve &s, int tile, int cur, int strip, int ys,
                                             int ye, unsigned char *smem,
                                             StreamAcc<V, T / G> &acc) {
    constexpr int TS = T / G, H = Strip<KIND>::H, PD = STREAM_PD;
    constexpr int NT = SW * G;          // threads; also the pack count of one shared row
    using P = Pack<V, TS>;
    // shared: [ps: 2 rows | us: 2 rows | ring: PD x (r, w, p) rows + colours]; the ring
    // is per-thread private (each thread copies and reads back only its own packs), so
    // it needs no barrier.
    P *const ps = reinterpret_cast<P *>(smem);
    P *const us = ps + 2 * NT;
    P *const ring = ps + 4 * NT + threadIdx.x;
    int *const ringc = reinterpret_cast<int *>(ps + (4 + 3 * PD) * NT) + threadIdx.x;
    // diagonal terms of field / mask models ride in the ring too (one word a vertex)
    V *const ringd = reinterpret_cast<V *>(reinterpret_cast<int *>(ps + (4 + 3 * PD) * NT) + PD * NT) + threadIdx.x;
    const V *const diag = KIND == KIND_2D5 ? diag_ptr<V>(s.op) : nullptr;
    const int nx = s.op.nx, ny = s.op.ny;
    const bool per = s.op.periodic;
    const int xl = threadIdx.x / G, g = threadIdx.x - xl * G;
    constexpr int XH = Strip<KIND>::XH;
    const int gx = strip * Strip<KIND>::W - XH + xl;
    bool inx;
    const int gxw = wrap_coord(gx, nx, per, inx);
    const bool outx = xl >= XH && xl < XH + Strip<KIND>::W && gx < nx;
    const int cb = tile * T + g * TS;
    const int64_t off = (int64_t)tile * s.op.n * T + g * TS;
    const V *const r = static_cast<const V *>(cur ? s.rbuf[1] : s.rbuf[0]) + off;
    const V *const w = static_cast<const V *>(cur ? s.wbuf[1] : s.wbuf[0]) + off;
    const V *const p = static_cast<const V *>(cur ? s.pbuf[1] : s.pbuf[0]) + off;
    using M = PackMath<V, TS>;
    P na, b;                  // -alpha, beta per column
#pragma unroll
    for (int t = 0; t < TS; ++t) {
        na.v[t] = -(V)s.alpha[cb + t];
        b.v[t] = (V)s.beta[cb + t];
    }
    P pw0 = zero_pack<V, TS>(), pw1 = pw0, pw2 = pw0;   // p at rows y-2, y-1, y
    P uw0 = pw0, uw1 = pw0, uw2 = pw0;                   // u at rows y-3, y-2, y-1

    int y = ys - H;
    const int yend = ye + H;
    // Rows are loaded in order, so the vertex index of the next row to load advances
    // by nx per row (wrapping on a torus) instead of being recomputed.
    int lrow = y;
    int64_t lvtx;
    {
        bool iny;
        const int w0 = wrap_coord(lrow, ny, per, iny);
        lvtx = (per ? (int64_t)w0 : (int64_t)lrow) * nx + gxw;
    }
    const int64_t nvtx = (int64_t)nx * ny;
    // rows past the segment's last step are not needed: empty (zero-fill) group
    auto load_row = [&](int slot) {
        const int yr = lrow;
        const bool in = (per || (unsigned)yr < (unsigned)ny) && inx && yr < yend;
        const int64_t vtx = in ? lvtx : 0;
        const int64_t e = vtx * T;
        P *q = ring + slot * 3 * NT;
        cp_async_pack<V, TS>(q, r + e, in);
        cp_async_pack<V, TS>(q + NT, w + e, in);
        cp_async_pack<V, TS>(q + 2 * NT, p + e, in);
        {
            const unsigned dc = (unsigned)__cvta_generic_to_shared(ringc + slot * NT);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dc),
                         "l"(s.colour + vtx), "r"(in ? 4 : 0));
        }
        if (diag) cp_async_word<V>(ringd + slot * NT, diag + vtx, in);
        cp_async_commit();
        ++lrow;
        lvtx += nx;
        if (per && lvtx >= nvtx) lvtx -= nvtx;
    };
    V *const rn = static_cast<V *>(cur ? s.rbuf[0] : s.rbuf[1]) + off;
    V *const wn = static_cast<V *>(cur ? s.wbuf[0] : s.wbuf[1]) + off;
    V *const pn = static_cast<V *>(cur ? s.pbuf[0] : s.pbuf[1]) + off;
    V *const xs = KEEPX ? static_cast<V *>(s.x) + off : nullptr;
    P xpre = zero_pack<V, TS>();   // x of the row emitted next step, loaded a step ahead
    // outputs at vertex evtx (column gx of the row emitted this step), ring slot `slot`
    auto emit = [&](int64_t evtx, int slot, const P &pk, const P &wk) {
        const P *q = ring + slot * 3 * NT;
        const P rk = M::fma(na, q[NT], q[0]);
        const int64_t e = evtx * T;
        *reinterpret_cast<P *>(rn + e) = rk;
        *reinterpret_cast<P *>(pn + e) = pk;
        *reinterpret_cast<P *>(wn + e) = wk;
        if constexpr (KEEPX) *reinterpret_cast<P *>(xs + e) = M::fma(M::neg(na), q[2 * NT], xpre);
        const int lc = ringc[slot * NT] - cb;
        acc.rr = M::fma(rk, rk, acc.rr);
        acc.pw = M::fma(pk, wk, acc.pw);
        acc.rw = M::fma(rk, wk, acc.rw);
        acc.ww = M::fma(wk, wk, acc.ww);
#pragma unroll
        for (int t = 0; t < TS; ++t) {
            if (lc == t) {
                acc.vr[t] += rk.v[t];
                acc.vw[t] += wk.v[t];
            }
        }
    };

    // ring slot of row yr is (yr - y0) mod PD.  A row is live from its p-step to its
    // emit step H rows later; at the end of step y the slot of row y - H takes row
    // y - H + PD, so the prologue queues rows y0 .. y0 + PD - H - 1 and row y's
    // copy group is always the (y - y0 + 1)-th: waiting with PD - H - 1 groups
    // pending completes it.
#pragma unroll
    for (int k = 0; k < PD - H; ++k) load_row(k);
    const P sc = M::splat(op_scale<V>(s.op)), k2 = M::splat(op_kappa2<V>(s.op));
    int64_t evtx = (int64_t)(y - H) * nx + gx;   // vertex of row y - H in column gx
    int slot = 0;            // slot of row y
    for (; y < yend; ++y) {
        cp_async_wait<PD - 1 - H>();
        {
            const P *q = ring + slot * 3 * NT;
            const P pk = M::fma(b, q[2 * NT], M::fma(na, q[NT], q[0]));
            ps[(y & 1) * NT + threadIdx.x] = pk;
            pw0 = pw1;
            pw1 = pw2;
            pw2 = pk;
        }
        const int slot_h = slot - H < 0 ? slot - H + PD : slot - H;   // slot of row y - H
        if constexpr (KIND == KIND_2D13_SQ) {
            // u = Q1 p at (x, y-1): p row y-1 was shared last step
            if (y >= ys) {
                P u = zero_pack<V, TS>();
                const bool uin = per || (unsigned)(y - 1) < (unsigned)ny;
                if (uin && inx && xl >= 1 && xl < SW - 1) {
                    const P *row = ps + ((y - 1) & 1) * NT;
                    u = diff5p<V, TS>(k2, pw1, row[threadIdx.x - G], row[threadIdx.x + G], pw0, pw2);
                }
                us[((y - 1) & 1) * NT + threadIdx.x] = u;
                uw0 = uw1;
                uw1 = uw2;
                uw2 = u;
            }
            // w = Q1 u at (x, y-2): u row y-2 was shared last step
            if (y - 2 >= ys && y - 2 < ye && outx) {
                const P *row = us + ((y - 2) & 1) * NT;
                const P wk = M::mul(sc, diff5p<V, TS>(k2, uw1, row[threadIdx.x - G], row[threadIdx.x + G], uw0, uw2));
                emit(evtx, slot_h, pw0, wk);
            }
        } else {
            // w = Q p at (x, y-1): p row y-1 was shared last step
            if (y - 1 >= ys && y - 1 < ye && outx) {
                const V dg = diag ? ringd[slot_h * NT] : op_kappa2<V>(s.op);
                const P *row = ps + ((y - 1) & 1) * NT;
                const P wk = M::mul(sc, diff5p<V, TS>(M::splat(dg), pw1, row[threadIdx.x - G], row[threadIdx.x + G], pw0, pw2));
                emit(evtx, slot_h, pw1, wk);
            }
        }
        // row y - H is done: its slot takes row y - H + PD (the next row in order)
        load_row(slot_h);
        evtx += nx;
        if constexpr (KEEPX) {
            const int yo = y + 1 - H;       // row emitted by the next step
            if (yo >= ys && yo < ye && outx) xpre = *reinterpret_cast<const P *>(xs + evtx * T);
        }
        slot = slot + 1 == PD ? 0 : slot + 1;
        __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
}

// ------------------------------------------------------------------ bulk-copy rows
// Rows of r, w, p move global -> shared as whole strip rows by the bulk copy
// engine (cp.async.bulk, completion counted on an mbarrier per ring slot), issued
// by one thread; per-thread 8..32-byte cp.async copies of the same rows keep the
// load/store units and L1 busy and reach about two thirds of HBM bandwidth on
// this access pattern, the bulk copies nearly all of it.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes) : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}
// wait for phase `parity` of the barrier; gives up after limit_ns (false)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          uint64_t limit_ns = 1000000000ull) {
    const unsigned a = smem_u32(bar);
    uint64_t t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 63) == 0) {
            const uint64_t t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}

constexpr int STREAM_PD_BULK = 8;   // ring depth of the bulk-copy sweep

template <typename V, int T>
constexpr size_t stream_bulk_smem_bytes() {
    constexpr size_t pk = sizeof(Pack<V, T>);
    constexpr size_t rows = (4 + 3 * STREAM_PD_BULK) * SW * pk + STREAM_PD_BULK * SW * sizeof(int);
    constexpr size_t part = (size_t)SW * NDOT * T * sizeof(V);
    constexpr size_t red = (size_t)SW * sizeof(double);
    return rows > part ? (rows > red ? rows : red) : (part > red ? part : red);
}

// Host-side test of the bulk path's alignment rules: every strip row piece must
// start on a 16-byte boundary and be a multiple of 16 bytes long, and a torus
// wraps a strip at most once.  Row pieces start at column strip*W - XH (even) and
// rows at y*nx: a pack of 16 or 32 bytes always qualifies, 8 or 24 bytes need an
// even nx.
inline bool stream_bulk_ok(int nx, int pack_bytes) {
    if (nx < SW) return false;
    if (pack_bytes % 16 == 0) return true;
    return pack_bytes % 8 == 0 && nx % 2 == 0;
}

// The sweep of stream_sweep with rows of r, w, p arriving by bulk copies into a
// ring shared by the CTA (slot rows [r | w | p] of SW packs).  Thread 0 issues
// row y - H + PD into the slot of row y - H after the barrier that ends step y
// (every thread has then finished reading it); each row completes one phase of
// its slot's mbarrier (an arrival without bytes when the row is outside the grid
// or past the segment).  Out-of-grid entries read as zero.  Colours still move by
// per-thread cp.async (4 bytes a vertex, own columns only matter).  bars: PD
// mbarriers in static shared memory.
template <typename V, int T, int KIND, bool KEEPX>
__device__ __forceinline__ void stream_sweep_bulk(const Solve &s, int tile, int cur, int strip, int ys,
                                                  int ye, unsigned char *smem, uint64_t *bars,
                                                  StreamAcc<V, T> &acc) {
    constexpr int H = Strip<KIND>::H, XH = Strip<KIND>::XH, PD = STREAM_PD_BULK, NT = SW;
    constexpr unsigned PB = sizeof(Pack<V, T>);
    static_assert(PB == T * sizeof(V), "packs are unpadded rows of T values");
    using P = Pack<V, T>;
    using M = PackMath<V, T>;
    P *const ps = reinterpret_cast<P *>(smem);
    P *const us = ps + 2 * NT;
    P *const ring = ps + 4 * NT;     // [PD][3][NT], shared by the CTA
    int *const ringc = reinterpret_cast<int *>(ps + (4 + 3 * PD) * NT) + threadIdx.x;
    const int nx = s.op.nx, ny = s.op.ny;
    const bool per = s.op.periodic;
    const int xl = threadIdx.x;
    const int gx0 = strip * Strip<KIND>::W - XH;
    const int gx = gx0 + xl;
    bool inx;
    const int gxw = wrap_coord(gx, nx, per, inx);
    const bool outx = xl >= XH && xl < XH + Strip<KIND>::W && gx < nx;
    const int cb = tile * T;
    const int64_t off = (int64_t)tile * s.op.n * T;
    const V *const r = static_cast<const V *>(cur ? s.rbuf[1] : s.rbuf[0]) + off;
    const V *const w = static_cast<const V *>(cur ? s.wbuf[1] : s.wbuf[0]) + off;
    const V *const p = static_cast<const V *>(cur ? s.pbuf[1] : s.pbuf[0]) + off;
    P na, b;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        na.v[t] = -(V)s.alpha[cb + t];
        b.v[t] = (V)s.beta[cb + t];
    }
    P pw0 = zero_pack<V, T>(), pw1 = pw0, pw2 = pw0;   // p at rows y-2, y-1, y
    P uw0 = pw0, uw1 = pw0, uw2 = pw0;                 // u at rows y-3, y-2, y-1
    int y = ys - H;
    const int yend = ye + H;
    // column pieces of every row copy: [c0, c1) of the row, and on a torus the
    // wrapped columns left of 0 (to slot offset 0) and right of nx - 1
    const int c0 = gx0 < 0 ? 0 : gx0;
    const int c1 = gx0 + SW > nx ? nx : gx0 + SW;
    const int lw = per && gx0 < 0 ? -gx0 : 0;
    const int rw = per && gx0 + SW > nx ? gx0 + SW - nx : 0;
    const unsigned row_bytes = (unsigned)(c1 - c0 + lw + rw) * PB;

    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PD; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int yr, int slot) {   // thread 0
        bool iny;
        const int gyw = wrap_coord(yr, ny, per, iny);
        if (!iny || yr >= yend) {
            mbar_arrive(&bars[slot]);
            return;
        }
        mbar_arrive_tx(&bars[slot], 3 * row_bytes);
        const int64_t re = (int64_t)gyw * nx * T;
        const V *src[3] = {r + re, w + re, p + re};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            P *dst = ring + (slot * 3 + a) * NT;
            bulk_g2s(dst + (c0 - gx0), src[a] + (int64_t)c0 * T, (unsigned)(c1 - c0) * PB, &bars[slot]);
            if (lw) bulk_g2s(dst, src[a] + (int64_t)(nx - lw) * T, (unsigned)lw * PB, &bars[slot]);
            if (rw) bulk_g2s(dst + (nx - gx0), src[a], (unsigned)rw * PB, &bars[slot]);
        }
    };
    auto load_colour = [&](int yr, int slot) {
        bool iny;
        const int gyw = wrap_coord(yr, ny, per, iny);
        const bool in = iny && inx && yr < yend;
        const unsigned dc = smem_u32(ringc + slot * NT);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dc),
                     "l"(s.colour + (in ? (int64_t)gyw * nx + gxw : 0)), "r"(in ? 4 : 0));
        cp_async_commit();
    };
    auto emit = [&](int yo, int slot, const P &pk, const P &wk) {
        const P *q = ring + slot * 3 * NT + xl;
        const P rk = M::fma(na, q[NT], q[0]);
        const int64_t e = ((int64_t)yo * nx + gx) * T;
        V *rn = static_cast<V *>(cur ? s.rbuf[0] : s.rbuf[1]) + off;
        V *wn = static_cast<V *>(cur ? s.wbuf[0] : s.wbuf[1]) + off;
        V *pn = static_cast<V *>(cur ? s.pbuf[0] : s.pbuf[1]) + off;
        *reinterpret_cast<P *>(rn + e) = rk;
        *reinterpret_cast<P *>(pn + e) = pk;
        *reinterpret_cast<P *>(wn + e) = wk;
        if constexpr (KEEPX) {
            V *x = static_cast<V *>(s.x) + off;
            const P xo = *reinterpret_cast<const P *>(x + e);
            *reinterpret_cast<P *>(x + e) = M::fma(M::neg(na), q[2 * NT], xo);
        }
        const int lc = ringc[slot * NT] - cb;
        acc.rr = M::fma(rk, rk, acc.rr);
        acc.pw = M::fma(pk, wk, acc.pw);
        acc.rw = M::fma(rk, wk, acc.rw);
        acc.ww = M::fma(wk, wk, acc.ww);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (lc == t) {
                acc.vr[t] += rk.v[t];
                acc.vw[t] += wk.v[t];
            }
        }
    };

    // ring slot of row yr is (yr - y0) mod PD, its n-th fill completes phase n of the
    // slot's barrier (parity bit kept per slot); see stream_sweep for the schedule
    for (int k = 0; k < PD - H; ++k) {
        if (threadIdx.x == 0) issue(y + k, k);
        load_colour(y + k, k);
    }
    const P sc = M::splat(op_scale<V>(s.op)), k2 = M::splat(op_kappa2<V>(s.op));
    int slot = 0;
    unsigned parity = 0;
    bool ok = true;
    for (; y < yend; ++y) {
        cp_async_wait<PD - 1 - H>();
        ok &= mbar_wait(&bars[slot], (parity >> slot) & 1u);
        parity ^= 1u << slot;
        {
            bool iny;
            wrap_coord(y, ny, per, iny);
            const bool in = iny && inx;
            const P *q = ring + slot * 3 * NT + xl;
            const P z = zero_pack<V, T>();
            const P rv = in ? q[0] : z, wv = in ? q[NT] : z, pv = in ? q[2 * NT] : z;
            const P pk = M::fma(b, pv, M::fma(na, wv, rv));
            ps[(y & 1) * NT + threadIdx.x] = pk;
            pw0 = pw1;
            pw1 = pw2;
            pw2 = pk;
        }
        const int slot_h = slot - H < 0 ? slot - H + PD : slot - H;   // slot of row y - H
        if constexpr (KIND == KIND_2D13_SQ) {
            if (y >= ys) {
                P u = zero_pack<V, T>();
                bool uin;
                wrap_coord(y - 1, ny, per, uin);
                if (uin && inx && xl >= 1 && xl < SW - 1) {
                    const P *row = ps + ((y - 1) & 1) * NT;
                    u = diff5p<V, T>(k2, pw1, row[threadIdx.x - 1], row[threadIdx.x + 1], pw0, pw2);
                }
                us[((y - 1) & 1) * NT + threadIdx.x] = u;
                uw0 = uw1;
                uw1 = uw2;
                uw2 = u;
            }
            if (y - 2 >= ys && y - 2 < ye && outx) {
                const P *row = us + ((y - 2) & 1) * NT;
                const P wk = M::mul(sc, diff5p<V, T>(k2, uw1, row[threadIdx.x - 1], row[threadIdx.x + 1], uw0, uw2));
                emit(y - 2, slot_h, pw0, wk);
            }
        } else {
            if (y - 1 >= ys && y - 1 < ye && outx) {
                const V dg = diag_at<V>(s.op, (int64_t)(y - 1) * nx + gx);
                const P *row = ps + ((y - 1) & 1) * NT;
                const P wk = M::mul(sc, diff5p<V, T>(M::splat(dg), pw1, row[threadIdx.x - 1], row[threadIdx.x + 1], pw0, pw2));
                emit(y - 1, slot_h, pw1, wk);
            }
        }
        load_colour(y - H + PD, slot_h);
        slot = slot + 1 == PD ? 0 : slot + 1;
        __syncthreads();
        if (threadIdx.x == 0) issue(y - H + PD, slot_h);
    }
    cp_async_wait<0>();
    if (!ok) set_status(s.status, DEV_TIMEOUT);
    __syncthreads();
}

// CTA sums of the sweep accumulators into cta[NDOT*T] (shared), dot-major
// (k = dot * T + column).  smem: >= (blockDim / 32) * NDOT * T doubles.  Ends with a
// barrier.
template <typename V, int T, int G>
__device__ __forceinline__ void stream_cta_sums(const StreamAcc<V, T / G> &acc, unsigned char *smem,
                                                double *cta) {
    static_assert(G == 1, "one thread per lattice column");
    V flat[NDOT * T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        flat[0 * T + t] = acc.rr.v[t];
        flat[1 * T + t] = acc.pw.v[t];
        flat[2 * T + t] = acc.rw.v[t];
        flat[3 * T + t] = acc.ww.v[t];
        flat[4 * T + t] = acc.vr[t];
        flat[5 * T + t] = acc.vw[t];
    }
    block_sum_to<V, NDOT * T>(flat, reinterpret_cast<double *>(smem), cta);
}

template <typename V, int T, int G, int KIND, bool KEEPX, bool BULK>
__global__ void __launch_bounds__(SW * G, stream_min_blocks_t<V, T>()) k_stream2d(Solve s, int cur) {
    constexpr int K = NDOT * T;
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int strip = blockIdx.x % s.strips, sg = blockIdx.x / s.strips;
    const int ys = sg * s.seg, ye = min(ys + s.seg, s.op.ny);
    StreamAcc<V, T / G> acc;
    acc.zero();
    if constexpr (BULK) {
        static_assert(G == 1, "bulk rows: one thread per lattice column");
        __shared__ uint64_t bars[STREAM_PD_BULK];
        stream_sweep_bulk<V, T, KIND, KEEPX>(s, tile, cur, strip, ys, ye, smem, bars, acc);
    } else {
        stream_sweep<V, T, G, KIND, KEEPX>(s, tile, cur, strip, ys, ye, smem, acc);
    }
    __shared__ double cta[K];
    stream_cta_sums<V, T, G>(acc, smem, cta);
    publish_and_tail<K>(s, tile, cur, cta, reinterpret_cast<double *>(smem));
}

// ------------------------------------------------------------------ streaming 3D engine
// The 7-point kind streams along z: a CTA owns a P3X x P3Y tile of lattice columns
// (a 1-wide halo all around, (P3X-2) x (P3Y-2) of its own) and a segment of
// planes, one thread per lattice column holding all T probing columns.  Per plane
// step: (r, w, p) of plane z arrive from the per-thread cp.async ring, p_k(z) goes
// to a double-buffered shared plane, and w = Q p_k at plane z-1 takes its in-plane
// neighbours from the shared plane written last step and its z neighbours from the
// thread's register window.  Out-of-grid entries are zero (Dirichlet ghosts of the
// difference form); a torus wraps.
constexpr int P3X = 32, P3Y = 8, P3T = P3X * P3Y;
// plane ring depth: a plane step moves 256 lattice columns, so two planes in flight
// suffice, and the smaller ring lets three CTAs share an SM for packs up to 16 bytes
constexpr int P3_PD = 4;

template <typename V, int T>
constexpr size_t stream3d_smem_bytes() {
    constexpr size_t pk = sizeof(Pack<V, T>);
    constexpr size_t rows = (2 + 3 * P3_PD) * P3T * pk + P3_PD * P3T * (sizeof(int) + sizeof(V));
    constexpr size_t part = (size_t)P3T * NDOT * T * sizeof(V);
    constexpr size_t red = (size_t)P3T * sizeof(double);
    return rows > part ? (rows > red ? rows : red) : (part > red ? part : red);
}

template <typename V, int T>
__host__ __device__ constexpr int stream3d_min_blocks() { return sizeof(V) * T <= 16 ? 3 : 2; }

template <typename V, int T, bool KEEPX>
__global__ void __launch_bounds__(P3T, stream3d_min_blocks<V, T>()) k_stream3d(Solve s, int cur) {
    constexpr int K = NDOT * T, PD = P3_PD, H = 1;
    using P = Pack<V, T>;
    using M = PackMath<V, T>;
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    P *const ps = reinterpret_cast<P *>(smem);                    // 2 planes
    P *const ring = ps + 2 * P3T + threadIdx.x;
    int *const ringc = reinterpret_cast<int *>(ps + (2 + 3 * PD) * P3T) + threadIdx.x;
    V *const ringd = reinterpret_cast<V *>(reinterpret_cast<int *>(ps + (2 + 3 * PD) * P3T) + PD * P3T) + threadIdx.x;
    const V *const diag = diag_ptr<V>(s.op);
    const int nx = s.op.nx, ny = s.op.ny, nz = s.op.nz;
    const bool per = s.op.periodic;
    const int xl = threadIdx.x % P3X, yl = threadIdx.x / P3X;
    const int tx = (nx + P3X - 3) / (P3X - 2);                    // x tiles
    const int xy = blockIdx.x % s.strips, sg = blockIdx.x / s.strips;
    const int bx = xy % tx, by = xy / tx;
    const int gx = bx * (P3X - 2) - 1 + xl, gy = by * (P3Y - 2) - 1 + yl;
    bool inx, iny;
    const int gxw = wrap_coord(gx, nx, per, inx);
    const int gyw = wrap_coord(gy, ny, per, iny);
    const bool inxy = inx && iny;
    const bool out = xl >= 1 && xl < P3X - 1 && yl >= 1 && yl < P3Y - 1 && gx < nx && gy < ny;
    const int zs = sg * s.seg, ze = min(zs + s.seg, nz);
    const int cb = tile * T;
    const int64_t off = (int64_t)tile * s.op.n * T;
    const int64_t plane = (int64_t)nx * ny;
    const V *const r = static_cast<const V *>(cur ? s.rbuf[1] : s.rbuf[0]) + off;
    const V *const w = static_cast<const V *>(cur ? s.wbuf[1] : s.wbuf[0]) + off;
    const V *const p = static_cast<const V *>(cur ? s.pbuf[1] : s.pbuf[0]) + off;
    P na, b;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        na.v[t] = -(V)s.alpha[cb + t];
        b.v[t] = (V)s.beta[cb + t];
    }
    StreamAcc<V, T> acc;
    acc.zero();
    int z = zs - H;
    const int zend = ze + H;
    const int64_t col_off = (int64_t)gyw * nx + gxw;
    auto load_plane = [&](int zr, int slot) {
        bool inz;
        const int gzw = wrap_coord(zr, nz, per, inz);
        const bool in = inz && inxy && zr < zend;
        const int64_t vtx = in ? (int64_t)gzw * plane + col_off : 0;
        const int64_t e = vtx * T;
        P *q = ring + slot * 3 * P3T;
        cp_async_pack<V, T>(q, r + e, in);
        cp_async_pack<V, T>(q + P3T, w + e, in);
        cp_async_pack<V, T>(q + 2 * P3T, p + e, in);
        const unsigned dc = (unsigned)__cvta_generic_to_shared(ringc + slot * P3T);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dc),
                     "l"(s.colour + vtx), "r"(in ? 4 : 0));
        if (diag) cp_async_word<V>(ringd + slot * P3T, diag + vtx, in);
        cp_async_commit();
    };
    P pw0 = zero_pack<V, T>(), pw1 = pw0, pw2 = pw0;   // p at planes z-2, z-1, z
    P xpre = zero_pack<V, T>();   // x of the plane emitted next step, loaded a step ahead
    const P sc = M::splat(op_scale<V>(s.op));
    // ring slot of plane zr is (zr - z0) mod PD (see the 2D sweep for the schedule)
#pragma unroll
    for (int k = 0; k < PD - H; ++k) load_plane(z + k, k);
    int slot = 0;
    for (; z < zend; ++z) {
        cp_async_wait<PD - 1 - H>();
        {
            const P *q = ring + slot * 3 * P3T;
            const P pk = M::fma(b, q[2 * P3T], M::fma(na, q[P3T], q[0]));
            ps[(z & 1) * P3T + threadIdx.x] = pk;
            pw0 = pw1;
            pw1 = pw2;
            pw2 = pk;
        }
        const int slot_h = slot - H < 0 ? slot - H + PD : slot - H;
        if (z - 1 >= zs && z - 1 < ze && out) {
            const int64_t gi = (int64_t)(z - 1) * plane + (int64_t)gy * nx + gx;
            const V dg = diag ? ringd[slot_h * P3T] : op_kappa2<V>(s.op);
            const P *pl = ps + ((z - 1) & 1) * P3T;
            const P c = pw1;
            P wk;
            if constexpr (sizeof(V) == 8) {   // direct form in FP64 (see diff5p)
                const P &l = pl[threadIdx.x - 1], &rr = pl[threadIdx.x + 1];
                const P &d = pl[threadIdx.x - P3X], &u = pl[threadIdx.x + P3X];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    wk.v[t] = sc.v[t] * fma(dg + (V)6, c.v[t],
                                            -(((l.v[t] + rr.v[t]) + (d.v[t] + u.v[t])) + (pw0.v[t] + pw2.v[t])));
            } else {
                const P h = M::add(M::add(M::sub(c, pl[threadIdx.x - 1]), M::sub(c, pl[threadIdx.x + 1])),
                                   M::add(M::sub(c, pl[threadIdx.x - P3X]), M::sub(c, pl[threadIdx.x + P3X])));
                const P v = M::add(M::sub(c, pw0), M::sub(c, pw2));
                wk = M::mul(sc, M::fma(M::splat(dg), c, M::add(h, v)));
            }
            // outputs at (gx, gy, z-1)
            const P *q = ring + slot_h * 3 * P3T;
            const P rk = M::fma(na, q[P3T], q[0]);
            const int64_t e = gi * T;
            *reinterpret_cast<P *>(static_cast<V *>(cur ? s.rbuf[0] : s.rbuf[1]) + off + e) = rk;
            *reinterpret_cast<P *>(static_cast<V *>(cur ? s.pbuf[0] : s.pbuf[1]) + off + e) = c;
            *reinterpret_cast<P *>(static_cast<V *>(cur ? s.wbuf[0] : s.wbuf[1]) + off + e) = wk;
            if constexpr (KEEPX)
                *reinterpret_cast<P *>(static_cast<V *>(s.x) + off + e) = M::fma(M::neg(na), q[2 * P3T], xpre);
            const int lc = ringc[slot_h * P3T] - cb;
            acc.rr = M::fma(rk, rk, acc.rr);
            acc.pw = M::fma(c, wk, acc.pw);
            acc.rw = M::fma(rk, wk, acc.rw);
            acc.ww = M::fma(wk, wk, acc.ww);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if (lc == t) {
                    acc.vr[t] += rk.v[t];
                    acc.vw[t] += wk.v[t];
                }
            }
        }
        load_plane(z - H + PD, slot_h);
        if constexpr (KEEPX) {
            if (z >= zs && z < ze && out)   // plane z is emitted by the next step
                xpre = *reinterpret_cast<const P *>(static_cast<const V *>(s.x) + off +
                                                    ((int64_t)z * plane + (int64_t)gy * nx + gx) * T);
        }
        slot = slot + 1 == PD ? 0 : slot + 1;
        __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
    // CTA sums (warp trees, then the warps in a fixed order)
    V flat[K];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        flat[0 * T + t] = acc.rr.v[t];
        flat[1 * T + t] = acc.pw.v[t];
        flat[2 * T + t] = acc.rw.v[t];
        flat[3 * T + t] = acc.ww.v[t];
        flat[4 * T + t] = acc.vr[t];
        flat[5 * T + t] = acc.vw[t];
    }
    __shared__ double cta[K];
    block_sum_to<V, K>(flat, reinterpret_cast<double *>(smem), cta);
    publish_and_tail<K>(s, tile, cur, cta, reinterpret_cast<double *>(smem));
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

// tile widths: FP64 T in {1, 2, 3, 4}, FP32 (mixed) T in {2, 4, 6, 8}
template <typename V, template <typename, int, int> class Launcher, class... A>
static int dispatch_v(int T, int kind, A &&...args) {
    if constexpr (std::is_same<V, double>::value) {
        switch (T) {
            case 1: return dispatch_kind<double, 1, Launcher>(kind, args...);
            case 2: return dispatch_kind<double, 2, Launcher>(kind, args...);
            case 3: return dispatch_kind<double, 3, Launcher>(kind, args...);
            case 4: return dispatch_kind<double, 4, Launcher>(kind, args...);
        }
    } else {
        switch (T) {
            case 2: return dispatch_kind<float, 2, Launcher>(kind, args...);
            case 4: return dispatch_kind<float, 4, Launcher>(kind, args...);
            case 6: return dispatch_kind<float, 6, Launcher>(kind, args...);
            case 8: return dispatch_kind<float, 8, Launcher>(kind, args...);
        }
    }
    return (int)cudaErrorInvalidValue;
}

template <template <typename, int, int> class Launcher, class... A>
static int dispatch(int precision, int T, int kind, A &&...args) {
    return precision == 0 ? dispatch_v<double, Launcher>(T, kind, args...)
                          : dispatch_v<float, Launcher>(T, kind, args...);
}

// The per-iteration pass kernels are compiled in one translation unit per
// precision (engine_iter_f32.cu, engine_iter_f64.cu).
template <typename V>
int iteration_launch(const Solve &s, int cur, cudaStream_t st);
template <typename V>
int iteration_occupancy(int T, int kind, bool bulk, int lean, bool keepx, int *occ);

}  // namespace ld
