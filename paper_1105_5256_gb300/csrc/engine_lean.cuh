// Lean fused CG-M pass for 2D lattices, FP32 vectors: four words of state traffic per
// vertex and probing vector per CG iteration (read r and one direction-like vector,
// write both), instead of the six of the stored-w pass.
//
// The one-reduction CG of the fused pass (Sec. 2.1: the real seed CG on Q x = v_c drives
// every shifted system) needs, per iteration k, r_k = r_{k-1} - alpha_{k-1} w_{k-1},
// p_k = r_k + beta_{k-1} p_{k-1}, w_k = Q p_k and the six dots of r_k, p_k, w_k.  The
// stored-w pass keeps w_{k-1} in HBM; here it is recomputed from the state instead,
// which costs stencil arithmetic but no bytes:
//
//   5-point kind, state (r, p):   q = Q p_{k-1}            (level 1, = w_{k-1})
//                                 r_k = r_{k-1} - alpha q,  p_k = r_k + beta p_{k-1}
//                                 w_k = Q p_k               (level 2)
//   Matern kind Q = s Q1^2, state (r, u = Q1 p):
//                                 q = s Q1 u_{k-1}          (level 1, = w_{k-1})
//                                 r_k = r_{k-1} - alpha q
//                                 u_k = Q1 r_k + beta u_{k-1}   (level 2, = Q1 p_k)
//                                 w_k = s Q1 u_k            (level 3)
//                                 p_k . w_k = s |u_k|^2     (Q1 symmetric)
//
// The Matern state never holds p itself, so its seed solution x (which needs p) is not
// available: contexts that keep x use the stored-w pass for that kind.  Both forms are
// the same CG in exact arithmetic; each level is the FP32-safe difference-form 5-point
// operator c m + ((m - l) + (m - r)) + ((m - d) + (m - u)) of the stored-w pass, applied
// unscaled (the scale s multiplies the update coefficient and the dot products).
//
// A CTA of LEAN_NT threads owns a strip of LEAN_NT X lattice columns (X = 1 or 2 per
// thread, XH halo columns on each side: the pipeline's reach rounded up to even) and a
// segment of rows, and marches down the rows.  Each row of the state (r and p or u, x
// when kept), of the diagonal terms and of the lane codes arrives through a shared ring
// LEAN_PD rows deep, filled by per-thread asynchronous copies (each thread copies its own
// columns; SWL / 16 threads copy the row's lane codes), so that the HBM latency is
// covered by rows in flight.  The row loop is unrolled by three so that the three-row
// register windows of every level rotate by renaming.  Level l at step y produces row
// y - l from the previous step's shared exchange row of level l - 1 (horizontal
// neighbours: each thread publishes its leftmost and rightmost vertex in two arrays, so
// neighbour reads are conflict-free) and its register window (vertical neighbours): one
// barrier per row for all levels.  Outputs of rows or columns outside a Dirichlet grid
// are zero (the ghost values of the difference form; copies of such rows zero-fill); a
// torus wraps.  The colour of a vertex enters only through a per-tile lane code (one
// byte: its column in the tile in the low seven bits, or LEAN_NONE), read for the rows whose
// dots are taken; for the 5-point kind with a scalar kappa^2 and an observation mask the
// code's high bit carries the vertex's mask bit, and the diagonal kappa^2 + tau mask_i is
// formed from it instead of read as a word.
#pragma once
#include "engine_device.cuh"

namespace ld {

constexpr int LEAN_NT = 96;       // threads per CTA (3 warps: strips of 192 columns at X = 2)
constexpr int LEAN_PD = 8;        // ring depth (rows; a power of two)
constexpr uint8_t LEAN_NONE = 0x7F;      // lane code of a vertex outside the tile's columns
constexpr uint8_t LEAN_MASK_BIT = 0x80;  // high bit of a lane code: the vertex is observed

template <int KIND>
struct LeanGeom {
    static constexpr int R = KIND == KIND_2D13_SQ ? 3 : 2;    // rows/columns of reach
    static constexpr int XH = KIND == KIND_2D13_SQ ? 4 : 2;   // halo columns (even)
    static constexpr int NLEV = R;                              // stencil levels per pass
};

template <int X, int KIND>
struct LeanStrip {
    static constexpr int SWL = LEAN_NT * X;                    // lattice columns per strip
    static constexpr int W = SWL - 2 * LeanGeom<KIND>::XH;     // owned columns per strip
};

// one thread's X vertices of one lattice row: T values each, as T/2 float2 (vertex j,
// pair q at index j * T/2 + q: the order of the values in memory)
template <int T, int X>
struct LRow {
    static constexpr int NP = X * T / 2;
    float2 f[NP];
};

// Shared memory of one CTA: the exchange arrays (per level, two buffers by row parity,
// EL = each thread's leftmost vertex and ER = its rightmost (the same array when X = 1),
// LEAN_NT + 2 vertex slots with a zero pad on both ends), then the ring: LEAN_PD slots of
// [r | p or u | x (kept) | diagonal terms (5-point) | lane codes], each one strip row.
template <int T, int X, int KIND, bool KEEPX>
struct LeanSmem {
    static constexpr int NE = X == 1 ? 1 : 2;
    static constexpr int SWL = LEAN_NT * X;
    static constexpr size_t arr = (size_t)(LEAN_NT + 2) * T * sizeof(float);
    static constexpr size_t xch = (size_t)LeanGeom<KIND>::NLEV * 2 * NE * arr;
    static constexpr size_t vrow = (size_t)SWL * T * sizeof(float);
    static constexpr size_t o_s = vrow;
    static constexpr size_t o_x = 2 * vrow;
    static constexpr size_t o_d = o_x + (KEEPX ? vrow : 0);
    static constexpr size_t o_c = o_d + (KIND == KIND_2D5 ? (size_t)SWL * sizeof(float) : 0);
    static constexpr size_t slot = o_c + (size_t)SWL;
    static constexpr size_t ring = (size_t)LEAN_PD * slot;
    static constexpr size_t red = (size_t)LEAN_NT * sizeof(double);
    static constexpr size_t bytes = xch + ring > red ? xch + ring : red;
    static_assert(xch % 16 == 0 && slot % 16 == 0 && vrow % 16 == 0, "16-byte aligned ring rows");
};

// resident CTAs per SM the register budget is sized for (x adds a stream and registers)
template <int T, int X, bool KEEPX>
__host__ __device__ constexpr int lean_min_blocks() { return KEEPX ? 3 : (T * X <= 2 ? 5 : 4); }

// asynchronous copy of BYTES (4, 8, 16 or a multiple of 16) from global to shared memory;
// src-size 0 zero-fills
template <int BYTES>
__device__ __forceinline__ void lean_cp(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *g = static_cast<const char *>(src);
    if constexpr (BYTES >= 16) {
        static_assert(BYTES % 16 == 0, "whole 16-byte pieces");
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d + 16 * k), "l"(g + 16 * k),
                         "r"(valid ? 16 : 0));
    } else if constexpr (BYTES == 8) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(g), "r"(valid ? 8 : 0));
    } else {
        static_assert(BYTES == 4, "copy sizes 4, 8, 16k");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(g), "r"(valid ? 4 : 0));
    }
}

template <int T, int X>
__device__ __forceinline__ void lrow_st(float *p, const LRow<T, X> &v) {
    constexpr int NF = X * T;
    if constexpr (NF == 2) {
        *reinterpret_cast<float2 *>(p) = v.f[0];
    } else {
#pragma unroll
        for (int k = 0; k < NF / 4; ++k)
            reinterpret_cast<float4 *>(p)[k] = make_float4(v.f[2 * k].x, v.f[2 * k].y, v.f[2 * k + 1].x,
                                                           v.f[2 * k + 1].y);
    }
}

// the thread's packs of one ring row (shared memory, aligned to X T 4 bytes)
template <int T, int X>
__device__ __forceinline__ LRow<T, X> lrow_sh(const unsigned char *p) {
    LRow<T, X> o;
    constexpr int NF = X * T;
    if constexpr (NF == 2) {
        o.f[0] = *reinterpret_cast<const float2 *>(p);
    } else {
#pragma unroll
        for (int k = 0; k < NF / 4; ++k) {
            const float4 a = reinterpret_cast<const float4 *>(p)[k];
            o.f[2 * k] = make_float2(a.x, a.y);
            o.f[2 * k + 1] = make_float2(a.z, a.w);
        }
    }
    return o;
}

template <int T, int X>
__device__ __forceinline__ LRow<T, X> lrow_zero() {
    LRow<T, X> o;
#pragma unroll
    for (int k = 0; k < LRow<T, X>::NP; ++k) o.f[k] = make_float2(0.f, 0.f);
    return o;
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);        // a - b, rounded once
}

// one difference-form level for the thread's X vertices; c: per-vertex diagonal term
// (the same for the vertex's columns); l/r of the outer vertices from the exchange arrays
template <int T, int X>
__device__ __forceinline__ LRow<T, X> lean_level(const float (&c)[X], const LRow<T, X> &dn,
                                                 const LRow<T, X> &mid, const LRow<T, X> &up,
                                                 const float2 (&lft)[T / 2], const float2 (&rgt)[T / 2]) {
    constexpr int H = T / 2;
    LRow<T, X> o;
#pragma unroll
    for (int j = 0; j < X; ++j) {
        const float2 cc = make_float2(c[j], c[j]);
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const float2 m = mid.f[j * H + q];
            const float2 l = j == 0 ? lft[q] : mid.f[(j - 1) * H + q];
            const float2 r = j == X - 1 ? rgt[q] : mid.f[(j + 1) * H + q];
            const float2 h = __fadd2_rn(f2sub(m, l), f2sub(m, r));
            const float2 v = __fadd2_rn(f2sub(m, dn.f[j * H + q]), f2sub(m, up.f[j * H + q]));
            o.f[j * H + q] = __ffma2_rn(cc, m, __fadd2_rn(h, v));
        }
    }
    return o;
}

template <int T>
struct LeanAcc {
    float2 rr[T / 2], pw[T / 2], rw[T / 2], ww[T / 2];
    float vr[T], vw[T];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < T / 2; ++q) rr[q] = pw[q] = rw[q] = ww[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < T; ++t) vr[t] = vw[t] = 0.f;
    }
};

// dots of one emitted row: r.r, (p.w), r.w, w.w over the thread's vertices, v.r and v.w
// for the vertices whose lane code names a column of the tile
template <int T, int X, bool PW>
__device__ __forceinline__ void lean_dots(LeanAcc<T> &acc, const LRow<T, X> &rk, const LRow<T, X> &pk,
                                          const LRow<T, X> &w, const uint8_t *codes) {
    constexpr int H = T / 2;
#pragma unroll
    for (int j = 0; j < X; ++j) {
        const int lc = codes[j] & 0x7F;
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const int k = j * H + q;
            acc.rr[q] = __ffma2_rn(rk.f[k], rk.f[k], acc.rr[q]);
            if constexpr (PW) acc.pw[q] = __ffma2_rn(pk.f[k], w.f[k], acc.pw[q]);
            acc.rw[q] = __ffma2_rn(rk.f[k], w.f[k], acc.rw[q]);
            acc.ww[q] = __ffma2_rn(w.f[k], w.f[k], acc.ww[q]);
            if (lc == 2 * q) {
                acc.vr[2 * q] += rk.f[k].x;
                acc.vw[2 * q] += w.f[k].x;
            }
            if (lc == 2 * q + 1) {
                acc.vr[2 * q + 1] += rk.f[k].y;
                acc.vw[2 * q + 1] += w.f[k].y;
            }
        }
    }
}

// Exchange arrays: write this thread's outer vertices of a row into (level, parity), or
// read its neighbours' (the previous thread's rightmost, the next thread's leftmost).
template <int T, int X>
struct LeanXch {
    static constexpr int NE = X == 1 ? 1 : 2;
    static constexpr size_t ARR = (size_t)(LEAN_NT + 2) * T * sizeof(float);
    unsigned char *base;
    __device__ __forceinline__ float2 *arr(int lev, int par, int side) const {
        return reinterpret_cast<float2 *>(base + ((size_t)(lev * 2 + par) * NE + side) * ARR);
    }
    __device__ __forceinline__ void put(int lev, int par, const LRow<T, X> &v) const {
        constexpr int H = T / 2;
        const int t = threadIdx.x + 1;
        float2 *el = arr(lev, par, 0) + t * H;
#pragma unroll
        for (int q = 0; q < H; ++q) el[q] = v.f[q];
        if constexpr (X > 1) {
            float2 *er = arr(lev, par, 1) + t * H;
#pragma unroll
            for (int q = 0; q < H; ++q) er[q] = v.f[(X - 1) * H + q];
        }
    }
    __device__ __forceinline__ void get(int lev, int par, float2 (&lft)[T / 2], float2 (&rgt)[T / 2]) const {
        constexpr int H = T / 2;
        const int t = threadIdx.x + 1;
        const float2 *er = arr(lev, par, X > 1 ? 1 : 0) + (t - 1) * H;
        const float2 *el = arr(lev, par, 0) + (t + 1) * H;
#pragma unroll
        for (int q = 0; q < H; ++q) {
            lft[q] = er[q];
            rgt[q] = el[q];
        }
    }
};

// One lean pass of one tile's strip segment, rows [ys, ye): per-thread dot accumulators.
template <int T, int X, int KIND, bool KEEPX>
__device__ __forceinline__ void lean_sweep(const Solve &s, int tile, int cur, int strip, int ys, int ye,
                                           unsigned char *smem, LeanAcc<T> &acc) {
    using Row = LRow<T, X>;
    using S = LeanSmem<T, X, KIND, KEEPX>;
    constexpr int R = LeanGeom<KIND>::R, XH = LeanGeom<KIND>::XH, H = T / 2, NP = Row::NP;
    constexpr int W = LeanStrip<X, KIND>::W, SWL = LeanStrip<X, KIND>::SWL, PD = LEAN_PD;
    constexpr bool MAT = KIND == KIND_2D13_SQ;
    static_assert(KIND == KIND_2D5 || KIND == KIND_2D13_SQ, "2D lattice kinds");
    static_assert(!(KEEPX && MAT), "the Matern state holds no p for x");
    const int tid = threadIdx.x;
    const int nx = s.op.nx, ny = s.op.ny;
    const bool per = s.op.periodic;
    const int xl0 = tid * X;
    const int gx = strip * W - XH + xl0;
    bool inx;
    const int gxw = wrap_coord(gx, nx, per, inx);
    if (!per) inx = gx >= 0 && gx + X - 1 < nx;        // X = 2 needs nx even: both or none
    const bool owned = xl0 >= XH && xl0 < XH + W && gx < nx;
    // a warp whose columns all lie outside a Dirichlet grid keeps only the barriers: its
    // values are the zero ghosts the exchange arrays already hold
    const bool wact = per || __any_sync(0xffffffffu, gx < nx && gx + X > 0);
    const int64_t off = (int64_t)tile * s.op.n * T;
    const float *const rg = static_cast<const float *>(cur ? s.rbuf[1] : s.rbuf[0]) + off;
    const float *const sg = static_cast<const float *>(cur ? s.pbuf[1] : s.pbuf[0]) + off;
    float *const rn = static_cast<float *>(cur ? s.rbuf[0] : s.rbuf[1]) + off;
    float *const sn = static_cast<float *>(cur ? s.pbuf[0] : s.pbuf[1]) + off;
    float *const xs = KEEPX ? static_cast<float *>(s.x) + off : nullptr;
    // 5-point diagonal: from the codes' mask bit (scalar kappa^2 with a mask), the FP32 word
    // array (kappa^2 field), or the scalar kappa^2
    const bool mbit = !MAT && s.lane_mask;
    const float *const diag = MAT || mbit ? nullptr : s.op.diag_f;
    const float tauf = s.op.tau_f;
    const uint8_t *const code = s.lane + ((int64_t)tile * s.strips + strip) * (int64_t)ny * SWL;
    const int cb = tile * T;
    // per-column coefficients: -alpha s (level-1 update), beta, alpha (seed solution)
    float2 nas[H], bb[H], aa[H];
#pragma unroll
    for (int q = 0; q < H; ++q) {
        const float a0 = (float)s.alpha[cb + 2 * q], a1 = (float)s.alpha[cb + 2 * q + 1];
        nas[q] = make_float2(-a0 * s.op.scale_f, -a1 * s.op.scale_f);
        aa[q] = make_float2(a0, a1);
        bb[q] = make_float2((float)s.beta[cb + 2 * q], (float)s.beta[cb + 2 * q + 1]);
    }
    const float k2 = s.op.kappa2_f;
    const LeanXch<T, X> xc{smem};
    unsigned char *const ring = smem + S::xch;
    // zero the exchange arrays (pads included) and the ring: every value a level reads is
    // then finite, whether or not its row was ever loaded
    for (int k = tid; k < (int)((S::xch + S::ring) / 16); k += LEAN_NT)
        reinterpret_cast<float4 *>(smem)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    const int y0 = ys - R;
    const int yend = ye + R;
    const int nsteps = yend - y0;
    // Ring: row r of the sweep lives in slot (r - y0) mod PD from its arrival (step r)
    // until its last reader, step r + R (the lane codes of the row it emits; r and x are
    // read at step r + 1, the diagonal at r + 1 and r + 2).  After the barrier that ends
    // step y the slot of row y - R takes row y - R + PD: the prologue queues PD - R rows,
    // and row y's copy group is complete once at most PD - R - 1 younger groups are pending.
    int lrow = y0;
    int lwr = per ? ((y0 % ny) + ny) % ny : y0;
    auto load_row = [&](int sl) {
        const bool in = lrow < yend && (per || (unsigned)lrow < (unsigned)ny) && inx;
        const int64_t v = in ? (int64_t)lwr * nx + gxw : 0;
        unsigned char *base = ring + (size_t)sl * S::slot;
        if (wact) {
            lean_cp<X * T * 4>(base + (size_t)xl0 * T * 4, rg + v * T, in);
            lean_cp<X * T * 4>(base + S::o_s + (size_t)xl0 * T * 4, sg + v * T, in);
            if constexpr (KEEPX) lean_cp<X * T * 4>(base + S::o_x + (size_t)xl0 * T * 4, xs + v * T, in && owned);
            if constexpr (!MAT) {
                if (diag) lean_cp<X * 4>(base + S::o_d + (size_t)xl0 * 4, diag + v, in);
            }
        }
        if (tid < SWL / 16) {
            const bool cin = lrow < yend && (per || (unsigned)lrow < (unsigned)ny);
            lean_cp<16>(base + S::o_c + tid * 16, code + (int64_t)(cin ? lwr : 0) * SWL + tid * 16, cin);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        ++lrow;
        ++lwr;
        if (per && lwr >= ny) lwr -= ny;
    };
#pragma unroll
    for (int k = 0; k < PD - R; ++k) load_row(k);

    Row U[3], RK[3], K[3];      // windows by lattice row, slot = (row - y0) mod 3
#pragma unroll
    for (int k = 0; k < 3; ++k) U[k] = RK[k] = K[k] = lrow_zero<T, X>();
    // store offset of lattice row y - 1 in the thread's column (rows y - 2: minus nx T)
    int64_t st1 = ((int64_t)(y0 - 1) * nx + gx) * T;

    // one row step; PH = (y - y0) mod 3 fixes the register roles at compile time
    auto step = [&](auto ph, int y) {
        constexpr int PH = decltype(ph)::value;
        constexpr int P1 = (PH + 2) % 3, P2 = (PH + 1) % 3;       // slots of rows y - 1, y - 2
        asm volatile("cp.async.wait_group %0;\n" ::"n"(PD - R - 1));
        const int jr = y - y0;
        const unsigned char *sy = ring + (size_t)(jr & (PD - 1)) * S::slot;
        const unsigned char *s1 = ring + (size_t)((jr - 1) & (PD - 1)) * S::slot;
        const unsigned char *sR = ring + (size_t)((jr - R) & (PD - 1)) * S::slot;
        if (wact) {
            const bool in1 = (per || (unsigned)(y - 1) < (unsigned)ny) && inx;
            const int par0 = y & 1, par1 = (y - 1) & 1;
            const bool own1 = owned && (unsigned)(y - 1 - ys) < (unsigned)(ye - ys);
            const bool own2 = owned && (unsigned)(y - 2 - ys) < (unsigned)(ye - ys);
            const Row unew = lrow_sh<T, X>(sy + S::o_s + (size_t)xl0 * T * 4);
            const Row rprev = lrow_sh<T, X>(s1 + (size_t)xl0 * T * 4);      // r_{k-1}, row y - 1
            U[PH] = unew;
            xc.put(0, par0, unew);
            float2 lf[H], rt[H];
            xc.get(0, par1, lf, rt);
            if constexpr (MAT) {
                const bool in2 = (per || (unsigned)(y - 2) < (unsigned)ny) && inx;
                float cc[X];
#pragma unroll
                for (int j = 0; j < X; ++j) cc[j] = k2;
                // level 1: q = Q1 u_{k-1} at row y - 1; r_k = r_{k-1} - alpha s q
                const Row q = lean_level<T, X>(cc, U[P2], U[P1], U[PH], lf, rt);
                Row rk;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const float2 na = in1 ? nas[k % H] : make_float2(0.f, 0.f);
                    rk.f[k] = __ffma2_rn(na, q.f[k], rprev.f[k]);
                }
                RK[P1] = rk;
                xc.put(1, par1, rk);
                if (own1) lrow_st<T, X>(rn + st1, rk);
                // level 2: u_k = Q1 r_k + beta u_{k-1} at row y - 2 (zero outside the grid)
                xc.get(1, par0, lf, rt);            // row y - 2 has the parity of y
                const Row t2 = lean_level<T, X>(cc, RK[PH], RK[P2], RK[P1], lf, rt);
                const float2 m2 = in2 ? make_float2(1.f, 1.f) : make_float2(0.f, 0.f);
                Row uk;
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    uk.f[k] = __ffma2_rn(m2, t2.f[k], __fmul2_rn(bb[k % H], U[P2].f[k]));
                K[P2] = uk;
                xc.put(2, par0, uk);
                if (own2) {
                    lrow_st<T, X>(sn + st1 - (int64_t)nx * T, uk);
#pragma unroll
                    for (int k = 0; k < NP; ++k) acc.pw[k % H] = __ffma2_rn(uk.f[k], uk.f[k], acc.pw[k % H]);
                }
                // level 3: w_k / s = Q1 u_k at row y - 3, and that row's dots
                if (owned && (unsigned)(y - 3 - ys) < (unsigned)(ye - ys)) {
                    xc.get(2, par1, lf, rt);        // row y - 3 has the parity of y - 1
                    const Row w = lean_level<T, X>(cc, K[P1], K[PH], K[P2], lf, rt);
                    lean_dots<T, X, false>(acc, RK[PH], RK[PH], w, sR + S::o_c + xl0);
                }
            } else {
                // level 1: q = Q p_{k-1} at row y - 1 (that row's diagonal); r_k, p_k, x_k
                const unsigned char *s2 = ring + (size_t)((jr - 2) & (PD - 1)) * S::slot;
                float d1[X], d2[X];
#pragma unroll
                for (int j = 0; j < X; ++j) {
                    if (mbit) {
                        d1[j] = k2 + ((s1 + S::o_c)[xl0 + j] & LEAN_MASK_BIT ? tauf : 0.f);
                        d2[j] = k2 + ((s2 + S::o_c)[xl0 + j] & LEAN_MASK_BIT ? tauf : 0.f);
                    } else {
                        d1[j] = diag ? reinterpret_cast<const float *>(s1 + S::o_d)[xl0 + j] : k2;
                        d2[j] = diag ? reinterpret_cast<const float *>(s2 + S::o_d)[xl0 + j] : k2;
                    }
                }
                const Row q = lean_level<T, X>(d1, U[P2], U[P1], U[PH], lf, rt);
                Row rk, pk;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const float2 na = in1 ? nas[k % H] : make_float2(0.f, 0.f);
                    rk.f[k] = __ffma2_rn(na, q.f[k], rprev.f[k]);
                    pk.f[k] = __ffma2_rn(bb[k % H], U[P1].f[k], rk.f[k]);
                }
                RK[P1] = rk;
                K[P1] = pk;
                xc.put(1, par1, pk);
                if (own1) {
                    lrow_st<T, X>(rn + st1, rk);
                    lrow_st<T, X>(sn + st1, pk);
                    if constexpr (KEEPX) {
                        const Row xo = lrow_sh<T, X>(s1 + S::o_x + (size_t)xl0 * T * 4);
                        Row xn;
#pragma unroll
                        for (int k = 0; k < NP; ++k) xn.f[k] = __ffma2_rn(aa[k % H], U[P1].f[k], xo.f[k]);
                        lrow_st<T, X>(xs + st1, xn);
                    }
                }
                // level 2: w_k / s = Q p_k at row y - 2, and that row's dots
                if (own2) {
                    xc.get(1, par0, lf, rt);        // row y - 2 has the parity of y
                    const Row w = lean_level<T, X>(d2, K[PH], K[P2], K[P1], lf, rt);
                    lean_dots<T, X, true>(acc, RK[P2], K[P2], w, sR + S::o_c + xl0);
                }
            }
        }
        st1 += (int64_t)nx * T;
        __syncthreads();
        load_row((jr - R) & (PD - 1));     // row y - R is done: its slot takes row y - R + PD
    };
    for (int j = 0; j < nsteps; j += 3) {
        const int y = y0 + j;
        step(std::integral_constant<int, 0>(), y);
        if (j + 1 < nsteps) step(std::integral_constant<int, 1>(), y + 1);
        if (j + 2 < nsteps) step(std::integral_constant<int, 2>(), y + 2);
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    // the levels ran unscaled: p.w and r.w carry one factor s, w.w two, v.w one
    const float sc = s.op.scale_f;
#pragma unroll
    for (int q = 0; q < H; ++q) {
        acc.pw[q] = make_float2(acc.pw[q].x * sc, acc.pw[q].y * sc);
        acc.rw[q] = make_float2(acc.rw[q].x * sc, acc.rw[q].y * sc);
        acc.ww[q] = make_float2(acc.ww[q].x * (sc * sc), acc.ww[q].y * (sc * sc));
    }
#pragma unroll
    for (int t = 0; t < T; ++t) acc.vw[t] *= sc;
    __syncthreads();
}

template <int T, int X, int KIND, bool KEEPX>
__global__ void __launch_bounds__(LEAN_NT, lean_min_blocks<T, X, KEEPX>()) k_lean2d(Solve s, int cur) {
    constexpr int K = NDOT * T;
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int strip = blockIdx.x % s.strips, sg = blockIdx.x / s.strips;
    const int ys = sg * s.seg, ye = min(ys + s.seg, s.op.ny);
    LeanAcc<T> acc;
    acc.zero();
    lean_sweep<T, X, KIND, KEEPX>(s, tile, cur, strip, ys, ye, smem, acc);
    float flat[K];
#pragma unroll
    for (int q = 0; q < T / 2; ++q) {
        flat[0 * T + 2 * q] = acc.rr[q].x;
        flat[0 * T + 2 * q + 1] = acc.rr[q].y;
        flat[1 * T + 2 * q] = acc.pw[q].x;
        flat[1 * T + 2 * q + 1] = acc.pw[q].y;
        flat[2 * T + 2 * q] = acc.rw[q].x;
        flat[2 * T + 2 * q + 1] = acc.rw[q].y;
        flat[3 * T + 2 * q] = acc.ww[q].x;
        flat[3 * T + 2 * q + 1] = acc.ww[q].y;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        flat[4 * T + t] = acc.vr[t];
        flat[5 * T + t] = acc.vw[t];
    }
    __shared__ double cta[K];
    block_sum_to<float, K>(flat, reinterpret_cast<double *>(smem), cta);
    publish_and_tail<K>(s, tile, cur, cta, reinterpret_cast<double *>(smem));
}

}  // namespace ld
