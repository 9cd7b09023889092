// Lean 3D pass: the 7-point kind in FP32 with four state words per vertex and column
// (r and p read and written; x two more in gradient mode), Q p recomputed instead of stored.
//
// The one-reduction CG step of the seed system (Sec. 2.1) needs w_k = Q p_k and the
// update r_k = r - alpha Q p_{k-1}; the stored-w pass keeps Q p_{k-1} as a third vector.
// Here it is recomputed: with q = Q p_{k-1},
//   r_k = r - alpha q,   p_k = r_k + beta p_{k-1},   w_k = Q p_k,   x += alpha p_{k-1},
// so w_k at a vertex needs p_k at its six neighbours, hence q there, hence p_{k-1} two
// steps away.  The CTA streams along z over a 32 x 16 tile of lattice columns with a
// 2-wide halo (28 x 12 of its own): per plane step every thread takes p_{k-1} of its
// column from a per-thread cp.async ring into a shared plane; the threads up to one column
// into the halo form q and p_k one plane behind (their in-plane neighbours from that shared
// plane, their z neighbours from a register window) and put p_k into a second shared plane;
// the own threads form w_k another plane behind and write r_k, p_k (and x, which rides in
// the ring) there.  One
// barrier per plane step; the shared planes are double-buffered.  Out-of-grid entries are
// zero (Dirichlet ghosts of the difference form); a torus wraps.
#pragma once
#include "engine_device.cuh"

namespace ld {

constexpr int L3X = 32, L3Y = 16, L3T = L3X * L3Y;
constexpr int L3_HALO = 2;
constexpr int L3_OWNX = L3X - 2 * L3_HALO, L3_OWNY = L3Y - 2 * L3_HALO;
constexpr int LEAN_3D = 3;   // Solve::lean value of this pass (the 2D pass uses 1 and 2)

// ring depth in planes (even: see the unrolled step loop): as deep as the shared memory of
// one (T = 4) or two (T = 2) CTAs per SM allows, so that the copies in flight cover DRAM
// latency
template <int T>
__host__ __device__ constexpr int lean3d_pd() { return T == 2 ? 4 : 6; }
template <int T>
__host__ __device__ constexpr int lean3d_min_blocks() { return T == 2 ? 2 : 1; }

template <typename V, int T>
constexpr size_t lean3d_smem_bytes() {
    constexpr size_t pk = sizeof(Pack<V, T>);
    constexpr size_t planes = 4 * (size_t)L3T * pk;   // p_{k-1} and p_k, two planes each
    constexpr size_t ring = (size_t)lean3d_pd<T>() * L3T * (3 * pk + sizeof(int) + sizeof(V));
    constexpr size_t red = (size_t)L3T * sizeof(double);
    return planes + ring > red ? planes + ring : red;
}

template <typename V, int T, bool KEEPX>
__global__ void __launch_bounds__(L3T, lean3d_min_blocks<T>()) k_lean3d(Solve s, int cur) {
    constexpr int K = NDOT * T, PD = lean3d_pd<T>();
    using P = Pack<V, T>;
    using M = PackMath<V, T>;
    const int tile = launch_tile(s);
    if (s.tile_done[tile]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    P *const pa = reinterpret_cast<P *>(smem);                       // p_{k-1}: 2 planes
    P *const pb = pa + 2 * L3T;                                        // p_k: 2 planes
    P *const ring = pb + 2 * L3T + threadIdx.x;                        // PD x (r, p, x)
    int *const ringc = reinterpret_cast<int *>(pb + 2 * L3T + 3 * PD * L3T) + threadIdx.x;
    V *const ringd = reinterpret_cast<V *>(reinterpret_cast<int *>(pb + 2 * L3T + 3 * PD * L3T) + PD * L3T) +
                     threadIdx.x;
    const V *const diag = diag_ptr<V>(s.op);
    const int nx = s.op.nx, ny = s.op.ny, nz = s.op.nz;
    const bool per = s.op.periodic;
    const int xl = threadIdx.x % L3X, yl = threadIdx.x / L3X;
    const int tx = (nx + L3_OWNX - 1) / L3_OWNX;
    const int xy = blockIdx.x % s.strips, sg = blockIdx.x / s.strips;
    const int bx = xy % tx, by = xy / tx;
    const int gx = bx * L3_OWNX - L3_HALO + xl, gy = by * L3_OWNY - L3_HALO + yl;
    bool inx, iny;
    const int gxw = wrap_coord(gx, nx, per, inx);
    const int gyw = wrap_coord(gy, ny, per, iny);
    const bool inxy = inx && iny;
    const int ring_d = min(min(xl, L3X - 1 - xl), min(yl, L3Y - 1 - yl));   // 0, 1: halo
    const bool lvl1 = ring_d >= 1;                                        // forms q and p_k
    const bool own = ring_d >= 2 && gx < nx && gy < ny;                   // forms w, writes
    const int zs = sg * s.seg, ze = min(zs + s.seg, nz);
    const int cb = tile * T;
    const int64_t off = (int64_t)tile * s.op.n * T;
    const int64_t plane = (int64_t)nx * ny;
    const V *const r = static_cast<const V *>(cur ? s.rbuf[1] : s.rbuf[0]) + off;
    const V *const p = static_cast<const V *>(cur ? s.pbuf[1] : s.pbuf[0]) + off;
    V *const rn = static_cast<V *>(cur ? s.rbuf[0] : s.rbuf[1]) + off;
    V *const pn = static_cast<V *>(cur ? s.pbuf[0] : s.pbuf[1]) + off;
    // the stencil levels run unscaled (Q = s Q~): r_k = r - (alpha s) Q~ p_{k-1}, and the dots
    // with w = s Q~ p_k take their factors of s at the end
    const V scale = op_scale<V>(s.op);
    P nas, b, a;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        a.v[t] = (V)s.alpha[cb + t];
        nas.v[t] = -a.v[t] * scale;
        b.v[t] = (V)s.beta[cb + t];
    }
    const V k2 = op_kappa2<V>(s.op);
    const int64_t col_off = inxy ? (int64_t)gyw * nx + gxw : 0;
    const V *const rc = r + col_off * T, *const pcol = p + col_off * T;
    const V *const xc = KEEPX ? static_cast<const V *>(s.x) + off + col_off * T : nullptr;
    const int32_t *const cc = s.colour + col_off;
    const V *const dcol = diag ? diag + col_off : nullptr;
    // planes zs-2 .. ze+1 are read (q on zs-1 .. ze, w on zs .. ze-1)
    auto load_plane = [&](int zr, int slot) {
        bool inz;
        const int gzw = wrap_coord(zr, nz, per, inz);
        const bool in = inz && inxy && zr <= ze + 1;
        const int64_t zo = in ? (int64_t)gzw * plane : 0;
        P *q = ring + slot * 3 * L3T;
        cp_async_pack<V, T>(q, rc + zo * T, in && lvl1);
        cp_async_pack<V, T>(q + L3T, pcol + zo * T, in);
        if constexpr (KEEPX) cp_async_pack<V, T>(q + 2 * L3T, xc + zo * T, in && own && zr >= zs && zr < ze);
        const unsigned dsm = (unsigned)__cvta_generic_to_shared(ringc + slot * L3T);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dsm), "l"(cc + zo),
                     "r"(in && own ? 4 : 0));
        if (dcol) cp_async_word<V>(ringd + slot * L3T, dcol + zo, in && lvl1);
        cp_async_commit();
    };
    StreamAcc<V, T> acc;
    acc.zero();
    P pm0 = zero_pack<V, T>(), pm1 = pm0, pm2 = pm0;   // p_{k-1} at planes t-2, t-1, t
    P pk0 = pm0, pk1 = pm0, pk2 = pm0;                 // p_k at planes t-3, t-2, t-1
    P rkp = pm0;                                       // r_k at plane t-2
    P xpre = pm0;                                      // x at plane t-2 (own threads)
    V dgp = (V)0;                                      // diagonal term at plane t-2
    int cp = -1;                                       // colour at plane t-2
    const int t0 = zs - L3_HALO;
    const int tend = ze + L3_HALO;
    const int64_t oe = ((int64_t)gy * nx + gx) * T;      // this column within a plane
    const int64_t pt = plane * T;                       // one plane of a vector
#pragma unroll
    for (int k = 0; k < PD - 1; ++k) load_plane(t0 + k, k);
    // One plane step; the loop is unrolled PD times so that the ring slots (plane t in slot
    // (t - t0) mod PD) and the shared planes (plane t in buffer (t - t0) mod 2; PD is even)
    // are compile-time constants.
    static_assert(PD % 2 == 0, "the shared planes alternate within the unrolled ring cycle");
    int t = t0;
    auto step = [&](auto jc) {
        constexpr int J = decltype(jc)::value;
        constexpr int SP = (J + PD - 1) % PD;           // ring slot of plane t-1
        constexpr int B0 = J & 1, B1 = (J + 1) & 1;     // shared buffers of planes t (and t-2), t-1
        const int tt = t + J;
        cp_async_wait<PD - 2>();
        pm0 = pm1;
        pm1 = pm2;
        pm2 = ring[J * 3 * L3T + L3T];
        pa[B0 * L3T + threadIdx.x] = pm2;
        // q = Q p_{k-1}, r_k and p_k at plane t-1 (own columns and the inner halo ring)
        P rkn = zero_pack<V, T>(), pkn = rkn;
        V dgn = (V)0;
        const bool in1 = per || (unsigned)(tt - 1) < (unsigned)nz;
        if (lvl1 && inxy && in1 && tt - 1 >= zs - 1) {
            dgn = diag ? ringd[SP * L3T] : k2;
            const P *pl = pa + B1 * L3T;
            const P c = pm1;
            const P h = M::add(M::add(M::sub(c, pl[threadIdx.x - 1]), M::sub(c, pl[threadIdx.x + 1])),
                               M::add(M::sub(c, pl[threadIdx.x - L3X]), M::sub(c, pl[threadIdx.x + L3X])));
            const P v = M::add(M::sub(c, pm0), M::sub(c, pm2));
            const P q = M::fma(M::splat(dgn), c, M::add(h, v));
            rkn = M::fma(nas, q, ring[SP * 3 * L3T]);
            pkn = M::fma(b, c, rkn);
        }
        pb[B1 * L3T + threadIdx.x] = pkn;
        pk0 = pk1;
        pk1 = pk2;
        pk2 = pkn;
        // w_k = Q p_k at plane t-2 and the outputs there (own columns)
        if (own && tt - 2 >= zs && tt - 2 < ze) {
            const P *pl = pb + B0 * L3T;
            const P c = pk1;
            const P h = M::add(M::add(M::sub(c, pl[threadIdx.x - 1]), M::sub(c, pl[threadIdx.x + 1])),
                               M::add(M::sub(c, pl[threadIdx.x - L3X]), M::sub(c, pl[threadIdx.x + L3X])));
            const P v = M::add(M::sub(c, pk0), M::sub(c, pk2));
            const P wk = M::fma(M::splat(dgp), c, M::add(h, v));   // w / s
            const int64_t e = (int64_t)(tt - 2) * pt + oe;
            *reinterpret_cast<P *>(rn + e) = rkp;
            *reinterpret_cast<P *>(pn + e) = c;
            if constexpr (KEEPX) *reinterpret_cast<P *>(static_cast<V *>(s.x) + off + e) = M::fma(a, pm0, xpre);
            const int lc = cp - cb;
            acc.rr = M::fma(rkp, rkp, acc.rr);
            acc.pw = M::fma(c, wk, acc.pw);
            acc.rw = M::fma(rkp, wk, acc.rw);
            acc.ww = M::fma(wk, wk, acc.ww);
#pragma unroll
            for (int k = 0; k < T; ++k) {
                if (lc == k) {
                    acc.vr[k] += rkp.v[k];
                    acc.vw[k] += wk.v[k];
                }
            }
        }
        rkp = rkn;
        dgp = dgn;
        cp = ringc[SP * L3T];
        if constexpr (KEEPX) xpre = ring[SP * 3 * L3T + 2 * L3T];   // x at plane t-1, emitted next step
        load_plane(tt + PD - 1, SP);
        __syncthreads();
    };
    for (; t < tend; t += PD) {
        step(std::integral_constant<int, 0>{});
        if (t + 1 < tend) step(std::integral_constant<int, 1>{});
        if (t + 2 < tend) step(std::integral_constant<int, 2>{});
        if (t + 3 < tend) step(std::integral_constant<int, 3>{});
        if constexpr (PD > 4) {
            if (t + 4 < tend) step(std::integral_constant<int, (PD > 4 ? 4 : 0)>{});
            if (t + 5 < tend) step(std::integral_constant<int, (PD > 5 ? 5 : 0)>{});
        }
        if constexpr (PD > 6) {
            if (t + 6 < tend) step(std::integral_constant<int, (PD > 6 ? 6 : 0)>{});
            if (t + 7 < tend) step(std::integral_constant<int, (PD > 7 ? 7 : 0)>{});
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    V flat[K];
#pragma unroll
    for (int k = 0; k < T; ++k) {
        flat[0 * T + k] = acc.rr.v[k];
        flat[1 * T + k] = scale * acc.pw.v[k];
        flat[2 * T + k] = scale * acc.rw.v[k];
        flat[3 * T + k] = scale * scale * acc.ww.v[k];
        flat[4 * T + k] = acc.vr[k];
        flat[5 * T + k] = scale * acc.vw[k];
    }
    __shared__ double cta[K];
    block_sum_to<V, K>(flat, reinterpret_cast<double *>(smem), cta);
    publish_and_tail<K>(s, tile, cur, cta, reinterpret_cast<double *>(smem));
}

}  // namespace ld
