#pragma once
// lf2_tblock.cuh -- temporal blocking: `T` leapfrog steps per pass over HBM.
//
// A block owns an output tile of TX x TY sites in the x-y plane and a chunk of z-planes.  It
// loads the tile plus a T-site halo on every side (the region, RX x RY columns) and streams
// the region along z.  Stage s (s = 1..T) computes step s for plane i - s while plane i is
// being loaded, so the T steps form a wavefront that lags one plane per stage:
//
//     iteration i:  load phi_0, pi, comp of plane i
//                   stage 1 -> phi_1(i-1), stage 2 -> phi_2(i-2), ..., stage T -> phi_T(i-T)
//
// Each thread owns CX adjacent columns of one region row for every stage, so for its own
// columns the centre and the z-neighbours of level s-1 (planes q-1, q, q+1) and the queues of
// pi and comp (planes i .. i-T) stay in registers.  The x-y neighbours of level s-1 come from
// shared memory, where every level keeps two plane buffers: stage s reads the plane that
// stage s-1 wrote in the previous iteration and writes its own into the other buffer, so one
// __syncthreads per iteration orders everything.  Level s is exact on the region shrunk by s
// sites on each side (the periodic images of the halo were loaded, Sec. 3.3.1); the values
// outside are never read by an exact site, and only the centre tile of level T is stored.
//
// The z-direction works the same way: to produce planes [z0, z1) at level T the chunk loads
// planes [z0 - T, z1 + T) (wrapped) and each stage computes the planes it is exact on.
//
// pi and comp of halo columns are read by the neighbouring blocks too, so this kernel reads
// phi, pi, comp from the front buffers and writes all three to the back buffers.
#include "lf2_bounds.cuh"
#include "lf2_internal.cuh"

namespace lf2 {
namespace tb {

constexpr int kTbMaxThreads = 512;

template <int BYTES>
struct VecOf;
template <>
struct VecOf<4> {
    using T = float;
};
template <>
struct VecOf<8> {
    using T = float2;
};
template <>
struct VecOf<16> {
    using T = float4;
};

// N contiguous elements of R as vector accesses of CH bytes, CH the largest of 16, 8, 4 that
// divides the N elements' size: one access for 4, 8 or 16 bytes (every 1- and 2-component
// case), three for the 12 and 24 bytes of a 3- or 6-component site, whose address is only
// 4- or 8-byte aligned.
template <typename R, int N>
struct VecChunk {
    static constexpr int BYTES = N * (int)sizeof(R);
    static constexpr int CH = BYTES % 16 == 0 ? 16 : (BYTES % 8 == 0 ? 8 : 4);
    static constexpr int COUNT = BYTES / CH;
    static constexpr int E = CH / (int)sizeof(R);
    using V = typename VecOf<CH>::T;
};

template <typename R, int N>
__device__ __forceinline__ void vload_g(const R *__restrict__ p, R (&v)[N]) {
    using C = VecChunk<R, N>;
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        typename C::V t = __ldg(reinterpret_cast<const typename C::V *>(p) + q);
        memcpy(&v[q * C::E], &t, C::CH);
    }
}
template <typename R, int N>
__device__ __forceinline__ void vload_cg(const R *__restrict__ p, R (&v)[N]) {
    using C = VecChunk<R, N>;
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        typename C::V t = __ldcg(reinterpret_cast<const typename C::V *>(p) + q);
        memcpy(&v[q * C::E], &t, C::CH);
    }
}
template <typename R, int N>
__device__ __forceinline__ void vstore_g(R *__restrict__ p, const R (&v)[N]) {
    using C = VecChunk<R, N>;
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        typename C::V t;
        memcpy(&t, &v[q * C::E], C::CH);
        reinterpret_cast<typename C::V *>(p)[q] = t;
    }
}
template <typename R, int N>
__device__ __forceinline__ void vload_s(const R *p, R (&v)[N]) {
    using C = VecChunk<R, N>;
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        typename C::V t = reinterpret_cast<const typename C::V *>(p)[q];
        memcpy(&v[q * C::E], &t, C::CH);
    }
}
template <typename R, int N>
__device__ __forceinline__ void vstore_s(R *p, const R (&v)[N]) {
    using C = VecChunk<R, N>;
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        typename C::V t;
        memcpy(&t, &v[q * C::E], C::CH);
        reinterpret_cast<typename C::V *>(p)[q] = t;
    }
}

__device__ __forceinline__ int wrap_any(int v, int n) {
    int w = v % n;
    return w < 0 ? w + n : w;
}

// Thread-block clusters: the CTAs of a cluster stack along y and each keeps its band of the
// cluster's region rows.  A band's first and last rows are the y-neighbours of the bands next
// to it; after each level's plane is written, those rows are also stored into the neighbour
// CTA's halo row (distributed shared memory), and one cluster-wide barrier per iteration orders
// the stores before the reads of the next iteration, as __syncthreads does for one CTA.
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Stores N elements at the address that `p` (this CTA's shared memory) has in CTA `rank` of
// the cluster.
template <typename R, int N>
__device__ __forceinline__ void vstore_cluster(const R *p, unsigned rank, const R (&v)[N]) {
    using C = VecChunk<R, N>;
    unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
    unsigned w[N * sizeof(R) / 4];
    memcpy(w, v, sizeof w);
#pragma unroll
    for (int q = 0; q < C::COUNT; ++q) {
        const unsigned d = ra + q * C::CH;
        const unsigned *u = w + q * (C::CH / 4);
        if constexpr (C::CH == 16)
            asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(d), "r"(u[0]), "r"(u[1]), "r"(u[2]),
                         "r"(u[3])
                         : "memory");
        else if constexpr (C::CH == 8)
            asm volatile("st.shared::cluster.v2.b32 [%0], {%1, %2};\n" ::"r"(d), "r"(u[0]), "r"(u[1]) : "memory");
        else
            asm volatile("st.shared::cluster.b32 [%0], %1;\n" ::"r"(d), "r"(u[0]) : "memory");
    }
}
// Own plane value v at `p`: also into the halo row of the band above (push & 1: this is the
// band's first row; the neighbour's halo row is `band` rows below p) and of the band below
// (push & 2: last row; `band` rows above p).
template <typename R, int W, int CL>
__device__ __forceinline__ void push_edges(const R *p, unsigned push, unsigned rank, int band, const R (&v)[W]) {
    if constexpr (CL > 1) {
        if (push & 1u) vstore_cluster<R, W>(p + band, rank - 1, v);
        if (push & 2u) vstore_cluster<R, W>(p - band, rank + 1, v);
    }
}

// Per-thread state of the wavefront, kept in registers across iterations.
template <typename R, int T, int W>
struct TbState {
    R lv[T][3][W];  // level l (0..T-1) of own columns at planes q-1, q, q+1 of stage l+1
    R pq[T + 1][W]; // pi of own columns at planes i, i-1, ..., i-T (updated stage by stage)
    R cq[T + 1][W]; // Kahan compensation, same planes
    R pf_phi[W], pf_pi[W], pf_c[W];  // plane i+1, loaded one iteration ahead
};

// One z-iteration of the wavefront.  Level l of the plane written in this iteration lives at
// cur + l * ps2, the one written in the previous iteration at prev + l * ps2 (both already
// offset to this thread's own columns).
// CL > 1: the CTA is one band of a cluster (push, rank, band as for push_edges).
template <typename R, int NC, int MODE, int T, int CX, typename CoefT, int CL = 1>
__device__ __forceinline__ void tb_iteration(TbState<R, T, CX * NC> &st, R *__restrict__ cur, const R *__restrict__ prev,
                                             int ps2, int row_e, const CoefT &k, bool load_next,
                                             const R *__restrict__ nphi, const R *__restrict__ npi,
                                             const float *__restrict__ ncomp, bool store, R *__restrict__ ophi,
                                             R *__restrict__ opi, float *__restrict__ ocomp, bool shfl_x,
                                             unsigned push = 0, unsigned rank = 0, int band = 0) {
    constexpr int W = CX * NC;
    R in_phi[W], in_pi[W], in_c[W];
#pragma unroll
    for (int e = 0; e < W; ++e) {
        in_phi[e] = st.pf_phi[e];
        in_pi[e] = st.pf_pi[e];
        in_c[e] = st.pf_c[e];
    }
    if (load_next) {
        vload_g<R, W>(nphi, st.pf_phi);
        vload_cg<R, W>(npi, st.pf_pi);
        if (MODE == 1) vload_cg<R, W>(reinterpret_cast<const R *>(ncomp), st.pf_c);
    }
#pragma unroll
    for (int e = 0; e < W; ++e) {
        st.lv[0][0][e] = st.lv[0][1][e];
        st.lv[0][1][e] = st.lv[0][2][e];
        st.lv[0][2][e] = in_phi[e];
    }
#pragma unroll
    for (int l = T; l > 0; --l)
#pragma unroll
        for (int e = 0; e < W; ++e) {
            st.pq[l][e] = st.pq[l - 1][e];
            if (MODE == 1) st.cq[l][e] = st.cq[l - 1][e];
        }
#pragma unroll
    for (int e = 0; e < W; ++e) {
        st.pq[0][e] = in_pi[e];
        if (MODE == 1) st.cq[0][e] = in_c[e];
    }
    vstore_s<R, W>(cur, in_phi);
    push_edges<R, W, CL>(cur, push, rank, band, in_phi);

#pragma unroll
    for (int s = 1; s <= T; ++s) {
        const R *src = prev + (s - 1) * ps2;
        R up[W], dn[W], left[NC], right[NC], out[W];
        vload_s<R, W>(src + row_e, up);
        vload_s<R, W>(src - row_e, dn);
        if (shfl_x) {
            // region rows are whole lane groups: the x-neighbours are the adjacent lanes' own
            // columns (at a row's ends the values are from another row, but those columns are
            // outside every stage's exact region and their results are never read)
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                left[a] = __shfl_up_sync(0xffffffffu, st.lv[s - 1][1][(CX - 1) * NC + a], 1);
                right[a] = __shfl_down_sync(0xffffffffu, st.lv[s - 1][1][a], 1);
            }
        } else {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                left[a] = src[a - NC];
                right[a] = src[W + a];
            }
        }
        if constexpr (MODE != 3 && NC == 2) {
            // FP32 complex: the two components of a site form one f32x2 pair
            const Coef32x2 k2 = make_coef32x2(k, k.zero);
            const R *L = st.lv[s - 1][1];
#pragma unroll
            for (int j = 0; j < CX; ++j) {
                const int e = 2 * j;
                f32x2 p = pk2(st.pq[s][e], st.pq[s][e + 1]);
                f32x2 cm = (MODE == 1) ? pk2(st.cq[s][e], st.cq[s][e + 1]) : 0ull;
                f32x2 o;
                update_f32_site2<MODE == 1>(
                    pk2(L[e], L[e + 1]), (j == 0) ? pk2(left[0], left[1]) : pk2(L[e - 2], L[e - 1]),
                    (j == CX - 1) ? pk2(right[0], right[1]) : pk2(L[e + 2], L[e + 3]), pk2(dn[e], dn[e + 1]),
                    pk2(up[e], up[e + 1]), pk2(st.lv[s - 1][0][e], st.lv[s - 1][0][e + 1]),
                    pk2(st.lv[s - 1][2][e], st.lv[s - 1][2][e + 1]), p, cm, o, k2, k);
                up2(o, out[e], out[e + 1]);
                up2(p, st.pq[s][e], st.pq[s][e + 1]);
                if (MODE == 1) up2(cm, st.cq[s][e], st.cq[s][e + 1]);
            }
        } else if constexpr (MODE != 3 && CX % 2 == 0) {
            // FP32: two columns per packed f32x2 instruction stream
            const Coef32x2 k2 = make_coef32x2(k, k.zero);
#pragma unroll
            for (int m = 0; m < CX / 2; ++m) {
                const int j0 = 2 * m, j1 = 2 * m + 1;
                f32x2 c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], o[NC];
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e0 = j0 * NC + a, e1 = j1 * NC + a;
                    const R *L = st.lv[s - 1][1];
                    c[a] = pk2(L[e0], L[e1]);
                    xm[a] = pk2((j0 == 0) ? left[a] : L[e0 - NC], L[e0]);
                    xp[a] = pk2(L[e1], (j1 == CX - 1) ? right[a] : L[e1 + NC]);
                    ym[a] = pk2(dn[e0], dn[e1]);
                    yp[a] = pk2(up[e0], up[e1]);
                    zm[a] = pk2(st.lv[s - 1][0][e0], st.lv[s - 1][0][e1]);
                    zp[a] = pk2(st.lv[s - 1][2][e0], st.lv[s - 1][2][e1]);
                    p[a] = pk2(st.pq[s][e0], st.pq[s][e1]);
                    cm[a] = (MODE == 1) ? pk2(st.cq[s][e0], st.cq[s][e1]) : 0ull;
                }
                update_f32x2<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, o, k2);
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e0 = j0 * NC + a, e1 = j1 * NC + a;
                    up2(o[a], out[e0], out[e1]);
                    up2(p[a], st.pq[s][e0], st.pq[s][e1]);
                    if (MODE == 1) up2(cm[a], st.cq[s][e0], st.cq[s][e1]);
                }
            }
        } else if constexpr (MODE != 3 && NC >= 3) {
            // FP32 with 3 to 6 components: the components of a site in packed pairs
            const Coef32x2 k2 = make_coef32x2(k, k.zero);
#pragma unroll
            for (int j = 0; j < CX; ++j) {
                float c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], o[NC];
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    c[a] = st.lv[s - 1][1][e];
                    xm[a] = (j == 0) ? left[a] : st.lv[s - 1][1][e - NC];
                    xp[a] = (j == CX - 1) ? right[a] : st.lv[s - 1][1][e + NC];
                    ym[a] = dn[e];
                    yp[a] = up[e];
                    zm[a] = st.lv[s - 1][0][e];
                    zp[a] = st.lv[s - 1][2][e];
                    p[a] = st.pq[s][e];
                    cm[a] = (MODE == 1) ? st.cq[s][e] : 0.0f;
                }
                update_f32_siteN<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, o, k2, k);
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    out[e] = o[a];
                    st.pq[s][e] = p[a];
                    if (MODE == 1) st.cq[s][e] = cm[a];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < CX; ++j) {
                R c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], o[NC];
    #pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    c[a] = st.lv[s - 1][1][e];
                    xm[a] = (j == 0) ? left[a] : st.lv[s - 1][1][e - NC];
                    xp[a] = (j == CX - 1) ? right[a] : st.lv[s - 1][1][e + NC];
                    ym[a] = dn[e];
                    yp[a] = up[e];
                    zm[a] = st.lv[s - 1][0][e];
                    zp[a] = st.lv[s - 1][2][e];
                    p[a] = st.pq[s][e];
                    cm[a] = (MODE == 1) ? (float)st.cq[s][e] : 0.0f;
                }
                if constexpr (MODE == 3) {
                    update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, o, k);
                } else {
                    update_f32<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, o, k);
                }
    #pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    out[e] = o[a];
                    st.pq[s][e] = p[a];
                    if (MODE == 1) st.cq[s][e] = cm[a];
                }
            }
        }
        if (s < T) {
#pragma unroll
            for (int e = 0; e < W; ++e) {
                st.lv[s][0][e] = st.lv[s][1][e];
                st.lv[s][1][e] = st.lv[s][2][e];
                st.lv[s][2][e] = out[e];
            }
            vstore_s<R, W>(cur + s * ps2, out);
            push_edges<R, W, CL>(cur + s * ps2, push, rank, band, out);
        } else if (store) {
            vstore_g<R, W>(ophi, out);
            vstore_g<R, W>(opi, st.pq[T]);
            if (MODE == 1) vstore_g<R, W>(reinterpret_cast<R *>(ocomp), st.cq[T]);
        }
    }
    if constexpr (CL > 1)
        cluster_sync();
    else
        __syncthreads();
}

// MODE: 0 = FP32 plain drift, 1 = FP32 Kahan drift, 3 = FP64.
// Light configurations (shallow, narrow) are held to 64 registers so two blocks fit per SM.
template <typename R, int NC, int T, int CX>
constexpr int tb_min_blocks() {
    return (T <= 4 && CX * NC * sizeof(R) <= 8) ? 2 : 1;
}

// One tile x z-chunk of a temporal-blocking pass: (bx, by) is the tile, bz the chunk.  With
// CL > 1 the tile's region rows (TY + 2T) are split into CL bands of equal height, one per CTA
// of a cluster, and `rank` is this CTA's band; CL = 1 is one CTA per tile.
template <typename R, int NC, int MODE, int T, int CX, typename CoefT, int CL = 1>
__device__ __forceinline__ void tb_block(const R *__restrict__ phi, R *__restrict__ phi_out, const R *__restrict__ pi,
                                         R *__restrict__ pi_out, const float *__restrict__ comp,
                                         float *__restrict__ comp_out, const Geom &g, const CoefT &k, int TX, int TY,
                                         int zchunk, int bx, int by, int bz, unsigned rank = 0) {
    constexpr int TP = ((T + CX - 1) / CX) * CX;  // x halo, rounded to whole thread groups
    constexpr int W = CX * NC;                     // elements per thread per plane
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);

    const int RX = TX + 2 * TP, RY = (TY + 2 * T) / CL;  // RY: this CTA's rows
    const int RXT = RX / CX;
    const int ps = (RY + 2) * RX * NC;  // elements per shared plane (one halo row above and below)
    const int t = threadIdx.x;
    const int tx = t % RXT, ry = t / RXT;
    const int ryg = (int)rank * RY + ry;  // row within the tile's region
    const int rx0 = tx * CX;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);

    const int gx0 = wrap_any(x0 - TP + rx0, g.nx);
    const int gy = wrap_any(y0 - T + ryg, g.ny);
    const long long planeE = (long long)g.nx * g.ny * NC;
#ifdef LF2_DEBUG_BOUNDS
    const long long total = planeE * g.nz;  // elements of every field buffer
#endif
    const int colE = (gy * g.nx + gx0) * NC;  // offset within a plane (< 2^31 for every lattice run here)
    const bool out_col =
        rx0 >= TP && rx0 < TP + TX && x0 + rx0 - TP < g.nx && ryg >= T && ryg < T + TY && y0 + ryg - T < g.ny;
    const int s_own = ((ry + 1) * RX + rx0) * NC;
    const int row_e = RX * NC;
    // edge rows of a band with a neighbouring band in the cluster
    const unsigned push = CL > 1 ? ((ry == 0 && rank > 0) ? 1u : 0u) | ((ry == RY - 1 && rank + 1 < CL) ? 2u : 0u) : 0u;

    TbState<R, T, W> st;
#pragma unroll
    for (int l = 0; l < T; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int e = 0; e < W; ++e) st.lv[l][m][e] = R(0);
#pragma unroll
    for (int l = 0; l <= T; ++l)
#pragma unroll
        for (int e = 0; e < W; ++e) st.pq[l][e] = st.cq[l][e] = R(0);
#pragma unroll
    for (int e = 0; e < W; ++e) st.pf_c[e] = R(0);

    // plane index of the next load, advanced with a compare instead of a modulo
    int pl = wrap_any(z0 - T, g.nz);
    {
#ifdef LF2_DEBUG_BOUNDS
        const long long off = checked((long long)pl * planeE + colE, W, total);
#else
        const long long off = (long long)pl * planeE + colE;
#endif
        vload_g<R, W>(phi + off, st.pf_phi);
        vload_cg<R, W>(pi + off, st.pf_pi);
        if (MODE == 1) vload_cg<R, W>(reinterpret_cast<const R *>(comp) + off, st.pf_c);
    }
    const int ibeg = z0 - T, iend = z1 + T;
    // output plane of stage T in iteration i is i - T; stores start at i = z0 + T
    long long out_off = (long long)(z0 - 2 * T - 1) * planeE + colE;  // advanced before each use
#ifdef LF2_DEBUG_BOUNDS
    // every shared access of this thread lies in [s_own - row_e, s_own + ps + 2 ps (T - 1) +
    // row_e + W) of the 2 T ps elements the block holds
    const long long s_lo = checked((long long)s_own - row_e, (long long)ps + 2LL * ps * (T - 1) + 2LL * row_e + W,
                                   2LL * T * ps);
    R *const base = sm + (s_lo + row_e);
#else
    R *const base = sm + s_own;
#endif
    // x-neighbours by warp shuffle when every region row is a whole group of lanes within one
    // warp and the block is whole warps
    const bool shfl_x = (32 % RXT == 0) && ((RXT * RY) % 32 == 0);
    for (int i = ibeg; i < iend; ++i) {
        pl = (pl + 1 == g.nz) ? 0 : pl + 1;
#ifdef LF2_DEBUG_BOUNDS
        const long long noff = checked((long long)pl * planeE + colE, W, total);
#else
        const long long noff = (long long)pl * planeE + colE;
#endif
        out_off += planeE;
        const int par = i & 1;
#ifdef LF2_DEBUG_BOUNDS
        const bool store = out_col && i - T >= z0;
        const long long oo = store ? checked(out_off, W, total) : out_off;
        tb_iteration<R, NC, MODE, T, CX, CoefT, CL>(st, base + par * ps, base + (par ^ 1) * ps, 2 * ps, row_e, k,
                                                    i + 1 < iend, phi + noff, pi + noff, comp + noff, store,
                                                    phi_out + oo, pi_out + oo, comp_out + oo, shfl_x, push, rank,
                                                    RY * row_e);
#else
        tb_iteration<R, NC, MODE, T, CX, CoefT, CL>(st, base + par * ps, base + (par ^ 1) * ps, 2 * ps, row_e, k,
                                                    i + 1 < iend, phi + noff, pi + noff, comp + noff,
                                                    out_col && i - T >= z0, phi_out + out_off, pi_out + out_off,
                                                    comp_out + out_off, shfl_x, push, rank, RY * row_e);
#endif
    }
}

template <typename R, int NC, int MODE, int T, int CX, typename CoefT>
__global__ void __launch_bounds__(kTbMaxThreads, (tb_min_blocks<R, NC, T, CX>()))
    k_tblock(const R *__restrict__ phi, R *__restrict__ phi_out, const R *__restrict__ pi, R *__restrict__ pi_out,
             const float *__restrict__ comp, float *__restrict__ comp_out, Geom g, CoefT k, int TX, int TY,
             int zchunk) {
    tb_block<R, NC, MODE, T, CX, CoefT>(phi, phi_out, pi, pi_out, comp, comp_out, g, k, TX, TY, zchunk, blockIdx.x,
                                        blockIdx.y, blockIdx.z);
}

// The same pass with CL CTAs per tile, one cluster each (cluster dimensions (1, CL, 1)):
// blockIdx.y / CL is the tile row and the cluster rank the band.
template <typename R, int NC, int MODE, int T, int CX, typename CoefT, int CL>
__global__ void __launch_bounds__(kTbMaxThreads, 1)
    k_tblock_cluster(const R *__restrict__ phi, R *__restrict__ phi_out, const R *__restrict__ pi,
                     R *__restrict__ pi_out, const float *__restrict__ comp, float *__restrict__ comp_out, Geom g,
                     CoefT k, int TX, int TY, int zchunk) {
    tb_block<R, NC, MODE, T, CX, CoefT, CL>(phi, phi_out, pi, pi_out, comp, comp_out, g, k, TX, TY, zchunk, blockIdx.x,
                                            blockIdx.y / CL, blockIdx.z, cluster_rank());
}

// Ensemble pass: one launch covers the tiles of every member lattice, items ordered longest
// chunk first.  Which block computes an item does not change its result, so the dynamic
// assignment keeps the output bitwise deterministic.
template <typename R, int NC, int MODE, int T, int CX, typename CoefT>
__global__ void __launch_bounds__(kTbMaxThreads, (tb_min_blocks<R, NC, T, CX>()))
    k_tblock_ensemble(const TbMember *__restrict__ members, const int4 *__restrict__ items, int nitems, int flip,
                      int TX, int TY, int *__restrict__ counter) {
    // Each block takes the next item from a shared counter (zeroed before the launch), so the
    // longest-first work list is scheduled greedily.  The loop ends when the counter passes
    // the last item; no block waits on another.
    __shared__ int s_item;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int4 w = items[it];
        const TbMember &m = members[w.x];
        const int f = m.front ^ flip;
        CoefT k;
        if constexpr (MODE == 3)
            k = m.k64;
        else
            k = m.k32;
        tb_block<R, NC, MODE, T, CX, CoefT>((const R *)m.phi[f], (R *)m.phi[f ^ 1], (const R *)m.pi[f],
                                            (R *)m.pi[f ^ 1], m.comp[f], const_cast<float *>(m.comp[f ^ 1]), m.g, k, TX, TY, m.zchunk,
                                            w.y, w.z, w.w);
        __syncthreads();
    }
}

template <typename R, int NC, int MODE, int T, int CX, typename CoefT>
cudaError_t launch_t(const TbArgs &a, const TbConfig &c, const CoefT &k, cudaStream_t s) {
    constexpr int TP = ((T + CX - 1) / CX) * CX;
    const int RX = c.tile_x + 2 * TP, RY = c.tile_y + 2 * T;
    const int threads = (RX / CX) * RY;
    const size_t smem = (size_t)2 * T * (RY + 2) * RX * NC * sizeof(R);
    auto kern = k_tblock<R, NC, MODE, T, CX, CoefT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.g.nx + c.tile_x - 1) / c.tile_x, (a.g.ny + c.tile_y - 1) / c.tile_y,
              (a.g.nz + c.zchunk - 1) / c.zchunk);
    kern<<<grid, threads, smem, s>>>((const R *)a.phi, (R *)a.phi_out, (const R *)a.pi, (R *)a.pi_out, a.comp,
                                     a.comp_out, a.g, k, c.tile_x, c.tile_y, c.zchunk);
    return cudaGetLastError();
}

// A clustered pass: tiles of tile_x x tile_y output sites, CL CTAs per tile (a cluster of
// dimensions (1, CL, 1)), each with (tile_y + 2T) / CL region rows.
template <typename R, int NC, int MODE, int T, int CX, typename CoefT, int CL>
cudaError_t launch_cluster_t(const TbArgs &a, const TbConfig &c, const CoefT &k, cudaStream_t s) {
    constexpr int TP = ((T + CX - 1) / CX) * CX;
    const int RX = c.tile_x + 2 * TP, RY = (c.tile_y + 2 * T) / CL;
    const int threads = (RX / CX) * RY;
    const size_t smem = (size_t)2 * T * (RY + 2) * RX * NC * sizeof(R);
    auto kern = k_tblock_cluster<R, NC, MODE, T, CX, CoefT, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && CL > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.g.nx + c.tile_x - 1) / c.tile_x, ((a.g.ny + c.tile_y - 1) / c.tile_y) * CL,
                       (a.g.nz + c.zchunk - 1) / c.zchunk);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CL;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorNotSupported;
    return cudaLaunchKernelEx(&cfg, kern, (const R *)a.phi, (R *)a.phi_out, (const R *)a.pi, (R *)a.pi_out, a.comp,
                              a.comp_out, a.g, k, c.tile_x, c.tile_y, c.zchunk);
}

// The clustered kernels that are built: FP32 storage, 1 or 2 components, depth 3 or 4, one
// vector of at most 16 bytes per thread and plane, 2, 4 or 8 CTAs per cluster.
template <typename R, int NC, int MODE, typename CoefT>
cudaError_t launch_cluster_prec(const TbArgs &a, const TbConfig &c, const CoefT &k, cudaStream_t s) {
    if constexpr (NC <= 2 && sizeof(R) == 4) {
        switch (c.cx * 1000 + c.depth * 100 + c.cluster) {
#define LF2_TBC_CASE(CXV, TV, CLV)                                                                     \
            case CXV * 1000 + TV * 100 + CLV:                                                          \
                if constexpr (CXV * NC * sizeof(R) <= 16) return launch_cluster_t<R, NC, MODE, TV, CXV, CoefT, CLV>(a, c, k, s); \
                return cudaErrorNotSupported;
            LF2_TBC_CASE(1, 3, 2) LF2_TBC_CASE(1, 3, 4) LF2_TBC_CASE(1, 3, 8)
            LF2_TBC_CASE(1, 4, 2) LF2_TBC_CASE(1, 4, 4) LF2_TBC_CASE(1, 4, 8)
            LF2_TBC_CASE(2, 3, 2) LF2_TBC_CASE(2, 3, 4) LF2_TBC_CASE(2, 3, 8)
            LF2_TBC_CASE(2, 4, 2) LF2_TBC_CASE(2, 4, 4) LF2_TBC_CASE(2, 4, 8)
            LF2_TBC_CASE(4, 3, 2) LF2_TBC_CASE(4, 3, 4) LF2_TBC_CASE(4, 3, 8)
            LF2_TBC_CASE(4, 4, 2) LF2_TBC_CASE(4, 4, 4) LF2_TBC_CASE(4, 4, 8)
#undef LF2_TBC_CASE
            default: return cudaErrorNotSupported;
        }
    }
    return cudaErrorNotSupported;
}

template <typename R, int NC, int MODE, int T, int CX, typename CoefT>
cudaError_t launch_ens_t(const TbEnsembleLaunch &e, cudaStream_t s) {
    constexpr int TP = ((T + CX - 1) / CX) * CX;
    const int RX = e.c.tile_x + 2 * TP, RY = e.c.tile_y + 2 * T;
    const int threads = (RX / CX) * RY;
    const size_t smem = (size_t)2 * T * (RY + 2) * RX * NC * sizeof(R);
    auto kern = k_tblock_ensemble<R, NC, MODE, T, CX, CoefT>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (per_sm > 0 ? per_sm : 1) * sms;
    if (grid > e.nitems) grid = e.nitems;
    if (grid < 1) return cudaSuccess;
    err = cudaMemsetAsync(e.counter, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    kern<<<grid, threads, smem, s>>>(e.members, e.items, e.nitems, e.flip, e.c.tile_x, e.c.tile_y, e.counter);
    return cudaGetLastError();
}


// Launches a depth-T pass (single lattice) or an ensemble pass for one storage type and mode;
// each precision's instantiations live in their own translation unit.
template <typename R, int NC, int MODE, typename CoefT>
cudaError_t launch_prec(const TbArgs &a, const TbConfig &c, const CoefT &k, cudaStream_t s) {
    if (c.cluster > 1) return launch_cluster_prec<R, NC, MODE, CoefT>(a, c, k, s);
    if constexpr (NC >= 3) {
        // 3 to 6 components: one column per thread; the per-column state grows with NC, so
        // 6 components run at depth 2 only (within the 128 registers of a 512-thread block)
        if (c.cx != 1) return cudaErrorNotSupported;
        switch (c.depth) {
            case 2: return launch_t<R, NC, MODE, 2, 1, CoefT>(a, c, k, s);
            case 3:
                if constexpr (NC <= 4) return launch_t<R, NC, MODE, 3, 1, CoefT>(a, c, k, s);
                return cudaErrorNotSupported;
            case 4:
                if constexpr (NC <= 4) return launch_t<R, NC, MODE, 4, 1, CoefT>(a, c, k, s);
                return cudaErrorNotSupported;
            default: return cudaErrorNotSupported;
        }
    } else {
        switch (c.cx * 16 + c.depth) {
#define LF2_TB_CASE(CXV, TV)                                                                      \
        case CXV * 16 + TV:                                                                           \
            if constexpr (CXV * NC * sizeof(R) <= 16) return launch_t<R, NC, MODE, TV, CXV, CoefT>(a, c, k, s); \
            return cudaErrorNotSupported;
            LF2_TB_CASE(1, 2) LF2_TB_CASE(1, 3) LF2_TB_CASE(1, 4) LF2_TB_CASE(1, 6) LF2_TB_CASE(1, 8)
            LF2_TB_CASE(2, 2) LF2_TB_CASE(2, 3) LF2_TB_CASE(2, 4) LF2_TB_CASE(2, 6) LF2_TB_CASE(2, 8)
            LF2_TB_CASE(4, 2) LF2_TB_CASE(4, 3) LF2_TB_CASE(4, 4) LF2_TB_CASE(4, 6) LF2_TB_CASE(4, 8)
#undef LF2_TB_CASE
            default: return cudaErrorNotSupported;
        }
    }
}

template <typename R, int NC, int MODE, typename CoefT>
cudaError_t launch_ens_prec(const TbEnsembleLaunch &e, cudaStream_t s) {
    if constexpr (NC >= 3) {
        // 3 to 6 components: one column per thread, depth 2 to 4 (2 for 6 components), as for
        // a single lattice
        if (e.c.cx != 1) return cudaErrorNotSupported;
        switch (e.c.depth) {
            case 2: return launch_ens_t<R, NC, MODE, 2, 1, CoefT>(e, s);
            case 3:
                if constexpr (NC <= 4) return launch_ens_t<R, NC, MODE, 3, 1, CoefT>(e, s);
                return cudaErrorNotSupported;
            case 4:
                if constexpr (NC <= 4) return launch_ens_t<R, NC, MODE, 4, 1, CoefT>(e, s);
                return cudaErrorNotSupported;
            default: return cudaErrorNotSupported;
        }
    } else {
        switch (e.c.cx * 16 + e.c.depth) {
#define LF2_TB_CASE(CXV, TV)                                                                          \
            case CXV * 16 + TV:                                                                       \
                if constexpr (CXV * NC * sizeof(R) <= 16) return launch_ens_t<R, NC, MODE, TV, CXV, CoefT>(e, s); \
                return cudaErrorNotSupported;
            LF2_TB_CASE(1, 2) LF2_TB_CASE(1, 3) LF2_TB_CASE(1, 4) LF2_TB_CASE(1, 6) LF2_TB_CASE(1, 8)
            LF2_TB_CASE(2, 2) LF2_TB_CASE(2, 3) LF2_TB_CASE(2, 4) LF2_TB_CASE(2, 6) LF2_TB_CASE(2, 8)
            LF2_TB_CASE(4, 2) LF2_TB_CASE(4, 3) LF2_TB_CASE(4, 4) LF2_TB_CASE(4, 6) LF2_TB_CASE(4, 8)
#undef LF2_TB_CASE
            default: return cudaErrorNotSupported;
        }
    }
}

}  // namespace tb
}  // namespace lf2
