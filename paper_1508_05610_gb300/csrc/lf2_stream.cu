// lf2_stream.cu -- z-streaming leapfrog kernel: one HBM pass per step.
//
// A block owns an x-y tile of the lattice and walks a chunk of z-planes.  Each thread holds
// 16 bytes of a row (4 floats or 2 doubles: S = 16 / (sizeof(R) * ncomp) sites) of three
// consecutive planes in registers (z-1, z, z+1), so the z-neighbours of the 7-point stencil
// cost nothing after the first load.  The current plane is also written to shared memory
// with one halo row above and below the tile, from which the y-neighbours are read; the
// x-neighbours come from the thread's own registers and from the adjacent lanes by warp
// shuffle, with only the two edge lanes of a warp reading one site from global memory.
// Periodic wrap (the torus of Sec. 3.3.1) is index arithmetic on plane, row and column.
//
// Requirements (else the one-thread-per-site kernel runs): rows of 16-byte multiples
// (Nx * ncomp * sizeof(R) % 16 == 0) and Ny a multiple of the tile height.
#include "lf2_bounds.cuh"
#include "lf2_internal.cuh"

namespace lf2 {
namespace {

template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
};
template <>
struct Vec16<double> {
    using T = double2;
};

// NV consecutive 16-byte vectors (E = NV * 16 / sizeof(R) elements).
template <typename R, int E>
__device__ __forceinline__ void ld16(const R *__restrict__ p, R (&v)[E]) {
    using VT = typename Vec16<R>::T;
#pragma unroll
    for (int q = 0; q < (int)(E * sizeof(R) / 16); ++q) {
        VT t = __ldg(reinterpret_cast<const VT *>(p) + q);
        memcpy(&v[q * (16 / sizeof(R))], &t, 16);
    }
}

template <typename R, int E>
__device__ __forceinline__ void ldcg16(const R *__restrict__ p, R (&v)[E]) {
    using VT = typename Vec16<R>::T;
#pragma unroll
    for (int q = 0; q < (int)(E * sizeof(R) / 16); ++q) {
        VT t = __ldcg(reinterpret_cast<const VT *>(p) + q);
        memcpy(&v[q * (16 / sizeof(R))], &t, 16);
    }
}

template <typename R, int E>
__device__ __forceinline__ void st16(R *__restrict__ p, const R (&v)[E]) {
    using VT = typename Vec16<R>::T;
#pragma unroll
    for (int q = 0; q < (int)(E * sizeof(R) / 16); ++q) {
        VT t;
        memcpy(&t, &v[q * (16 / sizeof(R))], 16);
        reinterpret_cast<VT *>(p)[q] = t;
    }
}

template <typename R>
__device__ __forceinline__ R shfl_up1(R v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename R>
__device__ __forceinline__ R shfl_dn1(R v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// NV 16-byte vectors per thread and plane: 1 for one or two components; 3 for 3 or 6
// components (and 2 for 4 FP64 components), so each thread holds whole sites.
template <typename R, int NC>
__host__ __device__ constexpr int stream_nv() {
    return (16 / (int)sizeof(R)) % NC == 0 ? 1 : ((32 / (int)sizeof(R)) % NC == 0 ? 2 : 3);
}

// MODE: 0 = FP32 plain drift, 1 = FP32 Kahan drift, 3 = FP64.
template <typename R, int NC, int MODE, int BY, typename CoefT>
__global__ void __launch_bounds__(32 * BY) k_stream(const R *__restrict__ phi, R *__restrict__ phi_out,
                                                    R *__restrict__ pi, float *__restrict__ comp, Geom g, CoefT k,
                                                    int zchunk) {
    constexpr int NV = stream_nv<R, NC>();
    constexpr int E = NV * 16 / sizeof(R);  // elements per thread
    constexpr int S = E / NC;               // sites per thread
    static_assert(E % NC == 0, "whole sites per thread");
    using VT = typename Vec16<R>::T;
    __shared__ VT sm[2][BY + 2][32 * NV];

    const int lane = threadIdx.x, ty = threadIdx.y;
    const int xs = (blockIdx.x * 32 + lane) * S;  // first site of this thread
    const bool active = xs < g.nx;
    const bool right_in_warp = (lane < 31) && (xs + S < g.nx);
    const int y = blockIdx.y * BY + ty;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const long long rowE = (long long)g.nx * NC;
    const long long planeE = rowE * g.ny;
    const long long col = (long long)xs * NC;
    const long long off_y = (long long)y * rowE + col;
    // halo rows of the tile: the row below (thread row 0) and above (last thread row)
    int yh = -1, hslot = 0;
    if (ty == 0) {
        yh = wrap_dn(blockIdx.y * BY, g.ny);
        hslot = 0;
    } else if (ty == BY - 1) {
        yh = wrap_up(y, g.ny);
        hslot = BY + 1;
    }
    const long long off_h = (long long)yh * rowE + col;
    // edge sites reached outside the warp
    const int xl = wrap_dn(xs, g.nx);
    const int xr = wrap_up(xs + S - 1, g.nx);
    const long long off_l = (long long)y * rowE + (long long)xl * NC;
    const long long off_r = (long long)y * rowE + (long long)xr * NC;

    const long long cnt = (long long)g.sites * NC;  // elements of every field buffer
    R below[E], cur[E], above[E];
#pragma unroll
    for (int e = 0; e < E; ++e) below[e] = cur[e] = above[e] = R(0);
    if (active) {
        ld16<R, E>(phi + checked((long long)wrap_dn(z0, g.nz) * planeE + off_y, E, cnt), below);
        ld16<R, E>(phi + checked((long long)z0 * planeE + off_y, E, cnt), cur);
    }

    for (int z = z0; z < z1; ++z) {
        const long long pz = (long long)z * planeE;
        R halo[E], pv[E], cv[E], lft[NC], rgt[NC];
        if (active) {
            ld16<R, E>(phi + checked((long long)wrap_up(z, g.nz) * planeE + off_y, E, cnt), above);
            if (yh >= 0) ld16<R, E>(phi + checked(pz + off_h, E, cnt), halo);
            const long long oy = checked(pz + off_y, E, cnt);
            ldcg16<R, E>(pi + oy, pv);
            if (MODE == 1) ldcg16<R, E>(reinterpret_cast<const R *>(comp) + oy, cv);
            if (lane == 0) {
                const long long ol = checked(pz + off_l, NC, cnt);
#pragma unroll
                for (int a = 0; a < NC; ++a) lft[a] = __ldg(phi + ol + a);
            }
            if (!right_in_warp) {
                const long long orr = checked(pz + off_r, NC, cnt);
#pragma unroll
                for (int a = 0; a < NC; ++a) rgt[a] = __ldg(phi + orr + a);
            }
        }
        const int buf = (z - z0) & 1;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            VT t;
            memcpy(&t, &cur[q * (16 / sizeof(R))], 16);
            sm[buf][ty + 1][lane * NV + q] = t;
            if (yh >= 0) {
                memcpy(&t, &halo[q * (16 / sizeof(R))], 16);
                sm[buf][hslot][lane * NV + q] = t;
            }
        }
        // x-neighbours across lanes
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const R fromleft = shfl_up1(cur[(S - 1) * NC + a]);
            const R fromright = shfl_dn1(cur[a]);
            if (lane > 0) lft[a] = fromleft;
            if (right_in_warp) rgt[a] = fromright;
        }
        __syncthreads();
        R ymv[E], ypv[E];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            VT t = sm[buf][ty][lane * NV + q];
            memcpy(&ymv[q * (16 / sizeof(R))], &t, 16);
            t = sm[buf][ty + 2][lane * NV + q];
            memcpy(&ypv[q * (16 / sizeof(R))], &t, 16);
        }
        if (active) {
            R outv[E];
#pragma unroll
            for (int j = 0; j < S; ++j) {
                R c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], o[NC];
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    c[a] = cur[e];
                    xm[a] = (j == 0) ? lft[a] : cur[e - NC];
                    xp[a] = (j == S - 1) ? rgt[a] : cur[e + NC];
                    ym[a] = ymv[e];
                    yp[a] = ypv[e];
                    zm[a] = below[e];
                    zp[a] = above[e];
                    p[a] = pv[e];
                    cm[a] = (MODE == 1) ? (float)cv[e] : 0.0f;
                }
                if constexpr (MODE == 3) {
                    update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, o, k);
                } else {
                    update_f32<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, o, k);
                }
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const int e = j * NC + a;
                    outv[e] = o[a];
                    pv[e] = p[a];
                    if (MODE == 1) cv[e] = cm[a];
                }
            }
            const long long oy = checked(pz + off_y, E, cnt);
            st16<R, E>(phi_out + oy, outv);
            st16<R, E>(pi + oy, pv);
            if (MODE == 1) st16<R, E>(reinterpret_cast<R *>(comp) + oy, cv);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            below[e] = cur[e];
            cur[e] = above[e];
        }
    }
}

constexpr int kDefaultBY = 4;

template <typename R, int NC, int MODE, int BY, typename CoefT>
cudaError_t launch_t(const StepArgs &a, int zchunk, const CoefT &k, cudaStream_t s) {
    constexpr int S = stream_nv<R, NC>() * 16 / (int)sizeof(R) / NC;
    dim3 block(32, BY);
    dim3 grid((a.g.nx + 32 * S - 1) / (32 * S), a.g.ny / BY, (a.g.nz + zchunk - 1) / zchunk);
    k_stream<R, NC, MODE, BY, CoefT><<<grid, block, 0, s>>>((const R *)a.phi, (R *)a.phi_out, (R *)a.pi, a.comp, a.g,
                                                             k, zchunk);
    return cudaGetLastError();
}

template <typename R, int MODE, int BY, typename CoefT>
cudaError_t launch_nc(const StepArgs &a, int zchunk, const CoefT &k, cudaStream_t s) {
    switch (a.ncomp) {
        case 1: return launch_t<R, 1, MODE, BY>(a, zchunk, k, s);
        case 2: return launch_t<R, 2, MODE, BY>(a, zchunk, k, s);
        case 3: return launch_t<R, 3, MODE, BY>(a, zchunk, k, s);
        case 4: return launch_t<R, 4, MODE, BY>(a, zchunk, k, s);
        case 6: return launch_t<R, 6, MODE, BY>(a, zchunk, k, s);
        default: return cudaErrorNotSupported;
    }
}

template <int BY>
cudaError_t launch_by(const StepArgs &a, int zchunk, cudaStream_t s) {
    if (a.prec == LF2_F64) return launch_nc<double, 3, BY>(a, zchunk, make_coef64(a.p, a.dt), s);
    const Coef32 k = make_coef32(a.p, a.dt);
    if (a.prec == LF2_F32_KAHAN) return launch_nc<float, 1, BY>(a, zchunk, k, s);
    return launch_nc<float, 0, BY>(a, zchunk, k, s);
}

// sites per thread of the streaming kernel for this precision and component count
int sites_per_thread(int esz, int ncomp) {
    const int e1 = 16 / esz;
    const int nv = e1 % ncomp == 0 ? 1 : ((2 * e1) % ncomp == 0 ? 2 : 3);
    return nv * e1 / ncomp;
}

int default_zchunk(const StepArgs &a, int by) {
    // Short chunks give many blocks, so the last partial wave of blocks (the tail) is a small
    // share of the launch; each chunk re-reads only two extra planes, mostly from L2.
    // Measured on the 256^3 complex and 1024^3 real lattices: 4 planes for FP64, 8 for FP32.
    (void)by;
    const int zc = a.prec == LF2_F64 ? 4 : 8;
    return zc < a.g.nz ? zc : a.g.nz;
}

}  // namespace

cudaError_t bounds_violations_stream(unsigned long long *n, bool reset) { return bounds_violations_here(n, reset); }

bool stream_supported(const StepArgs &a, int tile_y, int zchunk) {
    const int by = tile_y ? tile_y : kDefaultBY;
    if (by != 2 && by != 4 && by != 8 && by != 16) return false;
    if (a.ncomp == 5 || a.ncomp > 6) return false;
    const int esz = a.prec == LF2_F64 ? 8 : 4;
    if (((long long)a.g.nx * a.ncomp * esz) % 16) return false;
    if (a.g.nx % sites_per_thread(esz, a.ncomp)) return false;  // whole thread chunks per row
    if (a.g.ny % by) return false;
    if (zchunk < 0) return false;
    if (!a.drift) return false;
    // 16-byte alignment of every buffer
    if (((uintptr_t)a.phi | (uintptr_t)a.phi_out | (uintptr_t)a.pi | (uintptr_t)a.comp) % 16) return false;
    return true;
}

cudaError_t launch_stream_step(const StepArgs &a, int tile_y, int zchunk, int, cudaStream_t s) {
    if (a.g.sites == 0) return cudaSuccess;
    const int by = tile_y ? tile_y : kDefaultBY;
    const int zc = zchunk > 0 ? zchunk : default_zchunk(a, by);
    switch (by) {
        case 2: return launch_by<2>(a, zc, s);
        case 4: return launch_by<4>(a, zc, s);
        case 8: return launch_by<8>(a, zc, s);
        default: return launch_by<16>(a, zc, s);
    }
}

}  // namespace lf2
