// lf2_site.cu -- one thread per site: the shape-agnostic leapfrog kernel (any Nx, Ny, Nz),
// plus the precision conversions used by upload/download.
//
// Each thread owns one site (x, y, z) of the row-major lattice and reads its six periodic
// neighbours x+-i (the Site jumps of Sec. 3.4 with the torus wrap of Sec. 3.3.1 done by
// index arithmetic instead of a stored halo).
#include <atomic>
#include <type_traits>

#include "lf2_bounds.cuh"
#include "lf2_internal.cuh"

namespace lf2 {
namespace {

constexpr int kThreads = 256;

template <typename R, int NC>
__device__ __forceinline__ void load_site(const R *__restrict__ f, long long s, long long sites, R (&v)[NC]) {
    const long long i = checked(s * NC, NC, sites * NC);
#pragma unroll
    for (int a = 0; a < NC; ++a) v[a] = __ldg(f + i + a);
}

template <int NC>
__global__ void __launch_bounds__(kThreads) k_site_f64(const double *__restrict__ phi, double *__restrict__ phi_out,
                                                       double *__restrict__ pi, Geom g, Coef64 k, int drift) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride) {
        const int x = (int)(s % g.nx);
        const long long r = s / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long row = (long long)g.nx;
        const long long plane = row * g.ny;
        double c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], out[NC];
        const long long o = checked(s * NC, NC, g.sites * NC);
        load_site<double, NC>(phi, s, g.sites, c);
        load_site<double, NC>(phi, s - x + wrap_dn(x, g.nx), g.sites, xm);
        load_site<double, NC>(phi, s - x + wrap_up(x, g.nx), g.sites, xp);
        load_site<double, NC>(phi, s + (wrap_dn(y, g.ny) - y) * row, g.sites, ym);
        load_site<double, NC>(phi, s + (wrap_up(y, g.ny) - y) * row, g.sites, yp);
        load_site<double, NC>(phi, s + (wrap_dn(z, g.nz) - z) * plane, g.sites, zm);
        load_site<double, NC>(phi, s + (wrap_up(z, g.nz) - z) * plane, g.sites, zp);
#pragma unroll
        for (int a = 0; a < NC; ++a) p[a] = pi[o + a];
        update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, out, k);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            pi[o + a] = p[a];
            if (drift) phi_out[o + a] = out[a];
        }
    }
}

// MODE 0: plain FP32 drift, 1: Kahan drift, 2: kick only.
template <int NC, int MODE>
__global__ void __launch_bounds__(kThreads) k_site_f32(const float *__restrict__ phi, float *__restrict__ phi_out,
                                                       float *__restrict__ pi, float *__restrict__ comp, Geom g,
                                                       Coef32 k) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride) {
        const int x = (int)(s % g.nx);
        const long long r = s / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long row = (long long)g.nx;
        const long long plane = row * g.ny;
        float c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], out[NC];
        const long long o = checked(s * NC, NC, g.sites * NC);
        load_site<float, NC>(phi, s, g.sites, c);
        load_site<float, NC>(phi, s - x + wrap_dn(x, g.nx), g.sites, xm);
        load_site<float, NC>(phi, s - x + wrap_up(x, g.nx), g.sites, xp);
        load_site<float, NC>(phi, s + (wrap_dn(y, g.ny) - y) * row, g.sites, ym);
        load_site<float, NC>(phi, s + (wrap_up(y, g.ny) - y) * row, g.sites, yp);
        load_site<float, NC>(phi, s + (wrap_dn(z, g.nz) - z) * plane, g.sites, zm);
        load_site<float, NC>(phi, s + (wrap_up(z, g.nz) - z) * plane, g.sites, zp);
#pragma unroll
        for (int a = 0; a < NC; ++a) p[a] = pi[o + a];
        if constexpr (MODE == 2) {
            kick_f32<NC>(c, xm, xp, ym, yp, zm, zp, p, k);
#pragma unroll
            for (int a = 0; a < NC; ++a) pi[o + a] = p[a];
        } else {
#pragma unroll
            for (int a = 0; a < NC; ++a) cm[a] = (MODE == 1) ? comp[o + a] : 0.0f;
            update_f32<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, out, k);
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                pi[o + a] = p[a];
                phi_out[o + a] = out[a];
                if (MODE == 1) comp[o + a] = cm[a];
            }
        }
    }
}

int grid_for(long long sites) {
    long long b = (sites + kThreads - 1) / kThreads;
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

__global__ void k_from_f64_f32(const double *__restrict__ src, float *__restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_f32_to_f64(const float *__restrict__ src, double *__restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

}  // namespace

cudaError_t bounds_violations_site(unsigned long long *n, bool reset) { return bounds_violations_here(n, reset); }

template <int NC>
void site_launch(const StepArgs &a, int grid, cudaStream_t s) {
    if (a.prec == LF2_F64) {
        k_site_f64<NC><<<grid, kThreads, 0, s>>>((const double *)a.phi, (double *)a.phi_out, (double *)a.pi, a.g,
                                                 make_coef64(a.p, a.dt), a.drift ? 1 : 0);
        return;
    }
    const Coef32 k = make_coef32(a.p, a.dt);
    const float *phi = (const float *)a.phi;
    float *out = (float *)a.phi_out, *pi = (float *)a.pi;
    if (!a.drift)
        k_site_f32<NC, 2><<<grid, kThreads, 0, s>>>(phi, out, pi, a.comp, a.g, k);
    else if (a.prec == LF2_F32_KAHAN)
        k_site_f32<NC, 1><<<grid, kThreads, 0, s>>>(phi, out, pi, a.comp, a.g, k);
    else
        k_site_f32<NC, 0><<<grid, kThreads, 0, s>>>(phi, out, pi, a.comp, a.g, k);
}

cudaError_t launch_site_step(const StepArgs &a, cudaStream_t s) {
    if (a.g.sites == 0) return cudaSuccess;
    const int grid = grid_for(a.g.sites);
    switch (a.ncomp) {
        case 1: site_launch<1>(a, grid, s); break;
        case 2: site_launch<2>(a, grid, s); break;
        case 3: site_launch<3>(a, grid, s); break;
        case 4: site_launch<4>(a, grid, s); break;
        case 5: site_launch<5>(a, grid, s); break;
        case 6: site_launch<6>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ symmetric difference
namespace {

template <typename R>
__global__ void __launch_bounds__(kThreads) k_derivative(const R *__restrict__ src, R *__restrict__ dst, Geom g,
                                                         int ncomp, int dim, R inv2dx) {
    // one thread per element (site, component): neighbouring threads read neighbouring
    // elements, so every access is coalesced whatever the dimension
    const long long n = g.sites * ncomp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const long long s = e / ncomp;
        const int a = (int)(e - s * ncomp);
        const int x = (int)(s % g.nx);
        const long long r = s / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        long long up, dn;
        if (dim == 0) {
            up = s - x + wrap_up(x, g.nx);
            dn = s - x + wrap_dn(x, g.nx);
        } else if (dim == 1) {
            up = s + (long long)(wrap_up(y, g.ny) - y) * g.nx;
            dn = s + (long long)(wrap_dn(y, g.ny) - y) * g.nx;
        } else {
            const long long plane = (long long)g.nx * g.ny;
            up = s + (long long)(wrap_up(z, g.nz) - z) * plane;
            dn = s + (long long)(wrap_dn(z, g.nz) - z) * plane;
        }
        dst[e] = (__ldg(src + up * ncomp + a) - __ldg(src + dn * ncomp + a)) * inv2dx;
    }
}

}  // namespace

namespace {

// Row-vectorised symmetric difference for rows made of whole 16-byte vectors.  Blocks are
// (x-chunk, y, z), so there is no division; each lane holds E = 16 / sizeof(R) elements of a
// row.  Along y and z the two neighbours are whole-row vector loads.  Along x (template NC,
// which must divide E) they are within the lane's vector or in the adjacent lane's (warp
// shuffle); the first lane of a warp and the last lane of a row read the wrapped neighbour
// from memory.
template <typename R, int NC>
__global__ void __launch_bounds__(128) k_derivative_rows(const R *__restrict__ src, R *__restrict__ dst, Geom g,
                                                         int dim, R inv2dx) {
    constexpr int E = 16 / sizeof(R);
    static_assert(E % NC == 0, "components must divide the vector");
    using V = typename std::conditional<sizeof(R) == 8, double2, float4>::type;
    const long long rowE = (long long)g.nx * NC;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long e0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * E;
    const bool active = e0 < rowE;
    const long long base = ((long long)z * g.ny + y) * rowE;
    R up[E], dn[E];
    if (dim == 0) {
        R v[E];
        V t{};
        if (active) t = __ldg(reinterpret_cast<const V *>(src + base + e0));
        memcpy(v, &t, 16);
        R left[NC], right[NC];
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            left[a] = __shfl_up_sync(0xffffffffu, v[E - NC + a], 1);
            right[a] = __shfl_down_sync(0xffffffffu, v[a], 1);
        }
        if (active && lane == 0) {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                long long e = e0 - NC + a;
                if (e < 0) e += rowE;
                left[a] = __ldg(src + base + e);
            }
        }
        if (active && (lane == 31 || e0 + E >= rowE)) {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                long long e = e0 + E + a;
                if (e >= rowE) e -= rowE;
                right[a] = __ldg(src + base + e);
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) {
            dn[j] = j < NC ? left[j] : v[j - NC];
            up[j] = j + NC < E ? v[j + NC] : right[j + NC - E];
        }
    } else {
        if (!active) return;
        long long du, dd;
        if (dim == 1) {
            du = (long long)(wrap_up(y, g.ny) - y) * rowE;
            dd = (long long)(wrap_dn(y, g.ny) - y) * rowE;
        } else {
            const long long plane = rowE * g.ny;
            du = (long long)(wrap_up(z, g.nz) - z) * plane;
            dd = (long long)(wrap_dn(z, g.nz) - z) * plane;
        }
        V a = __ldg(reinterpret_cast<const V *>(src + base + du + e0));
        V b = __ldg(reinterpret_cast<const V *>(src + base + dd + e0));
        memcpy(up, &a, 16);
        memcpy(dn, &b, 16);
    }
    if (!active) return;
    R out[E];
#pragma unroll
    for (int j = 0; j < E; ++j) out[j] = (up[j] - dn[j]) * inv2dx;
    V o;
    memcpy(&o, out, 16);
    __stcs(reinterpret_cast<V *>(dst + base + e0), o);
}

template <typename R>
cudaError_t launch_rows(const void *src, void *dst, const Geom &g, int ncomp, int dim, R inv2dx, cudaStream_t s) {
    const long long vecs = (long long)g.nx * ncomp * sizeof(R) / 16;
    dim3 grid((unsigned)((vecs + 127) / 128), g.ny, g.nz);
    // along y and z the component count does not matter (whole rows): use the NC = 1 instance
    const int nc = dim == 0 ? ncomp : 1;
    const Geom gg = dim == 0 ? g : Geom{g.nx * ncomp, g.ny, g.nz, g.sites * ncomp};
    switch (nc) {
        case 1: k_derivative_rows<R, 1><<<grid, 128, 0, s>>>((const R *)src, (R *)dst, gg, dim, inv2dx); break;
        case 2: k_derivative_rows<R, 2><<<grid, 128, 0, s>>>((const R *)src, (R *)dst, gg, dim, inv2dx); break;
        case 4:
            if constexpr (sizeof(R) == 4) {
                k_derivative_rows<R, 4><<<grid, 128, 0, s>>>((const R *)src, (R *)dst, gg, dim, inv2dx);
                break;
            }
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_derivative(const void *src, void *dst, const Geom &g, int ncomp, lf2_precision prec, int dim,
                              double dx, cudaStream_t s) {
    if (g.sites == 0) return cudaSuccess;
    const int esz = prec == LF2_F64 ? 8 : 4;
    const int E = 16 / esz;
    const bool rows_ok = ((long long)g.nx * ncomp * esz) % 16 == 0 && ((uintptr_t)src | (uintptr_t)dst) % 16 == 0 &&
                         g.ny <= 65535 && g.nz <= 65535 && (dim != 0 || (ncomp <= E && E % ncomp == 0));
    if (rows_ok) {
        return prec == LF2_F64 ? launch_rows<double>(src, dst, g, ncomp, dim, 0.5 / dx, s)
                               : launch_rows<float>(src, dst, g, ncomp, dim, (float)(0.5 / dx), s);
    }
    const int grid = grid_for(g.sites * ncomp);
    if (prec == LF2_F64)
        k_derivative<double><<<grid, kThreads, 0, s>>>((const double *)src, (double *)dst, g, ncomp, dim, 0.5 / dx);
    else
        k_derivative<float><<<grid, kThreads, 0, s>>>((const float *)src, (float *)dst, g, ncomp, dim,
                                                      (float)(0.5 / dx));
    return cudaGetLastError();
}

cudaError_t launch_convert_from_f64(const double *src, void *dst, long long n, lf2_precision prec, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == LF2_F64) return cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_from_f64_f32<<<grid_for(n), kThreads, 0, s>>>(src, (float *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_to_f64(const void *src, double *dst, long long n, lf2_precision prec, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == LF2_F64) return cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_f32_to_f64<<<grid_for(n), kThreads, 0, s>>>((const float *)src, dst, n);
    return cudaGetLastError();
}

int device_sm_count() {
    // one entry per device ordinal; concurrent first calls store the same value
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        return 152;
    }
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

}  // namespace lf2
