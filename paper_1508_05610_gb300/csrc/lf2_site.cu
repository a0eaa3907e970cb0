// lf2_site.cu -- one thread per site: the shape-agnostic leapfrog kernel (any Nx, Ny, Nz),
// plus the precision conversions used by upload/download.
//
// Each thread owns one site (x, y, z) of the row-major lattice and reads its six periodic
// neighbours x+-i (the Site jumps of Sec. 3.4 with the torus wrap of Sec. 3.3.1 done by
// index arithmetic instead of a stored halo).
#include "lf2_internal.cuh"

namespace lf2 {
namespace {

constexpr int kThreads = 256;

template <typename R, int NC>
__device__ __forceinline__ void load_site(const R *__restrict__ f, long long s, R (&v)[NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a) v[a] = __ldg(f + s * NC + a);
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
        load_site<double, NC>(phi, s, c);
        load_site<double, NC>(phi, s - x + wrap_dn(x, g.nx), xm);
        load_site<double, NC>(phi, s - x + wrap_up(x, g.nx), xp);
        load_site<double, NC>(phi, s + (wrap_dn(y, g.ny) - y) * row, ym);
        load_site<double, NC>(phi, s + (wrap_up(y, g.ny) - y) * row, yp);
        load_site<double, NC>(phi, s + (wrap_dn(z, g.nz) - z) * plane, zm);
        load_site<double, NC>(phi, s + (wrap_up(z, g.nz) - z) * plane, zp);
#pragma unroll
        for (int a = 0; a < NC; ++a) p[a] = pi[s * NC + a];
        update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, out, k);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            pi[s * NC + a] = p[a];
            if (drift) phi_out[s * NC + a] = out[a];
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
        load_site<float, NC>(phi, s, c);
        load_site<float, NC>(phi, s - x + wrap_dn(x, g.nx), xm);
        load_site<float, NC>(phi, s - x + wrap_up(x, g.nx), xp);
        load_site<float, NC>(phi, s + (wrap_dn(y, g.ny) - y) * row, ym);
        load_site<float, NC>(phi, s + (wrap_up(y, g.ny) - y) * row, yp);
        load_site<float, NC>(phi, s + (wrap_dn(z, g.nz) - z) * plane, zm);
        load_site<float, NC>(phi, s + (wrap_up(z, g.nz) - z) * plane, zp);
#pragma unroll
        for (int a = 0; a < NC; ++a) p[a] = pi[s * NC + a];
        if (MODE == 2) {
            kick_f32<NC>(c, xm, xp, ym, yp, zm, zp, p, k);
#pragma unroll
            for (int a = 0; a < NC; ++a) pi[s * NC + a] = p[a];
            continue;
        }
#pragma unroll
        for (int a = 0; a < NC; ++a) cm[a] = (MODE == 1) ? comp[s * NC + a] : 0.0f;
        update_f32<NC, MODE == 1>(c, xm, xp, ym, yp, zm, zp, p, cm, out, k);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            pi[s * NC + a] = p[a];
            phi_out[s * NC + a] = out[a];
            if (MODE == 1) comp[s * NC + a] = cm[a];
        }
    }
}

int grid_for(long long sites) {
    long long b = (sites + kThreads - 1) / kThreads;
    const long long cap = 152LL * 16;
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

cudaError_t launch_site_step(const StepArgs &a, cudaStream_t s) {
    if (a.g.sites == 0) return cudaSuccess;
    const int grid = grid_for(a.g.sites);
    if (a.prec == LF2_F64) {
        const Coef64 k = make_coef64(a.p, a.dt);
        const double *phi = (const double *)a.phi;
        double *out = (double *)a.phi_out, *pi = (double *)a.pi;
        if (a.ncomp == 1)
            k_site_f64<1><<<grid, kThreads, 0, s>>>(phi, out, pi, a.g, k, a.drift ? 1 : 0);
        else
            k_site_f64<2><<<grid, kThreads, 0, s>>>(phi, out, pi, a.g, k, a.drift ? 1 : 0);
    } else {
        const Coef32 k = make_coef32(a.p, a.dt);
        const float *phi = (const float *)a.phi;
        float *out = (float *)a.phi_out, *pi = (float *)a.pi;
        const int mode = !a.drift ? 2 : (a.prec == LF2_F32_KAHAN ? 1 : 0);
#define LF2_SITE_F32(NC, M) k_site_f32<NC, M><<<grid, kThreads, 0, s>>>(phi, out, pi, a.comp, a.g, k)
        if (a.ncomp == 1) {
            if (mode == 0) LF2_SITE_F32(1, 0);
            else if (mode == 1) LF2_SITE_F32(1, 1);
            else LF2_SITE_F32(1, 2);
        } else {
            if (mode == 0) LF2_SITE_F32(2, 0);
            else if (mode == 1) LF2_SITE_F32(2, 1);
            else LF2_SITE_F32(2, 2);
        }
#undef LF2_SITE_F32
    }
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

}  // namespace lf2
