// lf2_energy.cu -- FP64 energy and checksum reduction (all precisions).
//
// Energy at integer step n from phi_n and pi_{n-1/2}:
//   pi_n       = pi_{n-1/2} + (dt/2) F(phi_n)          (synchronised momentum)
//   kinetic    = sum_x 1/2 sum_a pi_{a,n}^2
//   gradient   = sum_x sum_a sum_i (phi_a(x+i) - phi_a(x))^2 / (2 dx^2)
//                (forward differences: the discrete gradient energy whose variation is the
//                 7-point Laplacian built from the Site neighbours x+i, x-i of Sec. 3.4)
//   potential  = sum_x [lambda/4 (|phi|^2 - eta^2)^2 + m2/2 |phi|^2]
// plus sum_x phi_a and sum_x phi_a^2.  The dx^3 volume element is applied by the caller.
//
// Two passes with a fixed reduction order, so the result is bitwise reproducible: a
// grid-stride pass over sites leaves one partial row per block (at most kEnergyBlocks rows of
// kEnergySlots doubles, one block per 1024 sites), then one block sums the rows.  The scratch array lives in
// global memory owned by the caller of launch_energy.
#include <mutex>

#include "lf2_internal.cuh"

namespace lf2 {
namespace {

constexpr int kSlots = kEnergySlots;

template <typename R, int NC>
__device__ __forceinline__ void load_d(const R *__restrict__ f, long long s, double (&v)[NC]) {
#pragma unroll
    for (int a = 0; a < NC; ++a) v[a] = (double)__ldg(f + s * NC + a);
}

__device__ __forceinline__ void block_reduce_store(double (&acc)[kSlots], double *__restrict__ dst) {
    __shared__ double sh[kSlots][kEnergyThreads];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int j = 0; j < kSlots; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < kSlots) dst[threadIdx.x] = sh[threadIdx.x][0];
}

template <typename R, int NC>
__global__ void __launch_bounds__(kEnergyThreads) k_energy(const R *__restrict__ phi, const R *__restrict__ pi, Geom g,
                                                           CoefE k, double *__restrict__ partials) {
    double acc[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) acc[j] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long row = g.nx, plane = (long long)g.nx * g.ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride) {
        const int x = (int)(s % g.nx);
        const long long r = s / g.nx;
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        double c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC];
        load_d<R, NC>(phi, s, c);
        load_d<R, NC>(phi, s - x + wrap_dn(x, g.nx), xm);
        load_d<R, NC>(phi, s - x + wrap_up(x, g.nx), xp);
        load_d<R, NC>(phi, s + (wrap_dn(y, g.ny) - y) * row, ym);
        load_d<R, NC>(phi, s + (wrap_up(y, g.ny) - y) * row, yp);
        load_d<R, NC>(phi, s + (wrap_dn(z, g.nz) - z) * plane, zm);
        load_d<R, NC>(phi, s + (wrap_up(z, g.nz) - z) * plane, zp);
        load_d<R, NC>(pi, s, p);
        double s2 = 0.0;
#pragma unroll
        for (int a = 0; a < NC; ++a) s2 += c[a] * c[a];
        const double w = s2 - k.eta2;
        const double gpot = k.lam * w + k.m2;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const double nb = ((xm[a] + xp[a]) + (ym[a] + yp[a])) + (zm[a] + zp[a]);
            const double F = (nb - 6.0 * c[a]) * k.inv_dx2 - gpot * c[a];
            const double pin = p[a] + k.half_dt * F;
            acc[0] += 0.5 * pin * pin;
            const double ex = xp[a] - c[a], ey = yp[a] - c[a], ez = zp[a] - c[a];
            acc[1] += 0.5 * k.inv_dx2 * ((ex * ex + ey * ey) + ez * ez);
            acc[3 + a] += c[a];
            acc[3 + kMaxComp + a] += c[a] * c[a];
        }
        acc[2] += 0.25 * k.lam * w * w + 0.5 * k.m2 * s2;
    }
    block_reduce_store(acc, partials + (size_t)blockIdx.x * kSlots);
}

__global__ void __launch_bounds__(kEnergyThreads) k_energy_final(const double *__restrict__ partials, int nblocks,
                                                                 double *__restrict__ result) {
    double acc[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) acc[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < kSlots; ++j) acc[j] += partials[(size_t)b * kSlots + j];
    }
    block_reduce_store(acc, result);
}

template <typename R>
cudaError_t launch_typed(const void *phi, const void *pi, const Geom &g, int ncomp, const CoefE &k, double *partials,
                         double *result, cudaStream_t s) {
    // One block per 1024 sites up to the fixed maximum: small lattices (the 32^3 run with an
    // energy every step) reduce in few blocks; the grid depends only on the lattice, so the
    // result is bitwise reproducible for a given lattice.
    long long want = (g.sites + 1023) / 1024;
    const int nb = (int)(want < 1 ? 1 : (want > kEnergyBlocks ? kEnergyBlocks : want));
    switch (ncomp) {
#define LF2_E(NC) \
    case NC: k_energy<R, NC><<<nb, kEnergyThreads, 0, s>>>((const R *)phi, (const R *)pi, g, k, partials); break;
        LF2_E(1) LF2_E(2) LF2_E(3) LF2_E(4) LF2_E(5) LF2_E(6)
#undef LF2_E
        default: return cudaErrorInvalidValue;
    }
    k_energy_final<<<1, kEnergyThreads, 0, s>>>(partials, nb, result);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_energy(const void *phi, const void *pi, const Geom &g, int ncomp, lf2_precision prec,
                          const lf2_params &p, double *partials, double *result, cudaStream_t s) {
    const CoefE k = make_coefE(p);
    if (prec == LF2_F64) return launch_typed<double>(phi, pi, g, ncomp, k, partials, result, s);
    return launch_typed<float>(phi, pi, g, ncomp, k, partials, result, s);
}

// ------------------------------------------------------ device-side energy record
// Turns the raw result row into an lf2_energy_t-shaped record in device memory: kinetic,
// gradient, potential (times dx^3), total, sum[kMaxComp], sum_sq[kMaxComp].
__global__ void k_energy_record(const double *__restrict__ r, double vol, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    out[0] = vol * r[0];
    out[1] = vol * r[1];
    out[2] = vol * r[2];
    out[3] = out[0] + out[1] + out[2];
    for (int a = 0; a < kMaxComp; ++a) {
        out[4 + a] = r[3 + a];
        out[4 + kMaxComp + a] = r[3 + kMaxComp + a];
    }
}

cudaError_t launch_energy_record(const double *result, double vol, double *out, cudaStream_t s) {
    k_energy_record<<<1, 32, 0, s>>>(result, vol, out);
    return cudaGetLastError();
}

// ------------------------------------------------- fixed scratch for lf2_energy_noalloc
// Some callers cannot allocate device memory: code that runs while a memory pool or another
// framework owns the device allocator, or that must not make allocation calls at all.
// lf2_energy allocates its partial-sum scratch on first use; lf2_energy_noalloc uses this
// file-scope array instead.  Every GPU that loads the library holds it until process exit.
// It holds the per-block partials of the reduction's grid plus one result row; the grid has at
// most kEnergyBlocks blocks whatever the lattice, so the capacity is a constant.
static __device__ __align__(256) double g_energy_noalloc[kEnergyNoallocDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// The device address of g_energy_noalloc on the current device.  The first call on a device
// asks the runtime for it (host code cannot use the array's name as a device address) and
// caches it; later calls only read the cache.
cudaError_t energy_noalloc_scratch(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_energy_noalloc);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<double *>(addr);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace lf2
