// lf2_spectrum.cu -- binned power spectrum of one field component, or of all components
// summed (a diagnostic; the paper's PlanFFT role, Sec. 3.6, for cubic lattices as there).
//
// P(k) = |phi~(k)|^2 / V with phi~(k) = sum_x phi(x) exp(-i k.x), k_i = 2 pi m_i / (N dx).
// Mode (m_x, m_y, m_z) goes to shell b = floor(sqrt(m_x^2 + m_y^2 + m_z^2)), an exact integer
// square root, so the shell of every mode is the same whatever the rounding of |k|.  The
// transform is cuFFT's real-to-complex FFT (a library call); the half spectrum it returns
// stands for each mode k != -k twice.  The binning kernel accumulates (power, |k|, count) per
// shell in a per-block shared histogram, writes one row per block, and a second kernel sums
// the rows in a fixed order.  Shared-memory accumulation order varies between runs, so results
// are reproducible to FP64 rounding, not bitwise.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>

#include "lf2_handles.h"

using namespace lf2;

namespace {

constexpr int kBinThreads = 256;
constexpr int kMaxBins = 1024;

template <typename R>
__global__ void k_extract(const R *__restrict__ f, R *__restrict__ out, long long sites, int ncomp, int comp) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < sites; s += (long long)gridDim.x * blockDim.x)
        out[s] = f[s * ncomp + comp];
}

__device__ __forceinline__ int isqrt_exact(long long s) {
    long long b = (long long)sqrt((double)s);
    while (b * b > s) --b;
    while ((b + 1) * (b + 1) <= s) ++b;
    return (int)b;
}

// add_power: add this component's power to the rows a previous component's binning wrote,
// leaving the |k| sums and mode counts (the same for every component) as they are.
template <typename C>
__global__ void __launch_bounds__(kBinThreads) k_bin(const C *__restrict__ spec, int n, int nbins, double kunit,
                                                     double inv_volume, double *__restrict__ partials, int add_power) {
    extern __shared__ double hist[];  // 3 * nbins: power, |k| sum, count
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) hist[i] = 0.0;
    __syncthreads();
    const int hx = n / 2 + 1;
    const long long total = (long long)n * n * hx;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(e % hx);
        const long long r = e / hx;
        const int ky = (int)(r % n);
        const int kz = (int)(r / n);
        const int mx = kx, my = ky <= n / 2 ? ky : ky - n, mz = kz <= n / 2 ? kz : kz - n;
        const long long s2 = (long long)mx * mx + (long long)my * my + (long long)mz * mz;
        const int b = isqrt_exact(s2);
        if (b >= nbins) continue;
        const double w = (kx == 0 || (n % 2 == 0 && kx == n / 2)) ? 1.0 : 2.0;
        const double re = (double)spec[e].x, im = (double)spec[e].y;
        atomicAdd(&hist[b], w * (re * re + im * im) * inv_volume);
        atomicAdd(&hist[nbins + b], w * kunit * sqrt((double)s2));
        atomicAdd(&hist[2 * nbins + b], w);
    }
    __syncthreads();
    double *row = partials + (size_t)blockIdx.x * 3 * nbins;
    if (add_power) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) row[i] += hist[i];
    } else {
        for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) row[i] = hist[i];
    }
}

__global__ void k_bin_final(const double *__restrict__ partials, int nblocks, int nbins, double *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nbins; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * 3 * nbins + i];
        out[i] = s;
    }
}

}  // namespace

extern "C" lf2_status lf2_power_spectrum(lf2_field f, int comp, int nbins, double dx, double *power, double *kmean,
                                         double *count, void *stream) {
    if (!f || !power || !kmean || !count) return set_error(LF2_ERR_INVALID, "NULL argument");
    const int *n3 = f->lat->n;
    if (n3[0] != n3[1] || n3[1] != n3[2])
        return set_error(LF2_ERR_UNSUPPORTED, "the power spectrum needs a cubic lattice (as the paper's FFT)");
    if (comp < -1 || comp >= f->ncomp) return set_error(LF2_ERR_INVALID, "component %d out of range", comp);
    if (nbins < 1 || nbins > kMaxBins) return set_error(LF2_ERR_INVALID, "nbins must be 1 to %d", kMaxBins);
    if (!(dx > 0.0)) return set_error(LF2_ERR_INVALID, "dx must be > 0");
    const int n = n3[0];
    const long long sites = f->lat->sites;
    const bool dbl = f->prec == LF2_F64;
    const size_t rsz = dbl ? sizeof(double) : sizeof(float);
    const size_t csz = 2 * rsz;
    cudaStream_t s = (cudaStream_t)stream;
    void *real = nullptr, *spec = nullptr;
    double *partials = nullptr, *out = nullptr;
    cufftHandle plan = 0;
    bool have_plan = false;
    lf2_status st = LF2_OK;
    const int kBinBlocks = 2 * device_sm_count();  // two histogram blocks per SM
    cudaError_t e = cudaMalloc(&real, (size_t)sites * rsz);
    if (e == cudaSuccess) e = cudaMalloc(&spec, (size_t)n * n * (n / 2 + 1) * csz);
    if (e == cudaSuccess) e = cudaMalloc(&partials, (size_t)kBinBlocks * 3 * nbins * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)3 * nbins * sizeof(double));
    if (e != cudaSuccess) st = cuda_error(e, "spectrum buffers");
    if (st == LF2_OK) {
        cufftResult r = cufftPlan3d(&plan, n, n, n, dbl ? CUFFT_D2Z : CUFFT_R2C);
        have_plan = r == CUFFT_SUCCESS;
        if (r == CUFFT_SUCCESS) r = cufftSetStream(plan, s);
        if (r != CUFFT_SUCCESS) st = set_error(r == CUFFT_ALLOC_FAILED ? LF2_ERR_NOMEM : LF2_ERR_CUDA, "cuFFT error %d", (int)r);
    }
    // one component, or every component in order with their powers added bin by bin
    const int c0 = comp < 0 ? 0 : comp, c1 = comp < 0 ? f->ncomp : comp + 1;
    const double kunit = 2.0 * M_PI / (n * dx);
    const double inv_volume = 1.0 / ((double)n * n * n);
    const size_t smem = (size_t)3 * nbins * sizeof(double);
    for (int c = c0; c < c1 && st == LF2_OK; ++c) {
        const long long cap = 16LL * device_sm_count();
        const int g = (int)((sites + 255) / 256 < cap ? (sites + 255) / 256 : cap);
        if (dbl)
            k_extract<double><<<g, 256, 0, s>>>((const double *)f->val[f->front], (double *)real, sites, f->ncomp, c);
        else
            k_extract<float><<<g, 256, 0, s>>>((const float *)f->val[f->front], (float *)real, sites, f->ncomp, c);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            st = cuda_error(e, "component copy");
            break;
        }
        const cufftResult r = dbl ? cufftExecD2Z(plan, (cufftDoubleReal *)real, (cufftDoubleComplex *)spec)
                                  : cufftExecR2C(plan, (cufftReal *)real, (cufftComplex *)spec);
        if (r != CUFFT_SUCCESS) {
            st = set_error(LF2_ERR_CUDA, "cuFFT error %d", (int)r);
            break;
        }
        const int add = c > c0;
        if (dbl)
            k_bin<double2><<<kBinBlocks, kBinThreads, smem, s>>>((const double2 *)spec, n, nbins, kunit, inv_volume, partials,
                                                                 add);
        else
            k_bin<float2><<<kBinBlocks, kBinThreads, smem, s>>>((const float2 *)spec, n, nbins, kunit, inv_volume, partials,
                                                                add);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_error(e, "binning");
    }
    if (st == LF2_OK) {
        k_bin_final<<<(3 * nbins + 255) / 256, 256, 0, s>>>(partials, kBinBlocks, nbins, out);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(power, out, nbins * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(kmean, out + nbins, nbins * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(count, out + 2 * nbins, nbins * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "binning");
    }
    if (have_plan) cufftDestroy(plan);
    if (real) cudaFree(real);
    if (spec) cudaFree(spec);
    if (partials) cudaFree(partials);
    if (out) cudaFree(out);
    if (st != LF2_OK) return st;
    for (int b = 0; b < nbins; ++b) {  // sums -> means
        if (count[b] > 0) {
            power[b] /= count[b];
            kmean[b] /= count[b];
        }
    }
    return LF2_OK;
}
