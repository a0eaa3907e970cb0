// lf2_api.cu -- the C ABI of liblf2: handles, argument checks, status mapping, dispatch.
//
// Lattice and Field follow LATfield2's model (arXiv:1508.05610): Lattice(dim, sizes, h) of
// Sec. 3.2 and Field<T>(lat, comp) of Sec. 3.3, with updateHalo() of Sec. 3.3.1 reduced to a
// check because the kernels read periodic images by wrapped indexing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "lf2_internal.cuh"

using namespace lf2;

#include "lf2_handles.h"

namespace {

thread_local std::string g_last_error;

lf2_status fail(lf2_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
lf2_status fail(lf2_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

lf2_status cuda_fail(cudaError_t e, const char *what) {
    const lf2_status s = (e == cudaErrorMemoryAllocation) ? LF2_ERR_NOMEM : LF2_ERR_CUDA;
    return fail(s, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define LF2_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return cuda_fail(_e, (what));   \
    } while (0)

size_t elem_size(lf2_precision p) { return p == LF2_F64 ? sizeof(double) : sizeof(float); }

bool valid_prec(int p) { return p == LF2_F64 || p == LF2_F32_KAHAN || p == LF2_F32; }


lf2_status check_params(const lf2_params *p) {
    if (!p) return fail(LF2_ERR_INVALID, "params is NULL");
    if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return fail(LF2_ERR_INVALID, "dx must be finite and > 0");
    if (!std::isfinite(p->dt) || !std::isfinite(p->lambda) || !std::isfinite(p->eta) || !std::isfinite(p->m2))
        return fail(LF2_ERR_INVALID, "non-finite parameter");
    return LF2_OK;
}

lf2_status check_pair(lf2_field phi, lf2_field pi) {
    if (!phi || !pi) return fail(LF2_ERR_INVALID, "field handle is NULL");
    if (phi == pi) return fail(LF2_ERR_INVALID, "phi and pi must be different fields");
    if (phi->lat != pi->lat) return fail(LF2_ERR_INVALID, "phi and pi live on different lattices");
    if (phi->ncomp != pi->ncomp) return fail(LF2_ERR_INVALID, "phi and pi have different ncomp");
    if (phi->prec != pi->prec) return fail(LF2_ERR_INVALID, "phi and pi have different precision");
    return LF2_OK;
}

lf2_status new_field(lf2_lattice lat, int ncomp, int prec, lf2_field *out) {
    if (!lat || !out) return fail(LF2_ERR_INVALID, "lattice or output pointer is NULL");
    if (!valid_prec(prec)) return fail(LF2_ERR_INVALID, "unknown precision %d", prec);
    if (ncomp < 1) return fail(LF2_ERR_INVALID, "ncomp must be >= 1");
    if (ncomp > kMaxComp) return fail(LF2_ERR_UNSUPPORTED, "ncomp %d not built (1 to %d)", ncomp, kMaxComp);
    return LF2_OK;
}

}  // namespace

namespace lf2 {
lf2_status set_error(lf2_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}
lf2_status cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

bool fault_injected(const char *what) {
    const char *f = getenv("LF2_FAULT");
    return f && !strcmp(f, what);
}

// LF2_TUNE: "off" -- lf2_leapfrog ignores tuned plans; "force" -- it tunes a shape without a
// plan on first use; unset or anything else -- it uses a plan once lf2_tune made one.
TuneMode tune_mode() {
    const char *t = getenv("LF2_TUNE");
    if (t && !strcmp(t, "off")) return TuneMode::Off;
    if (t && !strcmp(t, "force")) return TuneMode::Force;
    return TuneMode::On;
}

lf2_status alloc_back(lf2_field f, const char *what) {
    if (f->val[1 - f->front]) return LF2_OK;
    if (fault_injected("alloc")) return fail(LF2_ERR_NOMEM, "allocation failure injected by LF2_FAULT=alloc");
    void *b = nullptr;
    const size_t bytes = (size_t)f->count * f->esize;
    LF2_CUDA(cudaMalloc(&b, bytes ? bytes : 16), what);
    f->val[1 - f->front] = b;
    f->own_val[1 - f->front] = true;
    return LF2_OK;
}

lf2_status alloc_comp(lf2_field phi, int which, cudaStream_t s) {
    if (phi->comp[which]) return LF2_OK;
    if (fault_injected("alloc")) return fail(LF2_ERR_NOMEM, "allocation failure injected by LF2_FAULT=alloc");
    void *c = nullptr;
    const size_t cb = (size_t)phi->count * sizeof(float);
    LF2_CUDA(cudaMalloc(&c, cb ? cb : 16), "cudaMalloc(compensation)");
    phi->comp[which] = (float *)c;
    phi->own_comp[which] = true;
    LF2_CUDA(cudaMemsetAsync(c, 0, cb, s), "cudaMemsetAsync(compensation)");
    return LF2_OK;
}

// Back buffer and compensation of a field used as phi.
lf2_status ensure_dynamic(lf2_field phi, cudaStream_t s) {
    lf2_status st = alloc_back(phi, "cudaMalloc(phi back buffer)");
    if (st == LF2_OK && phi->prec == LF2_F32_KAHAN) st = alloc_comp(phi, phi->cfront, s);
    return st;
}

// Temporal blocking also writes pi and the compensation out of place.
lf2_status ensure_tblock(lf2_field phi, lf2_field pi, cudaStream_t s) {
    lf2_status st = ensure_dynamic(phi, s);
    if (st == LF2_OK) st = alloc_back(pi, "cudaMalloc(pi back buffer)");
    if (st == LF2_OK && phi->prec == LF2_F32_KAHAN) st = alloc_comp(phi, 1 - phi->cfront, s);
    return st;
}

lf2_status ensure_energy_scratch(lf2_field f) {
    if (!f->energy_scratch) {
        void *d = nullptr;
        LF2_CUDA(cudaMalloc(&d, sizeof(double) * kFieldScratchDoubles), "cudaMalloc(energy scratch)");
        // the finished-block counter must start at zero (each reduction leaves it at zero)
        const double zero = 0.0;
        cudaError_t e = cudaMemcpy((double *)d + kEnergyCounterOffset, &zero, sizeof zero, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "energy scratch counter");
        }
        f->energy_scratch = (double *)d;
    }
    if (!f->energy_host) {
        void *h = nullptr;
        LF2_CUDA(cudaMallocHost(&h, sizeof(double) * kEnergySlots), "cudaMallocHost(energy result)");
        f->energy_host = (double *)h;
    }
    return LF2_OK;
}

StepArgs step_args(lf2_field phi, lf2_field pi, const lf2_params *p, double dt, bool drift) {
    StepArgs a;
    a.phi = phi->val[phi->front];
    a.phi_out = phi->val[1 - phi->front];
    a.pi = pi->val[pi->front];
    a.comp = phi->comp[phi->cfront];
    a.g = geom_of(phi->lat);
    a.ncomp = phi->ncomp;
    a.prec = phi->prec;
    a.p = *p;
    a.dt = dt;
    a.drift = drift;
    return a;
}

TbArgs tb_args(lf2_field phi, lf2_field pi, const lf2_params *p) {
    TbArgs a;
    a.phi = phi->val[phi->front];
    a.phi_out = phi->val[1 - phi->front];
    a.pi = pi->val[pi->front];
    a.pi_out = pi->val[1 - pi->front];
    a.comp = phi->comp[phi->cfront];
    a.comp_out = phi->comp[1 - phi->cfront];
    a.g = geom_of(phi->lat);
    a.ncomp = phi->ncomp;
    a.prec = phi->prec;
    a.p = *p;
    a.dt = p->dt;
    return a;
}

}  // namespace lf2

extern "C" {

const char *lf2_status_string(lf2_status s) {
    switch (s) {
        case LF2_OK: return "LF2_OK";
        case LF2_ERR_INVALID: return "LF2_ERR_INVALID";
        case LF2_ERR_UNSUPPORTED: return "LF2_ERR_UNSUPPORTED";
        case LF2_ERR_NOMEM: return "LF2_ERR_NOMEM";
        case LF2_ERR_CUDA: return "LF2_ERR_CUDA";
        case LF2_ERR_TIMEOUT: return "LF2_ERR_TIMEOUT";
        case LF2_ERR_STATE: return "LF2_ERR_STATE";
    }
    return "LF2_ERR_UNKNOWN";
}

const char *lf2_last_error(void) { return g_last_error.c_str(); }

const char *lf2_version(void) { return "lf2 0.1 (sm_103a)"; }

lf2_status lf2_lattice_create(int dim, const int *sizes, int halo, lf2_lattice *out) {
    if (!sizes || !out) return fail(LF2_ERR_INVALID, "sizes or output pointer is NULL");
    if (dim < 2) return fail(LF2_ERR_INVALID, "dim must be >= 2 (got %d)", dim);
    if (dim != 3) return fail(LF2_ERR_UNSUPPORTED, "only 3-D lattices are built (got dim=%d)", dim);
    if (halo < 1) return fail(LF2_ERR_INVALID, "halo must be >= 1 (got %d)", halo);
    long long sites = 1;
    for (int i = 0; i < 3; ++i) {
        if (sizes[i] < 1) return fail(LF2_ERR_INVALID, "sizes[%d] = %d must be >= 1", i, sizes[i]);
        sites *= sizes[i];
        if (sites > (1LL << 40)) return fail(LF2_ERR_INVALID, "lattice too large");
    }
    lf2_lattice_s *l = new (std::nothrow) lf2_lattice_s;
    if (!l) return fail(LF2_ERR_NOMEM, "host allocation failed");
    l->dim = dim;
    for (int i = 0; i < 3; ++i) l->n[i] = sizes[i];
    l->halo = halo;
    l->sites = sites;
    *out = l;
    return LF2_OK;
}

lf2_status lf2_lattice_destroy(lf2_lattice lat) {
    if (!lat) return fail(LF2_ERR_INVALID, "lattice is NULL");
    if (lat->users.load() != 0) return fail(LF2_ERR_STATE, "lattice still used by %d field(s)", lat->users.load());
    delete lat;
    return LF2_OK;
}

lf2_status lf2_lattice_sites(lf2_lattice lat, long long *out) {
    if (!lat || !out) return fail(LF2_ERR_INVALID, "NULL argument");
    *out = lat->sites;
    return LF2_OK;
}

lf2_status lf2_field_alloc(lf2_lattice lat, int ncomp, lf2_precision prec, lf2_field *out) {
    lf2_status st = new_field(lat, ncomp, prec, out);
    if (st != LF2_OK) return st;
    lf2_field_s *f = new (std::nothrow) lf2_field_s;
    if (!f) return fail(LF2_ERR_NOMEM, "host allocation failed");
    f->lat = lat;
    f->ncomp = ncomp;
    f->prec = prec;
    f->esize = elem_size(prec);
    f->count = lat->sites * ncomp;
    const size_t bytes = (size_t)f->count * f->esize;
    if (getenv("LF2_FAULT") && !strcmp(getenv("LF2_FAULT"), "alloc")) {
        delete f;
        return fail(LF2_ERR_NOMEM, "allocation failure injected by LF2_FAULT=alloc");
    }
    cudaError_t e = cudaMalloc(&f->val[0], bytes);
    if (e == cudaSuccess) e = cudaMemset(f->val[0], 0, bytes);
    if (e != cudaSuccess) {
        if (f->val[0]) cudaFree(f->val[0]);
        delete f;
        return cuda_fail(e, "cudaMalloc(field)");
    }
    f->own_val[0] = true;
    lat->users++;
    *out = f;
    return LF2_OK;
}

lf2_status lf2_field_wrap(lf2_lattice lat, int ncomp, lf2_precision prec, void *const *dev_ptrs, int nptrs,
                          lf2_field *out) {
    lf2_status st = new_field(lat, ncomp, prec, out);
    if (st != LF2_OK) return st;
    if (!dev_ptrs || nptrs < 1 || nptrs > 4) return fail(LF2_ERR_INVALID, "nptrs must be 1 to 4");
    if (nptrs >= 3 && prec != LF2_F32_KAHAN) return fail(LF2_ERR_INVALID, "a compensation buffer needs LF2_F32_KAHAN");
    for (int i = 0; i < nptrs; ++i) {
        if (!dev_ptrs[i]) return fail(LF2_ERR_INVALID, "dev_ptrs[%d] is NULL", i);
        if ((uintptr_t)dev_ptrs[i] % 16) return fail(LF2_ERR_INVALID, "dev_ptrs[%d] is not 16-byte aligned", i);
    }
    lf2_field_s *f = new (std::nothrow) lf2_field_s;
    if (!f) return fail(LF2_ERR_NOMEM, "host allocation failed");
    f->lat = lat;
    f->ncomp = ncomp;
    f->prec = prec;
    f->esize = elem_size(prec);
    f->count = lat->sites * ncomp;
    f->val[0] = dev_ptrs[0];
    if (nptrs >= 2) f->val[1] = dev_ptrs[1];
    if (nptrs >= 3) f->comp[0] = (float *)dev_ptrs[2];
    if (nptrs >= 4) f->comp[1] = (float *)dev_ptrs[3];
    lat->users++;
    *out = f;
    return LF2_OK;
}

lf2_status lf2_field_free(lf2_field f) {
    if (!f) return fail(LF2_ERR_INVALID, "field is NULL");
    if (f->ensemble) return fail(LF2_ERR_STATE, "field is a member of an ensemble: destroy the ensemble first");
    for (int i = 0; i < 2; ++i)
        if (f->own_val[i] && f->val[i]) cudaFree(f->val[i]);
    for (int i = 0; i < 2; ++i)
        if (f->own_comp[i] && f->comp[i]) cudaFree(f->comp[i]);
    if (f->energy_scratch) cudaFree(f->energy_scratch);
    if (f->energy_host) cudaFreeHost(f->energy_host);
    f->lat->users--;
    delete f;
    return LF2_OK;
}

lf2_status lf2_field_buffer(lf2_field f, int which, void **out) {
    if (!f || !out) return fail(LF2_ERR_INVALID, "NULL argument");
    switch (which) {
        case 0: *out = f->val[f->front]; break;
        case 1: *out = f->val[1 - f->front]; break;
        case 2: *out = f->comp[f->cfront]; break;
        case 3: *out = f->comp[1 - f->cfront]; break;
        default: return fail(LF2_ERR_INVALID, "which must be 0, 1, 2 or 3");
    }
    return LF2_OK;
}

lf2_status lf2_field_upload(lf2_field f, const double *host, void *stream) {
    if (!f || !host) return fail(LF2_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t total = (size_t)f->count;
    if (f->prec == LF2_F64) {
        LF2_CUDA(cudaMemcpyAsync(f->val[f->front], host, total * sizeof(double), cudaMemcpyHostToDevice, s),
                 "upload copy");
    } else {
        // Stage chunks of doubles on the device and convert there.
        const size_t chunk = std::min(total, (size_t)1 << 24);
        double *stage = nullptr;
        if (chunk) LF2_CUDA(cudaMalloc(&stage, chunk * sizeof(double)), "cudaMalloc(upload staging)");
        for (size_t off = 0; off < total; off += chunk) {
            const size_t n = std::min(chunk, total - off);
            cudaError_t e = cudaMemcpyAsync(stage, host + off, n * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = launch_convert_from_f64(stage, (float *)f->val[f->front] + off, (long long)n, f->prec, s);
            if (e != cudaSuccess) {
                cudaFree(stage);
                return cuda_fail(e, "upload");
            }
        }
        if (f->comp[f->cfront]) {
            cudaError_t e = cudaMemsetAsync(f->comp[f->cfront], 0, total * sizeof(float), s);
            if (e != cudaSuccess) {
                cudaFree(stage);
                return cuda_fail(e, "reset compensation");
            }
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (stage) cudaFree(stage);
        if (e != cudaSuccess) return cuda_fail(e, "upload sync");
        return LF2_OK;
    }
    if (f->comp[f->cfront])
        LF2_CUDA(cudaMemsetAsync(f->comp[f->cfront], 0, total * sizeof(float), s), "reset compensation");
    LF2_CUDA(cudaStreamSynchronize(s), "upload sync");
    return LF2_OK;
}

lf2_status lf2_field_download(lf2_field f, double *host, void *stream) {
    if (!f || !host) return fail(LF2_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t total = (size_t)f->count;
    if (f->prec == LF2_F64) {
        LF2_CUDA(cudaMemcpyAsync(host, f->val[f->front], total * sizeof(double), cudaMemcpyDeviceToHost, s),
                 "download copy");
        LF2_CUDA(cudaStreamSynchronize(s), "download sync");
        return LF2_OK;
    }
    const size_t chunk = std::min(total, (size_t)1 << 24);
    double *stage = nullptr;
    if (chunk) LF2_CUDA(cudaMalloc(&stage, chunk * sizeof(double)), "cudaMalloc(download staging)");
    for (size_t off = 0; off < total; off += chunk) {
        const size_t n = std::min(chunk, total - off);
        cudaError_t e = launch_convert_to_f64((const float *)f->val[f->front] + off, stage, (long long)n, f->prec, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host + off, stage, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(stage);
            return cuda_fail(e, "download");
        }
    }
    if (stage) cudaFree(stage);
    return LF2_OK;
}

lf2_status lf2_field_derivative(lf2_field src, lf2_field dst, int dim, double dx, void *stream) {
    if (!src || !dst) return fail(LF2_ERR_INVALID, "field handle is NULL");
    if (src == dst) return fail(LF2_ERR_INVALID, "src and dst must be different fields");
    if (src->lat != dst->lat || src->ncomp != dst->ncomp || src->prec != dst->prec)
        return fail(LF2_ERR_INVALID, "src and dst differ in lattice, components or precision");
    if (dim < 0 || dim > 2) return fail(LF2_ERR_INVALID, "dim must be 0, 1 or 2");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(LF2_ERR_INVALID, "dx must be finite and > 0");
    LF2_CUDA(launch_derivative(src->val[src->front], dst->val[dst->front], geom_of(src->lat), src->ncomp, src->prec,
                               dim, dx, (cudaStream_t)stream),
             "derivative launch");
    return LF2_OK;
}

lf2_status lf2_field_update_halo(lf2_field f, void *stream) {
    (void)stream;
    if (!f) return fail(LF2_ERR_INVALID, "field is NULL");
    return LF2_OK;
}

lf2_status lf2_leapfrog_init(lf2_field phi, lf2_field pi, const lf2_params *p, void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_dynamic(phi, s);
    if (st != LF2_OK) return st;
    st = ensure_energy_scratch(phi);
    if (st != LF2_OK) return st;
    const StepArgs a = step_args(phi, pi, p, -0.5 * p->dt, false);
    LF2_CUDA(launch_site_step(a, s), "half-kick launch");
    return LF2_OK;
}

lf2_status lf2_leapfrog_ex(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps, const lf2_step_config *cfg,
                           void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    if (nsteps < 0) return fail(LF2_ERR_INVALID, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int kernel = cfg ? cfg->kernel : LF2_KERNEL_AUTO;
    if (kernel < LF2_KERNEL_AUTO || kernel > LF2_KERNEL_TBLOCK) return fail(LF2_ERR_INVALID, "unknown kernel %d", kernel);
    if (fault_injected("launch")) return fail(LF2_ERR_CUDA, "launch failure injected by LF2_FAULT=launch");
    lf2_step_config tuned{};
    if (kernel == LF2_KERNEL_AUTO && tune_mode() != TuneMode::Off) {
        bool have = plan_lookup(phi->lat->n, phi->ncomp, phi->prec, &tuned);
        if (!have && tune_mode() == TuneMode::Force) {
            st = lf2_tune(phi, pi, p, 0, &tuned, stream);
            if (st != LF2_OK) return st;
            have = true;
        }
        if (have) {
            cfg = &tuned;
            kernel = tuned.kernel;
        }
    }
    const int tile_y = cfg ? cfg->tile_y : 0;
    const int zchunk = cfg ? cfg->zchunk : 0;
    st = (kernel == LF2_KERNEL_TBLOCK) ? ensure_tblock(phi, pi, s) : ensure_dynamic(phi, s);
    if (st != LF2_OK) return st;

    // one-step kernel used for single steps (and for what temporal blocking leaves over)
    const StepArgs probe = step_args(phi, pi, p, p->dt, true);
    const bool stream_ok = stream_supported(probe, kernel == LF2_KERNEL_STREAM ? tile_y : 0,
                                            kernel == LF2_KERNEL_STREAM ? zchunk : 0);
    if (kernel == LF2_KERNEL_STREAM && !stream_ok)
        return fail(LF2_ERR_UNSUPPORTED, "streaming kernel does not fit this lattice/config");
    const bool use_stream = (kernel == LF2_KERNEL_STREAM || kernel == LF2_KERNEL_AUTO || kernel == LF2_KERNEL_TBLOCK) &&
                            stream_ok;
    auto one_step = [&]() -> lf2_status {
        const StepArgs a = step_args(phi, pi, p, p->dt, true);
        cudaError_t e = use_stream ? launch_stream_step(a, kernel == LF2_KERNEL_STREAM ? tile_y : 0,
                                                        kernel == LF2_KERNEL_STREAM ? zchunk : 0, 1, s)
                                   : launch_site_step(a, s);
        if (e != cudaSuccess) return cuda_fail(e, "leapfrog launch");
        phi->front = 1 - phi->front;
        return LF2_OK;
    };

    int done = 0;
    if (kernel == LF2_KERNEL_TBLOCK) {
        TbConfig c{cfg->depth, cfg->cx, cfg->tile_x, tile_y, zchunk, cfg->cluster};
        TbArgs ta = tb_args(phi, pi, p);
        if (!tblock_supported(ta, c))
            return fail(LF2_ERR_UNSUPPORTED,
                        "temporal blocking config (depth %d, cx %d, tile %dx%d, cluster %d) does not fit", c.depth,
                        c.cx, c.tile_x, c.tile_y, c.cluster);
        for (; done + c.depth <= nsteps; done += c.depth) {
            ta = tb_args(phi, pi, p);
            cudaError_t e = launch_tblock(ta, c, s);
            if (e != cudaSuccess) return cuda_fail(e, "temporal-blocking launch");
            phi->front = 1 - phi->front;
            pi->front = 1 - pi->front;
            if (phi->prec == LF2_F32_KAHAN) phi->cfront = 1 - phi->cfront;
        }
    }
    for (; done < nsteps; ++done) {
        st = one_step();
        if (st != LF2_OK) return st;
    }
    return LF2_OK;
}

lf2_status lf2_leapfrog(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps, void *stream) {
    return lf2_leapfrog_ex(phi, pi, p, nsteps, nullptr, stream);
}

lf2_status lf2_energy(lf2_field phi, lf2_field pi, const lf2_params *p, lf2_energy_t *out, void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    if (!out) return fail(LF2_ERR_INVALID, "output pointer is NULL");
    st = ensure_energy_scratch(phi);
    if (st != LF2_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    LF2_CUDA(launch_energy(phi->val[phi->front], pi->val[pi->front], geom_of(phi->lat), phi->ncomp, phi->prec, *p,
                           phi->energy_scratch, nullptr, s),
             "energy launch");
    LF2_CUDA(cudaMemcpyAsync(phi->energy_host, phi->energy_scratch + kEnergyRecordOffset, sizeof(lf2_energy_t),
                             cudaMemcpyDeviceToHost, s),
             "energy copy");
    LF2_CUDA(cudaStreamSynchronize(s), "energy sync");
    memcpy(out, phi->energy_host, sizeof(lf2_energy_t));
    return LF2_OK;
}

lf2_status lf2_energy_device(lf2_field phi, lf2_field pi, const lf2_params *p, double *dev_out, void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    if (!dev_out) return fail(LF2_ERR_INVALID, "output pointer is NULL");
    if (!phi->energy_scratch)
        return fail(LF2_ERR_STATE, "no energy scratch yet: call lf2_leapfrog_init or lf2_energy on phi first");
    LF2_CUDA(launch_energy(phi->val[phi->front], pi->val[pi->front], geom_of(phi->lat), phi->ncomp, phi->prec, *p,
                           phi->energy_scratch, dev_out, (cudaStream_t)stream),
             "energy launch");
    return LF2_OK;
}

lf2_status lf2_leapfrog_energy(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps, double *dev_records,
                               void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    if (nsteps < 0) return fail(LF2_ERR_INVALID, "nsteps must be >= 0");
    if (nsteps > 0 && !dev_records) return fail(LF2_ERR_INVALID, "records pointer is NULL");
    if (nsteps > 0 && fault_injected("launch")) return fail(LF2_ERR_CUDA, "launch failure injected by LF2_FAULT=launch");
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_dynamic(phi, s);
    if (st == LF2_OK) st = ensure_energy_scratch(phi);
    if (st != LF2_OK) return st;
    // small lattices: all steps in one cooperative launch (bitwise the per-step launches)
    const cudaError_t e = launch_steps_energy(step_args(phi, pi, p, p->dt, true), nsteps, phi->energy_scratch,
                                              dev_records, fault_injected("timeout"), s);
    if (e == cudaSuccess) {
        if (nsteps & 1) phi->front = 1 - phi->front;
        return LF2_OK;
    }
    if (e != cudaErrorNotSupported) return cuda_fail(e, "multi-step step+energy launch");
    for (int k = 0; k < nsteps; ++k) {
        const StepArgs a = step_args(phi, pi, p, p->dt, true);
        LF2_CUDA(launch_step_energy(a, phi->energy_scratch, dev_records + (size_t)k * kEnergySlots, s),
                 "step+energy launch");
        phi->front = 1 - phi->front;
    }
    return LF2_OK;
}

lf2_status lf2_field_compare(lf2_field f, int which, const void *ref, lf2_precision ref_prec, double *out,
                             void *stream) {
    if (!f || !ref || !out) return fail(LF2_ERR_INVALID, "NULL argument");
    if (ref_prec != LF2_F64 && ref_prec != LF2_F32_KAHAN && ref_prec != LF2_F32)
        return fail(LF2_ERR_INVALID, "unknown reference precision %d", (int)ref_prec);
    void *buf = nullptr;
    lf2_status st = lf2_field_buffer(f, which, &buf);
    if (st != LF2_OK) return st;
    if (!buf) return fail(LF2_ERR_STATE, "buffer %d of this field does not exist", which);
    st = ensure_energy_scratch(f);
    if (st != LF2_OK) return st;
    // values are in the storage type; compensation buffers (2, 3) are float
    const bool a_double = which < 2 && f->prec == LF2_F64;
    cudaStream_t s = (cudaStream_t)stream;
    LF2_CUDA(launch_compare(buf, a_double, ref, ref_prec == LF2_F64, f->count, f->energy_scratch, s), "compare launch");
    LF2_CUDA(cudaMemcpyAsync(f->energy_host, f->energy_scratch + kEnergyRecordOffset, 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, s),
             "compare copy");
    LF2_CUDA(cudaStreamSynchronize(s), "compare sync");
    memcpy(out, f->energy_host, 4 * sizeof(double));
    return LF2_OK;
}

lf2_status lf2_field_check(lf2_field phi, void *stream) {
    if (!phi) return fail(LF2_ERR_INVALID, "field is NULL");
    if (!phi->energy_scratch) return LF2_OK;  // no multi-step run yet
    bool timed_out = false;
    LF2_CUDA(steps_energy_timed_out(phi->energy_scratch, &timed_out, (cudaStream_t)stream), "status read");
    if (timed_out)
        return fail(LF2_ERR_TIMEOUT,
                    "a grid barrier of the last multi-step lf2_leapfrog_energy run gave up: its records from that step "
                    "on are NaN and the fields are not a valid state");
    return LF2_OK;
}

lf2_status lf2_debug_bounds(unsigned long long *violations, int reset) {
    if (!violations) return fail(LF2_ERR_INVALID, "NULL argument");
#ifdef LF2_DEBUG_BOUNDS
    using Fn = cudaError_t (*)(unsigned long long *, bool);
    const Fn units[] = {bounds_violations_site,        bounds_violations_stream,       bounds_violations_tblock_f64,
                        bounds_violations_tblock_f32k, bounds_violations_tblock_f32, bounds_violations_energy};
    unsigned long long total = 0;
    for (Fn f : units) {
        unsigned long long n = 0;
        LF2_CUDA(f(&n, reset != 0), "bounds counter");
        total += n;
    }
    *violations = total;
    return LF2_OK;
#else
    (void)reset;
    *violations = 0;
    return fail(LF2_ERR_UNSUPPORTED, "built without LF2_DEBUG_BOUNDS (build the debug library to count index violations)");
#endif
}

lf2_status lf2_energy_noalloc(lf2_field phi, lf2_field pi, const lf2_params *p, lf2_energy_t *out, void *stream) {
    lf2_status st = check_pair(phi, pi);
    if (st == LF2_OK) st = check_params(p);
    if (st != LF2_OK) return st;
    if (!out) return fail(LF2_ERR_INVALID, "output pointer is NULL");
    // The reduction grid is capped at kEnergyBlocks whatever the lattice, so its partial rows,
    // record and counter always fit the fixed array (checked at compile time next to it).
    double *scratch = nullptr;
    LF2_CUDA(energy_noalloc_scratch(&scratch), "cudaGetSymbolAddress(energy scratch)");
    cudaStream_t s = (cudaStream_t)stream;
    // The last block of a reduction returns the finished-block counter to zero.  An earlier
    // call that overlapped another on the GPU (a documented race) could leave it non-zero, so
    // it is cleared on this call's stream first: the damage of an overlap stays in that call.
    LF2_CUDA(cudaMemsetAsync(scratch + kEnergyCounterOffset, 0, sizeof(unsigned int), s), "counter reset");
    // The reduction writes every partial row it reads and the record read back below.
    LF2_CUDA(launch_energy(phi->val[phi->front], pi->val[pi->front], geom_of(phi->lat), phi->ncomp, phi->prec, *p,
                           scratch, nullptr, s),
             "energy launch");
    double r[kEnergySlots];
    LF2_CUDA(cudaMemcpyAsync(r, scratch + kEnergyRecordOffset, sizeof r, cudaMemcpyDeviceToHost, s), "energy copy");
    LF2_CUDA(cudaStreamSynchronize(s), "energy sync");
    memcpy(out, r, sizeof(lf2_energy_t));
    return LF2_OK;
}

}  // extern "C"
