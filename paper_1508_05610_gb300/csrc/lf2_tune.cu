// lf2_tune.cu -- autotuner for the leapfrog kernel configuration.
//
// Every kernel variant computes bitwise the same result, so the tuner only has to find the
// fastest one.  It times candidate configurations (one-step streaming tiles and temporal
// blocking of several depths, column widths and tiles) on a proxy lattice with the same x-y
// plane as the real one and at most kProxyPlanes z-planes, filled with a copy of the real
// fields' first planes: the caller's fields are never modified.  The winner is kept in a
// process-wide table keyed by (shape, components, precision, SM count) that lf2_leapfrog
// consults, and is appended to the file named by LF2_TUNE_CACHE if that variable is set
// (that file is also read on first use).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lf2_handles.h"

namespace lf2 {
namespace {

constexpr int kProxyPlanes = 256;           // at most this many z-planes
constexpr size_t kProxyBytes = 8ull << 30;  // and at most this much device memory
constexpr int kTuneSteps = 24;  // divisible by every depth 2, 3, 4, 6, 8

using Key = std::tuple<int, int, int, int, int, int>;  // nx, ny, nz, ncomp, prec, sm count
std::mutex g_mu;
std::map<Key, lf2_step_config> g_plans;
bool g_file_read = false;

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

Key key_of(const int n[3], int ncomp, lf2_precision prec) { return Key{n[0], n[1], n[2], ncomp, (int)prec, sm_count()}; }

void read_file_locked() {
    if (g_file_read) return;
    g_file_read = true;
    const char *path = getenv("LF2_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    // one plan per line: the key's 6 integers, then kernel, tile_x, tile_y, zchunk, depth, cx,
    // cluster
    int v[13];
    char line[512];
    while (fgets(line, sizeof line, f)) {
        v[12] = 0;
        const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                               &v[6], &v[7], &v[8], &v[9], &v[10], &v[11], &v[12]);
        if (got < 12) continue;
        g_plans[Key{v[0], v[1], v[2], v[3], v[4], v[5]}] = lf2_step_config{v[6], v[7], v[8], v[9], v[10], v[11], v[12]};
    }
    fclose(f);
}

void append_file(const Key &k, const lf2_step_config &c) {
    const char *path = getenv("LF2_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
            std::get<3>(k), std::get<4>(k), std::get<5>(k), c.kernel, c.tile_x, c.tile_y, c.zchunk, c.depth, c.cx,
            c.cluster);
    fclose(f);
}

std::vector<lf2_step_config> candidates(lf2_precision prec, int flags) {
    std::vector<lf2_step_config> out;
    for (int ty : {4, 8})
        for (int zc : {4, 8, 16}) out.push_back(lf2_step_config{LF2_KERNEL_STREAM, 0, ty, zc, 0, 0});
    if (flags & LF2_TUNE_ONE_STEP) return out;
    const int depths64[] = {2, 4};
    const int depths32[] = {2, 3, 4, 6, 8};
    const bool f64 = prec == LF2_F64;
    for (int depth : f64 ? std::vector<int>(depths64, depths64 + 2) : std::vector<int>(depths32, depths32 + 5)) {
        for (int cx : {1, 2, 4}) {
            const int tp = ((depth + cx - 1) / cx) * cx;
            for (int rxt : {16, 32}) {
                const int tx = rxt * cx - 2 * tp;
                if (tx < cx) continue;
                for (int ty : {8, 16, 24}) {
                    if (rxt * (ty + 2 * depth) > 512) continue;
                    out.push_back(lf2_step_config{LF2_KERNEL_TBLOCK, tx, ty, 0, depth, cx});
                }
            }
            out.push_back(lf2_step_config{LF2_KERNEL_TBLOCK, 32, 16, 0, depth, cx});
        }
    }
    if (!f64) {
        // thread-block clusters: a warp per region row (32 threads x cx columns), 16 rows per
        // CTA, 2 to 8 CTAs stacked along y; fewer halo rows per output row than one CTA holds
        for (int depth : {3, 4})
            for (int cx : {1, 2, 4})
                for (int cl : {2, 4, 8}) {
                    const int tp = ((depth + cx - 1) / cx) * cx;
                    out.push_back(lf2_step_config{LF2_KERNEL_TBLOCK, 32 * cx - 2 * tp, 16 * cl - 2 * depth, 0, depth, cx,
                                                  cl});
                }
    }
    return out;
}

}  // namespace

bool plan_lookup(const int n[3], int ncomp, lf2_precision prec, lf2_step_config *out) {
    std::lock_guard<std::mutex> lock(g_mu);
    read_file_locked();
    auto it = g_plans.find(key_of(n, ncomp, prec));
    if (it == g_plans.end()) return false;
    *out = it->second;
    return true;
}

}  // namespace lf2

using namespace lf2;

extern "C" lf2_status lf2_tune(lf2_field phi, lf2_field pi, const lf2_params *p, int flags, lf2_step_config *chosen,
                               void *stream) {
    if (!phi || !pi || !p) return set_error(LF2_ERR_INVALID, "NULL argument");
    if (phi->lat != pi->lat || phi->ncomp != pi->ncomp || phi->prec != pi->prec)
        return set_error(LF2_ERR_INVALID, "phi and pi do not match");
    const int *n = phi->lat->n;
    const Key key = key_of(n, phi->ncomp, phi->prec);
    if (!(flags & LF2_TUNE_FORCE)) {
        lf2_step_config c;
        if (plan_lookup(n, phi->ncomp, phi->prec, &c)) {
            if (chosen) *chosen = c;
            return LF2_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    // proxy lattice: same x-y plane, first planes of the real fields
    // six buffers (phi, pi, compensation, each with a back buffer) of one plane
    const size_t plane_bytes = (size_t)n[0] * n[1] * phi->ncomp * 4 * sizeof(float) * 2;
    int pz = n[2] < kProxyPlanes ? n[2] : kProxyPlanes;
    while (pz > 32 && (size_t)pz * plane_bytes > kProxyBytes) pz /= 2;
    const int psizes[3] = {n[0], n[1], pz};
    lf2_lattice plat = nullptr;
    lf2_field pphi = nullptr, ppi = nullptr;
    lf2_status st = lf2_lattice_create(3, psizes, 1, &plat);
    if (st == LF2_OK) st = lf2_field_alloc(plat, phi->ncomp, phi->prec, &pphi);
    if (st == LF2_OK) st = lf2_field_alloc(plat, phi->ncomp, phi->prec, &ppi);
    auto cleanup = [&]() {
        if (pphi) lf2_field_free(pphi);
        if (ppi) lf2_field_free(ppi);
        if (plat) lf2_lattice_destroy(plat);
    };
    if (st != LF2_OK) {
        cleanup();
        return st;
    }
    const size_t bytes = (size_t)n[0] * n[1] * pz * phi->ncomp * phi->esize;
    cudaError_t e = cudaMemcpyAsync(pphi->val[pphi->front], phi->val[phi->front], bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ppi->val[ppi->front], pi->val[pi->front], bytes, cudaMemcpyDeviceToDevice, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cleanup();
        return cuda_error(e, "tuner set-up");
    }
    lf2_step_config best{LF2_KERNEL_STREAM, 0, 0, 0, 0, 0};
    float best_ms = -1.0f;
    for (const lf2_step_config &c : candidates(phi->prec, flags)) {
        // warm-up (also rejects configurations that do not fit this lattice)
        if (lf2_leapfrog_ex(pphi, ppi, p, kTuneSteps, &c, stream) != LF2_OK) continue;
        float ms = -1.0f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            if (lf2_leapfrog_ex(pphi, ppi, p, kTuneSteps, &c, stream) != LF2_OK) break;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (ms < 0.0f || t < ms) ms = t;
        }
        if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "tuning runs");
    if (best_ms < 0.0f) return set_error(LF2_ERR_UNSUPPORTED, "no kernel configuration ran on this lattice");
    {
        std::lock_guard<std::mutex> lock(g_mu);
        read_file_locked();
        g_plans[key] = best;
    }
    append_file(key, best);
    if (chosen) *chosen = best;
    return LF2_OK;
}

extern "C" lf2_status lf2_tune_lookup(const int *sizes, int ncomp, lf2_precision prec, lf2_step_config *out) {
    if (!sizes || !out) return set_error(LF2_ERR_INVALID, "NULL argument");
    if (!plan_lookup(sizes, ncomp, prec, out)) return set_error(LF2_ERR_STATE, "no tuned plan for this shape");
    return LF2_OK;
}
