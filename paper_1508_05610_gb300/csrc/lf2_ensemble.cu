// lf2_ensemble.cu -- batched ensembles of independent lattices of uneven sizes.
//
// An ensemble groups (phi, pi) field pairs of one precision and component count, each on its
// own lattice and with its own parameters.  lf2_ensemble_run advances all of them by nsteps
// with one CUDA-graph launch: the graph holds nsteps / depth temporal-blocking passes, each a
// single persistent kernel launch whose blocks take (member, tile, z-chunk) items, longest
// chunks first, from a counter zeroed before the pass, followed by the leftover single steps
// per member.  Members
// are independent, so no block ever waits for another; the graph is captured once per
// (nsteps, buffer parities) and relaunched.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lf2_handles.h"

using namespace lf2;

namespace {

struct CapturedRun {
    int nsteps = 0;
    std::vector<int> signature;  // fronts of every member before the run
    cudaGraphExec_t exec = nullptr;
    TbMember *d_members = nullptr;
};

}  // namespace

struct lf2_ensemble_s {
    int n = 0;
    std::vector<lf2_field> phi, pi;
    std::vector<lf2_params> params;
    lf2_precision prec = LF2_F64;
    int ncomp = 1;
    TbConfig cfg{0, 0, 0, 0, 0};
    bool tblock = false;  // temporal-blocking passes usable for every member
    int4 *d_items = nullptr;
    int nitems = 0;
    int *d_counter = nullptr;  // work-list position of the running pass
    cudaStream_t capture = nullptr;
    std::vector<CapturedRun> runs;
};

namespace {

void free_runs(lf2_ensemble e) {
    for (CapturedRun &r : e->runs) {
        if (r.exec) cudaGraphExecDestroy(r.exec);
        if (r.d_members) cudaFree(r.d_members);
    }
    e->runs.clear();
}

std::vector<int> signature_of(lf2_ensemble e) {
    std::vector<int> s;
    for (int i = 0; i < e->n; ++i) {
        s.push_back(e->phi[i]->front);
        s.push_back(e->pi[i]->front);
        s.push_back(e->phi[i]->cfront);
    }
    return s;
}

int member_zchunk(const lf2_lattice_s *lat) { return lat->n[2]; }

// Builds the work list for configuration c (longest z-chunks first, then member order).
lf2_status build_items(lf2_ensemble e, const TbConfig &c) {
    std::vector<int4> items;
    for (int m = 0; m < e->n; ++m) {
        const int *n = e->phi[m]->lat->n;
        const int tx = (n[0] + c.tile_x - 1) / c.tile_x, ty = (n[1] + c.tile_y - 1) / c.tile_y;
        const int zc = member_zchunk(e->phi[m]->lat);
        const int nzc = (n[2] + zc - 1) / zc;
        for (int bz = 0; bz < nzc; ++bz)
            for (int by = 0; by < ty; ++by)
                for (int bx = 0; bx < tx; ++bx) items.push_back(int4{m, bx, by, bz});
    }
    auto zlen = [&](const int4 &w) {
        const int nz = e->phi[w.x]->lat->n[2], zc = member_zchunk(e->phi[w.x]->lat);
        return std::min(zc, nz - w.w * zc);
    };
    std::stable_sort(items.begin(), items.end(), [&](const int4 &a, const int4 &b) { return zlen(a) > zlen(b); });
    if (e->d_items) cudaFree(e->d_items);
    e->d_items = nullptr;
    e->nitems = (int)items.size();
    if (items.empty()) return LF2_OK;
    cudaError_t err = cudaMalloc(&e->d_items, items.size() * sizeof(int4));
    if (err == cudaSuccess)
        err = cudaMemcpy(e->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_error(err, "ensemble work list");
    return LF2_OK;
}

// Checks that configuration c runs on every member (temporarily filling defaults).
bool config_fits(lf2_ensemble e, TbConfig c) {
    // every member must fit the pass (temporal blocking of 3, 4 and 6 components is FP32 only,
    // one column per thread, depth 2 to 4 -- 2 for 6 components -- as for a single lattice)
    for (int m = 0; m < e->n; ++m) {
        TbArgs a = tb_args(e->phi[m], e->pi[m], &e->params[m]);
        TbConfig cm = c;
        cm.zchunk = member_zchunk(e->phi[m]->lat);
        if (!tblock_supported(a, cm)) return false;
    }
    return true;
}

lf2_status set_config(lf2_ensemble e, const TbConfig &c) {
    e->cfg = c;
    e->tblock = config_fits(e, c);
    free_runs(e);
    return e->tblock ? build_items(e, c) : LF2_OK;
}

TbMember member_entry(lf2_ensemble e, int m) {
    lf2_field phi = e->phi[m], pi = e->pi[m];
    TbMember t;
    memset(&t, 0, sizeof t);
    // index 0 is the front at capture time, 1 the back
    t.phi[0] = phi->val[phi->front];
    t.phi[1] = phi->val[1 - phi->front];
    t.pi[0] = pi->val[pi->front];
    t.pi[1] = pi->val[1 - pi->front];
    t.comp[0] = phi->comp[phi->cfront];
    t.comp[1] = phi->comp[1 - phi->cfront];
    t.g = geom_of(phi->lat);
    t.k32 = make_coef32(e->params[m], e->params[m].dt);
    t.k64 = make_coef64(e->params[m], e->params[m].dt);
    t.zchunk = member_zchunk(phi->lat);
    t.front = 0;
    return t;
}

// Enqueues nsteps for every member on stream s (used for capture and for the tuner).
lf2_status enqueue_run(lf2_ensemble e, int nsteps, const TbMember *d_members, cudaStream_t s) {
    const int depth = e->tblock ? e->cfg.depth : 0;
    const int passes = depth ? nsteps / depth : 0;
    for (int k = 0; k < passes; ++k) {
        TbEnsembleLaunch L{d_members, e->d_items, e->nitems, e->d_counter, k & 1, e->cfg, e->ncomp, e->prec};
        cudaError_t err = launch_tblock_ensemble(L, s);
        if (err != cudaSuccess) return cuda_error(err, "ensemble pass");
    }
    // leftover single steps per member, from the buffers the passes leave current
    const int rest = nsteps - passes * depth;
    for (int m = 0; m < e->n; ++m) {
        lf2_field phi = e->phi[m], pi = e->pi[m];
        const int pf = passes & 1;
        int fphi = phi->front ^ pf;
        const int fpi = pi->front ^ pf, fc = phi->cfront ^ pf;
        for (int r = 0; r < rest; ++r) {
            StepArgs a = step_args(phi, pi, &e->params[m], e->params[m].dt, true);
            a.phi = phi->val[fphi];
            a.phi_out = phi->val[1 - fphi];
            a.pi = pi->val[fpi];
            a.comp = phi->comp[fc];
            cudaError_t err = stream_supported(a, 0, 0) ? launch_stream_step(a, 0, 0, 1, s) : launch_site_step(a, s);
            if (err != cudaSuccess) return cuda_error(err, "ensemble single step");
            fphi ^= 1;
        }
    }
    return LF2_OK;
}

void advance_fronts(lf2_ensemble e, int nsteps) {
    const int depth = e->tblock ? e->cfg.depth : 0;
    const int passes = depth ? nsteps / depth : 0;
    const int rest = nsteps - passes * depth;
    for (int m = 0; m < e->n; ++m) {
        e->phi[m]->front ^= (passes + rest) & 1;
        e->pi[m]->front ^= passes & 1;
        if (e->prec == LF2_F32_KAHAN) e->phi[m]->cfront ^= passes & 1;
    }
}

lf2_status upload_members(lf2_ensemble e, TbMember **out) {
    std::vector<TbMember> tab;
    for (int m = 0; m < e->n; ++m) tab.push_back(member_entry(e, m));
    void *d = nullptr;
    cudaError_t err = cudaMalloc(&d, tab.size() * sizeof(TbMember));
    if (err == cudaSuccess) err = cudaMemcpy(d, tab.data(), tab.size() * sizeof(TbMember), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        if (d) cudaFree(d);
        return cuda_error(err, "ensemble member table");
    }
    *out = (TbMember *)d;
    return LF2_OK;
}

}  // namespace

extern "C" {

lf2_status lf2_ensemble_create(int n, const lf2_field *phis, const lf2_field *pis, const lf2_params *per_lattice,
                               lf2_ensemble *out) {
    if (n < 1 || !phis || !pis || !per_lattice || !out) return set_error(LF2_ERR_INVALID, "invalid ensemble arguments");
    for (int m = 0; m < n; ++m) {
        lf2_field a = phis[m], b = pis[m];
        if (!a || !b || a == b || a->lat != b->lat || a->ncomp != b->ncomp || a->prec != b->prec)
            return set_error(LF2_ERR_INVALID, "member %d: phi and pi do not form a pair", m);
        if (a->prec != phis[0]->prec || a->ncomp != phis[0]->ncomp)
            return set_error(LF2_ERR_INVALID, "member %d: all members need one precision and component count", m);
        const lf2_params &q = per_lattice[m];
        if (!(q.dx > 0.0) || !std::isfinite(q.dx) || !std::isfinite(q.dt) || !std::isfinite(q.lambda) ||
            !std::isfinite(q.eta) || !std::isfinite(q.m2))
            return set_error(LF2_ERR_INVALID, "member %d: dx must be finite and > 0, the other parameters finite", m);
        if (a->ensemble || b->ensemble)
            return set_error(LF2_ERR_STATE, "member %d: a field already belongs to another ensemble", m);
        for (int k = 0; k < m; ++k)
            if (phis[k] == a || pis[k] == b || phis[k] == b || pis[k] == a)
                return set_error(LF2_ERR_INVALID, "member %d shares a field with member %d", m, k);
    }
    lf2_ensemble_s *e = new (std::nothrow) lf2_ensemble_s;
    if (!e) return set_error(LF2_ERR_NOMEM, "host allocation failed");
    e->n = n;
    e->phi.assign(phis, phis + n);
    e->pi.assign(pis, pis + n);
    e->params.assign(per_lattice, per_lattice + n);
    e->prec = phis[0]->prec;
    e->ncomp = phis[0]->ncomp;
    lf2_status st = LF2_OK;
    for (int m = 0; m < n && st == LF2_OK; ++m) st = ensure_tblock(e->phi[m], e->pi[m], nullptr);
    cudaError_t err = cudaSuccess;
    if (st == LF2_OK) err = cudaDeviceSynchronize();
    if (st == LF2_OK && err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking);
    if (st == LF2_OK && err == cudaSuccess) err = cudaMalloc(&e->d_counter, sizeof(int));
    if (st == LF2_OK && err != cudaSuccess) st = cuda_error(err, "ensemble set-up");
    if (st == LF2_OK) {
        // default configuration: depth 4 with the widest packed columns that fit, else one-step
        const TbConfig tries[] = {{4, 4, 56, 24, 0}, {4, 2, 24, 24, 0}, {4, 1, 24, 8, 0}, {2, 1, 16, 8, 0}};
        bool ok = false;
        for (const TbConfig &c : tries)
            if (config_fits(e, c)) {
                st = set_config(e, c);
                ok = true;
                break;
            }
        if (!ok) e->tblock = false;
    }
    if (st != LF2_OK) {
        if (e->capture) cudaStreamDestroy(e->capture);
        if (e->d_items) cudaFree(e->d_items);
        if (e->d_counter) cudaFree(e->d_counter);
        delete e;
        return st;
    }
    for (int m = 0; m < n; ++m) {
        e->phi[m]->lat->users++;
        e->phi[m]->ensemble = e->pi[m]->ensemble = e;
    }
    *out = e;
    return LF2_OK;
}

lf2_status lf2_ensemble_destroy(lf2_ensemble e) {
    if (!e) return set_error(LF2_ERR_INVALID, "ensemble is NULL");
    free_runs(e);
    if (e->d_items) cudaFree(e->d_items);
    if (e->d_counter) cudaFree(e->d_counter);
    if (e->capture) cudaStreamDestroy(e->capture);
    for (int m = 0; m < e->n; ++m) {
        e->phi[m]->lat->users--;
        e->phi[m]->ensemble = e->pi[m]->ensemble = nullptr;
    }
    delete e;
    return LF2_OK;
}

lf2_status lf2_ensemble_set_config(lf2_ensemble e, const lf2_step_config *c) {
    if (!e || !c) return set_error(LF2_ERR_INVALID, "NULL argument");
    if (c->kernel == LF2_KERNEL_TBLOCK) {
        TbConfig t{c->depth ? c->depth : 4, c->cx, c->tile_x, c->tile_y, 0};
        if (!config_fits(e, t)) return set_error(LF2_ERR_UNSUPPORTED, "configuration does not fit every member");
        return set_config(e, t);
    }
    free_runs(e);
    e->tblock = false;
    return LF2_OK;
}

lf2_status lf2_ensemble_run(lf2_ensemble e, int nsteps, void *stream) {
    if (!e) return set_error(LF2_ERR_INVALID, "ensemble is NULL");
    if (nsteps < 0) return set_error(LF2_ERR_INVALID, "nsteps must be >= 0");
    if (nsteps == 0) return LF2_OK;
    const std::vector<int> sig = signature_of(e);
    CapturedRun *run = nullptr;
    for (CapturedRun &r : e->runs)
        if (r.nsteps == nsteps && r.signature == sig) run = &r;
    if (!run) {
        CapturedRun r;
        r.nsteps = nsteps;
        r.signature = sig;
        lf2_status st = upload_members(e, &r.d_members);
        if (st != LF2_OK) return st;
        cudaGraph_t graph = nullptr;
        cudaError_t err = cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) {
            cudaFree(r.d_members);
            return cuda_error(err, "begin capture");
        }
        st = enqueue_run(e, nsteps, r.d_members, e->capture);
        err = cudaStreamEndCapture(e->capture, &graph);
        if (st == LF2_OK && err == cudaSuccess) err = cudaGraphInstantiate(&r.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st != LF2_OK || err != cudaSuccess) {
            cudaFree(r.d_members);
            return st != LF2_OK ? st : cuda_error(err, "capture ensemble run");
        }
        if (e->runs.size() >= 4) {  // keep a few captured runs
            cudaGraphExecDestroy(e->runs.front().exec);
            cudaFree(e->runs.front().d_members);
            e->runs.erase(e->runs.begin());
        }
        e->runs.push_back(r);
        run = &e->runs.back();
    }
    cudaError_t err = cudaGraphLaunch(run->exec, (cudaStream_t)stream);
    if (err != cudaSuccess) return cuda_error(err, "graph launch");
    advance_fronts(e, nsteps);
    return LF2_OK;
}

lf2_status lf2_ensemble_tune(lf2_ensemble e, int flags, lf2_step_config *chosen, void *stream) {
    (void)flags;
    if (!e) return set_error(LF2_ERR_INVALID, "ensemble is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // Time candidate configurations on a copy of the ensemble (fields cloned), so the members'
    // state is untouched.
    std::vector<lf2_lattice> lats;
    std::vector<lf2_field> cphi, cpi;
    lf2_status st = LF2_OK;
    for (int m = 0; m < e->n && st == LF2_OK; ++m) {
        lf2_lattice l = nullptr;
        lf2_field a = nullptr, b = nullptr;
        st = lf2_lattice_create(3, e->phi[m]->lat->n, 1, &l);
        if (st == LF2_OK) st = lf2_field_alloc(l, e->ncomp, e->prec, &a);
        if (st == LF2_OK) st = lf2_field_alloc(l, e->ncomp, e->prec, &b);
        if (l) lats.push_back(l);
        if (a) cphi.push_back(a);
        if (b) cpi.push_back(b);
        if (st == LF2_OK) {
            const size_t bytes = (size_t)e->phi[m]->count * e->phi[m]->esize;
            cudaMemcpyAsync(a->val[0], e->phi[m]->val[e->phi[m]->front], bytes, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(b->val[0], e->pi[m]->val[e->pi[m]->front], bytes, cudaMemcpyDeviceToDevice, s);
        }
    }
    lf2_ensemble clone = nullptr;
    if (st == LF2_OK) st = lf2_ensemble_create(e->n, cphi.data(), cpi.data(), e->params.data(), &clone);
    TbConfig best = e->cfg;
    bool best_tb = e->tblock;
    float best_ms = -1.0f;
    if (st == LF2_OK) {
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        std::vector<TbConfig> cands;
        for (int depth : {2, 3, 4, 6, 8})
            for (int cx : {1, 2, 4}) {
                const int tp = ((depth + cx - 1) / cx) * cx;
                for (int rxt : {16, 32})
                    for (int ty : {8, 16, 24}) {
                        const int tx = rxt * cx - 2 * tp;
                        if (tx >= cx && rxt * (ty + 2 * depth) <= 512) cands.push_back(TbConfig{depth, cx, tx, ty, 0});
                    }
            }
        cands.push_back(TbConfig{0, 0, 0, 0, 0});  // one-step kernels only
        for (const TbConfig &c : cands) {
            if (c.depth) {
                if (!config_fits(clone, c) || set_config(clone, c) != LF2_OK) continue;
            } else {
                free_runs(clone);
                clone->tblock = false;
            }
            const int steps = 24;
            if (lf2_ensemble_run(clone, steps, stream) != LF2_OK) continue;  // capture + warm-up
            float ms = -1.0f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(t0, s);
                if (lf2_ensemble_run(clone, steps, stream) != LF2_OK) break;
                cudaEventRecord(t1, s);
                if (cudaEventSynchronize(t1) != cudaSuccess) break;
                float t = 0.0f;
                cudaEventElapsedTime(&t, t0, t1);
                if (ms < 0.0f || t < ms) ms = t;
            }
            if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                best = c;
                best_tb = c.depth != 0;
            }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    if (clone) lf2_ensemble_destroy(clone);
    for (lf2_field f : cphi) lf2_field_free(f);
    for (lf2_field f : cpi) lf2_field_free(f);
    for (lf2_lattice l : lats) lf2_lattice_destroy(l);
    if (st != LF2_OK) return st;
    if (best_ms < 0.0f) return set_error(LF2_ERR_UNSUPPORTED, "no configuration ran on this ensemble");
    if (best_tb) {
        st = set_config(e, best);
        if (st != LF2_OK) return st;
    } else {
        free_runs(e);
        e->tblock = false;
    }
    if (chosen) {
        if (best_tb)
            *chosen = lf2_step_config{LF2_KERNEL_TBLOCK, best.tile_x, best.tile_y, 0, best.depth, best.cx};
        else
            *chosen = lf2_step_config{LF2_KERNEL_STREAM, 0, 0, 0, 0, 0};
    }
    return LF2_OK;
}

}  // extern "C"
