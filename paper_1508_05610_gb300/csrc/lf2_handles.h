// lf2_handles.h -- host-side definitions of the opaque handles of the C ABI (lattice, field,
// ensemble) and small helpers shared by the API, tuner and ensemble sources.
#pragma once

#include <atomic>
#include <string>

#include "lf2_internal.cuh"

struct lf2_lattice_s {
    int dim;
    int n[3];
    int halo;
    long long sites;
    std::atomic<int> users{0};  // fields and ensembles still attached
};

struct lf2_field_s {
    lf2_lattice lat = nullptr;
    int ncomp = 0;
    lf2_precision prec = LF2_F64;
    size_t esize = 0;  // bytes per stored element
    long long count = 0;  // sites * ncomp
    void *val[2] = {nullptr, nullptr};  // value buffers; val[front] is current
    bool own_val[2] = {false, false};
    int front = 0;
    float *comp[2] = {nullptr, nullptr};  // Kahan compensation of phi (F32_KAHAN); comp[cfront] current
    bool own_comp[2] = {false, false};
    int cfront = 0;
    double *energy_scratch = nullptr;  // kFieldScratchDoubles: partial rows, record, counter, multi-step rows (device)
    double *energy_host = nullptr;     // one pinned lf2_energy_t
    lf2_ensemble ensemble = nullptr;   // the ensemble this field is a member of, if any
};

namespace lf2 {

// Sets the calling thread's last-error message and returns `s`.
lf2_status set_error(lf2_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
lf2_status cuda_error(cudaError_t e, const char *what);

// Host-side switches (lf2_api.cu): LF2_FAULT=<what> injects a failure; LF2_TUNE picks how
// lf2_leapfrog uses tuned plans.
bool fault_injected(const char *what);
enum class TuneMode { Off, On, Force };
TuneMode tune_mode();

// Field helpers (lf2_api.cu).
lf2_status ensure_dynamic(lf2_field phi, cudaStream_t s);               // phi back buffer (+ compensation)
lf2_status ensure_tblock(lf2_field phi, lf2_field pi, cudaStream_t s);  // + pi and compensation back buffers
StepArgs step_args(lf2_field phi, lf2_field pi, const lf2_params *p, double dt, bool drift);
TbArgs tb_args(lf2_field phi, lf2_field pi, const lf2_params *p);

// Tuned kernel plan for a lattice shape (filled by lf2_tune); false if none.
bool plan_lookup(const int n[3], int ncomp, lf2_precision prec, lf2_step_config *out);

inline Geom geom_of(const lf2_lattice_s *lat) { return Geom{lat->n[0], lat->n[1], lat->n[2], lat->sites}; }

}  // namespace lf2
