// lf2_internal.cuh -- launcher declarations and host-side types shared by the sources of
// liblf2; the device arithmetic the kernels compile lives in lf2_arith.cuh.
#pragma once

#include "lf2_arith.cuh"

namespace lf2 {

// ------------------------------------------------------------------ host launchers
// Arguments of one leapfrog pass over a lattice.
struct StepArgs {
    const void *phi;  // phi_n (storage type of prec)
    void *phi_out;    // phi_{n+1} (not touched by a kick-only pass)
    void *pi;         // updated in place
    float *comp;      // Kahan compensation (F32_KAHAN), updated in place
    Geom g;
    int ncomp;
    lf2_precision prec;
    lf2_params p;
    double dt;        // time step of this pass (the half-kick uses -dt/2)
    bool drift;       // false: kick only
};

cudaError_t launch_site_step(const StepArgs &a, cudaStream_t s);

// Streaming kernel (x-y tile, z-streaming); returns cudaErrorNotSupported when the shape
// does not fit its constraints.
bool stream_supported(const StepArgs &a, int tile_y, int zchunk);
cudaError_t launch_stream_step(const StepArgs &a, int tile_y, int zchunk, int nsteps_hint, cudaStream_t s);

// Multiprocessors of the current device (queried once per device, then cached); grid sizes
// and the temporal-blocking wave model are derived from it.
int device_sm_count();

// Energy reduction scratch (device, kEnergyScratchDoubles doubles): one partial row of
// kEnergySlots per block, then the record row (an lf2_energy_t), then an unsigned counter of
// finished blocks that must be zero before the first launch (every launch leaves it zero).
// The reduction grid is capped at a fixed 608 blocks (four per SM of a 152-SM GB300) rather
// than at a multiple of the queried SM count: the cap fixes the partial rows, and with them
// the order of the FP64 sums, so a record is the same bits on every device.
constexpr int kEnergyBlocks = 608;
constexpr int kEnergyThreads = 256;
constexpr int kEnergySlots = 16;
constexpr int kEnergyRecordOffset = kEnergyBlocks * kEnergySlots;
constexpr int kEnergyCounterOffset = kEnergyRecordOffset + kEnergySlots;
constexpr int kEnergyScratchDoubles = kEnergyCounterOffset + 1;
static_assert(3 + 2 * kMaxComp <= kEnergySlots, "energy slots");
// The multi-step step + energy kernel keeps, after that layout, three rotating sets of up to
// kEnergyStepsBlocks partial rows and one row of barrier words.  A field's scratch
// (kFieldScratchDoubles doubles) holds both parts; lf2_energy_noalloc's fixed array only the
// first, since it never runs that kernel.
// At most 303 site blocks (two 256-thread blocks per SM of a 152-SM GB300, less the reducing
// block): a size bound of the row sets; the launch itself checks co-residency on the device it
// runs on and falls back to one launch per step where the grid does not fit.
constexpr int kEnergyStepsBlocks = 303;
constexpr int kEnergyStepsRowSets = 3;
constexpr int kStepsRowsOffset = (kEnergyScratchDoubles + kEnergySlots - 1) / kEnergySlots * kEnergySlots;
constexpr int kFieldScratchDoubles = kStepsRowsOffset + (kEnergyStepsRowSets * kEnergyStepsBlocks + 1) * kEnergySlots;
// Energy of (phi, pi) as an lf2_energy_t record: written to scratch + kEnergyRecordOffset and,
// when `record` is not NULL, also to `record` (device).  One launch.
cudaError_t launch_energy(const void *phi, const void *pi, const Geom &g, int ncomp, lf2_precision prec,
                          const lf2_params &p, double *scratch, double *record, cudaStream_t s);
// One leapfrog step (kick + drift, as launch_site_step) that also writes the energy record of
// the state it starts from to `record`, with the site order and reduction of launch_energy, so
// the record is bitwise the one launch_energy gives for that state.  One launch.
cudaError_t launch_step_energy(const StepArgs &a, double *scratch, double *record, cudaStream_t s);
// nsteps such steps in one cooperative launch (grid barriers between steps), writing
// records[0 .. nsteps) and leaving phi in a.phi_out if nsteps is odd, else in a.phi;
// cudaErrorNotSupported (nothing launched) unless the lattice is small enough for every block
// of the reduction grid to be resident at once and nsteps >= 2.  Bitwise the per-step launches.
// no_wait: the grid barrier gives up at once (host-side timeout injection, LF2_FAULT=timeout).
cudaError_t launch_steps_energy(const StepArgs &a, int nsteps, double *scratch, double *records, bool no_wait,
                                cudaStream_t s);
// Whether the last multi-step run on this scratch had a barrier give up (the flag is then
// cleared); synchronises `s`.
cudaError_t steps_energy_timed_out(double *scratch, bool *out, cudaStream_t s);

// Temporal blocking: `depth` fused steps per pass over x-y tiles of tile_x x tile_y output
// sites (plus a depth-site halo), z-chunks of `zchunk` planes.  Unlike the one-step kernels it
// reads phi, pi and the compensation from the front buffers and writes all three to the back
// buffers, because neighbouring tiles read each other's halo columns of pi and comp too.
struct TbArgs {
    const void *phi;
    void *phi_out;
    const void *pi;
    void *pi_out;
    const float *comp;  // F32_KAHAN only
    float *comp_out;
    Geom g;
    int ncomp;
    lf2_precision prec;
    lf2_params p;
    double dt;
};
struct TbConfig {
    int depth, cx, tile_x, tile_y, zchunk;
    int cluster;  // CTAs per tile (a thread-block cluster of bands along y); 0 or 1: one CTA
};
// One member lattice of an ensemble pass (device table entry).  Buffer f ^ 1 is written
// when buffer f = front ^ flip is read.
struct TbMember {
    const void *phi[2];
    const void *pi[2];
    const float *comp[2];
    Geom g;
    Coef32 k32;
    Coef64 k64;
    int zchunk;
    int front;
};
struct TbEnsembleLaunch {
    const TbMember *members;  // device
    const int4 *items;        // device: (member, tile x, tile y, z-chunk), longest chunks first
    int nitems;
    int *counter;             // device: next item, zeroed by the launcher before each pass
    int flip;
    TbConfig c;
    int ncomp;
    lf2_precision prec;
};
cudaError_t launch_tblock_ensemble(const TbEnsembleLaunch &e, cudaStream_t s);

// Whether a clustered temporal-blocking kernel exists for this storage size, component count,
// depth, columns per thread and cluster size (FP32 storage, 1 or 2 components).
bool tblock_cluster_built(int esz, int ncomp, int depth, int cx, int cluster);

// Shape/configuration check; fills defaults for zero fields of `c`.
bool tblock_supported(const TbArgs &a, TbConfig &c);
cudaError_t launch_tblock(const TbArgs &a, const TbConfig &c, cudaStream_t s);

// Writes an lf2_energy_t-shaped record (16 doubles) from a result row to device memory.
static_assert(sizeof(lf2_energy_t) == kEnergySlots * sizeof(double), "energy record layout");
// Error norms of n elements a against ref (FP64): max |a - ref|, max |ref|, sum (a - ref)^2,
// sum ref^2, written to scratch + kEnergyRecordOffset (energy scratch layout).  One launch.
cudaError_t launch_compare(const void *a, bool a_double, const void *ref, bool ref_double, long long n,
                           double *scratch, cudaStream_t s);

// Index-check violations counted by each kernel translation unit of a -DLF2_DEBUG_BOUNDS build
// (0 otherwise), optionally reset.
cudaError_t bounds_violations_site(unsigned long long *n, bool reset);
cudaError_t bounds_violations_stream(unsigned long long *n, bool reset);
cudaError_t bounds_violations_tblock_f64(unsigned long long *n, bool reset);
cudaError_t bounds_violations_tblock_f32k(unsigned long long *n, bool reset);
cudaError_t bounds_violations_tblock_f32(unsigned long long *n, bool reset);
cudaError_t bounds_violations_energy(unsigned long long *n, bool reset);

// Fixed-size scratch of lf2_energy_noalloc (kEnergyScratchDoubles doubles, 78 KB).
cudaError_t energy_noalloc_scratch(double **out);

// Conversions between host-side doubles and storage precision.
cudaError_t launch_convert_from_f64(const double *src, void *dst, long long n, lf2_precision prec, cudaStream_t s);
cudaError_t launch_convert_to_f64(const void *src, double *dst, long long n, lf2_precision prec, cudaStream_t s);

// First-order symmetric difference along `dim` into dst (same layout), in storage precision.
cudaError_t launch_derivative(const void *src, void *dst, const Geom &g, int ncomp, lf2_precision prec, int dim,
                              double dx, cudaStream_t s);

}  // namespace lf2
