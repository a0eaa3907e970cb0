/*
 * lf2.h -- C ABI of liblf2, a GB300 (sm_103a) implementation of the leapfrog evolution of a
 * classical scalar field on a periodic 3-D cartesian lattice, following the Lattice / Field /
 * Site / updateHalo model of LATfield2 (Daverio, Hindmarsh & Bevis, arXiv:1508.05610).
 *
 * The method (the paper describes the data model; the equation of motion is the standard one
 * for the classical field simulations the library was written for, Sec. 1 and Sec. 5):
 *
 *   field      phi_a(x), a = 0 .. ncomp-1 (ncomp = 1: real, 2: complex as two reals,
 *              up to LF2_MAX_COMP: an O(N)-symmetric N-component field)
 *   potential  V = lambda/4 (sum_b phi_b^2 - eta^2)^2 + m2/2 sum_a phi_a^2
 *   force      F_a(x) = (1/dx^2) sum_{i=0..2} [phi_a(x+i) + phi_a(x-i) - 2 phi_a(x)]
 *                       - lambda phi_a (sum_b phi_b^2 - eta^2) - m2 phi_a
 *              (the 7-point Laplacian built from the Site neighbours x+i, x-i, Sec. 3.4)
 *   leapfrog   pi_{n+1/2} = pi_{n-1/2} + dt F(phi_n);   phi_{n+1} = phi_n + dt pi_{n+1/2}
 *              (staggered: pi lives at half steps; one force evaluation per step)
 *   start      pi_{-1/2} = pi_0 - (dt/2) F(phi_0)
 *
 * Boundary conditions are periodic, the only ones LATfield2 has (Sec. 3.2, Sec. 3.3.1): the
 * lattice is a torus.  LATfield2 stores a halo of h sites around the local block and fills it
 * with updateHalo(); on one GPU the same periodic images are read in-kernel by wrapped
 * indexing, so no halo is stored and lf2_field_update_halo() only validates its argument.
 *
 * Memory layout of every field buffer (device and host): row-major with x (dimension 0)
 * fastest, then y, then z, and the ncomp components of a site next to each other -- the
 * Site order and the per-site component lists of the paper's binary files (Sec. 3.4, 3.5).
 * Element (x, y, z, a) is at offset ((z * Ny + y) * Nx + x) * ncomp + a.
 *
 * Precisions:
 *   LF2_F64        phi, pi in double; all arithmetic in double.
 *   LF2_F32_KAHAN  phi, pi in float; the drift phi += dt pi is Kahan-compensated with a
 *                  per-site float compensation term owned by the phi field; energies and
 *                  checksums are accumulated in double.
 *   LF2_F32        phi, pi in float with an uncompensated drift (ablation).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an lf2_status; LF2_OK is 0.  No C++ exception crosses the ABI.
 *   - On error the output handle is left untouched and lf2_last_error() returns a
 *     human-readable message for the calling thread.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *     Calls enqueue work on the stream and return without waiting unless stated otherwise.
 *   - Handles are opaque and owned by the caller, who frees them with the matching
 *     destroy/free call.  Handles are not thread-safe; use one handle from one thread at a time.
 *   - All device memory belongs to the current CUDA device at creation time.
 */
#ifndef LF2_H
#define LF2_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LF2_OK = 0,
    LF2_ERR_INVALID = 1,     /* bad argument: NULL pointer, size, mismatched fields ... */
    LF2_ERR_UNSUPPORTED = 2, /* valid in the paper's model but not built here (dim != 3, ncomp > 6),
                              * or a kernel variant that cannot run this shape (lf2_leapfrog_ex) */
    LF2_ERR_NOMEM = 3,       /* a device or host allocation failed */
    LF2_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    LF2_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (reported by lf2_field_check) */
    LF2_ERR_STATE = 6        /* call not allowed in the object's current state */
} lf2_status;

typedef enum { LF2_F64 = 0, LF2_F32_KAHAN = 1, LF2_F32 = 2 } lf2_precision;

/* Most components a field may have.  1 and 2 run on every kernel.  3, 4 and 6 run on the
 * one-thread-per-site and the one-step streaming kernels in every precision, and on the
 * temporal-blocking kernel in FP32 storage (depth 2-4; 2 for 6 components).  5 runs on the
 * one-thread-per-site kernel only. */
#define LF2_MAX_COMP 6

typedef struct lf2_lattice_s *lf2_lattice;
typedef struct lf2_field_s *lf2_field;
typedef struct lf2_ensemble_s *lf2_ensemble;

/* Model and integrator parameters (double for every precision; converted once per call). */
typedef struct {
    double dx;     /* lattice spacing, > 0 */
    double dt;     /* time step; may be negative (time reversal) */
    double lambda; /* quartic coupling */
    double eta;    /* vacuum expectation value */
    double m2;     /* mass term m^2 (0 for the pure phi^4 potential) */
} lf2_params;

/* Energy and checksums at integer step n (see lf2_energy).  All values are FP64. */
typedef struct {
    double kinetic;   /* dx^3 sum_x 1/2 sum_a pi_{a,n}^2 */
    double gradient;  /* dx^3 sum_x sum_a sum_i (phi_a(x+i) - phi_a(x))^2 / (2 dx^2) */
    double potential; /* dx^3 sum_x V(phi(x)) */
    double total;     /* kinetic + gradient + potential */
    double sum[LF2_MAX_COMP];    /* sum_x phi_a(x) per component (unused entries 0) */
    double sum_sq[LF2_MAX_COMP]; /* sum_x phi_a(x)^2 per component (unused entries 0) */
} lf2_energy_t;

/* Kernel selection for lf2_leapfrog_ex.  Every variant computes bitwise the same result. */
typedef enum {
    LF2_KERNEL_AUTO = 0,     /* tuned choice (the one lf2_leapfrog uses) */
    LF2_KERNEL_SITE = 1,     /* one thread per site, any lattice shape */
    LF2_KERNEL_STREAM = 2,   /* x-y tile streaming along z, one step per pass */
    LF2_KERNEL_TBLOCK = 3    /* temporal blocking: `depth` steps per pass */
} lf2_kernel;

typedef struct {
    int kernel; /* lf2_kernel */
    int tile_x; /* output sites of the x-y tile along x (TBLOCK); 0 = default */
    int tile_y; /* rows of the x-y tile (STREAM, TBLOCK); 0 = default */
    int zchunk; /* z-planes per block (STREAM, TBLOCK); 0 = default */
    int depth;  /* temporal-blocking depth, steps fused per pass: 2, 3, 4, 6 or 8 (TBLOCK); 0 = 4 */
    int cx;     /* adjacent x-columns per thread, 1, 2 or 4 (TBLOCK; 4 for real FP32 fields); 0 = default */
    int cluster; /* TBLOCK, FP32 storage, 1 or 2 components: CTAs per tile, 2, 4 or 8, one thread-block
                  * cluster that splits the tile's tile_y + 2 depth region rows into equal bands and
                  * exchanges the bands' edge rows through distributed shared memory (Blackwell);
                  * 0 or 1 = one CTA per tile */
} lf2_step_config;

/* ---------------------------------------------------------------------- lattice */

/* Lattice(dim, sizes, h) of Sec. 3.2: a dim-dimensional periodic cartesian lattice with
 * sizes[0..dim) sites per dimension (sizes[0] is x, the fastest) and a halo of `halo` sites.
 * Returns LF2_ERR_UNSUPPORTED for dim != 3 (the paper allows dim >= 2; this build is 3-D),
 * LF2_ERR_INVALID for halo < 1, any size < 1, or more than 2^40 sites.  The halo width is
 * recorded for fidelity with the paper's model; the 7-point stencil needs 1. */
lf2_status lf2_lattice_create(int dim, const int *sizes, int halo, lf2_lattice *out);

/* Frees the lattice.  LF2_ERR_STATE while any field or ensemble still uses it. */
lf2_status lf2_lattice_destroy(lf2_lattice lat);

/* Number of sites Nx*Ny*Nz. */
lf2_status lf2_lattice_sites(lf2_lattice lat, long long *out);

/* ------------------------------------------------------------------------ field */

/* Field<T>(lat, comp) of Sec. 3.3: allocates one device buffer of sites*ncomp elements of
 * the precision's storage type, zero-filled.  1 <= ncomp <= LF2_MAX_COMP
 * (LF2_ERR_UNSUPPORTED above).  A field used as phi by lf2_leapfrog also gets a back buffer and, for
 * LF2_F32_KAHAN, a zeroed float compensation buffer; they are allocated by
 * lf2_leapfrog_init or, failing that, by the first lf2_leapfrog on the field -- before any
 * stream capture.  The library owns these buffers. */
lf2_status lf2_field_alloc(lf2_lattice lat, int ncomp, lf2_precision prec, lf2_field *out);

/* Like lf2_field_alloc, but the buffers are borrowed from the caller (for example torch
 * tensors), who must keep them alive and contiguous until lf2_field_free.  dev_ptrs[0] is
 * the value buffer; dev_ptrs[1] (optional) the back buffer; dev_ptrs[2] and dev_ptrs[3]
 * (optional, LF2_F32_KAHAN only) the float compensation buffer and its back buffer.  nptrs is
 * 1 to 4.  Every pointer must be 16-byte aligned.  Buffers not given are allocated by the
 * library when first needed (temporal blocking needs back buffers for pi and the compensation
 * as well as for phi). */
lf2_status lf2_field_wrap(lf2_lattice lat, int ncomp, lf2_precision prec, void *const *dev_ptrs,
                          int nptrs, lf2_field *out);

/* Frees the field and every buffer the library allocated for it.  LF2_ERR_STATE (nothing
 * freed) while the field is a member of an ensemble. */
lf2_status lf2_field_free(lf2_field f);

/* Device address of one of the field's buffers: which = 0 the current value buffer, 1 the
 * back buffer, 2 the current compensation buffer, 3 its back buffer.  Front and back swap
 * as the leapfrog runs (phi's every step; pi's and the compensation's after each
 * temporal-blocking pass), so ask again after each call.  *out is NULL if that buffer does
 * not exist. */
lf2_status lf2_field_buffer(lf2_field f, int which, void **out);

/* Copies sites*ncomp doubles from host memory (the layout above) into the field, converting
 * to the storage precision on the device; for LF2_F32_KAHAN the compensation is reset to 0.
 * Returns after the host buffer may be reused (the call synchronises `stream`). */
lf2_status lf2_field_upload(lf2_field f, const double *host, void *stream);

/* Copies the field's current values to sites*ncomp host doubles; synchronises `stream`. */
lf2_status lf2_field_download(lf2_field f, double *host, void *stream);

/* Binary snapshot in LATfield2's write/read format (Sec. 3.5): one file, no header, sites in
 * row-major order with each site's components together.  Elements are written in the field's
 * storage type (double for LF2_F64, float otherwise), so a snapshot is exact.  which = 0
 * writes the current values, which = 2 the Kahan compensation of an LF2_F32_KAHAN phi field.
 * Synchronises `stream`; LF2_ERR_INVALID on I/O errors (message in lf2_last_error). */
lf2_status lf2_field_write(lf2_field f, int which, const char *path, void *stream);

/* Reads a snapshot written by lf2_field_write (or any file of that layout and element type)
 * into the current values (which = 0) or the compensation (which = 2).  The file size must
 * match the field exactly (else LF2_ERR_INVALID before anything is copied).  Reading values
 * resets the compensation to zero; read the compensation afterwards for an exact restart.
 * A read error part-way (LF2_ERR_INVALID for a short read, LF2_ERR_CUDA for a copy) leaves
 * the buffer partly overwritten.  Synchronises `stream`. */
lf2_status lf2_field_read(lf2_field f, int which, const char *path, void *stream);

/* The first-order symmetric difference along dimension dim (0 = x, 1 = y, 2 = z), the
 * paper's example of Site neighbours (Sec. 3.4) and the field operation of its benchmarks
 * (Sec. 4.2): dst_a(x) = (src_a(x + dim) - src_a(x - dim)) / (2 dx) for every component, with
 * periodic wrap.  src and dst: same lattice, components and precision, different fields.
 * Computed in the storage precision. */
lf2_status lf2_field_derivative(lf2_field src, lf2_field dst, int dim, double dx, void *stream);

/* Binned power spectrum of component `comp` of a field on a cubic N^3 lattice (the paper's
 * FFT is for cubic lattices, Sec. 3.6): P(k) = |phi~(k)|^2 / N^3 with phi~(k) = sum_x phi(x)
 * exp(-i k.x), k_i = 2 pi m_i / (N dx); comp = -1 sums the components' powers,
 * sum_a |phi~_a(k)|^2 / N^3 (for a complex field, in every shell the mean of |FFT(phi_0 + i phi_1)|^2
 * / N^3, since the cross terms cancel between k and -k).  Mode (m_x, m_y, m_z) (signed integer frequencies)
 * belongs to shell b = floor(sqrt(m_x^2 + m_y^2 + m_z^2)); shells b < nbins (<= 1024) are
 * returned as host arrays of nbins doubles: mean power, mean |k|, mode count.  The transform is
 * cuFFT (single or double precision after the storage type); buffers and the plan are
 * allocated per call.  LF2_ERR_UNSUPPORTED for non-cubic lattices.  Synchronises `stream`. */
lf2_status lf2_power_spectrum(lf2_field f, int comp, int nbins, double dx, double *power, double *kmean,
                              double *count, void *stream);

/* updateHalo() of Sec. 3.3.1.  The GPU kernels read periodic images by wrapped indexing,
 * so there is no stored halo to refresh: this validates the handle and returns LF2_OK. */
lf2_status lf2_field_update_halo(lf2_field f, void *stream);

/* -------------------------------------------------------------------- leapfrog */

/* Start of the staggered leapfrog: pi <- pi - (dt/2) F(phi), turning pi_0 into pi_{-1/2}.
 * The paper (Sec. 1, Sec. 5) evolves classical fields but prints no integrator; the scheme
 * taken here is the staggered kick-drift leapfrog (velocity Verlet with its two half kicks of
 * consecutive steps merged): pi lives at half steps, one force evaluation per step, and this
 * half kick starts it.  The force F is the 7-point Laplacian of the Site neighbours x+i, x-i
 * (Sec. 3.4) minus dV/dphi_a, the equation of motion of the Lagrangian
 * 1/2 sum_a (d phi_a)^2 - V.
 * phi and pi must share the lattice, ncomp and precision.  Also allocates phi's back and
 * compensation buffers if missing (so that later lf2_leapfrog calls allocate nothing). */
lf2_status lf2_leapfrog_init(lf2_field phi, lf2_field pi, const lf2_params *p, void *stream);

/* nsteps >= 0 leapfrog steps of the staggered kick-drift scheme above (kick
 * pi_{n+1/2} = pi_{n-1/2} + dt F(phi_n), then drift phi_{n+1} = phi_n + dt pi_{n+1/2}, every
 * site reading the old phi_n; LF2_F32_KAHAN compensates the drift's rounding with the per-site
 * term c: y = dt pi - c, t = phi + y, c = (t - phi) - y, phi = t).
 * On entry phi holds phi_n and pi holds pi_{n-1/2}; on return
 * phi holds phi_{n+nsteps} and pi holds pi_{n+nsteps-1/2}.  phi's front and back buffers swap
 * after each step (no copy).  Uses the tuned kernel of lf2_tune when one was chosen for this
 * shape, else the default one; results are bitwise identical whichever kernel runs.  The
 * environment variable LF2_TUNE changes that: "off" ignores tuned plans, "force" tunes a shape
 * that has no plan on its first call (that call synchronises and allocates, so keep it out of
 * stream capture). */
lf2_status lf2_leapfrog(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps, void *stream);

/* lf2_leapfrog with an explicit kernel choice (testing and tuning).  LF2_ERR_UNSUPPORTED if the
 * chosen kernel cannot run this lattice (for example x rows not a multiple of 16 bytes). */
lf2_status lf2_leapfrog_ex(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps,
                           const lf2_step_config *cfg, void *stream);

/* Energy and checksums at integer step n from phi_n and pi_{n-1/2}: the synchronised momentum
 * pi_n = pi_{n-1/2} + (dt/2) F(phi_n) is formed on the fly (the staggered scheme keeps pi at
 * half steps, so the energy of an integer step needs it).  The paper prints no energy; the one
 * taken is E = dx^3 sum_x [1/2 sum_a pi_{a,n}^2 + 1/(2 dx^2) sum_a sum_i (phi_a(x+i) - phi_a(x))^2
 * + V(phi(x))], with forward differences along the Site neighbours x+i (Sec. 3.4): the gradient
 * energy whose variation is exactly the 7-point Laplacian of the force, so that E is the
 * quantity the leapfrog conserves to O(dt^2).  Accumulates in FP64 for every
 * precision, with a fixed reduction order (bitwise reproducible).  Writes *out and
 * synchronises `stream`. */
lf2_status lf2_energy(lf2_field phi, lf2_field pi, const lf2_params *p, lf2_energy_t *out, void *stream);

/* lf2_energy without synchronising: enqueues the reduction on `stream` and writes one
 * lf2_energy_t record (16 doubles, same layout) to the device memory at dev_out.  Allocates
 * nothing and never waits, so step and energy calls can be captured together into a CUDA
 * graph (for example a run with energies every step).  Uses the scratch that
 * lf2_leapfrog_init or a first lf2_energy allocated on phi (LF2_ERR_STATE before that).
 * Calls on one phi field share that scratch: order them on one stream. */
lf2_status lf2_energy_device(lf2_field phi, lf2_field pi, const lf2_params *p, double *dev_out, void *stream);

/* Advances nsteps exactly as lf2_leapfrog does (bitwise the same fields) and writes, for
 * k = 0 .. nsteps-1, the energy record of the state at the start of step k (phi_k and the
 * synchronised pi_k, as lf2_energy defines them) to dev_records + 16 k: nsteps lf2_energy_t
 * records in device memory, caller-owned.  The paper's programs report diagnostics every step;
 * here each step reads the stencil once for both the energy and the update (kick and drift),
 * visiting the sites in the order and with the arithmetic of lf2_energy, so each record is
 * bitwise the one lf2_energy_device gives for that state.  Meant for runs with an energy every
 * step: the kernel is the one-thread-per-site one, not the tiled kernels of lf2_leapfrog.
 * A lattice of at most 303 x 256 sites runs all nsteps (>= 2) in one cooperative launch with a
 * grid barrier between steps; larger ones run one launch per step.  Results are the same bits
 * either way.  A barrier that does not complete within about a second (all blocks of a
 * cooperative launch are resident, so it always completes) ends the run and leaves NaN in the
 * records from the step before that barrier on (a step's record is finished during the next
 * step); lf2_field_check(phi) then returns LF2_ERR_TIMEOUT.  Enqueues on `stream` without waiting; after the first call on phi (which may
 * allocate its back buffer and energy scratch, so make it outside a stream capture) calls
 * allocate nothing and can be captured into a CUDA graph.  Calls on one phi share its energy
 * scratch with lf2_energy and lf2_energy_device: order them on one stream.
 * LF2_ERR_INVALID for nsteps < 0 or dev_records NULL with nsteps > 0. */
lf2_status lf2_leapfrog_energy(lf2_field phi, lf2_field pi, const lf2_params *p, int nsteps, double *dev_records,
                               void *stream);

/* Error norms of a field against a reference array: the stated error of an FP32 run against
 * the FP64 run of the same state (the paper has no counterpart).  Compares buffer `which` of
 * f (as lf2_field_buffer: 0 = current value, 2 = current compensation) element by element
 * with `ref`: sites*ncomp values of precision ref_prec (LF2_F64 for doubles, LF2_F32 or
 * LF2_F32_KAHAN for floats) in the same layout, device memory, caller-owned.  Writes
 *   out[0] = max |f - ref|,  out[1] = max |ref|,  out[2] = sum (f - ref)^2,  out[3] = sum ref^2
 * (4 doubles, host), computed in FP64 on the device in a fixed order (bitwise reproducible);
 * a NaN in either operand makes out[0] NaN.  Uses f's energy scratch (order calls on one
 * stream, as for lf2_energy) and synchronises `stream`.  LF2_ERR_INVALID for NULL arguments,
 * `which` outside 0..3 or an unknown ref_prec; LF2_ERR_STATE if that buffer does not exist. */
lf2_status lf2_field_compare(lf2_field f, int which, const void *ref, lf2_precision ref_prec, double *out,
                             void *stream);

/* Status of the last multi-step lf2_leapfrog_energy run on phi: LF2_ERR_TIMEOUT (once; the
 * flag is then cleared) if one of its grid barriers gave up, else LF2_OK.  The paper has no
 * counterpart (its programs have no device-side waits).  Synchronises `stream`.  Host-side
 * failure injection for tests: with LF2_FAULT=timeout in the environment the barrier waits give
 * up at once; with LF2_FAULT=launch, lf2_leapfrog and lf2_leapfrog_energy return LF2_ERR_CUDA
 * without launching; with LF2_FAULT=alloc, the library's allocations fail with LF2_ERR_NOMEM. */
lf2_status lf2_field_check(lf2_field phi, void *stream);

/* Index checks of a debug build, an aid for the kernels' index arithmetic (the paper has no
 * counterpart).  The library built with -DLF2_DEBUG_BOUNDS
 * (lib/liblf2_debug.so) checks every element index the leapfrog, temporal-blocking, ensemble
 * and energy kernels compute against its allocation, replaces an index outside by a safe one
 * and counts it.  Writes the count since the last reset to *violations (reset != 0 clears it);
 * synchronises the device.  The release library returns LF2_ERR_UNSUPPORTED (*violations = 0). */
lf2_status lf2_debug_bounds(unsigned long long *violations, int reset);

/* lf2_energy for callers that cannot allocate device memory.  The paper has no counterpart;
 * this entry point exists for callers whose device allocator belongs to someone else (a memory
 * pool or host framework that forbids cudaMalloc while it runs) or that must make no
 * allocation call at all.  lf2_energy allocates scratch and a pinned result buffer on its
 * first call for a field; this variant allocates nothing: no cudaMalloc, cudaFree, pinned-host
 * or library allocation.  Its scratch is one fixed array inside the library (608 x 16 + 17
 * doubles, 78 KB) that every GPU which loads the library holds until the process exits.  The
 * reduction uses at most 608 blocks whatever the lattice, so every lattice the library accepts
 * fits (the library checks the array's layout when it is compiled); there is no size to
 * reject.  The first call on a device looks up the array's device address (make it before any
 * stream capture).  All calls share the array: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race and must be serialised by the caller.  Each call
 * first clears the array's finished-block counter on its stream, so an overlap spoils only the
 * overlapping calls' results, not later ones.  Arguments, result and synchronisation are those
 * of lf2_energy; the result is copied into *out. */
lf2_status lf2_energy_noalloc(lf2_field phi, lf2_field pi, const lf2_params *p, lf2_energy_t *out, void *stream);

/* -------------------------------------------------------------------- ensembles */

/* Groups n >= 1 independent (phi, pi) pairs -- one precision and component count, any
 * lattice sizes, per-member parameters -- into a batched ensemble.  The paper runs many
 * independent fields only as separate programs; here they share every kernel launch.
 * Allocates the members' back buffers (temporal blocking needs them) and device tables.
 * Until lf2_ensemble_destroy the fields cannot be freed or put into another ensemble, and
 * their lattices cannot be destroyed (each returns LF2_ERR_STATE). */
lf2_status lf2_ensemble_create(int n, const lf2_field *phis, const lf2_field *pis, const lf2_params *per_lattice,
                               lf2_ensemble *out);

/* Advances every member by nsteps (each member's phi_n / pi_{n-1/2} convention as in
 * lf2_leapfrog) with ONE CUDA-graph launch on `stream`: nsteps/depth temporal-blocking passes,
 * each a persistent kernel over a work list of (member, tile, z-chunk) items ordered longest
 * first, then the leftover single steps.  The graph is captured on first use for a given
 * nsteps and buffer state (this first call must not itself be inside a stream capture) and
 * relaunched afterwards.  Results are bitwise those of running each member alone. */
lf2_status lf2_ensemble_run(lf2_ensemble e, int nsteps, void *stream);

/* Chooses the ensemble's pass configuration (depth, cx, tile) by timing candidates on a
 * clone of the ensemble (members untouched); allocates the clone; synchronises `stream`. */
lf2_status lf2_ensemble_tune(lf2_ensemble e, int flags, lf2_step_config *chosen, void *stream);

/* Sets the pass configuration explicitly (kernel LF2_KERNEL_TBLOCK with depth/cx/tile_x/
 * tile_y, or any other kernel for one-step passes).  LF2_ERR_UNSUPPORTED if it does not fit
 * every member. */
lf2_status lf2_ensemble_set_config(lf2_ensemble e, const lf2_step_config *c);

/* Frees the ensemble's graphs and tables (not the member fields). */
lf2_status lf2_ensemble_destroy(lf2_ensemble e);

/* -------------------------------------------------------------------- autotuner */

/* lf2_tune flags */
#define LF2_TUNE_FORCE 1    /* re-tune even if a plan for this shape is cached */
#define LF2_TUNE_ONE_STEP 2 /* only one-step kernels (no temporal blocking) */

/* Picks the fastest kernel configuration for phi's lattice shape, component count and
 * precision by timing candidates (one-step streaming tiles; temporal blocking of depth 2-8
 * with several tiles and column widths) on a proxy lattice of the same x-y plane and at most
 * 256 z-planes (fewer for very large planes, to stay within about 8 GB), filled with a copy
 * of the fields' first planes -- phi and pi are not modified.
 * The plan is cached per process (and appended to the file named by the environment variable
 * LF2_TUNE_CACHE, which is read on first use) and used by every later lf2_leapfrog on a lattice
 * of that shape.  Results do not depend on the plan: all variants are bitwise identical.
 * Allocates the proxy fields and synchronises `stream`; call it before any stream capture.
 * *chosen (may be NULL) receives the plan. */
lf2_status lf2_tune(lf2_field phi, lf2_field pi, const lf2_params *p, int flags, lf2_step_config *chosen,
                    void *stream);

/* The cached plan for sizes[3] / ncomp / prec; LF2_ERR_STATE if none was tuned. */
lf2_status lf2_tune_lookup(const int *sizes, int ncomp, lf2_precision prec, lf2_step_config *out);

/* ------------------------------------------------------------------- utilities */

const char *lf2_status_string(lf2_status s);

/* Message of the last failed call on this thread ("" if none). */
const char *lf2_last_error(void);

/* Library version string. */
const char *lf2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LF2_H */
