// lf2_energy.cu -- FP64 energy and checksum reduction (all precisions), alone or fused into a
// leapfrog step.
//
// Energy at integer step n from phi_n and pi_{n-1/2}:
//   pi_n       = pi_{n-1/2} + (dt/2) F(phi_n)          (synchronised momentum: a half kick)
//   kinetic    = sum_x 1/2 sum_a pi_{a,n}^2
//   gradient   = sum_x sum_a sum_i (phi_a(x+i) - phi_a(x))^2 / (2 dx^2)
//                (forward differences: the discrete gradient energy whose variation is the
//                 7-point Laplacian built from the Site neighbours x+i, x-i of Sec. 3.4)
//   potential  = sum_x [lambda/4 (|phi|^2 - eta^2)^2 + m2/2 |phi|^2]
// plus sum_x phi_a and sum_x phi_a^2, all times the volume element dx^3 except the sums.
//
// Each site adds raw sums (pi_n^2, squared differences, (|phi|^2 - eta^2)^2, phi_a, phi_a^2)
// to per-thread FP64 accumulators; the constant factors are applied once to the totals
// (the potential's mass term is m2/2 times the sum of the phi_a^2 totals).  A grid-stride
// pass over sites leaves one partial row per block; the last block to finish (counted with
// an atomic) sums the rows in block order and writes the record.  The grid depends only on
// the lattice and every sum has a fixed order, so the result is bitwise reproducible, and the
// fused step kernels, which visit the sites in the same order with the same per-site
// arithmetic, give bitwise the record of the stand-alone reduction.
#include <mutex>

#include "lf2_bounds.cuh"
#include "lf2_internal.cuh"

namespace lf2 {
namespace {

// Raw sums per thread for NC components: 0 kinetic, 1 gradient, 2 potential, then sum_x phi_a
// (3 + a) and sum_x phi_a^2 (3 + NC + a).  Partial rows in the scratch keep kEnergySlots
// doubles of which the first kNs<NC> are used.
template <int NC>
constexpr int kNs = 3 + 2 * NC;
constexpr int kKin = 0, kGrad = 1, kPot = 2, kSum = 3;

// L2 loads (COHERENT) where other blocks of the same launch wrote the data; the read-only
// path otherwise.  The values are the same either way.
template <bool COHERENT, typename R>
__device__ __forceinline__ R ld_field(const R *p) {
    if constexpr (COHERENT)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Exact FP32 -> FP64 widening on the integer pipe, without a branch.  This GPU converts on its
// FP64 pipe, which the FP64 sums already keep busy: the 8 conversions per component-site of
// FP32 storage made the FP64 energy of FP32 data 1.4x slower than that of FP64 data.  Widening
// re-biases the exponent (bias 127 -> 1023) and moves the 23-bit significand to the top of the
// 52-bit one.  A subnormal (leading bit n places below the implicit one) is first shifted up by
// n and its exponent lowered by n; infinities and NaN keep the all-ones exponent, a NaN comes
// back quiet with its payload; a signed zero keeps only its sign.  The result is the one exact
// double (IEEE 754 widening), so FP64 and FP32 storage of the same values give the same sums.
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) {
    const unsigned u = __float_as_uint(v), mag = u & 0x7fffffffu;
    const int n = max(__clz(mag) - 8, 0);  // 0 for normal numbers, infinities and NaN
    const unsigned m = mag << n;
    unsigned hi = (m >> 3) + ((896u - (unsigned)n) << 20);
    hi += mag >= 0x7f800000u ? 896u << 20 : 0u;
    hi |= mag > 0x7f800000u ? 1u << 19 : 0u;
    hi = (mag ? hi : 0u) | (u & 0x80000000u);
    return __hiloint2double((int)hi, (int)(m << 29));
}

template <typename R, int NC, bool COHERENT = false>
__device__ __forceinline__ void load_d(const R *__restrict__ f, long long s, long long sites, double (&v)[NC]) {
    const long long i = checked(s * NC, NC, sites * NC);
#pragma unroll
    for (int a = 0; a < NC; ++a) v[a] = widen(ld_field<COHERENT>(f + i + a));
}

// Adds one site's raw sums to acc.  c: phi_n at the site, xm..zp: its neighbours in the order
// -x, +x, -y, +y, -z, +z; p: pi_{n-1/2}.  Explicit round-to-nearest operations keep the
// stand-alone and fused kernels bitwise equal; the half kick is the FP64 kick's arithmetic.
template <int NC>
__device__ __forceinline__ void energy_site(const double (&c)[NC], const double (&xm)[NC], const double (&xp)[NC],
                                            const double (&ym)[NC], const double (&yp)[NC], const double (&zm)[NC],
                                            const double (&zp)[NC], const double (&p)[NC], double (&acc)[kNs<NC>],
                                            const CoefE &k) {
    double s2 = __dmul_rn(c[0], c[0]);
#pragma unroll
    for (int b = 1; b < NC; ++b) s2 = __fma_rn(c[b], c[b], s2);
    const double gh = __fma_rn(k.hl, s2, k.hb0);
    const double w = __dsub_rn(s2, k.eta2);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        const double nb = __dadd_rn(__dadd_rn(xm[a], xp[a]), __dadd_rn(__dadd_rn(ym[a], yp[a]), __dadd_rn(zm[a], zp[a])));
        const double pin = __fma_rn(k.ah, nb, __fma_rn(-gh, c[a], p[a]));
        acc[kKin] = __fma_rn(pin, pin, acc[kKin]);
        const double ex = __dsub_rn(xp[a], c[a]), ey = __dsub_rn(yp[a], c[a]), ez = __dsub_rn(zp[a], c[a]);
        acc[kGrad] = __fma_rn(ez, ez, __fma_rn(ey, ey, __fma_rn(ex, ex, acc[kGrad])));
        acc[kSum + a] = __dadd_rn(acc[kSum + a], c[a]);
        acc[kSum + NC + a] = __fma_rn(c[a], c[a], acc[kSum + NC + a]);
    }
    acc[kPot] = __fma_rn(w, w, acc[kPot]);
}

// Block sum of acc, left in sh[j][0].  A pairwise tree whose additions at each level are packed
// onto consecutive threads: an FP64 warp instruction costs the same however few of its lanes
// are active, so the levels with fewer than 32 pairs per sum still fill whole warps.
template <int NS>
__device__ __forceinline__ void block_sum(const double (&acc)[NS], double (&sh)[NS][kEnergyThreads]) {
#pragma unroll
    for (int j = 0; j < NS; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
#pragma unroll
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        for (int t = threadIdx.x; t < NS * w; t += kEnergyThreads) {
            const int j = t / w, i = t % w;
            sh[j][i] = __dadd_rn(sh[j][i], sh[j][i + w]);
        }
        __syncthreads();
    }
}

// Sums `nrows` partial rows (L2 reads, in row order) with the block and writes the record
// (thread 0) to `record` and, when not NULL, to `own`.  All threads of the block take part.
template <int NC>
__device__ __forceinline__ void reduce_rows(const double *rows, int nrows, double (&sh)[kNs<NC>][kEnergyThreads],
                                            const CoefE &k, double *__restrict__ record, double *__restrict__ own) {
    constexpr int NS = kNs<NC>;
    double tot[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) tot[j] = 0.0;
    for (int b = threadIdx.x; b < nrows; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NS; ++j) tot[j] = __dadd_rn(tot[j], __ldcg(rows + (size_t)b * kEnergySlots + j));
    }
    block_sum<NS>(tot, sh);
    if (threadIdx.x == 0) {
        double r[kEnergySlots];
        double ssq = 0.0;
        for (int a = 0; a < NC; ++a) ssq += sh[kSum + NC + a][0];
        r[0] = k.vol * (0.5 * sh[kKin][0]);
        r[1] = k.vol * (0.5 * k.inv_dx2 * sh[kGrad][0]);
        r[2] = k.vol * (0.25 * k.lam * sh[kPot][0] + 0.5 * k.m2 * ssq);
        r[3] = r[0] + r[1] + r[2];
        for (int a = 0; a < kMaxComp; ++a) {
            r[4 + a] = a < NC ? sh[kSum + a][0] : 0.0;
            r[4 + kMaxComp + a] = a < NC ? sh[kSum + NC + a][0] : 0.0;
        }
        for (int j = 0; j < kEnergySlots; ++j) {
            if (own) own[j] = r[j];
            if (record) record[j] = r[j];
        }
    }
}

// End of every energy kernel: stores this block's partial row, and the last block to get here
// sums all rows (in block order) and writes the record.  No block waits for another.
template <int NC>
__device__ __forceinline__ void finish_energy(const double (&acc)[kNs<NC>], double (&sh)[kNs<NC>][kEnergyThreads],
                                              double *__restrict__ scratch, const CoefE &k,
                                              double *__restrict__ record) {
    constexpr int NS = kNs<NC>;
    __shared__ bool s_last;
    block_sum<NS>(acc, sh);
    if (threadIdx.x < NS) scratch[(size_t)blockIdx.x * kEnergySlots + threadIdx.x] = sh[threadIdx.x][0];
    __threadfence();  // this block's row is visible device-wide before the block is counted
    __syncthreads();
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kEnergyCounterOffset);
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // every other block's row is visible to this one
    reduce_rows<NC>(scratch, (int)gridDim.x, sh, k, record, scratch + kEnergyRecordOffset);
    if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch on this scratch
}

// Linear indices of the six periodic neighbours of site s.
struct Nbr {
    long long xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbr neighbours(long long s, const Geom &g) {
    const int x = (int)(s % g.nx);
    const long long r = s / g.nx;
    const int y = (int)(r % g.ny);
    const int z = (int)(r / g.ny);
    const long long row = g.nx, plane = (long long)g.nx * g.ny;
    return Nbr{s - x + wrap_dn(x, g.nx),       s - x + wrap_up(x, g.nx),       s + (wrap_dn(y, g.ny) - y) * row,
               s + (wrap_up(y, g.ny) - y) * row, s + (wrap_dn(z, g.nz) - z) * plane, s + (wrap_up(z, g.nz) - z) * plane};
}

template <typename R, int NC>
__global__ void __launch_bounds__(kEnergyThreads) k_energy(const R *__restrict__ phi, const R *__restrict__ pi, Geom g,
                                                           CoefE k, double *__restrict__ scratch, double *__restrict__ record) {
    __shared__ double sh[kNs<NC>][kEnergyThreads];
    double acc[kNs<NC>];
#pragma unroll
    for (int j = 0; j < kNs<NC>; ++j) acc[j] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride) {
        const Nbr n = neighbours(s, g);
        double c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC];
        load_d<R, NC>(phi, s, g.sites, c);
        load_d<R, NC>(phi, n.xm, g.sites, xm);
        load_d<R, NC>(phi, n.xp, g.sites, xp);
        load_d<R, NC>(phi, n.ym, g.sites, ym);
        load_d<R, NC>(phi, n.yp, g.sites, yp);
        load_d<R, NC>(phi, n.zm, g.sites, zm);
        load_d<R, NC>(phi, n.zp, g.sites, zp);
        load_d<R, NC>(pi, s, g.sites, p);
        energy_site<NC>(c, xm, xp, ym, yp, zm, zp, p, acc, k);
    }
    finish_energy<NC>(acc, sh, scratch, k, record);
}

// One site of a fused step + energy, FP64: adds the energy of (phi_n, pi_{n-1/2}) at site s
// to acc and writes the step to (phi_{n+1}, pi_{n+1/2}), from one read of the site's stencil.
template <int NC, bool COHERENT>
__device__ __forceinline__ void site_step_energy_f64(const double *__restrict__ phi, double *__restrict__ phi_out,
                                                     double *__restrict__ pi, long long s, const Geom &g,
                                                     const Coef64 &k, const CoefE &ke, double (&acc)[kNs<NC>]) {
    const Nbr n = neighbours(s, g);
    double c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], out[NC];
    load_d<double, NC, COHERENT>(phi, s, g.sites, c);
    load_d<double, NC, COHERENT>(phi, n.xm, g.sites, xm);
    load_d<double, NC, COHERENT>(phi, n.xp, g.sites, xp);
    load_d<double, NC, COHERENT>(phi, n.ym, g.sites, ym);
    load_d<double, NC, COHERENT>(phi, n.yp, g.sites, yp);
    load_d<double, NC, COHERENT>(phi, n.zm, g.sites, zm);
    load_d<double, NC, COHERENT>(phi, n.zp, g.sites, zp);
    const long long o = checked(s * NC, NC, g.sites * NC);
#pragma unroll
    for (int a = 0; a < NC; ++a) p[a] = pi[o + a];
    energy_site<NC>(c, xm, xp, ym, yp, zm, zp, p, acc, ke);
    update_f64<NC>(c, xm, xp, ym, yp, zm, zp, p, out, k);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        pi[o + a] = p[a];
        phi_out[o + a] = out[a];
    }
}

// The same for FP32 storage (KAHAN: compensated drift); the energy is computed in FP64 from
// the exact conversions of the stored values.
template <int NC, bool KAHAN, bool COHERENT>
__device__ __forceinline__ void site_step_energy_f32(const float *__restrict__ phi, float *__restrict__ phi_out,
                                                     float *__restrict__ pi, float *__restrict__ comp, long long s,
                                                     const Geom &g, const Coef32 &k, const CoefE &ke,
                                                     double (&acc)[kNs<NC>]) {
    const Nbr n = neighbours(s, g);
    const long long cnt = g.sites * NC;
    const long long o = checked(s * NC, NC, cnt), ixm = checked(n.xm * NC, NC, cnt), ixp = checked(n.xp * NC, NC, cnt),
                    iym = checked(n.ym * NC, NC, cnt), iyp = checked(n.yp * NC, NC, cnt),
                    izm = checked(n.zm * NC, NC, cnt), izp = checked(n.zp * NC, NC, cnt);
    float c[NC], xm[NC], xp[NC], ym[NC], yp[NC], zm[NC], zp[NC], p[NC], cm[NC], out[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        c[a] = ld_field<COHERENT>(phi + o + a);
        xm[a] = ld_field<COHERENT>(phi + ixm + a);
        xp[a] = ld_field<COHERENT>(phi + ixp + a);
        ym[a] = ld_field<COHERENT>(phi + iym + a);
        yp[a] = ld_field<COHERENT>(phi + iyp + a);
        zm[a] = ld_field<COHERENT>(phi + izm + a);
        zp[a] = ld_field<COHERENT>(phi + izp + a);
        p[a] = pi[o + a];
        cm[a] = KAHAN ? comp[o + a] : 0.0f;
    }
    double dc[NC], dxm[NC], dxp[NC], dym[NC], dyp[NC], dzm[NC], dzp[NC], dp[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        dc[a] = widen(c[a]);
        dxm[a] = widen(xm[a]);
        dxp[a] = widen(xp[a]);
        dym[a] = widen(ym[a]);
        dyp[a] = widen(yp[a]);
        dzm[a] = widen(zm[a]);
        dzp[a] = widen(zp[a]);
        dp[a] = widen(p[a]);
    }
    energy_site<NC>(dc, dxm, dxp, dym, dyp, dzm, dzp, dp, acc, ke);
    update_f32<NC, KAHAN>(c, xm, xp, ym, yp, zm, zp, p, cm, out, k);
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        pi[o + a] = p[a];
        phi_out[o + a] = out[a];
        if (KAHAN) comp[o + a] = cm[a];
    }
}

// Fused step + energy, one step per launch.
template <int NC>
__global__ void __launch_bounds__(kEnergyThreads)
    k_step_energy_f64(const double *__restrict__ phi, double *__restrict__ phi_out, double *__restrict__ pi, Geom g,
                      Coef64 k, CoefE ke, double *__restrict__ scratch, double *__restrict__ record) {
    __shared__ double sh[kNs<NC>][kEnergyThreads];
    double acc[kNs<NC>];
#pragma unroll
    for (int j = 0; j < kNs<NC>; ++j) acc[j] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride)
        site_step_energy_f64<NC, false>(phi, phi_out, pi, s, g, k, ke, acc);
    finish_energy<NC>(acc, sh, scratch, ke, record);
}

template <int NC, bool KAHAN>
__global__ void __launch_bounds__(kEnergyThreads)
    k_step_energy_f32(const float *__restrict__ phi, float *__restrict__ phi_out, float *__restrict__ pi,
                      float *__restrict__ comp, Geom g, Coef32 k, CoefE ke, double *__restrict__ scratch,
                      double *__restrict__ record) {
    __shared__ double sh[kNs<NC>][kEnergyThreads];
    double acc[kNs<NC>];
#pragma unroll
    for (int j = 0; j < kNs<NC>; ++j) acc[j] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride)
        site_step_energy_f32<NC, KAHAN, false>(phi, phi_out, pi, comp, s, g, k, ke, acc);
    finish_energy<NC>(acc, sh, scratch, ke, record);
}

// ------------------------------------------- many fused steps in one launch (small lattices)
// On a small lattice (the 32^3 run with an energy every step) a step costs a few microseconds
// of arithmetic and about as much again in launch gaps and in the serial reduction.  One
// cooperative launch runs all steps: the same grid, site order and per-site code as
// k_step_energy for the site blocks, a grid barrier between steps, and one extra block, which
// owns no sites and reduces the partial rows.  The fields and every record are bitwise those
// of one launch per step.
//
// The barrier is split in two halves.  A site block arrives as soon as its part of step k is
// written (that is all the next step needs), then sums its energy accumulators into its
// partial row of step k, then waits.  The block sums thus overlap the barrier instead of
// preceding it.  A site block writes its row of step k before it arrives at barrier k+1, so
// the reducing block sums the rows of step k once barrier k+1 has completed, while the site
// blocks run step k+2, and one more barrier after the last step completes its rows.  The rows
// rotate over three sets: a site block writes the set of step k+3 only after barrier k+2,
// which the reducing block joins only after it has read the rows of step k.

// The row sets (at most kStepsMaxBlocks rows each) start at kStepsRowsOffset of a field's
// scratch; the barrier slots (arrivals, generation, error) fill the row after them.
constexpr int kRowSets = kEnergyStepsRowSets;
constexpr int kStepsMaxBlocks = kEnergyStepsBlocks;
constexpr size_t kBarrierOffset = (size_t)kStepsRowsOffset + (size_t)kRowSets * kStepsMaxBlocks * kEnergySlots;
static_assert(kBarrierOffset + kEnergySlots == (size_t)kFieldScratchDoubles, "multi-step scratch layout");
// A barrier waits at most about a second (2^24 polls of >= 64 ns); co-residency, which the
// cooperative launch guarantees, keeps real waits to microseconds.
constexpr unsigned kBarrierPolls = 1u << 24;

// Arrival half of the grid barrier: once every thread of the block has made its writes,
// thread 0 publishes them (fence) and counts the block in; the last block to arrive resets
// the count and advances the generation.  Returns, in thread 0, the generation before the
// arrival, which grid_wait compares against.
__device__ __forceinline__ unsigned grid_arrive(unsigned *bar) {
    __syncthreads();
    unsigned g = 0u;
    if (threadIdx.x == 0) {
        g = *(volatile unsigned *)(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        }
    }
    return g;
}

// Waiting half: returns true once the generation has moved past g (every block arrived),
// false when the wait ran out after polls_max polls, here or in another block (error flag).
// The generation can move by one at most while a block waits, since no barrier completes
// without this block's next arrival.
__device__ __forceinline__ bool grid_wait(unsigned *bar, unsigned g, unsigned polls_max) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = bar + 1;
        unsigned polls = 0;
        while (*gen == g) {
            if (++polls > polls_max) {
                atomicExch(bar + 2, 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        if (*(volatile unsigned *)(bar + 2) != 0u) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// A run cut short by a barrier that did not complete leaves NaN records from `from` on (the
// record of a step is finished during the next step, so `from` is the step before that barrier).
__device__ __forceinline__ void poison_records(double *records, int from, int nsteps) {
    if (blockIdx.x != gridDim.x - 1 || threadIdx.x != 0) return;
    for (int j = from; j < nsteps; ++j)
        for (int i = 0; i < kEnergySlots; ++i) records[(size_t)j * kEnergySlots + i] = __longlong_as_double(0x7ff8000000000000LL);
}

// The step loop shared by the FP64 and FP32 kernels.  site(src, dst, s, acc) performs the
// fused step + energy of site s.
template <int NC, typename R, typename Site>
__device__ __forceinline__ void steps_energy_loop(R *phi_a, R *phi_b, Geom g, const CoefE &ke, int nsteps,
                                                  double *__restrict__ scratch, double *__restrict__ records,
                                                  unsigned polls, double (&sh)[kNs<NC>][kEnergyThreads], Site site) {
    constexpr int NS = kNs<NC>;
    unsigned *bar = reinterpret_cast<unsigned *>(scratch + kBarrierOffset);
    const int nsb = (int)gridDim.x - 1;  // site blocks; the last block reduces
    const bool reducer = (int)blockIdx.x == nsb;
    const long long stride = (long long)nsb * blockDim.x;
    // rows [first, first + count) of the set of `step`, inside the row-set region (checked in
    // the debug build against that region, so neither the reduction layout before it nor the
    // barrier row after it can be hit)
    auto rows_of = [&](int step, long long first, long long count) {
        const long long rel = checked((long long)(step % kRowSets) * nsb * kEnergySlots + first * kEnergySlots,
                                      count * kEnergySlots, (long long)kRowSets * kStepsMaxBlocks * kEnergySlots);
        return scratch + kStepsRowsOffset + rel;
    };
    for (int step = 0; step <= nsteps; ++step) {
        double acc[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) acc[j] = 0.0;
        if (!reducer && step < nsteps) {
            const R *src = (step & 1) ? phi_b : phi_a;
            R *dst = (step & 1) ? phi_a : phi_b;
            for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.sites; s += stride)
                site(src, dst, s, acc);
        }
        const unsigned gen = grid_arrive(bar);  // step's fields published (the final pass: rows only)
        if (!reducer && step < nsteps) {
            block_sum<NS>(acc, sh);
            if (threadIdx.x < NS) rows_of(step, blockIdx.x, 1)[threadIdx.x] = sh[threadIdx.x][0];
        }
        if (!grid_wait(bar, gen, polls)) {
            poison_records(records, step > 0 ? step - 1 : 0, nsteps);
            return;
        }
        if (reducer && step > 0)
            reduce_rows<NC>(rows_of(step - 1, 0, nsb), nsb, sh, ke, records + (size_t)(step - 1) * kEnergySlots, nullptr);
    }
}

template <int NC>
__global__ void __launch_bounds__(kEnergyThreads)
    k_steps_energy_f64(double *phi_a, double *phi_b, double *__restrict__ pi, Geom g, Coef64 k, CoefE ke, int nsteps,
                       double *__restrict__ scratch, double *__restrict__ records, unsigned polls) {
    __shared__ double sh[kNs<NC>][kEnergyThreads];
    steps_energy_loop<NC>(phi_a, phi_b, g, ke, nsteps, scratch, records, polls, sh,
                          [&](const double *src, double *dst, long long s, double (&acc)[kNs<NC>]) {
                              site_step_energy_f64<NC, true>(src, dst, pi, s, g, k, ke, acc);
                          });
}

template <int NC, bool KAHAN>
__global__ void __launch_bounds__(kEnergyThreads)
    k_steps_energy_f32(float *phi_a, float *phi_b, float *__restrict__ pi, float *__restrict__ comp, Geom g, Coef32 k,
                       CoefE ke, int nsteps, double *__restrict__ scratch, double *__restrict__ records,
                       unsigned polls) {
    __shared__ double sh[kNs<NC>][kEnergyThreads];
    steps_energy_loop<NC>(phi_a, phi_b, g, ke, nsteps, scratch, records, polls, sh,
                          [&](const float *src, float *dst, long long s, double (&acc)[kNs<NC>]) {
                              site_step_energy_f32<NC, KAHAN, true>(src, dst, pi, comp, s, g, k, ke, acc);
                          });
}

// One block per 256 sites up to kEnergyBlocks: small lattices (a 32^3 run with an energy every
// step) spread over many SMs, large ones keep at most kEnergyBlocks partial rows.
int energy_grid(long long sites) {
    const long long want = (sites + kEnergyThreads - 1) / kEnergyThreads;
    return (int)(want < 1 ? 1 : (want > kEnergyBlocks ? kEnergyBlocks : want));
}

template <typename R>
cudaError_t launch_typed(const void *phi, const void *pi, const Geom &g, int ncomp, const CoefE &k, double *scratch,
                         double *record, cudaStream_t s) {
    const int nb = energy_grid(g.sites);
    switch (ncomp) {
#define LF2_E(NC)                                                                                               \
    case NC:                                                                                                    \
        k_energy<R, NC><<<nb, kEnergyThreads, 0, s>>>((const R *)phi, (const R *)pi, g, k, scratch, record); \
        break;
        LF2_E(1) LF2_E(2) LF2_E(3) LF2_E(4) LF2_E(5) LF2_E(6)
#undef LF2_E
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NC>
void step_energy_nc(const StepArgs &a, const CoefE &ke, int nb, double *scratch, double *record, cudaStream_t s) {
    if (a.prec == LF2_F64) {
        k_step_energy_f64<NC><<<nb, kEnergyThreads, 0, s>>>((const double *)a.phi, (double *)a.phi_out, (double *)a.pi,
                                                            a.g, make_coef64(a.p, a.dt), ke, scratch, record);
        return;
    }
    const Coef32 k = make_coef32(a.p, a.dt);
    if (a.prec == LF2_F32_KAHAN)
        k_step_energy_f32<NC, true><<<nb, kEnergyThreads, 0, s>>>((const float *)a.phi, (float *)a.phi_out,
                                                                  (float *)a.pi, a.comp, a.g, k, ke, scratch, record);
    else
        k_step_energy_f32<NC, false><<<nb, kEnergyThreads, 0, s>>>((const float *)a.phi, (float *)a.phi_out,
                                                                   (float *)a.pi, a.comp, a.g, k, ke, scratch, record);
}

// ------------------------------------------------------------ error norms (a12)
// max |a - ref|, max |ref|, sum (a - ref)^2, sum ref^2 over n elements, FP64.  The maxima
// propagate NaN (a NaN difference must not vanish from an error report).  Per element they are
// taken on the integer pipe: with the sign bit cleared, the bit patterns of doubles order as
// unsigned integers exactly as their values do, and every NaN orders above +inf, so the
// largest pattern is the largest magnitude, or a NaN if one occurred.  Only the subtraction
// and the two squares use the FP64 pipe, which bounds this kernel.
__device__ __forceinline__ double nanmax(double m, double x) { return (x > m || x != x) ? x : m; }

constexpr int kCmp = 4;

// Running maximum of |x| as its bit pattern (sign cleared), compared as the pair (high word,
// low word) in 32-bit integer operations.  (A 64-bit unsigned max here kept the FP64 pipe as
// busy as the two FP64 comparisons it replaced: 0.36 ms against 0.20 ms for this kernel on a
// 256^3 complex field.)
struct MagMax {
    unsigned hi = 0u, lo = 0u;
    __device__ __forceinline__ void add(double x) {
        const unsigned h = (unsigned)__double2hiint(x) & 0x7fffffffu, l = (unsigned)__double2loint(x);
        const bool gt = h > hi || (h == hi && l > lo);
        hi = gt ? h : hi;
        lo = gt ? l : lo;
    }
    __device__ __forceinline__ double value() const { return __hiloint2double((int)hi, (int)lo); }
};

__device__ __forceinline__ void block_cmp(const double (&acc)[kCmp], double (&sh)[kCmp][kEnergyThreads]) {
#pragma unroll
    for (int j = 0; j < kCmp; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
#pragma unroll
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        for (int t = threadIdx.x; t < kCmp * w; t += kEnergyThreads) {
            const int j = t / w, i = t % w;
            sh[j][i] = j < 2 ? nanmax(sh[j][i], sh[j][i + w]) : __dadd_rn(sh[j][i], sh[j][i + w]);
        }
        __syncthreads();
    }
}

template <typename RA, typename RB>
__global__ void __launch_bounds__(kEnergyThreads) k_compare(const RA *__restrict__ a, const RB *__restrict__ ref,
                                                            long long n, double *__restrict__ scratch) {
    __shared__ double sh[kCmp][kEnergyThreads];
    __shared__ bool s_last;
    double acc[kCmp] = {0.0, 0.0, 0.0, 0.0};
    MagMax max_d, max_r;
    // The thread's elements i, i + stride, i + 2 stride, ... are taken kBatch at a time: all their
    // loads are issued before the first is used (the bound checks come first, so no load is
    // speculative), and the sums still run in element order.
    constexpr int kBatch = 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kBatch * stride) {
        RA av[kBatch];
        RB rv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const long long i = i0 + u * stride;
            av[u] = i < n ? __ldg(a + i) : RA(0);
            rv[u] = i < n ? __ldg(ref + i) : RB(0);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (i0 + u * stride >= n) break;
            const double r = widen(rv[u]);
            const double d = __dsub_rn(widen(av[u]), r);
            max_d.add(d);
            max_r.add(r);
            acc[2] = __fma_rn(d, d, acc[2]);
            acc[3] = __fma_rn(r, r, acc[3]);
        }
    }
    acc[0] = max_d.value();
    acc[1] = max_r.value();
    block_cmp(acc, sh);
    if (threadIdx.x < kCmp) scratch[(size_t)blockIdx.x * kEnergySlots + threadIdx.x] = sh[threadIdx.x][0];
    __threadfence();
    __syncthreads();
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kEnergyCounterOffset);
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[kCmp] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < kCmp; ++j) {
            const double v = __ldcg(scratch + (size_t)b * kEnergySlots + j);
            tot[j] = j < 2 ? nanmax(tot[j], v) : __dadd_rn(tot[j], v);
        }
    }
    block_cmp(tot, sh);
    if (threadIdx.x == 0) {
        for (int j = 0; j < kCmp; ++j) scratch[kEnergyRecordOffset + j] = sh[j][0];
        *counter = 0u;
    }
}

template <typename RA>
cudaError_t compare_ref(const RA *a, const void *ref, bool ref_double, long long n, int nb, double *scratch,
                        cudaStream_t s) {
    if (ref_double)
        k_compare<RA, double><<<nb, kEnergyThreads, 0, s>>>(a, (const double *)ref, n, scratch);
    else
        k_compare<RA, float><<<nb, kEnergyThreads, 0, s>>>(a, (const float *)ref, n, scratch);
    return cudaGetLastError();
}

// Cooperative launch of k (grid nb) when every block can be resident at once.
template <typename K, typename... Args>
cudaError_t launch_cooperative(K kern, int nb, cudaStream_t s, Args... args) {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEnergyThreads, 0);
    if (e != cudaSuccess) return e;
    if (!coop || (long long)per_sm * sms < nb) return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kEnergyThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t r = cudaLaunchKernelEx(&cfg, kern, args...);
    if (r == cudaErrorCooperativeLaunchTooLarge || r == cudaErrorNotSupported) {
        (void)cudaGetLastError();  // not launched: the caller runs one launch per step instead
        return cudaErrorNotSupported;
    }
    return r;
}

// nb site blocks plus the reducing block
template <int NC>
cudaError_t steps_energy_nc(const StepArgs &a, int nsteps, int nb, const CoefE &ke, double *scratch, double *records,
                            unsigned polls, cudaStream_t s) {
    nb += 1;
    if (a.prec == LF2_F64)
        return launch_cooperative(k_steps_energy_f64<NC>, nb, s, (double *)a.phi, (double *)a.phi_out, (double *)a.pi,
                                  a.g, make_coef64(a.p, a.dt), ke, nsteps, scratch, records, polls);
    const Coef32 k = make_coef32(a.p, a.dt);
    if (a.prec == LF2_F32_KAHAN)
        return launch_cooperative(k_steps_energy_f32<NC, true>, nb, s, (float *)a.phi, (float *)a.phi_out,
                                  (float *)a.pi, a.comp, a.g, k, ke, nsteps, scratch, records, polls);
    return launch_cooperative(k_steps_energy_f32<NC, false>, nb, s, (float *)a.phi, (float *)a.phi_out, (float *)a.pi,
                              a.comp, a.g, k, ke, nsteps, scratch, records, polls);
}

}  // namespace

cudaError_t launch_steps_energy(const StepArgs &a, int nsteps, double *scratch, double *records, bool no_wait,
                                cudaStream_t s) {
    const int nb = energy_grid(a.g.sites);  // site blocks, as for one launch per step
    if (!a.drift || nsteps < 2 || nb > kStepsMaxBlocks) return cudaErrorNotSupported;
    // the barrier's arrival count, generation and error flag start at zero
    cudaError_t e = cudaMemsetAsync(scratch + kBarrierOffset, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const CoefE ke = make_coefE(a.p);
    const unsigned polls = no_wait ? 0u : kBarrierPolls;
    switch (a.ncomp) {
        case 1: return steps_energy_nc<1>(a, nsteps, nb, ke, scratch, records, polls, s);
        case 2: return steps_energy_nc<2>(a, nsteps, nb, ke, scratch, records, polls, s);
        case 3: return steps_energy_nc<3>(a, nsteps, nb, ke, scratch, records, polls, s);
        case 4: return steps_energy_nc<4>(a, nsteps, nb, ke, scratch, records, polls, s);
        case 5: return steps_energy_nc<5>(a, nsteps, nb, ke, scratch, records, polls, s);
        case 6: return steps_energy_nc<6>(a, nsteps, nb, ke, scratch, records, polls, s);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t steps_energy_timed_out(double *scratch, bool *out, cudaStream_t s) {
    unsigned word[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(word, scratch + kBarrierOffset, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *out = word[2] != 0u;
    if (*out) {
        e = cudaMemsetAsync(scratch + kBarrierOffset, 0, sizeof word, s);  // reported once
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e;
}

cudaError_t bounds_violations_energy(unsigned long long *n, bool reset) { return bounds_violations_here(n, reset); }

cudaError_t launch_compare(const void *a, bool a_double, const void *ref, bool ref_double, long long n,
                           double *scratch, cudaStream_t s) {
    const int nb = energy_grid(n);
    if (a_double) return compare_ref<double>((const double *)a, ref, ref_double, n, nb, scratch, s);
    return compare_ref<float>((const float *)a, ref, ref_double, n, nb, scratch, s);
}

cudaError_t launch_energy(const void *phi, const void *pi, const Geom &g, int ncomp, lf2_precision prec,
                          const lf2_params &p, double *scratch, double *record, cudaStream_t s) {
    const CoefE k = make_coefE(p);
    if (prec == LF2_F64) return launch_typed<double>(phi, pi, g, ncomp, k, scratch, record, s);
    return launch_typed<float>(phi, pi, g, ncomp, k, scratch, record, s);
}

cudaError_t launch_step_energy(const StepArgs &a, double *scratch, double *record, cudaStream_t s) {
    if (!a.drift) return cudaErrorInvalidValue;
    const CoefE ke = make_coefE(a.p);
    const int nb = energy_grid(a.g.sites);
    switch (a.ncomp) {
        case 1: step_energy_nc<1>(a, ke, nb, scratch, record, s); break;
        case 2: step_energy_nc<2>(a, ke, nb, scratch, record, s); break;
        case 3: step_energy_nc<3>(a, ke, nb, scratch, record, s); break;
        case 4: step_energy_nc<4>(a, ke, nb, scratch, record, s); break;
        case 5: step_energy_nc<5>(a, ke, nb, scratch, record, s); break;
        case 6: step_energy_nc<6>(a, ke, nb, scratch, record, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------- fixed scratch for lf2_energy_noalloc
// Some callers cannot allocate device memory: code that runs while a memory pool or another
// framework owns the device allocator, or that must not make allocation calls at all.
// lf2_energy allocates its scratch on first use; lf2_energy_noalloc uses this file-scope array
// instead.  Every GPU that loads the library holds it until process exit.  Its size is fixed
// because the reduction grid has at most kEnergyBlocks blocks whatever the lattice: the
// partial rows, the record and the finished-block counter of any reduction fit, as the
// assertion below checks.  Static device memory starts zeroed; lf2_energy_noalloc also clears
// the counter before each launch.
static __device__ __align__(256) double g_energy_noalloc[kEnergyScratchDoubles];
static_assert(kEnergyRecordOffset >= kEnergyBlocks * kEnergySlots &&
                  kEnergyCounterOffset >= kEnergyRecordOffset + kEnergySlots &&
                  kEnergyCounterOffset + 1 <= kEnergyScratchDoubles,
              "the fixed scratch must hold kEnergyBlocks partial rows, the record and the counter");

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
