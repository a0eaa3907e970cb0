// lf2_tblock.cu -- temporal blocking: configuration checks and dispatch by precision.
// The kernels are in lf2_tblock.cuh, instantiated per precision in lf2_tblock_{f64,f32k,f32}.cu.
#include "lf2_internal.cuh"

namespace lf2 {

cudaError_t launch_tblock_f64(const TbArgs &a, const TbConfig &c, cudaStream_t s);
cudaError_t launch_tblock_f32k(const TbArgs &a, const TbConfig &c, cudaStream_t s);
cudaError_t launch_tblock_f32(const TbArgs &a, const TbConfig &c, cudaStream_t s);
cudaError_t launch_tblock_ensemble_f64(const TbEnsembleLaunch &e, cudaStream_t s);
cudaError_t launch_tblock_ensemble_f32k(const TbEnsembleLaunch &e, cudaStream_t s);
cudaError_t launch_tblock_ensemble_f32(const TbEnsembleLaunch &e, cudaStream_t s);

namespace {
constexpr int kTbMaxThreads = 512;  // the kernels' launch bound
}  // namespace

bool tblock_cluster_built(int esz, int ncomp, int depth, int cx, int cluster) {
    return esz == 4 && ncomp <= 2 && (depth == 3 || depth == 4) && (cx == 1 || cx == 2 || cx == 4) &&
           cx * ncomp * esz <= 16 && (cluster == 2 || cluster == 4 || cluster == 8);
}

bool tblock_supported(const TbArgs &a, TbConfig &c) {
    const int esz = a.prec == LF2_F64 ? 8 : 4;
    if (a.ncomp > 2) {
        // 3, 4 or 6 components, FP32 storage: one column per thread, depth 2 to 4 (2 for 6
        // components); FP64 stays on the one-step kernels, which its FP64 arithmetic bounds
        if (esz == 8 || (a.ncomp != 3 && a.ncomp != 4 && a.ncomp != 6)) return false;
        if (c.depth == 0) c.depth = a.ncomp == 6 ? 2 : 3;
        if (c.cx == 0) c.cx = 1;
        if (c.cx != 1 || c.depth < 2 || c.depth > (a.ncomp == 6 ? 2 : 4)) return false;
    } else {
        if (c.depth == 0) c.depth = 4;
        if (c.depth != 2 && c.depth != 3 && c.depth != 4 && c.depth != 6 && c.depth != 8) return false;
        if (c.cx == 0) c.cx = (esz == 8 && a.ncomp == 2) ? 1 : 2;
        if (c.cx != 1 && c.cx != 2 && c.cx != 4) return false;
        if (c.cx * a.ncomp * esz > 16) return false;  // one vector of at most 16 bytes per thread and plane
        if (c.cx == 4 && (esz != 4 || a.ncomp != 1)) return false;
    }
    if ((long long)a.g.nx * a.g.ny * a.ncomp >= (1LL << 31)) return false;
    if (c.tile_x == 0) c.tile_x = 32;
    if (c.tile_y == 0) c.tile_y = 16;
    if (c.tile_x < c.cx || c.tile_x % c.cx || c.tile_y < 1) return false;
    if (a.g.nx % c.cx) return false;
    if (c.cluster <= 1) c.cluster = 1;
    if (c.cluster > 1 && !tblock_cluster_built(esz, a.ncomp, c.depth, c.cx, c.cluster)) return false;
    const int TP = ((c.depth + c.cx - 1) / c.cx) * c.cx;
    const int RX = c.tile_x + 2 * TP;
    // region rows of one CTA: the whole region, or one of `cluster` equal bands of it
    if ((c.tile_y + 2 * c.depth) % c.cluster) return false;
    const int RY = (c.tile_y + 2 * c.depth) / c.cluster;
    if (c.cluster > 1 && RY < 2) return false;
    if ((RX / c.cx) * RY > kTbMaxThreads) return false;
    const size_t smem = (size_t)2 * c.depth * (RY + 2) * RX * a.ncomp * esz;
    if (smem > 227 * 1024) return false;
    if (c.zchunk == 0) {
        // Split z into m chunks, m minimising (waves of blocks) x (iterations per block): a
        // chunk of zc planes costs zc + 2 depth iterations, and with one block per SM a launch
        // takes ceil(blocks / SMs) waves.  More chunks shrink the last, partly filled wave
        // but add the 2 depth halo planes per chunk.
        const long long tiles = (long long)((a.g.nx + c.tile_x - 1) / c.tile_x) * ((a.g.ny + c.tile_y - 1) / c.tile_y);
        const long long sms = device_sm_count();
        long long best = -1;
        for (int m = 1; m <= 64; ++m) {
            const int zc = (a.g.nz + m - 1) / m;
            if (m > 1 && zc < 2 * c.depth) break;
            const long long blocks = tiles * c.cluster * ((a.g.nz + zc - 1) / zc);
            const long long cost = ((blocks + sms - 1) / sms) * (zc + 2 * c.depth);
            if (best < 0 || cost < best) {
                best = cost;
                c.zchunk = zc;
            }
        }
    }
    if (c.zchunk < 1) return false;
    // the accesses are chunks of the largest of 16, 8, 4 bytes dividing a thread's bytes
    const int bytes = c.cx * a.ncomp * esz;
    const uintptr_t align = bytes % 16 == 0 ? 16 : (bytes % 8 == 0 ? 8 : 4);
    if (((uintptr_t)a.phi | (uintptr_t)a.phi_out | (uintptr_t)a.pi | (uintptr_t)a.pi_out | (uintptr_t)a.comp |
         (uintptr_t)a.comp_out) % align)
        return false;
    if (a.prec == LF2_F32_KAHAN && (!a.comp || !a.comp_out)) return false;
    return true;
}

cudaError_t launch_tblock_ensemble(const TbEnsembleLaunch &e, cudaStream_t s) {
    if (e.nitems == 0) return cudaSuccess;
    if (e.prec == LF2_F64) return launch_tblock_ensemble_f64(e, s);
    return e.prec == LF2_F32_KAHAN ? launch_tblock_ensemble_f32k(e, s) : launch_tblock_ensemble_f32(e, s);
}

cudaError_t launch_tblock(const TbArgs &a, const TbConfig &c, cudaStream_t s) {
    if (a.g.sites == 0) return cudaSuccess;
    if (a.prec == LF2_F64) return launch_tblock_f64(a, c, s);
    return a.prec == LF2_F32_KAHAN ? launch_tblock_f32k(a, c, s) : launch_tblock_f32(a, c, s);
}

}  // namespace lf2
