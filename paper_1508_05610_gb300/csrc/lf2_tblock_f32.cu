// lf2_tblock_f32.cu -- temporal-blocking instantiations for plain FP32 (one translation unit per
// precision so that the kernels compile in parallel).
#include "lf2_tblock.cuh"

namespace lf2 {

cudaError_t bounds_violations_tblock_f32(unsigned long long *n, bool reset) { return bounds_violations_here(n, reset); }

cudaError_t launch_tblock_f32(const TbArgs &a, const TbConfig &c, cudaStream_t s) {
    const Coef32 k = make_coef32(a.p, a.dt);
    switch (a.ncomp) {
        case 1: return tb::launch_prec<float, 1, 0>(a, c, k, s);
        case 2: return tb::launch_prec<float, 2, 0>(a, c, k, s);
        case 3: return tb::launch_prec<float, 3, 0>(a, c, k, s);
        case 4: return tb::launch_prec<float, 4, 0>(a, c, k, s);
        case 6: return tb::launch_prec<float, 6, 0>(a, c, k, s);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_tblock_ensemble_f32(const TbEnsembleLaunch &e, cudaStream_t s) {
    switch (e.ncomp) {
        case 1: return tb::launch_ens_prec<float, 1, 0, Coef32>(e, s);
        case 2: return tb::launch_ens_prec<float, 2, 0, Coef32>(e, s);
        case 3: return tb::launch_ens_prec<float, 3, 0, Coef32>(e, s);
        case 4: return tb::launch_ens_prec<float, 4, 0, Coef32>(e, s);
        case 6: return tb::launch_ens_prec<float, 6, 0, Coef32>(e, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace lf2
