// lf2_tblock_f64.cu -- temporal-blocking instantiations for FP64 (one translation unit per
// precision so that the kernels compile in parallel).
#include "lf2_tblock.cuh"

namespace lf2 {

cudaError_t bounds_violations_tblock_f64(unsigned long long *n, bool reset) { return bounds_violations_here(n, reset); }

cudaError_t launch_tblock_f64(const TbArgs &a, const TbConfig &c, cudaStream_t s) {
    const Coef64 k = make_coef64(a.p, a.dt);
    if (a.ncomp > 2) return cudaErrorNotSupported;  // FP64 fields of 3+ components run one-step kernels
    return a.ncomp == 1 ? tb::launch_prec<double, 1, 3>(a, c, k, s) : tb::launch_prec<double, 2, 3>(a, c, k, s);
}

cudaError_t launch_tblock_ensemble_f64(const TbEnsembleLaunch &e, cudaStream_t s) {
    if (e.ncomp > 2) return cudaErrorNotSupported;
    return e.ncomp == 1 ? tb::launch_ens_prec<double, 1, 3, Coef64>(e, s)
                        : tb::launch_ens_prec<double, 2, 3, Coef64>(e, s);
}

}  // namespace lf2
