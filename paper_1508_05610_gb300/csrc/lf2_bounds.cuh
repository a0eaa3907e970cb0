#pragma once
// lf2_bounds.cuh -- bounds checks of computed element indices, for a debug build.
//
// Compiled with -DLF2_DEBUG_BOUNDS (python -m paper_1508_05610_gb300.build --debug-bounds,
// which writes lib/liblf2_debug.so), checked(i, n, count) verifies that elements [i, i + n) lie
// inside an allocation of `count` elements.  An index outside is counted in this translation
// unit's device word and replaced by 0, so the access stays inside the allocation instead of
// faulting; lf2_debug_bounds() reads the counts.  Without the macro checked() returns i and
// the kernels compile to the same code as before.
#include <cuda_runtime.h>

namespace lf2 {
namespace {

#ifdef LF2_DEBUG_BOUNDS
__device__ unsigned long long g_bounds_violations;  // one per translation unit

__device__ __forceinline__ long long checked(long long i, long long n, long long count) {
    if (i >= 0 && i + n <= count) return i;
    atomicAdd(&g_bounds_violations, 1ull);
    return 0;
}

// Host: this translation unit's count (optionally reset to zero).
inline cudaError_t bounds_violations_here(unsigned long long *n, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(n, g_bounds_violations, sizeof *n);
    if (e == cudaSuccess && reset) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_bounds_violations, &zero, sizeof zero);
    }
    return e;
}
#else
__device__ __forceinline__ long long checked(long long i, long long, long long) { return i; }

inline cudaError_t bounds_violations_here(unsigned long long *n, bool) {
    *n = 0;
    return cudaSuccess;
}
#endif

}  // namespace
}  // namespace lf2
