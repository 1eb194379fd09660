// placeholder until the tcgen05 kernels land
#include "tdk_internal.cuh"
namespace tdk {
int sketch_tc(tdk_ctx*, const Geom&, int, const void*, const double* const[], double*) { return TDK_ENOTSUP; }
int core_tc(tdk_ctx*, const Geom&, int, const void*, const double* const[], void*, double*) { return TDK_ENOTSUP; }
}  // namespace tdk
