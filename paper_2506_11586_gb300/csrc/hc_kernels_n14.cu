// hc_kernels_n14.cu -- kernels and launchers for N = 16384 (see hc_kernels.cuh).
#include "hc_kernels.cuh"

namespace hc {
template hc_status launch_n<14>(const hc_ctx *, int, int, const LaunchArgs &, cudaStream_t);
}  // namespace hc
