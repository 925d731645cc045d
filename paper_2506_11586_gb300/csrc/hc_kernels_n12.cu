// hc_kernels_n12.cu -- kernels and launchers for N = 4096 (see hc_kernels.cuh).
#include "hc_kernels.cuh"

namespace hc {
template hc_status launch_n<12>(const hc_ctx *, int, int, const LaunchArgs &, cudaStream_t);
}  // namespace hc
