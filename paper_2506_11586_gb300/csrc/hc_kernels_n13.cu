// hc_kernels_n13.cu -- kernels and launchers for N = 8192 (see hc_kernels.cuh).
#include "hc_kernels.cuh"

namespace hc {
template hc_status launch_n<13>(const hc_ctx *, int, int, const LaunchArgs &, cudaStream_t);
}  // namespace hc
