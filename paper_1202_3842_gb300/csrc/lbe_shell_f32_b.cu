// Explicit instantiations of the FP32 shell-force kernels.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<5, 3, 16>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
