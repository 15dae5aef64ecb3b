// Explicit instantiations of the FP32 shell-force kernels.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<8, 1, 8>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
