// Instantiation of the z-blocked FP32 shell-force kernel for pair diameters 1, 2, 3, 4.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<float, 1, 4>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_zb<float, 2, 4>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_zb<float, 3, 4>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_zb<float, 4, 4>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
