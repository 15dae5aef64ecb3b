// Instantiation of the z-blocked FP32 shell-force kernel for pair diameters 8.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<float, 8, 2>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
