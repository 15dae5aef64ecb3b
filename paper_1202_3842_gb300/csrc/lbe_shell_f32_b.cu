// Instantiation of the z-blocked FP32 shell-force kernel for pair diameters 5.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<float, 5, 4>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
