// Explicit instantiations of the FP32 shell-force kernels.
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_zb<5, LBE_SHELL_TZ, LBE_SHELL_TY>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_yb<5, LBE_SHELL_YTZ, LBE_SHELL_YTY>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
