// Instantiation of the FP64 shell-force kernel (one output per thread and plane).
#include "lbe_shell_kernels.cuh"

namespace lbe {
template cudaError_t launch_one<double, 1>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 2>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 3>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 4>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 5>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 6>(const ShellLaunch &, cudaStream_t);
template cudaError_t launch_one<double, 7>(const ShellLaunch &, cudaStream_t);
}  // namespace lbe
