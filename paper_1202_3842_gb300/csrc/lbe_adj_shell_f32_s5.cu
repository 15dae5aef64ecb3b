// Explicit instantiations of the shell-transpose kernels (adjoint of K3), one group per
// translation unit so that the builds run in parallel.
#include "lbe_adj_shell.cuh"

namespace lbe {
template cudaError_t launch_adj_tile2<5, 3, 16>(const AdjShellTile &, cudaStream_t);
}  // namespace lbe
