// Explicit instantiations of the shell-transpose kernels (adjoint of K3), one group per
// translation unit so that the builds run in parallel.  Pair diameter 6 is the costliest to
// compile: its three component kernels sit in lbe_adj_shell_f32_s6_c{0,1,2}.cu.
#include "lbe_adj_shell.cuh"

namespace lbe {
extern template cudaError_t launch_adj_tile2_cc<6, 3, 16, 0>(const AdjShellTile &, cudaStream_t);
extern template cudaError_t launch_adj_tile2_cc<6, 3, 16, 1>(const AdjShellTile &, cudaStream_t);
extern template cudaError_t launch_adj_tile2_cc<6, 3, 16, 2>(const AdjShellTile &, cudaStream_t);
template cudaError_t launch_adj_tile2<6, 3, 16>(const AdjShellTile &, cudaStream_t);
}  // namespace lbe
