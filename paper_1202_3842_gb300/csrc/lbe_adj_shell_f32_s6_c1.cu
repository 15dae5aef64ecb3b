// Shell-transpose kernel of pair diameter 6, component 1 (adjoint of K3).
#include "lbe_adj_shell.cuh"

namespace lbe {
template cudaError_t launch_adj_tile2_cc<6, 3, 16, 1>(const AdjShellTile &, cudaStream_t);
}  // namespace lbe
