// Dispatch of the shell-force kernels by precision and pair diameter, and the
// host-side shell helpers.  FP32 pair diameters up to 7 use the z-blocked
// kernel (32 x 16 threads; three outputs per thread along z up to diameter 6,
// two at 7, where three would not fit the shared-memory ring); diameter 8 and
// the FP64 path use the plain kernel (one output per thread and plane).  The kernels are instantiated in lbe_shell_f32_*.cu
// and lbe_shell_f64.cu.
#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_shell.cuh"

namespace lbe {

template <typename T, int S>
cudaError_t launch_one(const ShellLaunch &L, cudaStream_t st);
template <typename T, int S, int TZ, int TYB>
cudaError_t launch_zb(const ShellLaunch &L, cudaStream_t st);



cudaError_t launch_shell_force(bool fp64, int S, const ShellLaunch &L, cudaStream_t st) {
    if (!fp64) {
        switch (S) {
            case 1: return launch_zb<float, 1, 3, 16>(L, st);
            case 2: return launch_zb<float, 2, 3, 16>(L, st);
            case 3: return launch_zb<float, 3, 3, 16>(L, st);
            case 4: return launch_zb<float, 4, 3, 16>(L, st);
            case 5: return launch_zb<float, 5, 3, 16>(L, st);
            case 6: return launch_zb<float, 6, 3, 16>(L, st);
            case 7: return launch_zb<float, 7, 2, 16>(L, st);
            case 8: return launch_one<float, 8>(L, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (S) {
        case 1: return launch_one<double, 1>(L, st);
        case 2: return launch_one<double, 2>(L, st);
        case 3: return launch_one<double, 3>(L, st);
        case 4: return launch_one<double, 4>(L, st);
        case 5: return launch_one<double, 5>(L, st);
        case 6: return launch_one<double, 6>(L, st);
        case 7: return launch_one<double, 7>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

bool shell_supported(bool fp64, int S) { return S >= 1 && S <= (fp64 ? 7 : 8); }

void shell_box(bool fp64, int S, int *bx, int *by) {
    if (!fp64) {
        const int zb = S <= 7;  // z-blocked tiles are 32 x 16 outputs per plane, the plain ones 32 x 8
        *bx = ((32 + 2 * S + 3) + 3) / 4 * 4;  // same for ShellTile and ShellTileZ
        *by = (zb ? 16 : 8) + 2 * S;
        return;
    }
#define LBE_BOX(s)                              \
    case s:                                     \
        *bx = ShellTile<double, s>::BX;         \
        *by = ShellTile<double, s>::BY;         \
        return;
    switch (S) { LBE_BOX(1) LBE_BOX(2) LBE_BOX(3) LBE_BOX(4) LBE_BOX(5) LBE_BOX(6) LBE_BOX(7) default: break; }
#undef LBE_BOX
    *bx = 0;
    *by = 0;
}

}  // namespace lbe
