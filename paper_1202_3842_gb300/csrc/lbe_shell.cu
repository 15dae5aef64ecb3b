// Dispatch of the shell-force kernels by precision and pair diameter, and the
// host-side shell helpers.  FP32 reads the interleaved field (n_b, g_ab n_b):
// diameters 4 to 6 run the y-blocked kernel (32 x 8 threads, two rows and
// three planes of outputs per thread); 1 to 3 the z-blocked one with three
// outputs along z on 32 x 16 threads, 7 with two, 8 with one on 32 x 8.  The
// FP64 path uses the plain kernel (one output per thread and plane).  The
// kernels are instantiated in lbe_shell_f32_*.cu and lbe_shell_f64.cu.
#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_shell.cuh"

namespace lbe {

template <typename T, int S>
cudaError_t launch_one(const ShellLaunch &L, cudaStream_t st);
template <int S, int TZ, int TYB>
cudaError_t launch_zb(const ShellLaunch &L, cudaStream_t st);
template <int S, int TZ, int TYT>
cudaError_t launch_yb(const ShellLaunch &L, cudaStream_t st);

#if LBE_SHELL_YB
#define LBE_MID(S) launch_yb<S, LBE_SHELL_YTZ, LBE_SHELL_YTY>(L, st)
#else
#define LBE_MID(S) launch_zb<S, LBE_SHELL_TZ, LBE_SHELL_TY>(L, st)
#endif



cudaError_t launch_shell_force(bool fp64, int S, const ShellLaunch &L, cudaStream_t st) {
    if (!fp64) {
        switch (S) {
            case 1: return launch_zb<1, 3, 16>(L, st);
            case 2: return launch_zb<2, 3, 16>(L, st);
            case 3: return launch_zb<3, 3, 16>(L, st);
            case 4: return LBE_MID(4);
            case 5: return LBE_MID(5);
            case 6: return LBE_MID(6);
            case 7: return launch_zb<7, 2, 16>(L, st);
            case 8: return launch_zb<8, 1, 8>(L, st);
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

// Box of the shell-transpose tiles (lbe_adj_shell.cuh, dispatched in lbe_adjoint.cu).  FP32: the
// interleaved 8-byte (Lambda, g Lambda) elements of a 32 x 16 tile (32 x 8 at S = 8), the tile the
// transpose itself runs, which stays at 16 rows whatever the forward kernel's rows are; FP64: the
// forward kernel's box of two separate planes.
void adj_shell_box(bool fp64, int S, int *bx, int *by) {
    if (!fp64) {
        *bx = ((32 + 2 * S + 1) + 1) / 2 * 2;
        *by = (S <= 7 ? 16 : 8) + 2 * S;
        return;
    }
    shell_box(true, S, bx, by);
}

void shell_box(bool fp64, int S, int *bx, int *by) {
    if (!fp64) {  // interleaved 8-byte elements; 32 x 16 outputs per plane (32 x 8 at S = 8)
        *bx = ((32 + 2 * S + 1) + 1) / 2 * 2;
        *by = (S >= 4 && S <= 6 ? (LBE_SHELL_YB ? 2 * LBE_SHELL_YTY : LBE_SHELL_TY) : (S <= 7 ? 16 : 8)) + 2 * S;
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
