// K2 launchers (contact values); the kernel is in lbe_contact.cuh.
#include "lbe_contact.cuh"

namespace lbe {

cudaError_t launch_contact_tma(bool fp64, const ContactLaunch &L, cudaStream_t st) {
    return fp64 ? dispatch_m<double, 0>(L, st) : dispatch_m<float, 0>(L, st);
}

void contact_box(bool fp64, int M, int RB, int *bx, int *by) {
    const int es = fp64 ? 8 : 4, A = 16 / es;
    *bx = ((32 + 2 * RB + A - 1) + A - 1) / A * A;
    *by = 8 + 2 * RB;
    (void)M;
}

}  // namespace lbe
