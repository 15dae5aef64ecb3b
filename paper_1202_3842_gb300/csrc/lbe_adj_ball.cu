// Transposed ball average of the discrete adjoint (K2 transposed, second half):
// ln_b(r) += sum over the ball |d| <= sigma_b/2 of lnbar_b(r + d), zero on solid
// nodes.  The same TMA ring, ball rows and prefix rows as the contact-value
// kernel (lbe_contact.cuh, MODE 1).
#include "lbe_contact.cuh"

namespace lbe {

cudaError_t launch_adj_ball_tma(bool fp64, const ContactLaunch &L, cudaStream_t st) {
    return fp64 ? dispatch_m<double, 1>(L, st) : dispatch_m<float, 1>(L, st);
}

}  // namespace lbe
