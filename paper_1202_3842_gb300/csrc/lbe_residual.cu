// Steady-state residual: per node, the largest relative density change over
// the species since the recorded densities, and the update of the record.
#include "lbe_device.cuh"
#include "lbe_launch.h"

namespace lbe {

__global__ void k_residual(int M, long long N, InvN0 inv, const double *__restrict__ n, double *__restrict__ rec,
                           double *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double m = 0.0;
    for (int a = 0; a < M; ++a) {
        const double v = n[(long long)a * N + i];
        m = fmax(m, fabs(v - rec[(long long)a * N + i]) * inv.v[a]);
        rec[(long long)a * N + i] = v;
    }
    out[i] = m;
}

cudaError_t launch_residual(int M, long long N, const InvN0 &inv, const double *n, double *rec, double *out,
                            cudaStream_t st) {
    const unsigned nb = (unsigned)((N + 255) / 256);
    k_residual<<<nb, 256, 0, st>>>(M, N, inv, n, rec, out);
    return cudaGetLastError();
}

}  // namespace lbe
