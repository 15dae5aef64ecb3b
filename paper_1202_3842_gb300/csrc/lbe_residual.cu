// Diagnostics of the state: the steady-state residual (per node, the largest
// relative density change over the species since the recorded densities, and
// the update of the record) and the divergence of a velocity field.
#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

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

// div u = (1/c_s^2) sum_p w_p c_p . u(r + c_p) (the isotropic D3Q19 gradient of the force field),
// with u = 0 outside closed axes; solid nodes carry u = 0 from the velocity kernel.
__global__ void k_divergence(Grid g, const double *__restrict__ u, double *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double d = 0.0;
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        int X = x + cx(p), Y = y + cy(p), Z = z + cz(p);
        if (!(wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2]))) continue;
        const long long j = X + (long long)g.nx * (Y + (long long)g.ny * Z);
        d += wq(p) * (cx(p) * u[j] + cy(p) * u[g.N + j] + cz(p) * u[2 * g.N + j]);
    }
    out[i] = 3.0 * d;
}

cudaError_t launch_divergence(const Grid &g, const double *u, double *out, cudaStream_t st) {
    k_divergence<<<(unsigned)((g.N + 255) / 256), 256, 0, st>>>(g, u, out);
    return cudaGetLastError();
}

}  // namespace lbe
