// Quasi-pressure initialisation (Sec. "Stabilization", Eq. for the quasi-pressure Pi^alpha): the
// zeroth moment of the second distribution is chosen as
//   Pi^a(r) = n^a(r) - beta * integral up to r of ( C^{a,mf}(r') + n^a(r') F^a(r') / m ) . dr',
// with the integral taken by the trapezoidal rule along a lattice path.  The paper leaves the path
// open (the integral is path dependent and its constant never enters the evolution); here it runs
// from the origin along x at y = z = 0, then along y at z = 0, then along z:
//   I(x,0,0) = I(x-1,0,0) + (V_x(x-1,0,0) + V_x(x,0,0)) / 2,
//   I(x,y,0) = I(x,y-1,0) + (V_y(x,y-1,0) + V_y(x,y,0)) / 2,
//   I(x,y,z) = I(x,y,z-1) + (V_z(x,y,z-1) + V_z(x,y,z)) / 2,
// V = C^{a,mf} + n^a F^a (zero on solid nodes, where n = 0 and C = 0), I(0,0,0) = 0, Pi = n - 3 I.
// Each line is one thread's sequential sum in FP64: one thread per species, then one per (species,
// x), then one per (species, x, y).  Initialisation only.
#include "lbe_device.cuh"
#include "lbe_launch.h"

namespace lbe {

template <typename T>
__device__ __forceinline__ double integrand(const Grid &g, const double *n, const T *C, const T *F, int a, int c,
                                            long long i) {
    const long long k = ((long long)a * 3 + c) * g.N + i;
    return (double)C[k] + n[(long long)a * g.N + i] * (double)F[k];
}

template <typename T>
__global__ void k_qp_line_x(Grid g, int M, const double *__restrict__ n, const T *__restrict__ C,
                            const T *__restrict__ F, double *__restrict__ I) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= M) return;
    double acc = 0.0;
    I[(long long)a * g.N] = 0.0;
    for (int x = 1; x < g.nx; ++x) {
        acc += 0.5 * (integrand(g, n, C, F, a, 0, x - 1) + integrand(g, n, C, F, a, 0, x));
        I[(long long)a * g.N + x] = acc;
    }
}

template <typename T>
__global__ void k_qp_line_y(Grid g, int M, const double *__restrict__ n, const T *__restrict__ C,
                            const T *__restrict__ F, double *__restrict__ I) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)M * g.nx) return;
    const int a = (int)(t / g.nx), x = (int)(t % g.nx);
    double acc = I[(long long)a * g.N + x];
    for (int y = 1; y < g.ny; ++y) {
        const long long i0 = x + (long long)g.nx * (y - 1), i1 = i0 + g.nx;
        acc += 0.5 * (integrand(g, n, C, F, a, 1, i0) + integrand(g, n, C, F, a, 1, i1));
        I[(long long)a * g.N + i1] = acc;
    }
}

template <typename T>
__global__ void k_qp_line_z(Grid g, int M, const double *__restrict__ n, const T *__restrict__ C,
                            const T *__restrict__ F, double *__restrict__ I) {
    const long long plane = (long long)g.nx * g.ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)M * plane) return;
    const int a = (int)(t / plane);
    const long long xy = t % plane;
    double acc = I[(long long)a * g.N + xy];
    for (int z = 1; z < g.nz; ++z) {
        const long long i0 = xy + plane * (z - 1), i1 = i0 + plane;
        acc += 0.5 * (integrand(g, n, C, F, a, 2, i0) + integrand(g, n, C, F, a, 2, i1));
        I[(long long)a * g.N + i1] = acc;
    }
}

__global__ void k_qp_pi(long long total, const double *__restrict__ n, double *__restrict__ IPi) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    IPi[i] = n[i] - 3.0 * IPi[i];  // beta = 1 / k_B T = 3
}

cudaError_t launch_quasipressure(bool fp64, const Grid &g, int M, const double *n, const void *C, const void *F,
                                 double *Pi, cudaStream_t st) {
    constexpr int nt = 128;
    const long long ly = (long long)M * g.nx, lz = (long long)M * g.nx * g.ny, tot = (long long)M * g.N;
    if (fp64) {
        k_qp_line_x<double><<<1, nt, 0, st>>>(g, M, n, (const double *)C, (const double *)F, Pi);
        k_qp_line_y<double><<<(unsigned)((ly + nt - 1) / nt), nt, 0, st>>>(g, M, n, (const double *)C,
                                                                           (const double *)F, Pi);
        k_qp_line_z<double><<<(unsigned)((lz + nt - 1) / nt), nt, 0, st>>>(g, M, n, (const double *)C,
                                                                           (const double *)F, Pi);
    } else {
        k_qp_line_x<float><<<1, nt, 0, st>>>(g, M, n, (const float *)C, (const float *)F, Pi);
        k_qp_line_y<float><<<(unsigned)((ly + nt - 1) / nt), nt, 0, st>>>(g, M, n, (const float *)C,
                                                                         (const float *)F, Pi);
        k_qp_line_z<float><<<(unsigned)((lz + nt - 1) / nt), nt, 0, st>>>(g, M, n, (const float *)C,
                                                                         (const float *)F, Pi);
    }
    k_qp_pi<<<(unsigned)((tot + nt - 1) / nt), nt, 0, st>>>(tot, n, Pi);
    return cudaGetLastError();
}

}  // namespace lbe
