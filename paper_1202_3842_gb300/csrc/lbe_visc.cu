// Viscous part of the Enskog force (Appendix, C^{alpha,visc}), switched on by
// lbe_config.enable_visc:
//   C^{a,visc}(r) = n_a(r) sum_b 2 sigma_ab^2 sqrt(m k_B T / pi) w_ab
//                   sum_{e in K_ab} e^ g-bar_ab n_b(r + e) e^.(u~_b(r + e) - u~_b(r)),
// the shell, unit vectors, weight and endpoint-averaged contact value of the
// mean-field force, with the tilde velocities u~_b = J~_b / n_b of the streamed
// populations (the collision functional taken at the tilde moments, Sec.
// "Numerical solution").  In the DD-TR moment recovery and both sources the
// paper adds C^{visc} wherever n F appears (Sec. "Hard sphere fluid mixture":
// J, S_f, S_g), so the kernels here fold it into an effective force field
//   F_eff = F + C^{visc} / n   (F where n = 0),
// which the collide and the moment getters take in place of F.
//
// k_tilde_velocity pulls the g populations of every species; k_visc_force
// gathers the shell of every ordered pair from global memory (one thread per
// node; neighbours wrapped on periodic axes, skipped beyond closed axes and on
// solid nodes, where n_b = 0).  This is a plain gather, not a tiled stencil:
// the term is an option, about four times the mean-field stencil's work.
#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int VNT = 256;

template <typename S, typename T, int M>
__global__ void __launch_bounds__(VNT) k_tilde_velocity(Grid g, const S *__restrict__ pop,
                                                       const uint32_t *__restrict__ mask, const T *__restrict__ npad,
                                                       StepParams sp, T *__restrict__ ut) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = mask[i];
    const bool fluid = !(m & 1u);
    NbrOff o{};
    if (fluid) o = nbr_offsets(g, x, y, z);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        T J[3] = {0, 0, 0};
        if (fluid) {
            const S *gb = pop + pop_off(a, 1, 0, g.N);
            const T n0 = (T)sp.sp[a].n0;
            [&]<int... P>(std::integer_sequence<int, P...>) {
                (
                    [&] {
                        const T gv = pull<S, T, P, true>(gb, g.N, i, o, m, n0);
                        J[0] += (T)cx(P) * gv;
                        J[1] += (T)cy(P) * gv;
                        J[2] += (T)cz(P) * gv;
                    }(),
                    ...);
            }(std::make_integer_sequence<int, Q>{});
        }
        const T n = fluid ? npad[(long long)a * g.P + pidx(g, x, y, z)] : (T)0;
        for (int c = 0; c < 3; ++c) ut[((long long)a * 3 + c) * g.N + i] = n > (T)0 ? J[c] / n : (T)0;
    }
}

template <typename T>
__global__ void __launch_bounds__(VNT) k_visc_force(Grid g, const uint32_t *__restrict__ mask,
                                                   const T *__restrict__ npad, const T *__restrict__ gab,
                                                   const T *__restrict__ ut, const T *__restrict__ F, ViscPairs vp,
                                                   const int *__restrict__ eoff, const double *__restrict__ ehat,
                                                   T *__restrict__ Feff) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const bool fluid = !(mask[i] & 1u);
    for (int a = 0; a < vp.M; ++a) {
        T V[3] = {0, 0, 0};
        const T na = fluid ? npad[(long long)a * g.P + pidx(g, x, y, z)] : (T)0;
        if (na > (T)0) {
            for (int q = 0; q < vp.npairs; ++q) {
                if (vp.a[q] != a) continue;
                const int b = vp.b[q];
                const T *gq = gab + (long long)(a * vp.M + b) * g.N;
                const T *ub = ut + (long long)b * 3 * g.N;
                const T gr = gq[i];
                const T u0[3] = {ub[i], ub[g.N + i], ub[2 * (long long)g.N + i]};
                T sum[3] = {0, 0, 0};
                for (int k = vp.first[q]; k < vp.first[q] + vp.count[q]; ++k) {
                    int X = x + eoff[3 * k], Y = y + eoff[3 * k + 1], Z = z + eoff[3 * k + 2];
                    if (!wrap(X, g.nx, g.per[0]) || !wrap(Y, g.ny, g.per[1]) || !wrap(Z, g.nz, g.per[2])) continue;
                    const long long s = (long long)X + (long long)g.nx * ((long long)Y + (long long)g.ny * Z);
                    if (mask[s] & 1u) continue;
                    const T e0 = (T)ehat[3 * k], e1 = (T)ehat[3 * k + 1], e2 = (T)ehat[3 * k + 2];
                    const T edu = e0 * (ub[s] - u0[0]) + e1 * (ub[g.N + s] - u0[1]) + e2 * (ub[2 * (long long)g.N + s] - u0[2]);
                    const T w = (T)0.5 * (gr + gq[s]) * npad[(long long)b * g.P + pidx(g, X, Y, Z)] * edu;
                    sum[0] += e0 * w;
                    sum[1] += e1 * w;
                    sum[2] += e2 * w;
                }
                const T pre = (T)vp.pre[q];
                for (int c = 0; c < 3; ++c) V[c] += pre * sum[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            const long long k = ((long long)a * 3 + c) * g.N + i;
            Feff[k] = na > (T)0 ? F[k] + V[c] : F[k];  // V holds C^visc / n_a
        }
    }
}

template <typename S, typename T>
static cudaError_t tilde_m(const Grid &g, const void *pop, const uint32_t *mask, const void *npad,
                           const StepParams &sp, void *ut, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + VNT - 1) / VNT);
    switch (sp.M) {
        case 1: k_tilde_velocity<S, T, 1><<<nb, VNT, 0, st>>>(g, (const S *)pop, mask, (const T *)npad, sp, (T *)ut); break;
        case 2: k_tilde_velocity<S, T, 2><<<nb, VNT, 0, st>>>(g, (const S *)pop, mask, (const T *)npad, sp, (T *)ut); break;
        case 3: k_tilde_velocity<S, T, 3><<<nb, VNT, 0, st>>>(g, (const S *)pop, mask, (const T *)npad, sp, (T *)ut); break;
        case 4: k_tilde_velocity<S, T, 4><<<nb, VNT, 0, st>>>(g, (const S *)pop, mask, (const T *)npad, sp, (T *)ut); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_visc(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *npad,
                        const void *gab, const void *F, const StepParams &sp, const ViscPairs &vp, const int *eoff,
                        const double *ehat, void *ut, void *Feff, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    switch (p) {
        case Prec::F64: e = tilde_m<double, double>(g, pop, mask, npad, sp, ut, st); break;
        case Prec::F32: e = tilde_m<float, float>(g, pop, mask, npad, sp, ut, st); break;
        case Prec::BF16: e = tilde_m<__nv_bfloat16, float>(g, pop, mask, npad, sp, ut, st); break;
        case Prec::F16: e = tilde_m<__half, float>(g, pop, mask, npad, sp, ut, st); break;
    }
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((g.N + VNT - 1) / VNT);
    if (p == Prec::F64)
        k_visc_force<double><<<nb, VNT, 0, st>>>(g, mask, (const double *)npad, (const double *)gab,
                                                 (const double *)ut, (const double *)F, vp, eoff, ehat,
                                                 (double *)Feff);
    else
        k_visc_force<float><<<nb, VNT, 0, st>>>(g, mask, (const float *)npad, (const float *)gab, (const float *)ut,
                                                (const float *)F, vp, eoff, ehat, (float *)Feff);
    return cudaGetLastError();
}

}  // namespace lbe
