// Collision-streaming and moments of the scheme ablations (Sec. "Results"):
//   SD-TR  one distribution f; trapezoidal update; J = J~ + (h/2)(C + nF) with J~ = sum c f~;
//   SD-EU  one distribution; Euler update f* = f + (1/tau)(f_eq - f) + h S_f; J = sum c f;
//   DD-EU  two distributions; Euler update of f and g; J = sum c g, Pi = sum g.
// (DD-TR, the method itself, runs in k_collide.)  Both updates have the form
//   f* = f + omega_eff (f_eq - f) + inv S,   omega_eff = 1/tau,
// with inv = 1/(1 + omega h/2) for TR and inv = h for EU (set on the host).  f_eq, g_eq, S_f and
// S_g are those of the DD-TR kernel; in the SD schemes S_f carries the whole force C + nF and g is
// not evolved: it is written as a copy of f.  FP64 and FP32 storage, one or two species; every
// population is pulled once into registers.
#include <utility>

#include "../../include/lbe.h"
#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int NTA = 128;

template <typename S, typename T, int M, bool SOLID>
__global__ void __launch_bounds__(NTA)
    k_collide_ablation(Grid g, const S *__restrict__ src, S *__restrict__ dst, const uint32_t *__restrict__ mask,
                       const T *__restrict__ C, const T *__restrict__ F, StepParams sp,
                       double *__restrict__ flux_buf) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = SOLID ? mask[i] : 0u;
    const int coord = sp.flux_axis == 0 ? x : (sp.flux_axis == 1 ? y : z);
    const bool on_plane = sp.flux_axis >= 0 && coord == sp.flux_plane;
    const int psize = sp.flux_axis == 0 ? g.ny * g.nz : (sp.flux_axis == 1 ? g.nx * g.nz : g.nx * g.ny);
    if (m & 1u) {
        if (on_plane)
            for (int a = 0; a < M; ++a) flux_buf[(long long)a * psize + plane_index(g, sp.flux_axis, x, y, z)] = 0.0;
        return;
    }
    const bool sd = sp.scheme == LBE_SD_TR || sp.scheme == LBE_SD_EU;
    const bool eu = sp.scheme == LBE_SD_EU || sp.scheme == LBE_DD_EU;
    const NbrOff o = nbr_offsets(g, x, y, z);
    T fv[M][Q], gv[M][Q];
    T n[M], Pi[M], J[M][3], Cv[M][3], nF[M][3], ua[M][3];
    T ntot = 0, Jtot[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T n0 = (T)sp.sp[a].n0;
        const S *fb = src + pop_off(a, 0, 0, g.N);
        const S *gb = src + pop_off(a, 1, 0, g.N);
        [&]<int... P>(std::integer_sequence<int, P...>) {
            ((fv[a][P] = pull<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
            if (!sd) ((gv[a][P] = pull<S, T, P, SOLID>(gb, g.N, i, o, m, n0)), ...);
        }(std::make_integer_sequence<int, Q>{});
        const T *mom = sd ? fv[a] : gv[a];
        T na = 0, Pit = 0, Jt[3] = {0, 0, 0};
        [&]<int... P>(std::integer_sequence<int, P...>) {
            ((na += fv[a][P]), ...);
            ((Pit += mom[P]), ...);
            ((Jt[0] += (T)cx(P) * mom[P]), ...);
            ((Jt[1] += (T)cy(P) * mom[P]), ...);
            ((Jt[2] += (T)cz(P) * mom[P]), ...);
        }(std::make_integer_sequence<int, Q>{});
        const T inv_n = na > (T)0 ? (T)1 / na : (T)0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Cv[a][c] = C[((long long)a * 3 + c) * g.N + i];
            nF[a][c] = na * F[((long long)a * 3 + c) * g.N + i];
            J[a][c] = eu ? Jt[c] : Jt[c] + (T)0.5 * (Cv[a][c] + nF[a][c]);
            ua[a][c] = J[a][c] * inv_n;
            Jtot[c] += J[a][c];
        }
        n[a] = na;
        Pi[a] = sd ? na : Pit;
        ntot += na;
    }
    const T inv_tot = ntot > (T)0 ? (T)1 / ntot : (T)0;
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = Jtot[c] * inv_tot;
    if (on_plane) {
#pragma unroll
        for (int a = 0; a < M; ++a)
            flux_buf[(long long)a * psize + plane_index(g, sp.flux_axis, x, y, z)] = (double)J[a][sp.flux_axis];
    }
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T na = n[a];
        const T uau = ua[a][0] * u[0] + ua[a][1] * u[1] + ua[a][2] * u[2];
        const T iso = (T)1.5 * na * ((T)2 * uau - uu);
        const T A = na - iso, B = Pi[a] - iso;
        T X[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = Cv[a][c] + nF[a][c];
        const T sf0 = (T)-3 * (X[0] * ua[a][0] + X[1] * ua[a][1] + X[2] * ua[a][2]);
        const T om = (T)sp.sp[a].omega_eff, inv = (T)sp.sp[a].inv;
        const T n0a = (T)sp.sp[a].n0;
        const T in0 = sp.sp[a].n0 > 0.0 ? (T)(1.0 / sp.sp[a].n0) : (T)0;
        S *fo = dst + pop_off(a, 0, 0, g.N) + i;
        S *go = dst + pop_off(a, 1, 0, g.N) + i;
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    constexpr T w = (T)wq(P);
                    const T cua = cdot<T, P>(ua[a]);
                    const T cu = cdot<T, P>(u);
                    const T cX = cdot<T, P>(X);
                    const T t1 = (T)3 * na * cua + (T)4.5 * na * ((T)2 * cua * cu - cu * cu);
                    const T feq = w * (A + t1);
                    const T Sf = w * (sf0 + (T)3 * cX + (T)9 * cX * cua);
                    const T fs = fv[a][P] + om * (feq - fv[a][P]) + inv * Sf;
                    constexpr T iw = (T)(1.0 / wq(P));
                    Store<S, T>::store(fo + (long long)P * g.N, fs, w * n0a, iw * in0);
                    if (sd) {
                        Store<S, T>::store(go + (long long)P * g.N, fs, w * n0a, iw * in0);
                    } else {
                        const T cY = cdot<T, P>(nF[a]);
                        const T cC = cdot<T, P>(Cv[a]);
                        const T geq = w * (B + t1);
                        const T Sg = w * (sf0 + (T)3 * cY + (T)18 * cC * cua + (T)9 * cY * cua);
                        const T gs = gv[a][P] + om * (geq - gv[a][P]) + inv * Sg;
                        Store<S, T>::store(go + (long long)P * g.N, gs, w * n0a, iw * in0);
                    }
                }(),
                ...);
        }(std::make_integer_sequence<int, Q>{});
    }
}

// Moments of the current state for the getters (FP64 out): n [M][N], J [M][3][N] by the scheme's recovery.
template <typename S, typename T, int M>
__global__ void __launch_bounds__(NTA)
    k_moments_ablation(Grid g, const S *__restrict__ src, const uint32_t *__restrict__ mask, const T *__restrict__ C,
                       const T *__restrict__ F, StepParams sp, double *__restrict__ nout, double *__restrict__ Jout) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = mask[i];
    const bool sd = sp.scheme == LBE_SD_TR || sp.scheme == LBE_SD_EU;
    const bool eu = sp.scheme == LBE_SD_EU || sp.scheme == LBE_DD_EU;
    const NbrOff o = nbr_offsets(g, x, y, z);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        T na = 0, Jt[3] = {0, 0, 0};
        if (!(m & 1u)) {
            const T n0 = (T)sp.sp[a].n0;
            const S *fb = src + pop_off(a, 0, 0, g.N);
            const S *mb = src + pop_off(a, sd ? 0 : 1, 0, g.N);
            [&]<int... P>(std::integer_sequence<int, P...>) {
                ((na += pull<S, T, P, true>(fb, g.N, i, o, m, n0)), ...);
                (
                    [&] {
                        const T v = pull<S, T, P, true>(mb, g.N, i, o, m, n0);
                        Jt[0] += (T)cx(P) * v;
                        Jt[1] += (T)cy(P) * v;
                        Jt[2] += (T)cz(P) * v;
                    }(),
                    ...);
            }(std::make_integer_sequence<int, Q>{});
        }
        nout[(long long)a * g.N + i] = (double)na;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T Jc = Jt[c];
            if (!(m & 1u) && !eu)
                Jc += (T)0.5 * (C[((long long)a * 3 + c) * g.N + i] + na * F[((long long)a * 3 + c) * g.N + i]);
            Jout[((long long)a * 3 + c) * g.N + i] = (m & 1u) ? 0.0 : (double)Jc;
        }
    }
}

bool ablation_supported(Prec p, int M) { return (p == Prec::F64 || p == Prec::F32) && M >= 1 && M <= 2; }

#define LBE_ABL_DISPATCH(p, ...)                                                     \
    switch (p) {                                                                     \
        case Prec::F64: { using S = double; using T = double; __VA_ARGS__; break; }  \
        case Prec::F32: { using S = float; using T = float; __VA_ARGS__; break; }    \
        default: return cudaErrorInvalidValue;                                       \
    }

cudaError_t launch_collide_ablation(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask,
                                    bool solid, const void *C, const void *F, const StepParams &sp,
                                    double *flux_buf, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + NTA - 1) / NTA);
#define LBE_ABL(MM, SOL)                                                                                    \
    k_collide_ablation<S, T, MM, SOL><<<nb, NTA, 0, st>>>(g, (const S *)src, (S *)dst, mask, (const T *)C, \
                                                          (const T *)F, sp, flux_buf)
    LBE_ABL_DISPATCH(p, {
        if (sp.M == 1) {
            if (solid) LBE_ABL(1, true); else LBE_ABL(1, false);
        } else if (sp.M == 2) {
            if (solid) LBE_ABL(2, true); else LBE_ABL(2, false);
        } else {
            return cudaErrorInvalidValue;
        }
    });
#undef LBE_ABL
    return cudaGetLastError();
}

cudaError_t launch_moments_ablation(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *C,
                                    const void *F, const StepParams &sp, double *n, double *J, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + NTA - 1) / NTA);
    LBE_ABL_DISPATCH(p, {
        if (sp.M == 1)
            k_moments_ablation<S, T, 1><<<nb, NTA, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp,
                                                            n, J);
        else if (sp.M == 2)
            k_moments_ablation<S, T, 2><<<nb, NTA, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp,
                                                            n, J);
        else
            return cudaErrorInvalidValue;
    });
    return cudaGetLastError();
}

}  // namespace lbe
