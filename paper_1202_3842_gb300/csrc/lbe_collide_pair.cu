// K4 for one or two species: fused moments + DD-TR collision + pull
// streaming (Sec. "Hard sphere fluid mixture in a potential well"; the
// arithmetic is that of k_collide in lbe_kernels.cu).
//
// Two species: a CTA of 256 threads takes 128 consecutive nodes; warps 0-3
// take species 0 and warps 4-7 species 1 of the same nodes, 32 consecutive
// nodes per warp.  Each thread pulls only its own species' 38 populations and
// keeps them in registers, computes that species' moments, and gets the
// partner species' n and J through shared memory to form the barycentric
// velocity u = (J_0 + J_1)/(n_0 + n_1).  A warp's load of one population is
// one 128-byte run of one species' array (FP32), as in the one-species
// kernel.  Compared with one thread per node holding both species, the live
// state per thread halves, which lets three CTAs of 256 threads share an SM.
// One species: one thread per node, 32 consecutive nodes per warp, u = J/n.
// K1 (the pulled density) uses the same layout.
#include <math.h>

#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int NTP = 256;  // threads per CTA: 128 nodes (two species) or 256 (one)

// FP32 arithmetic: four CTAs of 256 threads per SM for one species (0.95 -> 0.88 ms on the 256^3
// well, with some spills at 64 registers), three for two (four made the two-species launch slower).
template <typename S, typename T, int M, bool SOLID>
__global__ void __launch_bounds__(NTP, sizeof(T) == 4 ? (M == 1 ? 4 : 3) : 1)
    k_collide_pair(Grid g, const S *__restrict__ src, S *__restrict__ dst, const uint32_t *__restrict__ mask,
                   const T *__restrict__ C, const T *__restrict__ F, StepParams sp, double *__restrict__ flux_buf) {
    static_assert(M == 1 || M == 2, "one or two species");
    const int a = M == 2 ? (int)(threadIdx.x >> 7) : 0;         // species of this thread
    const int loc = M == 2 ? (int)(threadIdx.x & 127) : 0;      // node within the CTA's 128
    const long long i = M == 2 ? (long long)blockIdx.x * (NTP / 2) + loc : (long long)blockIdx.x * NTP + threadIdx.x;
    const bool valid = i < g.N;
    int x = 0, y = 0, z = 0;
    if (valid) node_xyz(g, i, x, y, z);
    const uint32_t m = valid ? (SOLID ? mask[i] : 0u) : 1u;
    const bool fluid = !(m & 1u);
    const int coord = sp.flux_axis == 0 ? x : (sp.flux_axis == 1 ? y : z);
    const bool on_plane = valid && sp.flux_axis >= 0 && coord == sp.flux_plane;
    const int psize = sp.flux_axis == 0 ? g.ny * g.nz : (sp.flux_axis == 1 ? g.nx * g.nz : g.nx * g.ny);

    // this species' constants (selected, not indexed, so the parameter block stays in constant memory)
    // (16-bit storage takes the float copies rounded on the host; the doubles are then unused)
    const double n0d = a == 0 ? sp.sp[0].n0 : sp.sp[1].n0;
    const double omd = a == 0 ? sp.sp[0].omega_eff : sp.sp[1].omega_eff;
    const double invd = a == 0 ? sp.sp[0].inv : sp.sp[1].inv;
    // a warp none of whose nodes has a blocked link pulls without the bounce-back selects
    const bool plain = !SOLID || __all_sync(0xffffffffu, (m >> 1) == 0u);
    // moments of this thread's species (zero on solid nodes and past the end)
    constexpr bool DEV = Store<S, T>::shifted;
    T f[Q], gq[Q];
    T n = 0, dn = 0, Pi = 0, J[3] = {0, 0, 0}, Cv[3] = {0, 0, 0}, nF[3] = {0, 0, 0}, ua[3] = {0, 0, 0};
    NbrOff o{};
    if (fluid) {
        o = nbr_offsets(g, x, y, z);
        // FP32 storage, two species: C and F issue with the populations, so their latency is not paid
        // again after the moment sums (0.99 -> 0.90 ms on the 512x128x128 channel).  With 16-bit storage
        // or one species the early loads measured slower (0.89 -> 0.91, 0.87 -> 0.92 ms): they stay after
        // the sums there.
        constexpr bool CF_EARLY = sizeof(S) == 4 && M == 2;
        T Fv[3];
        if constexpr (CF_EARLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Cv[c] = C[((long long)a * 3 + c) * g.N + i];
                Fv[c] = F[((long long)a * 3 + c) * g.N + i];
            }
        }
        const T n0 = sc_float<S, T> ? (T)(a == 0 ? sp.sp[0].n0_f : sp.sp[1].n0_f) : (T)n0d;
        const S *fb = src + pop_off(a, 0, 0, g.N);
        const S *gb = src + pop_off(a, 1, 0, g.N);
        // DEV: the populations as deviations from w_p n0 (f, gq below hold f - w_p n0, g - w_p n0)
        if (plain) {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (DEV) {
                    ((f[P] = pull_dev<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
                    ((gq[P] = pull_dev<S, T, P, false>(gb, g.N, i, o, m, n0)), ...);
                } else {
                    ((f[P] = pull<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
                    ((gq[P] = pull<S, T, P, false>(gb, g.N, i, o, m, n0)), ...);
                }
            }(std::make_integer_sequence<int, Q>{});
        } else {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (DEV) {
                    ((f[P] = pull_dev<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
                    ((gq[P] = pull_dev<S, T, P, SOLID>(gb, g.N, i, o, m, n0)), ...);
                } else {
                    ((f[P] = pull<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
                    ((gq[P] = pull<S, T, P, SOLID>(gb, g.N, i, o, m, n0)), ...);
                }
            }(std::make_integer_sequence<int, Q>{});
        }
        // n and Pi~ (DEV: their deviations from n0; the rest values sum to n0, and to zero in J~)
        T Pit = 0, Jt[3] = {0, 0, 0};
        [&]<int... P>(std::integer_sequence<int, P...>) {
            ((n += f[P]), ...);
            ((Pit += gq[P]), ...);
            ((Jt[0] += (T)cx(P) * gq[P]), ...);
            ((Jt[1] += (T)cy(P) * gq[P]), ...);
            ((Jt[2] += (T)cz(P) * gq[P]), ...);
        }(std::make_integer_sequence<int, Q>{});
        if constexpr (DEV) {
            dn = n;
            n = n0 + dn;
        }
        const T inv_n = n > (T)0 ? (T)1 / n : (T)0;
        T Cu = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if constexpr (!CF_EARLY) {
                Cv[c] = C[((long long)a * 3 + c) * g.N + i];
                Fv[c] = F[((long long)a * 3 + c) * g.N + i];
            }
            nF[c] = n * Fv[c];
            J[c] = sp.consistent ? Jt[c] + (T)0.5 * nF[c] : Jt[c] + (T)0.5 * (Cv[c] + nF[c]);
            ua[c] = J[c] * inv_n;
            Cu += Cv[c] * ua[c];
        }
        Pi = sp.consistent ? Pit + (T)1.5 * Cu : Pit - (T)0.5 * Cu;  // DEV: Pi - n0
    }
    // the partner species of the same node, through shared memory; every thread takes part
    T np = 0, Jp[3] = {0, 0, 0};
    if constexpr (M == 2) {
        __shared__ T xch[2][4][NTP / 2];
        xch[a][0][loc] = n;
#pragma unroll
        for (int c = 0; c < 3; ++c) xch[a][c + 1][loc] = J[c];
        // only the two warps over the same 32 nodes (warp w of species 0, warp w + 4 of species 1) wait
        // for each other: named barrier 1 + w of 64 threads (barrier 0 is the block's); 0.897 -> 0.885 ms
        // on the 512x128x128 channel against the block barrier
        asm volatile("bar.sync %0, 64;" ::"r"(1 + (loc >> 5)) : "memory");
        np = xch[1 - a][0][loc];
#pragma unroll
        for (int c = 0; c < 3; ++c) Jp[c] = xch[1 - a][c + 1][loc];
    }
    if (on_plane)
        flux_buf[(long long)a * psize + plane_index(g, sp.flux_axis, x, y, z)] =
            fluid ? (double)J[sp.flux_axis] : 0.0;
    if (!fluid) return;
    // species order in the sums: n_0 + n_1, J_0 + J_1 (one species: 0 + n, 0 + J as in k_collide)
    const T ntot = a == 0 ? n + np : np + n;
    const T inv_tot = ntot > (T)0 ? (T)1 / ntot : (T)0;
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = (a == 0 ? J[c] + Jp[c] : Jp[c] + J[c]) * inv_tot;

    const T uau = ua[0] * u[0] + ua[1] * u[1] + ua[2] * u[2];
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T iso = (T)1.5 * n * ((T)2 * uau - uu);
    // A and B enter f_eq and g_eq as w_p A, w_p B; DEV: their deviations from n0, so that f_eq and g_eq
    // come out as deviations from w_p n0 like the populations
    const T A = (DEV ? dn : n) - iso;
    const T B = Pi - iso;
    T X[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) X[c] = Cv[c] + nF[c];
    const T sf0 = (T)-3 * (X[0] * ua[0] + X[1] * ua[1] + X[2] * ua[2]);
    T om, inv, in0, n0s;
    if constexpr (sc_float<S, T>) {
        om = a == 0 ? sp.sp[0].omega_eff_f : sp.sp[1].omega_eff_f;
        inv = a == 0 ? sp.sp[0].inv_f : sp.sp[1].inv_f;
        in0 = a == 0 ? sp.sp[0].in0_f : sp.sp[1].in0_f;
        n0s = a == 0 ? sp.sp[0].n0_f : sp.sp[1].n0_f;
    } else {
        om = (T)omd;
        inv = (T)invd;
        in0 = n0d > 0.0 ? (T)(1.0 / n0d) : (T)0;
        n0s = (T)n0d;
    }
    S *fo = dst + pop_off(a, 0, 0, g.N) + i;
    S *go = dst + pop_off(a, 1, 0, g.N) + i;
    [&]<int... P>(std::integer_sequence<int, P...>) {
        (
            [&] {
                constexpr T w = (T)wq(P);
                const T cua = cdot<T, P>(ua);
                const T cu = cdot<T, P>(u);
                const T cX = cdot<T, P>(X);
                const T cY = cdot<T, P>(nF);
                const T cC = cdot<T, P>(Cv);
                const T t1 = (T)3 * n * cua + (T)4.5 * n * ((T)2 * cua * cu - cu * cu);
                const T feq = w * (A + t1);
                const T geq = w * (B + t1);
                const T Sf = w * (sf0 + (T)3 * cX + (T)9 * cX * cua);
                const T Sg = w * (sf0 + (T)3 * cY + (T)18 * cC * cua + (T)9 * cY * cua);
                const T fs = f[P] + om * (feq - f[P]) + inv * Sf;
                const T gs = gq[P] + om * (geq - gq[P]) + inv * Sg;
                constexpr T iw = (T)(1.0 / wq(P));
                if constexpr (DEV) {
                    Store<S, T>::store_dev(fo + (long long)P * g.N, fs, w * n0s, iw * in0);
                    Store<S, T>::store_dev(go + (long long)P * g.N, gs, w * n0s, iw * in0);
                } else {
                    Store<S, T>::store(fo + (long long)P * g.N, fs, w * n0s, iw * in0);
                    Store<S, T>::store(go + (long long)P * g.N, gs, w * n0s, iw * in0);
                }
            }(),
            ...);
    }(std::make_integer_sequence<int, Q>{});
}

// K1 for one or two species with the same thread layout: n^a(r) = sum_p f~_p(r) pulled, 0 on solid nodes,
// into the padded stencil field with its periodic images (the arithmetic of k_density).
template <typename S, typename T, int M, bool SOLID>
__global__ void __launch_bounds__(NTP)
    k_density_pair(Grid g, const S *__restrict__ pop, const uint32_t *__restrict__ mask, double n00, double n01,
                   T *__restrict__ npad, int *err) {
    static_assert(M == 1 || M == 2, "one or two species");
    const int a = M == 2 ? (int)(threadIdx.x >> 7) : 0;
    const long long i = M == 2 ? (long long)blockIdx.x * (NTP / 2) + (threadIdx.x & 127)
                               : (long long)blockIdx.x * NTP + threadIdx.x;
    const bool valid = i < g.N;
    const uint32_t m = valid ? (SOLID ? mask[i] : 0u) : 1u;
    // a warp none of whose nodes has a blocked link pulls without the bounce-back selects
    const bool plain = !SOLID || __all_sync(0xffffffffu, (m >> 1) == 0u);
    if (!valid) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    T n = (T)0;
    if (!(m & 1u)) {
        const NbrOff o = nbr_offsets(g, x, y, z);
        const S *fb = pop + pop_off(a, 0, 0, g.N);
        const T n0 = (T)(a == 0 ? n00 : n01);
        // shifted storage: n = n0 + the sum of the deviations
        if (plain) {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (Store<S, T>::shifted)
                    ((n += pull_dev<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
                else
                    ((n += pull<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
            }(std::make_integer_sequence<int, Q>{});
        } else {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (Store<S, T>::shifted)
                    ((n += pull_dev<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
                else
                    ((n += pull<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
            }(std::make_integer_sequence<int, Q>{});
        }
        if constexpr (Store<S, T>::shifted) n = n0 + n;
        if (!(n >= (T)0) || !isfinite(n)) atomicOr(err, ERR_DENSITY);
    }
    write_padded<T>(g, npad + (long long)a * g.P, x, y, z, n);
}

#define LBE_PAIR_DISPATCH(p, ...)                                                      \
    switch (p) {                                                                       \
        case Prec::F64: { using S = double; using T = double; __VA_ARGS__; break; }    \
        case Prec::F32: { using S = float; using T = float; __VA_ARGS__; break; }      \
        case Prec::BF16: { using S = __nv_bfloat16; using T = float; __VA_ARGS__; break; } \
        case Prec::F16: { using S = __half; using T = float; __VA_ARGS__; break; }     \
    }

cudaError_t launch_collide_pair(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask, bool solid,
                                const void *C, const void *F, const StepParams &sp, double *flux_buf,
                                cudaStream_t st) {
    const int per_cta = sp.M == 2 ? NTP / 2 : NTP;
    const unsigned nb = (unsigned)((g.N + per_cta - 1) / per_cta);
#define LBE_PAIR(MM, SOL)                                                                                   \
    k_collide_pair<S, T, MM, SOL><<<nb, NTP, 0, st>>>(g, (const S *)src, (S *)dst, mask, (const T *)C,      \
                                                      (const T *)F, sp, flux_buf)
    if (sp.M == 1) {
        if (solid) {
            LBE_PAIR_DISPATCH(p, LBE_PAIR(1, true));
        } else {
            LBE_PAIR_DISPATCH(p, LBE_PAIR(1, false));
        }
    } else if (sp.M == 2) {
        if (solid) {
            LBE_PAIR_DISPATCH(p, LBE_PAIR(2, true));
        } else {
            LBE_PAIR_DISPATCH(p, LBE_PAIR(2, false));
        }
    } else {
        return cudaErrorInvalidValue;
    }
#undef LBE_PAIR
    return cudaGetLastError();
}

cudaError_t launch_density_pair(Prec p, const Grid &g, const void *pop, const uint32_t *mask, bool solid, int M,
                                const double *n0, void *npad, int *err, cudaStream_t st) {
    const int per_cta = M == 2 ? NTP / 2 : NTP;
    const unsigned nb = (unsigned)((g.N + per_cta - 1) / per_cta);
    const double a0 = n0[0], a1 = M > 1 ? n0[1] : 0.0;
#define LBE_DPAIR(MM, SOL) \
    k_density_pair<S, T, MM, SOL><<<nb, NTP, 0, st>>>(g, (const S *)pop, mask, a0, a1, (T *)npad, err)
    if (M == 1) {
        if (solid) {
            LBE_PAIR_DISPATCH(p, LBE_DPAIR(1, true));
        } else {
            LBE_PAIR_DISPATCH(p, LBE_DPAIR(1, false));
        }
    } else if (M == 2) {
        if (solid) {
            LBE_PAIR_DISPATCH(p, LBE_DPAIR(2, true));
        } else {
            LBE_PAIR_DISPATCH(p, LBE_DPAIR(2, false));
        }
    } else {
        return cudaErrorInvalidValue;
    }
#undef LBE_DPAIR
    return cudaGetLastError();
}

}  // namespace lbe
