// D3Q19 Lattice Boltzmann-Enskog kernels (sm_103a): geometry, force field,
// population set/get, K1 density, K2 contact values, K4 fused DD-TR
// collide-stream, moments and FP64 reductions.  The shell force (K3) is in
// lbe_shell.cu.
//
// Population storage: [M][2 (f, g)][19][N] of the storage type S, holding the
// post-collision populations f~*(r, t-1); the streamed populations of step t
// are pulled: f~_p(r, t) = f~*_p(r - c_p, t-1), or f~*_{opp(p)}(r, t-1) when
// the link is blocked (mid-point bounce-back, Sec. "Channel flow with a
// bottleneck").  Link mask bit 0 marks a solid node, bit p a blocked link p.
#include <math.h>

#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int NT = 256;

struct N0Vec {
    double v[MAXS];
};
struct N0VecF {  // the same rounded once on the host, read with 16-bit storage
    float v[MAXS];
};

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
__global__ void k_link_mask(Grid g, const uint8_t *__restrict__ solid, uint32_t *__restrict__ mask) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    uint32_t m = solid[i] ? 1u : 0u;
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        int X = x - cx(p), Y = y - cy(p), Z = z - cz(p);
        bool ok = wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2]);
        if (!ok || solid[X + (long long)g.nx * (Y + (long long)g.ny * Z)]) m |= (1u << p);
    }
    mask[i] = m;
}

cudaError_t launch_link_mask(const Grid &g, const uint8_t *solid, uint32_t *mask, cudaStream_t st) {
    k_link_mask<<<(unsigned)((g.N + NT - 1) / NT), NT, 0, st>>>(g, solid, mask);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// force field F = -grad_h V + g  (isotropic D3Q19 gradient, FP64 arithmetic)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_force_field(Grid g, const double *__restrict__ V, const double *__restrict__ phi,
                              const double *__restrict__ amp, double g0, double g1, double g2, T *__restrict__ F) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const double vi = V[i] + amp[i] * phi[i];
    double gr[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        int X = x + cx(p), Y = y + cy(p), Z = z + cz(p);
        bool ok = wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2]);
        double v = vi;
        if (ok) {
            long long j = X + (long long)g.nx * (Y + (long long)g.ny * Z);
            v = V[j] + amp[j] * phi[j];
        }
        gr[0] += wq(p) * cx(p) * v;
        gr[1] += wq(p) * cy(p) * v;
        gr[2] += wq(p) * cz(p) * v;
    }
    F[i] = (T)(-3.0 * gr[0] + g0);
    F[g.N + i] = (T)(-3.0 * gr[1] + g1);
    F[2 * g.N + i] = (T)(-3.0 * gr[2] + g2);
}

cudaError_t launch_force_field(Prec p, const Grid &g, const double *V, const double *phi, const double *amp,
                               const double gb[3], void *F, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    if (prec_fp64(p))
        k_force_field<double><<<nb, NT, 0, st>>>(g, V, phi, amp, gb[0], gb[1], gb[2], (double *)F);
    else
        k_force_field<float><<<nb, NT, 0, st>>>(g, V, phi, amp, gb[0], gb[1], gb[2], (float *)F);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// populations: streamed FP64 <-> stored post-collision form
// ---------------------------------------------------------------------------
// post_p(s) = streamed_p(s + c_p) when s + c_p is a fluid node inside the
// lattice, else streamed_{opp(p)}(s) (the population bounced back at s).
// A population given in FP64 (host data, rest state) stored in the storage form: the shifted forms take
// the deviation f - w_p n0 formed in FP64, so it keeps its precision.
template <typename S, typename T>
__device__ __forceinline__ void store_full(S *p, double v, double wn0) {
    if constexpr (Store<S, T>::shifted)
        Store<S, T>::store_dev(p, (T)(v - wn0), (T)wn0, wn0 > 0.0 ? (T)(1.0 / wn0) : (T)0);
    else
        Store<S, T>::store(p, (T)v, (T)wn0, (T)0);
}

// The FP64 value of a stored population (the shifted forms add w_p n0 in FP64).
template <typename S, typename T, int P>
__device__ __forceinline__ double pull_full(const S *fb, long long N, long long i, const NbrOff &o, uint32_t m,
                                            double n0) {
    if constexpr (Store<S, T>::shifted)
        return (double)pull_dev<S, T, P>(fb, N, i, o, m, (T)n0) + wq(P) * n0;
    else
        return (double)pull<S, T, P>(fb, N, i, o, m, (T)n0);
}

template <typename S, typename T>
__global__ void k_unstream(Grid g, const uint32_t *__restrict__ mask, const double *__restrict__ f,
                           const double *__restrict__ gq, S *__restrict__ pop, int a, double n0) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    node_xyz(g, s, x, y, z);
    const bool solid = mask[s] & 1u;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        double fv = 0.0, gv = 0.0;
        if (!solid) {
            int X = x + cx(p), Y = y + cy(p), Z = z + cz(p);
            bool ok = wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2]);
            long long t = ok ? X + (long long)g.nx * (Y + (long long)g.ny * Z) : 0;
            if (ok && !(mask[t] & 1u)) {
                fv = f[(long long)p * g.N + t];
                gv = gq[(long long)p * g.N + t];
            } else {
                fv = f[(long long)opp(p) * g.N + s];
                gv = gq[(long long)opp(p) * g.N + s];
            }
        }
        store_full<S, T>(pop + pop_off(a, 0, p, g.N) + s, fv, wq(p) * n0);
        store_full<S, T>(pop + pop_off(a, 1, p, g.N) + s, gv, wq(p) * n0);
    }
}

// Rest state: streamed f_p(r) = w_p n(r) and g_p(r) = w_p Pi(r) on fluid nodes (Pi = n without pi).
template <typename S, typename T>
__global__ void k_rest_state(Grid g, const uint32_t *__restrict__ mask, const double *__restrict__ n,
                             const double *__restrict__ pi, S *__restrict__ pop, int a, double n0) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    int x, y, z;
    node_xyz(g, s, x, y, z);
    const bool solid = mask[s] & 1u;
    const double *gsrc = pi ? pi : n;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        double v = 0.0, vg = 0.0;
        if (!solid) {
            int X = x + cx(p), Y = y + cy(p), Z = z + cz(p);
            bool ok = wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2]);
            long long t = ok ? X + (long long)g.nx * (Y + (long long)g.ny * Z) : 0;
            const long long u = (ok && !(mask[t] & 1u)) ? t : s;
            v = wq(p) * n[u];
            vg = wq(p) * gsrc[u];
        }
        store_full<S, T>(pop + pop_off(a, 0, p, g.N) + s, v, wq(p) * n0);
        store_full<S, T>(pop + pop_off(a, 1, p, g.N) + s, vg, wq(p) * n0);
    }
}

template <typename S, typename T>
__global__ void k_stream_out(Grid g, const uint32_t *__restrict__ mask, const S *__restrict__ pop, int a, double n0,
                             double *__restrict__ f, double *__restrict__ gq) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = mask[i];
    const NbrOff o = nbr_offsets(g, x, y, z);
    const S *fb = pop + pop_off(a, 0, 0, g.N);
    const S *gb = pop + pop_off(a, 1, 0, g.N);
    auto body = [&](auto Pc) {
        constexpr int P = decltype(Pc)::value;
        double fv = 0.0, gv = 0.0;
        if (!(m & 1u)) {
            fv = pull_full<S, T, P>(fb, g.N, i, o, m, n0);
            gv = pull_full<S, T, P>(gb, g.N, i, o, m, n0);
        }
        f[(long long)P * g.N + i] = fv;
        gq[(long long)P * g.N + i] = gv;
    };
    [&]<int... P>(std::integer_sequence<int, P...>) { (body(std::integral_constant<int, P>{}), ...); }
    (std::make_integer_sequence<int, Q>{});
}

#define LBE_DISPATCH_PREC(p, CALL)                                       \
    switch (p) {                                                         \
        case Prec::F64: { using S = double; using T = double; CALL; break; }      \
        case Prec::F32: { using S = float; using T = float; CALL; break; }        \
        case Prec::BF16: { using S = __nv_bfloat16; using T = float; CALL; break; } \
        case Prec::F16: { using S = __half; using T = float; CALL; break; }       \
    }

cudaError_t launch_unstream(Prec p, const Grid &g, const uint32_t *mask, const double *f, const double *gq,
                            void *pop, int a, double n0, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    LBE_DISPATCH_PREC(p, (k_unstream<S, T><<<nb, NT, 0, st>>>(g, mask, f, gq, (S *)pop, a, n0)));
    return cudaGetLastError();
}

cudaError_t launch_rest_state(Prec p, const Grid &g, const uint32_t *mask, const double *n, void *pop, int a,
                              double n0, cudaStream_t st, const double *pi) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    LBE_DISPATCH_PREC(p, (k_rest_state<S, T><<<nb, NT, 0, st>>>(g, mask, n, pi, (S *)pop, a, n0)));
    return cudaGetLastError();
}

cudaError_t launch_stream_out(Prec p, const Grid &g, const uint32_t *mask, const void *pop, int a, double n0,
                              double *f, double *gq, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    LBE_DISPATCH_PREC(p, (k_stream_out<S, T><<<nb, NT, 0, st>>>(g, mask, (const S *)pop, a, n0, f, gq)));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K1: density n^a(r) = sum_p f~_p(r) (streamed), 0 on solid nodes, written to
// the padded stencil field with its periodic images.
// ---------------------------------------------------------------------------
template <typename S, typename T, bool SOLID, int MC>
__global__ void __launch_bounds__(NT) k_density(Grid g, const S *__restrict__ pop, const uint32_t *__restrict__ mask,
                                                int M, N0Vec n0v, N0VecF n0f, T *__restrict__ npad,
                                                int *err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < g.N;
    const uint32_t m = valid ? (SOLID ? mask[i] : 0u) : 1u;
    // two species: a warp none of whose nodes has a blocked link pulls without the bounce-back selects
    // (0.257 -> 0.227 ms on the 512x128x128 channel)
    const bool plain = MC == 2 && (!SOLID || __all_sync(0xffffffffu, (m >> 1) == 0u));
    if (!valid) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const NbrOff o = nbr_offsets(g, x, y, z);  // (without solids every axis is periodic)
    auto n0_of = [&](int a) -> T {
        if constexpr (sc_float<S, T>)
            return n0f.v[a];
        else
            return (T)n0v.v[a];
    };
    // one species' pulled populations (shifted storage: their deviations from w_p n0)
    auto pull_all = [&](int a, T *v) {
        const S *fb = pop + pop_off(a, 0, 0, g.N);
        const T n0 = n0_of(a);
        if (plain) {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (Store<S, T>::shifted)
                    ((v[P] = pull_dev<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
                else
                    ((v[P] = pull<S, T, P, false>(fb, g.N, i, o, m, n0)), ...);
            }(std::make_integer_sequence<int, Q>{});
        } else {
            [&]<int... P>(std::integer_sequence<int, P...>) {
                if constexpr (Store<S, T>::shifted)
                    ((v[P] = pull_dev<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
                else
                    ((v[P] = pull<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
            }(std::make_integer_sequence<int, Q>{});
        }
    };
    // n = n0 + the sum of the deviations (shifted storage), the sum itself otherwise
    auto finish = [&](int a, const T *v) -> T {
        T n = (T)0;
#pragma unroll
        for (int p = 0; p < Q; ++p) n += v[p];
        if constexpr (Store<S, T>::shifted) n = n0_of(a) + n;
        if (!(n >= (T)0) || !isfinite(n)) atomicOr(err, ERR_DENSITY);
        return n;
    };
    if constexpr (MC == 2) {
        // two species: all 38 loads issue before either sum
        T n[2] = {(T)0, (T)0};
        if (!(m & 1u)) {
            T v0[Q], v1[Q];
            pull_all(0, v0);
            pull_all(1, v1);
            n[0] = finish(0, v0);
            n[1] = finish(1, v1);
        }
        write_padded<T>(g, npad, x, y, z, n[0]);
        write_padded<T>(g, npad + g.P, x, y, z, n[1]);
    } else {
        for (int a = 0; a < M; ++a) {
            T n = (T)0;
            if (!(m & 1u)) {
                T v[Q];
                pull_all(a, v);
                n = finish(a, v);
            }
            write_padded<T>(g, npad + (long long)a * g.P, x, y, z, n);
        }
    }
}

cudaError_t launch_density(Prec p, const Grid &g, const void *pop, const uint32_t *mask, bool solid, int M,
                           const double *n0, void *npad, int *err, cudaStream_t st) {
    // one species: one thread per node at 32-42 registers (lbe_collide_pair.cu); measured faster than this
    // kernel for one species (256^3 well 0.42 -> 0.31 ms) and slower for two (0.29 -> 0.31 ms)
    if (M == 1) return launch_density_pair(p, g, pop, mask, solid, M, n0, npad, err, st);
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    N0Vec n0v;
    N0VecF n0f;
    for (int a = 0; a < MAXS; ++a) {
        n0v.v[a] = a < M ? n0[a] : 0.0;
        n0f.v[a] = (float)n0v.v[a];
    }
#define LBE_K1(SOL, MC) \
    LBE_DISPATCH_PREC(p, (k_density<S, T, SOL, MC><<<nb, NT, 0, st>>>(g, (const S *)pop, mask, M, n0v, n0f, (T *)npad, err)))
    if (M == 2) {
        if (solid) {
            LBE_K1(true, 2);
        } else {
            LBE_K1(false, 2);
        }
    } else if (solid) {
        LBE_K1(true, 0);
    } else {
        LBE_K1(false, 0);
    }
#undef LBE_K1
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4: fused moments + DD-TR collision + streaming (Sec. "Hard sphere fluid
// mixture in a potential well"):
//   n = sum f~, Pi~ = sum g~, J~ = sum c g~;
//   printed recovery:    J = J~ + (C + nF)/2,  Pi = Pi~ - C.u^a/2;
//   consistent recovery: J = J~ + nF/2,        Pi = Pi~ + beta C.u^a/2;
//   u^a = J/n, u = sum J / sum n;
//   f_eq = w [n + n u^a.H1 + n (2 u^a u - u u):H2],  g_eq = same with Pi first;
//   S_f = w (C + nF).[H1 + 2 H2.u^a];
//   S_g = w { C.[u^a/v_T^2 + 4 H2.u^a] + nF.[H1 + 2 H2.u^a] };
//   f~* = f~ + [omega (f_eq - f~) + S_f] / (1 + omega/2)   (same for g~).
// With v_T^2 = 1/3 the Hermite contractions expand to the scalar forms below
// (A, B isotropic parts; sf0 = -3 (C + nF).u^a is shared by S_f and S_g).
// ---------------------------------------------------------------------------
// Per-node moments of every species.  With KEEP the pulled populations stay
// in registers for the collision (one species); otherwise they are pulled
// again species by species in the collision pass (the second pull hits L2).
template <typename S, typename T, int M, bool KEEP>
struct NodeState {
    T f[KEEP ? M : 1][Q], g[KEEP ? M : 1][Q];
    T n[M], Pi[M], J[M][3], C[M][3], nF[M][3], ua[M][3];
    T u[3];
};

template <typename S, typename T, bool SOLID>
__device__ __forceinline__ void pull_species(const Grid &g, const S *__restrict__ src, int a, T n0, long long i,
                                             const NbrOff &o, uint32_t m, T *f, T *gq) {
    const S *fb = src + pop_off(a, 0, 0, g.N);
    const S *gb = src + pop_off(a, 1, 0, g.N);
    [&]<int... P>(std::integer_sequence<int, P...>) {
        ((f[P] = pull<S, T, P, SOLID>(fb, g.N, i, o, m, n0)), ...);
        ((gq[P] = pull<S, T, P, SOLID>(gb, g.N, i, o, m, n0)), ...);
    }(std::make_integer_sequence<int, Q>{});
}

template <typename S, typename T, int M, bool SOLID, bool KEEP>
__device__ __forceinline__ void load_moments(const Grid &g, const S *__restrict__ src, const T *__restrict__ C,
                                             const T *__restrict__ F, const StepParams &sp, long long i,
                                             const NbrOff &o, uint32_t m, NodeState<S, T, M, KEEP> &st) {
    T ntot = 0, Jtot[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T n0 = sc_n0<S, T>(sp.sp[a]);
        T fl[Q], gl[Q];
        T *f = KEEP ? st.f[KEEP ? a : 0] : fl;
        T *gq = KEEP ? st.g[KEEP ? a : 0] : gl;
        pull_species<S, T, SOLID>(g, src, a, n0, i, o, m, f, gq);
        T n = 0, Pit = 0, Jt[3] = {0, 0, 0};
        [&]<int... P>(std::integer_sequence<int, P...>) {
            ((n += f[P]), ...);
            ((Pit += gq[P]), ...);
            ((Jt[0] += (T)cx(P) * gq[P]), ...);
            ((Jt[1] += (T)cy(P) * gq[P]), ...);
            ((Jt[2] += (T)cz(P) * gq[P]), ...);
        }(std::make_integer_sequence<int, Q>{});
        const T *Ca = C + (long long)a * 3 * g.N + i;
        const T *Fa = F + (long long)a * 3 * g.N + i;
        T Cu = 0;
        const T inv_n = n > (T)0 ? (T)1 / n : (T)0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st.C[a][c] = Ca[(long long)c * g.N];
            st.nF[a][c] = n * Fa[(long long)c * g.N];
            st.J[a][c] = sp.consistent ? Jt[c] + (T)0.5 * st.nF[a][c]
                                       : Jt[c] + (T)0.5 * (st.C[a][c] + st.nF[a][c]);
            st.ua[a][c] = st.J[a][c] * inv_n;
            Cu += st.C[a][c] * st.ua[a][c];
            Jtot[c] += st.J[a][c];
        }
        st.n[a] = n;
        st.Pi[a] = sp.consistent ? Pit + (T)1.5 * Cu : Pit - (T)0.5 * Cu;
        ntot += n;
    }
    const T inv_tot = ntot > (T)0 ? (T)1 / ntot : (T)0;
#pragma unroll
    for (int c = 0; c < 3; ++c) st.u[c] = Jtot[c] * inv_tot;
}

template <typename S, typename T, int M, bool SOLID>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (M == 1 ? 3 : 2) : 1)
    k_collide(Grid g, const S *__restrict__ src, S *__restrict__ dst,
                                                const uint32_t *__restrict__ mask, const T *__restrict__ C,
                                                const T *__restrict__ F, StepParams sp,
                                                double *__restrict__ flux_buf) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = SOLID ? mask[i] : 0u;
    const int coord = sp.flux_axis == 0 ? x : (sp.flux_axis == 1 ? y : z);
    const bool on_plane = sp.flux_axis >= 0 && coord == sp.flux_plane;
    const int psize = sp.flux_axis == 0 ? g.ny * g.nz : (sp.flux_axis == 1 ? g.nx * g.nz : g.nx * g.ny);
    if (m & 1u) {  // solid node: no fluid
        if (on_plane)
            for (int a = 0; a < M; ++a) flux_buf[(long long)a * psize + plane_index(g, sp.flux_axis, x, y, z)] = 0.0;
        return;
    }
    const NbrOff o = nbr_offsets(g, x, y, z);
    constexpr bool KEEP = (M == 1);
    NodeState<S, T, M, KEEP> st;
    load_moments<S, T, M, SOLID, KEEP>(g, src, C, F, sp, i, o, m, st);
    if (on_plane) {
#pragma unroll
        for (int a = 0; a < M; ++a)
            flux_buf[(long long)a * psize + plane_index(g, sp.flux_axis, x, y, z)] = (double)st.J[a][sp.flux_axis];
    }
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T n = st.n[a];
        const T *ua = st.ua[a];
        const T uau = ua[0] * st.u[0] + ua[1] * st.u[1] + ua[2] * st.u[2];
        const T uu = st.u[0] * st.u[0] + st.u[1] * st.u[1] + st.u[2] * st.u[2];
        const T iso = (T)1.5 * n * ((T)2 * uau - uu);
        const T A = n - iso;
        const T B = st.Pi[a] - iso;
        T X[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = st.C[a][c] + st.nF[a][c];
        const T sf0 = (T)-3 * (X[0] * ua[0] + X[1] * ua[1] + X[2] * ua[2]);
        const T om = sc_omega<S, T>(sp.sp[a]);
        const T inv = sc_inv<S, T>(sp.sp[a]);
        const T in0 = sc_in0<S, T>(sp.sp[a]);
        T fl[Q], gl[Q];
        const T *fa = st.f[0];
        const T *ga = st.g[0];
        if constexpr (KEEP) {
            fa = st.f[KEEP ? a : 0];
            ga = st.g[KEEP ? a : 0];
        } else {
            pull_species<S, T, SOLID>(g, src, a, sc_n0<S, T>(sp.sp[a]), i, o, m, fl, gl);
            fa = fl;
            ga = gl;
        }
        S *fo = dst + pop_off(a, 0, 0, g.N) + i;
        S *go = dst + pop_off(a, 1, 0, g.N) + i;
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    constexpr T w = (T)wq(P);
                    const T cua = cdot<T, P>(ua);
                    const T cu = cdot<T, P>(st.u);
                    const T cX = cdot<T, P>(X);
                    const T cY = cdot<T, P>(st.nF[a]);
                    const T cC = cdot<T, P>(st.C[a]);
                    const T t1 = (T)3 * n * cua + (T)4.5 * n * ((T)2 * cua * cu - cu * cu);
                    const T feq = w * (A + t1);
                    const T geq = w * (B + t1);
                    const T Sf = w * (sf0 + (T)3 * cX + (T)9 * cX * cua);
                    const T Sg = w * (sf0 + (T)3 * cY + (T)18 * cC * cua + (T)9 * cY * cua);
                    const T fs = fa[P] + om * (feq - fa[P]) + inv * Sf;
                    const T gs = ga[P] + om * (geq - ga[P]) + inv * Sg;
                    constexpr T iw = (T)(1.0 / wq(P));
                    Store<S, T>::store(fo + (long long)P * g.N, fs, w * sc_n0<S, T>(sp.sp[a]), iw * in0);
                    Store<S, T>::store(go + (long long)P * g.N, gs, w * sc_n0<S, T>(sp.sp[a]), iw * in0);
                }(),
                ...);
        }(std::make_integer_sequence<int, Q>{});
    }
}

template <typename S, typename T, bool SOLID>
static cudaError_t collide_m(int M, const Grid &g, const void *src, void *dst, const uint32_t *mask, const void *C,
                             const void *F, const StepParams &sp, double *flux_buf, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
#define LBE_COLLIDE(MM)                                                                                   \
    k_collide<S, T, MM, SOLID><<<nb, NT, 0, st>>>(g, (const S *)src, (S *)dst, mask, (const T *)C, (const T *)F, \
                                                  sp, flux_buf)
    switch (M) {  // one or two species: k_collide_pair (lbe_collide_pair.cu)
        case 3: LBE_COLLIDE(3); break;
        case 4: LBE_COLLIDE(4); break;
        default: return cudaErrorInvalidValue;
    }
#undef LBE_COLLIDE
    return cudaGetLastError();
}

cudaError_t launch_collide(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask, bool solid,
                           const void *C, const void *F, const StepParams &sp, double *flux_buf, cudaStream_t st) {
    if (sp.M <= 2) return launch_collide_pair(p, g, src, dst, mask, solid, C, F, sp, flux_buf, st);
    cudaError_t e = cudaSuccess;
    if (solid) {
        LBE_DISPATCH_PREC(p, (e = collide_m<S, T, true>(sp.M, g, src, dst, mask, C, F, sp, flux_buf, st)));
    } else {
        LBE_DISPATCH_PREC(p, (e = collide_m<S, T, false>(sp.M, g, src, dst, mask, C, F, sp, flux_buf, st)));
    }
    return e;
}

// Moments of the current state for the getters: n [M][N], J [M][3][N] (FP64).
template <typename S, typename T, int M>
__global__ void __launch_bounds__(NT) k_moments(Grid g, const S *__restrict__ src, const uint32_t *__restrict__ mask,
                                                const T *__restrict__ C, const T *__restrict__ F, StepParams sp,
                                                double *__restrict__ nout, double *__restrict__ Jout) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = mask[i];
    if (m & 1u) {
        for (int a = 0; a < M; ++a) {
            nout[(long long)a * g.N + i] = 0.0;
            for (int c = 0; c < 3; ++c) Jout[((long long)a * 3 + c) * g.N + i] = 0.0;
        }
        return;
    }
    const NbrOff o = nbr_offsets(g, x, y, z);
    NodeState<S, T, M, false> st;
    load_moments<S, T, M, true, false>(g, src, C, F, sp, i, o, m, st);
    for (int a = 0; a < M; ++a) {
        nout[(long long)a * g.N + i] = (double)st.n[a];
        for (int c = 0; c < 3; ++c) Jout[((long long)a * 3 + c) * g.N + i] = (double)st.J[a][c];
    }
}

template <typename S, typename T>
static cudaError_t moments_m(int M, const Grid &g, const void *pop, const uint32_t *mask, const void *C, const void *F,
                             const StepParams &sp, double *n, double *J, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    switch (M) {
        case 1: k_moments<S, T, 1><<<nb, NT, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp, n, J); break;
        case 2: k_moments<S, T, 2><<<nb, NT, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp, n, J); break;
        case 3: k_moments<S, T, 3><<<nb, NT, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp, n, J); break;
        case 4: k_moments<S, T, 4><<<nb, NT, 0, st>>>(g, (const S *)pop, mask, (const T *)C, (const T *)F, sp, n, J); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *C,
                           const void *F, const StepParams &sp, double *n, double *J, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    LBE_DISPATCH_PREC(p, (e = moments_m<S, T>(sp.M, g, pop, mask, C, F, sp, n, J, st)));
    return e;
}

// ---------------------------------------------------------------------------
// K5 and FP64 reductions (deterministic: fixed per-thread order, fixed tree).
// ---------------------------------------------------------------------------
template <int NTH>
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NTH / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;  // valid in thread 0
}
template <int NTH>
__device__ __forceinline__ double block_max(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NTH / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(1024) k_flux_reduce(int M, int psize, const double *__restrict__ buf,
                                                      double *__restrict__ acc, double *__restrict__ last) {
    __shared__ double sh[32];
    for (int a = 0; a < M; ++a) {
        double s = 0.0;
        for (int k = threadIdx.x; k < psize; k += 1024) s += buf[(long long)a * psize + k];
        s = block_sum<1024>(s, sh);
        if (threadIdx.x == 0) {
            acc[a] += s;
            last[a] = s;
        }
    }
}

cudaError_t launch_flux_reduce(int M, int plane_size, const double *buf, double *acc, double *last,
                               cudaStream_t st) {
    k_flux_reduce<<<1, 1024, 0, st>>>(M, plane_size, buf, acc, last);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) k_reduce_partial(const double *__restrict__ x, long long n, long long chunk,
                                                       double *__restrict__ partial) {
    __shared__ double sh[32];
    const long long b0 = (long long)blockIdx.x * chunk;
    const long long b1 = min(n, b0 + chunk);
    double s = 0.0, mx = 0.0;
    for (long long k = b0 + threadIdx.x; k < b1; k += NT) {
        s += x[k];
        mx = fmax(mx, fabs(x[k]));
    }
    s = block_sum<NT>(s, sh);
    mx = block_max<NT>(mx, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s;
        partial[2 * blockIdx.x + 1] = mx;
    }
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double *__restrict__ partial, int np,
                                                       double *__restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0, mx = 0.0;
    for (int k = threadIdx.x; k < np; k += 1024) {
        s += partial[2 * k];
        mx = fmax(mx, partial[2 * k + 1]);
    }
    s = block_sum<1024>(s, sh);
    mx = block_max<1024>(mx, sh);
    if (threadIdx.x == 0) {
        out[0] = s;
        out[1] = mx;
    }
}

cudaError_t launch_reduce(const double *x, long long n, double *partial, int npartial, double *out,
                          cudaStream_t st) {
    long long chunk = (n + npartial - 1) / npartial;
    if (chunk < 1) chunk = 1;
    int nb = (int)((n + chunk - 1) / chunk);
    if (nb < 1) nb = 1;
    k_reduce_partial<<<nb, NT, 0, st>>>(x, n, chunk, partial);
    k_reduce_final<<<1, 1024, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ src, long long n, double *__restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

cudaError_t launch_to_f64(bool fp64, const void *src, long long n, double *dst, cudaStream_t st) {
    unsigned nb = (unsigned)((n + NT - 1) / NT);
    if (fp64)
        k_to_f64<double><<<nb, NT, 0, st>>>((const double *)src, n, dst);
    else
        k_to_f64<float><<<nb, NT, 0, st>>>((const float *)src, n, dst);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_unpad(Grid g, const T *__restrict__ pad, double *__restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    dst[i] = (double)pad[pidx(g, x, y, z)];
}

cudaError_t launch_unpad(bool fp64, const Grid &g, const void *pad, double *dst, cudaStream_t st) {
    unsigned nb = (unsigned)((g.N + NT - 1) / NT);
    if (fp64)
        k_unpad<double><<<nb, NT, 0, st>>>(g, (const double *)pad, dst);
    else
        k_unpad<float><<<nb, NT, 0, st>>>(g, (const float *)pad, dst);
    return cudaGetLastError();
}

// Velocity u = sum_sel J / sum_sel n (sel: species s, or all for s < 0), 0 where n = 0.
__global__ void k_velocity(int M, long long N, int s, const double *__restrict__ n, const double *__restrict__ J,
                           double *__restrict__ u, double *__restrict__ speed) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double nn = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
    for (int a = 0; a < M; ++a) {
        if (s >= 0 && a != s) continue;
        nn += n[(long long)a * N + i];
        j0 += J[((long long)a * 3 + 0) * N + i];
        j1 += J[((long long)a * 3 + 1) * N + i];
        j2 += J[((long long)a * 3 + 2) * N + i];
    }
    const double r = nn > 0.0 ? 1.0 / nn : 0.0;
    if (u) {
        u[i] = j0 * r;
        u[N + i] = j1 * r;
        u[2 * N + i] = j2 * r;
    }
    if (speed) speed[i] = sqrt(j0 * j0 + j1 * j1 + j2 * j2) * r;
}

cudaError_t launch_velocity(int M, long long N, int s, const double *n, const double *J, double *u, double *speed,
                            cudaStream_t st) {
    k_velocity<<<(unsigned)((N + NT - 1) / NT), NT, 0, st>>>(M, N, s, n, J, u, speed);
    return cudaGetLastError();
}

// Self-test of the failure detector of the TMA kernels: one thread arms an mbarrier for 16 bytes that
// no copy will deliver (none is issued, so nothing is in flight) and waits on it with the kernels'
// bounded wait, limited to `polls` polls.  The wait gives up and records ERR_TMA_WAIT in the error
// word, as a kernel whose copy never completed would; the barrier is invalidated before the CTA exits.
__global__ void k_wait_probe(int *err, long long polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16u);
        mbar_wait_bounded(&bar, 0u, err, polls);
        mbar_inval(&bar);
    }
}

cudaError_t launch_wait_probe(int *err, long long polls, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(err, polls);
    return cudaGetLastError();
}

}  // namespace lbe
