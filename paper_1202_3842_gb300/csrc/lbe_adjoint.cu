// Discrete adjoint of the DD-TR step (reverse mode, hand-derived), for the
// gradient of the time-averaged plane flux
//   Phi = (1/T) sum_{t<T} sum_a sum_{plane, fluid} J^a_axis(t)
// with respect to the force field F^a(r) (and through it the wall-potential
// amplitude and the body force).  One reverse step at time t takes the adjoint
// of the streamed populations at t+1 and produces the adjoint at t:
//   K4^T  k_adj_collide   streaming transpose (push-gather), collision and moment
//                         recovery transposed node by node; emits lambda_C, adds lambda_F
//                         and the adjoint moments (ln, lPi, lJ) of each species;
//         k_adj_write     the adjoint of the pre-collision populations from them
//                         (three or four species; one or two species run all of K4^T
//                         in k_adj_collide_pair, lbe_adj_collide_pair.cu)
//   K3^T  k_adj_shell_prep / k_adj_shell_tile   shell force transposed: node-local
//                         terms, then divergence-type shell sums of the weighted
//                         adjoint from shared-memory tiles (lbe_adj_shell.cuh)
//   K2^T  k_adj_contact_prep / k_contact_tma<MODE 1>  BMCSL contact value and ball
//                         average transposed
//   K1^T  the density adjoint is kept as a field and added in the next push-gather
// All arithmetic in the precision T of the populations (FP32 or FP64).
#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int ANT = 256;
constexpr int ACT = 256;  // k_adj_collide: two CTAs per SM (FP32: 128 registers), one (FP64)

// Adjoint of the post-collision population p of species a at node i, gathered
// from the adjoint of the streamed populations at t+1 (the streaming is a
// permutation; its transpose sends post_p(r) to r + c_p, or back to opp(p) at r
// when that link is blocked).  For f the density-path adjoint ln is added.
template <typename T, int P>
__device__ __forceinline__ T gather_post(const T *__restrict__ lY, const T *__restrict__ ln, long long N, long long i,
                                         const NbrOff &o, uint32_t m) {
    if (m & (1u << opp(P))) {
        const T v = lY[(long long)opp(P) * N + i];
        return ln ? v + ln[i] : v;
    }
    const long long j = i + src_off<opp(P)>(o);  // r + c_P
    const T v = lY[(long long)P * N + j];
    return ln ? v + ln[j] : v;
}

template <typename S, typename T, int M>
__global__ void __launch_bounds__(ACT, sizeof(T) == 4 ? 2 : 1)
    k_adj_collide(Grid g, const S *__restrict__ post, const uint32_t *__restrict__ mask, const T *__restrict__ C,
                  const T *__restrict__ F, AdjParams ap, const T *__restrict__ lYf_in, const T *__restrict__ lYg_in,
                  const T *__restrict__ lnd_in, T *__restrict__ lmom, T *__restrict__ lC, T *__restrict__ lF) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const uint32_t m = mask[i];
    if (m & 1u) {
        for (int a = 0; a < M; ++a)
            for (int c = 0; c < 3; ++c) lC[((long long)a * 3 + c) * g.N + i] = (T)0;
        return;
    }
    const NbrOff o = nbr_offsets(g, x, y, z);
    // ---- forward moments (pass A)
    T n[M], inv_n[M], Pi[M], J[M][3], ua[M][3], Cv[M][3], Fv[M][3], nF[M][3];
    T ntot = 0, Jtot[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T n0 = (T)ap.sp[a].n0;
        const S *fb = post + pop_off(a, 0, 0, g.N);
        const S *gb = post + pop_off(a, 1, 0, g.N);
        T na = 0, Pit = 0, Jt[3] = {0, 0, 0};
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    const T fv = pull<S, T, P, true>(fb, g.N, i, o, m, n0);
                    const T gv = pull<S, T, P, true>(gb, g.N, i, o, m, n0);
                    na += fv;
                    Pit += gv;
                    Jt[0] += (T)cx(P) * gv;
                    Jt[1] += (T)cy(P) * gv;
                    Jt[2] += (T)cz(P) * gv;
                }(),
                ...);
        }(std::make_integer_sequence<int, Q>{});
        n[a] = na;
        inv_n[a] = na > (T)0 ? (T)1 / na : (T)0;
        T Cu = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Cv[a][c] = C[((long long)a * 3 + c) * g.N + i];
            Fv[a][c] = F[((long long)a * 3 + c) * g.N + i];
            nF[a][c] = na * Fv[a][c];
            J[a][c] = ap.consistent ? Jt[c] + (T)0.5 * nF[a][c] : Jt[c] + (T)0.5 * (Cv[a][c] + nF[a][c]);
            ua[a][c] = J[a][c] * inv_n[a];
            Cu += Cv[a][c] * ua[a][c];
            Jtot[c] += J[a][c];
        }
        Pi[a] = ap.consistent ? Pit + (T)1.5 * Cu : Pit - (T)0.5 * Cu;
        ntot += na;
    }
    (void)Pi;
    const T inv_tot = ntot > (T)0 ? (T)1 / ntot : (T)0;
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = Jtot[c] * inv_tot;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // ---- reverse of the collision (pass B)
    T lu[3] = {0, 0, 0};
    T lua[M][3], lCs[M][3], lnFs[M][3], lns[M], lPis[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T om = (T)ap.sp[a].omega_eff, inv = (T)ap.sp[a].inv;
        const T na = n[a];
        const T uau = ua[a][0] * u[0] + ua[a][1] * u[1] + ua[a][2] * u[2];
        T X[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = Cv[a][c] + nF[a][c];
        T lA = 0, lB = 0, lsf0 = 0, lnv = 0;
        T lX[3] = {0, 0, 0}, lnFv[3] = {0, 0, 0}, lCv[3] = {0, 0, 0}, luav[3] = {0, 0, 0}, lua_u[3] = {0, 0, 0};
        const T *lYf = lYf_in + (long long)a * Q * g.N;
        const T *lYg = lYg_in + (long long)a * Q * g.N;
        const T *lnd = lnd_in + (long long)a * g.N;
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    constexpr T w = (T)wq(P);
                    const T lfs = gather_post<T, P>(lYf, lnd, g.N, i, o, m);
                    const T lgs = gather_post<T, P>(lYg, nullptr, g.N, i, o, m);
                    const T cua = cdot<T, P>(ua[a]);
                    const T cu = cdot<T, P>(u);
                    const T cX = cdot<T, P>(X);
                    const T cY = cdot<T, P>(nF[a]);
                    const T cC = cdot<T, P>(Cv[a]);
                    const T lSf = inv * lfs, lSg = inv * lgs;
                    const T lt1 = w * om * (lfs + lgs);
                    lA += w * om * lfs;
                    lB += w * om * lgs;
                    lsf0 += w * (lSf + lSg);
                    const T lcX = w * lSf * ((T)3 + (T)9 * cua);
                    const T lcY = w * lSg * ((T)3 + (T)9 * cua);
                    const T lcC = (T)18 * w * lSg * cua;
                    const T lcua = (T)9 * w * lSf * cX + w * lSg * ((T)18 * cC + (T)9 * cY) +
                                   lt1 * ((T)3 * na + (T)9 * na * cu);
                    const T lcu = (T)9 * na * (cua - cu) * lt1;
                    lnv += lt1 * ((T)3 * cua + (T)4.5 * ((T)2 * cua * cu - cu * cu));
                    if constexpr (cx(P) != 0) {
                        luav[0] += (T)cx(P) * lcua; lua_u[0] += (T)cx(P) * lcu; lX[0] += (T)cx(P) * lcX;
                        lnFv[0] += (T)cx(P) * lcY; lCv[0] += (T)cx(P) * lcC;
                    }
                    if constexpr (cy(P) != 0) {
                        luav[1] += (T)cy(P) * lcua; lua_u[1] += (T)cy(P) * lcu; lX[1] += (T)cy(P) * lcX;
                        lnFv[1] += (T)cy(P) * lcY; lCv[1] += (T)cy(P) * lcC;
                    }
                    if constexpr (cz(P) != 0) {
                        luav[2] += (T)cz(P) * lcua; lua_u[2] += (T)cz(P) * lcu; lX[2] += (T)cz(P) * lcX;
                        lnFv[2] += (T)cz(P) * lcY; lCv[2] += (T)cz(P) * lcC;
                    }
                }(),
                ...);
        }(std::make_integer_sequence<int, Q>{});
        // sf0 = -3 X.u^a ; X = C + nF ; A = n - iso ; B = Pi - iso ; iso = 1.5 n (2 u^a.u - u.u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lX[c] += (T)-3 * ua[a][c] * lsf0;
            luav[c] += (T)-3 * X[c] * lsf0;
            lCv[c] += lX[c];
            lnFv[c] += lX[c];
        }
        const T liso = -lA - lB;
        lnv += lA + (T)1.5 * ((T)2 * uau - uu) * liso;
        const T luau = (T)3 * na * liso;
        const T luu = (T)-1.5 * na * liso;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            luav[c] += u[c] * luau;
            lu[c] += lua_u[c] + ua[a][c] * luau + (T)2 * u[c] * luu;
            lua[a][c] = luav[c];
            lCs[a][c] = lCv[c];
            lnFs[a][c] = lnFv[c];
        }
        lns[a] = lnv;
        lPis[a] = lB;
    }
    // ---- u = sum J / sum n
    T lJtot[3] = {0, 0, 0}, lntot = 0;
    if (ntot > (T)0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lJtot[c] = lu[c] * inv_tot;
            lntot -= lu[c] * u[c] * inv_tot;
        }
    }
    // ---- reverse of the moment recovery (pass C) and the outputs
    const int coord = ap.axis == 0 ? x : (ap.axis == 1 ? y : z);
    const bool on_plane = ap.axis >= 0 && coord == ap.plane;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const T om = (T)ap.sp[a].omega_eff;
        const T kPi = ap.consistent ? (T)1.5 : (T)-0.5;
        const T lPit = lPis[a];
        const T lCu = kPi * lPis[a];
        T lJ[3], lCv[3], luav[3];
        T ln = lns[a] + lntot;
        T dot = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lCv[c] = lCs[a][c] + ua[a][c] * lCu;
            luav[c] = lua[a][c] + Cv[a][c] * lCu;
            lJ[c] = lJtot[c] + luav[c] * inv_n[a];
            dot += luav[c] * ua[a][c];
        }
        ln -= dot * inv_n[a];
        if (on_plane) lJ[ap.axis] += (T)ap.wobj;
        T lnF[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lnF[c] = lnFs[a][c] + (T)0.5 * lJ[c];
            if (!ap.consistent) lCv[c] += (T)0.5 * lJ[c];
            ln += lnF[c] * Fv[a][c];
            lF[((long long)a * 3 + c) * g.N + i] += n[a] * lnF[c];
            lC[((long long)a * 3 + c) * g.N + i] = lCv[c];
        }
        // adjoint moments of the pre-collision populations, for k_adj_write
        T *lm = lmom + (long long)a * 5 * g.N + i;
        lm[0] = ln;
        lm[g.N] = lPit;
        lm[2 * g.N] = lJ[0];
        lm[3 * g.N] = lJ[1];
        lm[4 * g.N] = lJ[2];
    }
}

// Adjoint of the pre-collision populations of species a = blockIdx.y at time t:
//   lf_p = (1 - omega_eff) lf*_p + ln,   lg_p = (1 - omega_eff) lg*_p + lPi + c_p.lJ,
// lf*_p, lg*_p the push-gathered adjoint of the post-collision populations (density adjoint added
// to f) and (ln, lPi, lJ) the adjoint moments from k_adj_collide.  Zero on solid nodes.
template <typename T>
__global__ void __launch_bounds__(ANT)
    k_adj_write(Grid g, const uint32_t *__restrict__ mask, AdjParams ap, const T *__restrict__ lYf_in,
                const T *__restrict__ lYg_in, const T *__restrict__ lnd_in, const T *__restrict__ lmom,
                T *__restrict__ lYf_out, T *__restrict__ lYg_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const int a = blockIdx.y;
    T *of = lYf_out + (long long)a * Q * g.N + i;
    T *og = lYg_out + (long long)a * Q * g.N + i;
    const uint32_t m = mask[i];
    if (m & 1u) {
#pragma unroll
        for (int p = 0; p < Q; ++p) {
            of[(long long)p * g.N] = (T)0;
            og[(long long)p * g.N] = (T)0;
        }
        return;
    }
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const NbrOff o = nbr_offsets(g, x, y, z);
    const T om1 = (T)1 - (T)ap.sp[a].omega_eff;
    const T *lm = lmom + (long long)a * 5 * g.N + i;
    const T ln = lm[0], lPit = lm[g.N];
    const T lJ[3] = {lm[2 * g.N], lm[3 * g.N], lm[4 * g.N]};
    const T *lYf = lYf_in + (long long)a * Q * g.N;
    const T *lYg = lYg_in + (long long)a * Q * g.N;
    const T *lnd = lnd_in + (long long)a * g.N;
    [&]<int... P>(std::integer_sequence<int, P...>) {
        (
            [&] {
                const T lfs = gather_post<T, P>(lYf, lnd, g.N, i, o, m);
                const T lgs = gather_post<T, P>(lYg, nullptr, g.N, i, o, m);
                of[(long long)P * g.N] = om1 * lfs + ln;
                og[(long long)P * g.N] = om1 * lgs + lPit + cdot<T, P>(lJ);
            }(),
            ...);
    }(std::make_integer_sequence<int, Q>{});
}

// ---------------------------------------------------------------------------
// Shell force transposed, pair (a, b), node-local part.  C^a += coef n_a
// [g/2 P + Q/2] with P = sum_e e^ n_b(r+e), Q = sum_e e^ (g n_b)(r+e).  With
// Lambda = coef n_a lC^a / 2 this kernel writes the padded fields Lambda and
// g Lambda (read by the shell sums of lbe_adj_shell.cuh) and adds
//   lg(s)   += Lambda(s).P(s),
//   ln_a(s) += C^a(s).lC^a(s) / n_a(s)      (own = 1: once per species a;
// summed over b, coef/2 (g P + Q).lC^a is C^a.lC^a / n_a).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_shell_prep(Grid g, const T *__restrict__ npad_a, const T *__restrict__ gab,
                                 const T *__restrict__ lC_a, const T *__restrict__ P, const T *__restrict__ C_a,
                                 T coef, int own, T *__restrict__ Lpad, T *__restrict__ gLpad, T *__restrict__ ln_a,
                                 T *__restrict__ lg) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const T na = npad_a[pidx(g, x, y, z)];
    const T s = (T)0.5 * coef * na;
    const T gv = gab[i];
    T lp = 0, cl = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T lc = lC_a[(long long)c * g.N + i];
        const T L = s * lc;
        if (!Lpad) {  // the spectral transposes form Lambda themselves
        } else if constexpr (sizeof(T) == 4) {  // FP32: interleaved (Lambda_c, g Lambda_c), [3][P] float2 in Lpad
            write_padded<float2>(g, reinterpret_cast<float2 *>(Lpad) + (long long)c * g.P, x, y, z,
                                 make_float2(L, gv * L));
        } else {
            write_padded<T>(g, Lpad + (long long)c * g.P, x, y, z, L);
            write_padded<T>(g, gLpad + (long long)c * g.P, x, y, z, gv * L);
        }
        lp += L * P[(long long)c * g.N + i];
        cl += C_a[(long long)c * g.N + i] * lc;
    }
    lg[i] += lp;
    if (own && na != (T)0) ln_a[i] += cl / na;
}

// ---------------------------------------------------------------------------
// Contact value transposed (first half; the ball average's transpose is the
// TMA ball sum of lbe_adj_ball.cu).  From the xi2, xi3 kept by the forward
// contact kernel:
//   lxi2 = sum_ab lg_ab dg_ab/dxi2, lxi3 = sum_ab lg_ab dg_ab/dxi3,
//   lnbar_b = (pi/6)(sigma_b^2 lxi2 + sigma_b^3 lxi3) / |B_b|  (padded).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_contact_prep(Grid g, ContactParams cp, BallRows br, const T *__restrict__ xi,
                                   const T *__restrict__ lg, T *__restrict__ lnbar) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const T xi2 = xi[i], xi3 = xi[g.N + i];
    const T i1 = (T)1 / ((T)1 - xi3);
    T l2 = 0, l3 = 0;
    for (int a = 0; a < cp.M; ++a)
        for (int b = 0; b < cp.M; ++b) {
            const T s = (T)cp.s_ab[a][b];
            const T lgv = lg[(long long)(a * cp.M + b) * g.N + i];
            l2 += lgv * ((T)3 * s * i1 * i1 + (T)4 * s * s * xi2 * i1 * i1 * i1);
            l3 += lgv * (i1 * i1 + (T)6 * s * xi2 * i1 * i1 * i1 + (T)6 * s * s * xi2 * xi2 * i1 * i1 * i1 * i1);
        }
    for (int b = 0; b < cp.M; ++b) {
        const T v = ((T)cp.xi2c[b] * l2 + (T)cp.xi3c[b] * l3) / (T)br.count[b];
        write_padded<T>(g, lnbar + (long long)b * g.P, x, y, z, v);
    }
}

// ---------------------------------------------------------------------------
// Force field transposed: F^a_c(r) = -3 sum_p w_p c_pc (V^a + amp phi)(nb_p(r)) + g_c, nb_p(r) = r + c_p,
// or r itself when r + c_p leaves a closed axis.  dPhi/damp(s) = -3 phi(s) sum_a sum_p w_p
//   [ c_p . lF^a(s - c_p) if s - c_p is a node ] + [ c_p . lF^a(s) if s + c_p is outside ].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_amp(Grid g, int M, const T *__restrict__ lF, const double *__restrict__ phi,
                          double *__restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double acc = 0.0;
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        int X = x - cx(p), Y = y - cy(p), Z = z - cz(p);
        if (wrap(X, g.nx, g.per[0]) && wrap(Y, g.ny, g.per[1]) && wrap(Z, g.nz, g.per[2])) {
            const long long r = X + (long long)g.nx * (Y + (long long)g.ny * Z);
            for (int a = 0; a < M; ++a)
                acc += wq(p) * ((double)cx(p) * (double)lF[((long long)a * 3 + 0) * g.N + r] +
                                (double)cy(p) * (double)lF[((long long)a * 3 + 1) * g.N + r] +
                                (double)cz(p) * (double)lF[((long long)a * 3 + 2) * g.N + r]);
        }
        int X2 = x + cx(p), Y2 = y + cy(p), Z2 = z + cz(p);
        if (!(wrap(X2, g.nx, g.per[0]) && wrap(Y2, g.ny, g.per[1]) && wrap(Z2, g.nz, g.per[2]))) {
            for (int a = 0; a < M; ++a)
                acc += wq(p) * ((double)cx(p) * (double)lF[((long long)a * 3 + 0) * g.N + i] +
                                (double)cy(p) * (double)lF[((long long)a * 3 + 1) * g.N + i] +
                                (double)cz(p) * (double)lF[((long long)a * 3 + 2) * g.N + i]);
        }
    }
    out[i] = -3.0 * phi[i] * acc;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define LBE_ADJ_DISPATCH(p, ...)                                                  \
    switch (p) {                                                                  \
        case Prec::F64: { using S = double; using T = double; __VA_ARGS__; break; } \
        case Prec::F32: { using S = float; using T = float; __VA_ARGS__; break; }   \
        default: return cudaErrorInvalidValue;                                    \
    }

cudaError_t launch_adj_collide(Prec p, const Grid &g, const void *post, const uint32_t *mask, const void *C,
                               const void *F, const AdjParams &ap, const void *lYf_in, const void *lYg_in,
                               const void *lnd_in, void *lYf_out, void *lYg_out, void *lC, void *lF, void *lmom,
                               cudaStream_t st) {
    if (ap.M <= 2)  // species-parallel lanes, all three passes in one kernel (lbe_adj_collide_pair.cu)
        return launch_adj_collide_pair(p, g, post, mask, C, F, ap, lYf_in, lYg_in, lnd_in, lYf_out, lYg_out, lC, lF,
                                       st);
    const unsigned nb = (unsigned)((g.N + ANT - 1) / ANT);
    const unsigned nbc = (unsigned)((g.N + ACT - 1) / ACT);
#define LBE_ADJ_M(MM)                                                                                          \
    k_adj_collide<S, T, MM><<<nbc, ACT, 0, st>>>(g, (const S *)post, mask, (const T *)C, (const T *)F, ap,       \
                                                (const T *)lYf_in, (const T *)lYg_in, (const T *)lnd_in,       \
                                                (T *)lmom, (T *)lC, (T *)lF)
    LBE_ADJ_DISPATCH(p, {
        switch (ap.M) {
            case 3: LBE_ADJ_M(3); break;
            case 4: LBE_ADJ_M(4); break;
            default: return cudaErrorInvalidValue;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_adj_write<T><<<dim3(nb, (unsigned)ap.M), ANT, 0, st>>>(g, mask, ap, (const T *)lYf_in, (const T *)lYg_in,
                                                                 (const T *)lnd_in, (const T *)lmom, (T *)lYf_out,
                                                                 (T *)lYg_out);
    });
#undef LBE_ADJ_M
    return cudaGetLastError();
}

cudaError_t launch_adj_shell_prep(bool fp64, const Grid &g, const AdjShell &L, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + ANT - 1) / ANT);
    if (fp64)
        k_adj_shell_prep<double><<<nb, ANT, 0, st>>>(g, (const double *)L.npad_a, (const double *)L.gab,
                                                     (const double *)L.lC_a, (const double *)L.P,
                                                     (const double *)L.C_a, L.coef, L.own, (double *)L.Lpad,
                                                     (double *)L.gLpad, (double *)L.ln_a, (double *)L.lg);
    else
        k_adj_shell_prep<float><<<nb, ANT, 0, st>>>(g, (const float *)L.npad_a, (const float *)L.gab,
                                                    (const float *)L.lC_a, (const float *)L.P, (const float *)L.C_a,
                                                    (float)L.coef, L.own, (float *)L.Lpad, (float *)L.gLpad,
                                                    (float *)L.ln_a, (float *)L.lg);
    return cudaGetLastError();
}

template <typename T, int S, int TZ, int TYB>
cudaError_t launch_adj_tile(const AdjShellTile &L, cudaStream_t st);
template <int S, int TZ, int TYB>
cudaError_t launch_adj_tile2(const AdjShellTile &L, cudaStream_t st);

// FP32: interleaved (Lambda, g Lambda) tiles of 32 x 16 (32 x 8 at S = 8); FP64: two planes.  The
// tensor maps take their boxes from adj_shell_box, which must match these tiles.
cudaError_t launch_adj_shell_tile(bool fp64, int S, const AdjShellTile &L, cudaStream_t st) {
    if (!fp64) {
        switch (S) {
            case 1: return launch_adj_tile2<1, 3, 16>(L, st);
            case 2: return launch_adj_tile2<2, 3, 16>(L, st);
            case 3: return launch_adj_tile2<3, 3, 16>(L, st);
            case 4: return launch_adj_tile2<4, 3, 16>(L, st);
            case 5: return launch_adj_tile2<5, 3, 16>(L, st);
            case 6: return launch_adj_tile2<6, 3, 16>(L, st);
            case 7: return launch_adj_tile2<7, 2, 16>(L, st);
            case 8: return launch_adj_tile2<8, 1, 8>(L, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (S) {
        case 1: return launch_adj_tile<double, 1, 1, 8>(L, st);
        case 2: return launch_adj_tile<double, 2, 1, 8>(L, st);
        case 3: return launch_adj_tile<double, 3, 1, 8>(L, st);
        case 4: return launch_adj_tile<double, 4, 1, 8>(L, st);
        case 5: return launch_adj_tile<double, 5, 1, 4>(L, st);
        case 6: return launch_adj_tile<double, 6, 1, 4>(L, st);
        case 7: return launch_adj_tile<double, 7, 1, 4>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj_contact_prep(bool fp64, const Grid &g, const ContactParams &cp, const BallRows &br,
                                   const void *xi, const void *lg, void *lnbar, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + ANT - 1) / ANT);
    if (fp64)
        k_adj_contact_prep<double><<<nb, ANT, 0, st>>>(g, cp, br, (const double *)xi, (const double *)lg,
                                                       (double *)lnbar);
    else
        k_adj_contact_prep<float><<<nb, ANT, 0, st>>>(g, cp, br, (const float *)xi, (const float *)lg,
                                                      (float *)lnbar);
    return cudaGetLastError();
}

cudaError_t launch_adj_amp(bool fp64, const Grid &g, int M, const void *lF, const double *phi, double *out,
                           cudaStream_t st) {
    const unsigned nb = (unsigned)((g.N + ANT - 1) / ANT);
    if (fp64)
        k_adj_amp<double><<<nb, ANT, 0, st>>>(g, M, (const double *)lF, phi, out);
    else
        k_adj_amp<float><<<nb, ANT, 0, st>>>(g, M, (const float *)lF, phi, out);
    return cudaGetLastError();
}

}  // namespace lbe
