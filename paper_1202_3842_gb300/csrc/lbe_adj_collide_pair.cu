// K4 transposed for one or two species with species-parallel lanes (the
// arithmetic is that of k_adj_collide + k_adj_write in lbe_adjoint.cu).
//
// Two species: lanes 0-15 of a warp take species 0 and lanes 16-31 species 1
// of the same 16 consecutive nodes (one species: one thread per node).  Each
// thread
//   pass A  pulls its own species' populations and forms its moments; n and J
//           of the partner species (lane ^ 16) give the barycentric u;
//   pass B  push-gathers the adjoint of its post-collision populations (kept in
//           registers) and transposes the collision; the adjoint of u is the
//           sum over both species, again by one exchange with the partner;
//   pass C  transposes the moment recovery, adds lambda_F, writes lambda_C and
//           the adjoint of its pre-collision populations.
// Cross-species sums are formed in species order (0 then 1), as in the
// one-thread-per-node kernel.
#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_node.cuh"

namespace lbe {

constexpr int ACP = 256;  // threads per CTA: 128 nodes (two species) or 256 (one)

// adjoint of the post-collision population p (streaming transposed), density adjoint added for f
template <typename T, int P>
__device__ __forceinline__ T gather_post_pair(const T *__restrict__ lY, const T *__restrict__ ln, long long N,
                                              long long i, const NbrOff &o, uint32_t m) {
    if (m & (1u << opp(P))) {
        const T v = lY[(long long)opp(P) * N + i];
        return ln ? v + ln[i] : v;
    }
    const long long j = i + src_off<opp(P)>(o);  // r + c_P
    const T v = lY[(long long)P * N + j];
    return ln ? v + ln[j] : v;
}

template <typename T, int M>
__device__ __forceinline__ T partner(T v) {
    if constexpr (M == 2) return __shfl_xor_sync(0xffffffffu, v, 16);
    return (T)0;
}

template <typename S, typename T, int M>
__global__ void __launch_bounds__(ACP, sizeof(T) == 4 ? 3 : 1)
    k_adj_collide_pair(Grid g, const S *__restrict__ post, const uint32_t *__restrict__ mask,
                       const T *__restrict__ C, const T *__restrict__ F, AdjParams ap, const T *__restrict__ lYf_in,
                       const T *__restrict__ lYg_in, const T *__restrict__ lnd_in, T *__restrict__ lYf_out,
                       T *__restrict__ lYg_out, T *__restrict__ lC, T *__restrict__ lF) {
    static_assert(M == 1 || M == 2, "one or two species");
    const int lane = threadIdx.x & 31;
    const int a = M == 2 ? lane >> 4 : 0;
    const long long i = M == 2 ? (long long)blockIdx.x * (ACP / 2) + (threadIdx.x >> 5) * 16 + (lane & 15)
                               : (long long)blockIdx.x * ACP + threadIdx.x;
    const bool valid = i < g.N;
    int x = 0, y = 0, z = 0;
    if (valid) node_xyz(g, i, x, y, z);
    const uint32_t m = valid ? mask[i] : 1u;
    const bool fluid = !(m & 1u);
    const double n0d = a == 0 ? ap.sp[0].n0 : ap.sp[1].n0;
    const T om = (T)(a == 0 ? ap.sp[0].omega_eff : ap.sp[1].omega_eff);
    const T inv = (T)(a == 0 ? ap.sp[0].inv : ap.sp[1].inv);
    NbrOff o{};
    if (fluid) o = nbr_offsets(g, x, y, z);

    // ---- pass A: forward moments of this species
    T n = 0, inv_n = 0, J[3] = {0, 0, 0}, ua[3] = {0, 0, 0}, Cv[3] = {0, 0, 0}, Fv[3] = {0, 0, 0};
    T nF[3] = {0, 0, 0};
    if (fluid) {
        const T n0 = (T)n0d;
        const S *fb = post + pop_off(a, 0, 0, g.N);
        const S *gb = post + pop_off(a, 1, 0, g.N);
        T Jt[3] = {0, 0, 0};
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    const T fv = pull<S, T, P, true>(fb, g.N, i, o, m, n0);
                    const T gv = pull<S, T, P, true>(gb, g.N, i, o, m, n0);
                    n += fv;
                    Jt[0] += (T)cx(P) * gv;
                    Jt[1] += (T)cy(P) * gv;
                    Jt[2] += (T)cz(P) * gv;
                }(),
                ...);
        }(std::make_integer_sequence<int, Q>{});
        inv_n = n > (T)0 ? (T)1 / n : (T)0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Cv[c] = C[((long long)a * 3 + c) * g.N + i];
            Fv[c] = F[((long long)a * 3 + c) * g.N + i];
            nF[c] = n * Fv[c];
            J[c] = ap.consistent ? Jt[c] + (T)0.5 * nF[c] : Jt[c] + (T)0.5 * (Cv[c] + nF[c]);
            ua[c] = J[c] * inv_n;
        }
    }
    const T np = partner<T, M>(n);
    T Jp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Jp[c] = partner<T, M>(J[c]);
    const T ntot = a == 0 ? n + np : np + n;
    const T inv_tot = ntot > (T)0 ? (T)1 / ntot : (T)0;
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = (a == 0 ? J[c] + Jp[c] : Jp[c] + J[c]) * inv_tot;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // ---- pass B: collision transposed
    // FP32: the gathered adjoint populations wait for the last pass in shared memory (39 KB per CTA),
    // which leaves the registers for three CTAs per SM; FP64 keeps them in registers
    constexpr bool SMEM = sizeof(T) == 4;
    __shared__ T sl[SMEM ? 2 : 1][SMEM ? Q : 1][SMEM ? ACP : 1];
    T lfk[SMEM ? 1 : Q], lgk[SMEM ? 1 : Q];
    const int tid = threadIdx.x;
    T lu[3] = {0, 0, 0}, lua[3] = {0, 0, 0}, lCs[3] = {0, 0, 0}, lnFs[3] = {0, 0, 0}, lns = 0, lPis = 0;
    if (fluid) {
        const T uau = ua[0] * u[0] + ua[1] * u[1] + ua[2] * u[2];
        T X[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = Cv[c] + nF[c];
        T lA = 0, lB = 0, lsf0 = 0, lnv = 0;
        T lX[3] = {0, 0, 0}, lnFv[3] = {0, 0, 0}, lCv[3] = {0, 0, 0}, luav[3] = {0, 0, 0}, lua_u[3] = {0, 0, 0};
        const T *lYf = lYf_in + (long long)a * Q * g.N;
        const T *lYg = lYg_in + (long long)a * Q * g.N;
        const T *lnd = lnd_in + (long long)a * g.N;
        [&]<int... P>(std::integer_sequence<int, P...>) {
            (
                [&] {
                    constexpr T w = (T)wq(P);
                    const T lfs = gather_post_pair<T, P>(lYf, lnd, g.N, i, o, m);
                    const T lgs = gather_post_pair<T, P>(lYg, nullptr, g.N, i, o, m);
                    if constexpr (SMEM) {
                        sl[0][P][tid] = lfs;
                        sl[1][P][tid] = lgs;
                    } else {
                        lfk[P] = lfs;
                        lgk[P] = lgs;
                    }
                    const T cua = cdot<T, P>(ua);
                    const T cu = cdot<T, P>(u);
                    const T cX = cdot<T, P>(X);
                    const T cY = cdot<T, P>(nF);
                    const T cC = cdot<T, P>(Cv);
                    const T lSf = inv * lfs, lSg = inv * lgs;
                    const T lt1 = w * om * (lfs + lgs);
                    lA += w * om * lfs;
                    lB += w * om * lgs;
                    lsf0 += w * (lSf + lSg);
                    const T lcX = w * lSf * ((T)3 + (T)9 * cua);
                    const T lcY = w * lSg * ((T)3 + (T)9 * cua);
                    const T lcC = (T)18 * w * lSg * cua;
                    const T lcua = (T)9 * w * lSf * cX + w * lSg * ((T)18 * cC + (T)9 * cY) +
                                   lt1 * ((T)3 * n + (T)9 * n * cu);
                    const T lcu = (T)9 * n * (cua - cu) * lt1;
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
            lX[c] += (T)-3 * ua[c] * lsf0;
            luav[c] += (T)-3 * X[c] * lsf0;
            lCv[c] += lX[c];
            lnFv[c] += lX[c];
        }
        const T liso = -lA - lB;
        lnv += lA + (T)1.5 * ((T)2 * uau - uu) * liso;
        const T luau = (T)3 * n * liso;
        const T luu = (T)-1.5 * n * liso;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            luav[c] += u[c] * luau;
            lu[c] += lua_u[c] + ua[c] * luau + (T)2 * u[c] * luu;
            lua[c] = luav[c];
            lCs[c] = lCv[c];
            lnFs[c] = lnFv[c];
        }
        lns = lnv;
        lPis = lB;
    }
    // ---- u = sum J / sum n: the adjoint of u summed over both species (species order)
    T lJtot[3] = {0, 0, 0}, lntot = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T lp = partner<T, M>(lu[c]);
        const T lut = a == 0 ? lu[c] + lp : lp + lu[c];
        if (ntot > (T)0) {
            lJtot[c] = lut * inv_tot;
            lntot -= lut * u[c] * inv_tot;
        }
    }
    if (!valid) return;
    T *of = lYf_out + (long long)a * Q * g.N + i;
    T *og = lYg_out + (long long)a * Q * g.N + i;
    if (!fluid) {
#pragma unroll
        for (int c = 0; c < 3; ++c) lC[((long long)a * 3 + c) * g.N + i] = (T)0;
#pragma unroll
        for (int p = 0; p < Q; ++p) {
            of[(long long)p * g.N] = (T)0;
            og[(long long)p * g.N] = (T)0;
        }
        return;
    }
    // ---- pass C: moment recovery transposed, outputs
    const int coord = ap.axis == 0 ? x : (ap.axis == 1 ? y : z);
    const bool on_plane = ap.axis >= 0 && coord == ap.plane;
    const T kPi = ap.consistent ? (T)1.5 : (T)-0.5;
    const T lPit = lPis;
    const T lCu = kPi * lPis;
    T lJ[3], lCv[3], luav[3];
    T ln = lns + lntot;
    T dot = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lCv[c] = lCs[c] + ua[c] * lCu;
        luav[c] = lua[c] + Cv[c] * lCu;
        lJ[c] = lJtot[c] + luav[c] * inv_n;
        dot += luav[c] * ua[c];
    }
    ln -= dot * inv_n;
    if (on_plane) lJ[ap.axis] += (T)ap.wobj;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T lnF = lnFs[c] + (T)0.5 * lJ[c];
        if (!ap.consistent) lCv[c] += (T)0.5 * lJ[c];
        ln += lnF * Fv[c];
        lF[((long long)a * 3 + c) * g.N + i] += n * lnF;
        lC[((long long)a * 3 + c) * g.N + i] = lCv[c];
    }
    const T om1 = (T)1 - om;
    [&]<int... P>(std::integer_sequence<int, P...>) {
        (
            [&] {
                const T lfs = SMEM ? sl[0][P][tid] : lfk[SMEM ? 0 : P];
                const T lgs = SMEM ? sl[1][P][tid] : lgk[SMEM ? 0 : P];
                of[(long long)P * g.N] = om1 * lfs + ln;
                og[(long long)P * g.N] = om1 * lgs + lPit + cdot<T, P>(lJ);
            }(),
            ...);
    }(std::make_integer_sequence<int, Q>{});
}

cudaError_t launch_adj_collide_pair(Prec p, const Grid &g, const void *post, const uint32_t *mask, const void *C,
                                   const void *F, const AdjParams &ap, const void *lYf_in, const void *lYg_in,
                                   const void *lnd_in, void *lYf_out, void *lYg_out, void *lC, void *lF,
                                   cudaStream_t st) {
    const int per_cta = ap.M == 2 ? ACP / 2 : ACP;
    const unsigned nb = (unsigned)((g.N + per_cta - 1) / per_cta);
#define LBE_ADJ_PAIR(SS, TT, MM)                                                                                \
    k_adj_collide_pair<SS, TT, MM><<<nb, ACP, 0, st>>>(g, (const SS *)post, mask, (const TT *)C, (const TT *)F, \
                                                       ap, (const TT *)lYf_in, (const TT *)lYg_in,               \
                                                       (const TT *)lnd_in, (TT *)lYf_out, (TT *)lYg_out,         \
                                                       (TT *)lC, (TT *)lF)
    if (p == Prec::F64) {
        if (ap.M == 1) LBE_ADJ_PAIR(double, double, 1); else LBE_ADJ_PAIR(double, double, 2);
    } else if (p == Prec::F32) {
        if (ap.M == 1) LBE_ADJ_PAIR(float, float, 1); else LBE_ADJ_PAIR(float, float, 2);
    } else {
        return cudaErrorInvalidValue;
    }
#undef LBE_ADJ_PAIR
    return cudaGetLastError();
}

}  // namespace lbe
