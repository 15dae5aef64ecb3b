// Kernel templates of the mean-field shell force (K3) and their launchers.
// Included by the translation units that instantiate them (one group of pair
// diameters each, so the builds run in parallel).
//
// K3: mean-field Enskog force of one ordered species pair (a, b) (Appendix,
// hard-sphere C^{alpha,mf}):
//   C^a(r) (+)= -kT sigma_ab^2 w_ab n_a(r) sum_{e in K_ab} e^ (g_ab(r) + g_ab(r+e))/2 n_b(r+e)
//            =  coef * n_a(r) * [ g_ab(r)/2 * sum e^ n_b(r+e) + 1/2 * sum e^ (g_ab n_b)(r+e) ]
// with coef = -kT sigma_ab^2 w_ab.  Both sums run over the half shell as
// e^ [a(r+e) - a(r-e)].
//
// Data path: the padded fields are streamed plane by plane (z-marching) into a
// shared-memory ring by TMA (cp.async.bulk.tensor, 2-D boxes of
// (32 + 2S) x (TY + 2S) per plane, completion on an mbarrier per ring slot).
// The plain kernel (FP64) reads the padded density n_b and the padded product
// g_ab*n_b as two planes and gives each thread one output per plane.  The FP32
// kernels read the interleaved pair (n_b, g_ab n_b) as one 8-byte element per
// node and sum both fields with packed f32x2 instructions: the z-blocked one
// gives each thread TZ outputs along z and reuses every shared-memory read
// across them; the y-blocked one (pair diameters 4 to 6) gives each thread two
// output rows as well and carries shell rows in registers from one column of
// the half shell to the next.  The shell offsets and unit vectors are
// compile-time immediates.  When Pout is given, the kernels also store
// P = sum_e e^ n_b(r+e) of the pair ([3][N]), which the discrete adjoint needs.
#pragma once
#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_shell.cuh"

namespace lbe {

template <int S>
struct ShellTable {
    static constexpr auto hs = make_half_shell<S>();
    static constexpr int count = half_shell_count(S);
};

template <typename T, int S, int I>
__device__ __forceinline__ void shell_term(const T *const *sb, T *an, T *ag) {
    using Tl = ShellTile<T, S>;
    constexpr int ex = ShellTable<S>::hs.e[I][0];
    constexpr int ey = ShellTable<S>::hs.e[I][1];
    constexpr int ez = ShellTable<S>::hs.e[I][2];
    constexpr double len = ct_sqrt((double)(ex * ex + ey * ey + ez * ez));
    constexpr int off = ey * Tl::BX + ex;
    constexpr int GN = Tl::PLANE_BYTES / (int)sizeof(T);
    const T *pp = sb[S + ez] + off;
    const T *pm = sb[S - ez] - off;
    const T dn = pp[0] - pm[0];
    const T dg = pp[GN] - pm[GN];
    if constexpr (ex != 0) {
        constexpr T u = (T)(ex / len);
        an[0] += u * dn;
        ag[0] += u * dg;
    }
    if constexpr (ey != 0) {
        constexpr T u = (T)(ey / len);
        an[1] += u * dn;
        ag[1] += u * dg;
    }
    if constexpr (ez != 0) {
        constexpr T u = (T)(ez / len);
        an[2] += u * dn;
        ag[2] += u * dg;
    }
}

template <typename T, int S, int... I>
__device__ __forceinline__ void shell_sum(const T *const *sb, T *an, T *ag, std::integer_sequence<int, I...>) {
    (shell_term<T, S, I>(sb, an, ag), ...);
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename T, int S>
__global__ void __launch_bounds__(32 * ShellTile<T, S>::TY)
    k_shell_force(const __grid_constant__ CUtensorMap map_n, const __grid_constant__ CUtensorMap map_gn,
                  Grid g, int ox, const T *__restrict__ npad_a, const T *__restrict__ g_ab,
                  T *__restrict__ Cout, T *__restrict__ Pout, T coef, int accumulate, int *err) {
    using Tl = ShellTile<T, S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_align128(smem_raw);
    T *ring = reinterpret_cast<T *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Tl::R * Tl::SLOT_BYTES);
    constexpr int SLOT = Tl::SLOT_BYTES / (int)sizeof(T);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::LZ;
    const int zend = min(z0 + Tl::LZ, g.nz);
    const int nout = zend - z0;
    const int nplanes = nout + 2 * S;
    const bool leader = (tx == 0 && ty == 0);
    const int bx = x0 + g.H - S - ox;  // multiple of 16 bytes / sizeof(T)
    const int by = y0 + g.H - S;
    constexpr uint32_t tx_bytes = 2u * Tl::PLANE * (uint32_t)sizeof(T);

    if (leader) {
        prefetch_tensormap(&map_n);
        prefetch_tensormap(&map_gn);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int j) {  // plane j holds interior z = z0 - S + j
        const int slot = j % Tl::R;
        unsigned char *dst = base + slot * Tl::SLOT_BYTES;
        const int zp = z0 - S + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
        tma_load_3d(dst, &map_n, bx, by, zp, &bars[slot]);
        tma_load_3d(dst + Tl::PLANE_BYTES, &map_gn, bx, by, zp, &bars[slot]);
    };
    if (leader) {
        for (int j = 0; j < 2 * S + 1 && j < nplanes; ++j) issue(j);
    }
    for (int j = 0; j < 2 * S; ++j)
        if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
            mbar_drain(bars, Tl::R, j, min(2 * S + 1, nplanes));
            return;
        }

    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    const int toff = (ty + S) * Tl::BX + (tx + S + ox);
    const T half = (T)0.5;

    for (int iz = 0; iz < nout; ++iz) {
        if (leader && iz + 2 * S + 1 < nplanes) {
            fence_proxy_async_smem();
            issue(iz + 2 * S + 1);
        }
        const int jn = iz + 2 * S;
        if (!mbar_wait_bounded(&bars[jn % Tl::R], (jn / Tl::R) & 1, err)) {
            mbar_drain(bars, Tl::R, jn, min(iz + 2 * S + 2, nplanes));
            return;
        }
        if (active) {
            const T *sb[2 * S + 1];
#pragma unroll
            for (int k = 0; k <= 2 * S; ++k) sb[k] = ring + ((iz + k) % Tl::R) * SLOT + toff;
            T an[3] = {0, 0, 0}, ag[3] = {0, 0, 0};
            shell_sum<T, S>(sb, an, ag, std::make_integer_sequence<int, ShellTable<S>::count>{});
            const int z = z0 + iz;
            const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
            const T na = npad_a[pidx(g, x, y, z)];
            const T gr = g_ab[i];
            const T pre = coef * na;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T v = pre * (half * gr * an[c] + half * ag[c]);
                T *o = Cout + (long long)c * g.N + i;
                if (accumulate)
                    *o += v;
                else
                    *o = v;
                if (Pout) Pout[(long long)c * g.N + i] = an[c];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// z-blocked variant (FP32): each thread produces TZ outputs along z.  The half
// shell is walked as column pairs (ex, ey) / (-ex, -ey); every input value of
// a column within the planes t + D (t < TZ, D the column's z-offsets) is read
// from shared memory once and reused by all TZ outputs:
//   d_t(ez) = a(x+ex, y+ey, z+t+ez) - a(x-ex, y-ey, z+t-ez),  ez in D,
//   acc_t  += (ex, ey, ez)/|e| * d_t(ez).
// The centre column (0, 0, +-S) contributes only to the z component.
// ---------------------------------------------------------------------------
template <int S>
struct ColTable {
    static constexpr auto cols = make_columns<S>();
    static constexpr int count = column_count(S);
};

template <int S, int TZ>
__host__ __device__ constexpr bool col_needs(unsigned mask, int k) {
    // plane offset k (relative to the first output) is read by some output t
    for (int t = 0; t < TZ; ++t) {
        int ez = k - t;
        if (ez >= -S && ez <= S && (mask >> (ez + S)) & 1u) return true;
    }
    return false;
}

// Packed pairs of FP32 values (x in the low half): the two sums of the shell force, over n_b and g_ab n_b,
// run side by side as f32x2 instructions; each lane rounds like the scalar instruction.
using f2 = unsigned long long;
__device__ __forceinline__ f2 f2sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2splat(float u) {
    f2 d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(u));
    return d;
}
__device__ __forceinline__ float2 f2unpack(f2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

template <int S, int TZ, int TYB, int I>
__device__ __forceinline__ void column_pair2(const f2 *const *sb, f2 (*acc)[3]) {
    using Tl = ShellTileZ2<S, TZ, TYB>;
    constexpr int ex = ColTable<S>::cols.ex[I];
    constexpr int ey = ColTable<S>::cols.ey[I];
    constexpr unsigned mask = ColTable<S>::cols.mask[I];
    constexpr int offc = ey * Tl::BX + ex;
    constexpr int NK = 2 * S + TZ;  // plane offsets k = -S .. S + TZ - 1
    f2 cp[NK], cm[NK];
    [&]<int... K>(std::integer_sequence<int, K...>) {
        (
            [&] {
                if constexpr (col_needs<S, TZ>(mask, K - S)) {
                    cp[K] = sb[K][offc];
                    cm[K] = sb[K][-offc];
                }
            }(),
            ...);
    }(std::make_integer_sequence<int, NK>{});
    [&]<int... J>(std::integer_sequence<int, J...>) {
        (
            [&] {
                constexpr int t = J / (2 * S + 1);
                constexpr int ez = J % (2 * S + 1) - S;
                if constexpr ((mask >> (ez + S)) & 1u) {
                    constexpr double len = ct_sqrt((double)(ex * ex + ey * ey + ez * ez));
                    const f2 d = f2sub(cp[t + ez + S], cm[t - ez + S]);
                    if constexpr (ex != 0) acc[t][0] = f2fma(f2splat((float)(ex / len)), d, acc[t][0]);
                    if constexpr (ey != 0) acc[t][1] = f2fma(f2splat((float)(ey / len)), d, acc[t][1]);
                    if constexpr (ez != 0) acc[t][2] = f2fma(f2splat((float)(ez / len)), d, acc[t][2]);
                }
            }(),
            ...);
    }(std::make_integer_sequence<int, TZ *(2 * S + 1)>{});
}

template <int S, int TZ, int TYB, int... I>
__device__ __forceinline__ void all_columns2(const f2 *const *sb, f2 (*acc)[3], std::integer_sequence<int, I...>) {
    (column_pair2<S, TZ, TYB, I>(sb, acc), ...);
}

// ---------------------------------------------------------------------------
// z-blocked variant (FP32) on the interleaved field (n_b, g_ab n_b): each
// thread produces TZ outputs along z.  The half shell is walked as column
// pairs (ex, ey) / (-ex, -ey); every input pair of a column within the planes
// t + D (t < TZ, D the column's z-offsets) is read from shared memory once
// (one 8-byte load) and reused by all TZ outputs:
//   d_t(ez) = a(x+ex, y+ey, z+t+ez) - a(x-ex, y-ey, z+t-ez),  ez in D,
//   acc_t  += (ex, ey, ez)/|e| * d_t(ez),
// both fields at once.  The centre column (0, 0, +-S) contributes only to the
// z component.
// ---------------------------------------------------------------------------
template <int S, int TZ, int TYB>
__global__ void __launch_bounds__(32 * TYB, 1)
    k_shell_force_zb(const __grid_constant__ CUtensorMap map_gn2, Grid g, int ox, const float *__restrict__ npad_a,
                     const float *__restrict__ g_ab, float *__restrict__ Cout, float *__restrict__ Pout, float coef,
                     int accumulate, int *err) {
    using Tl = ShellTileZ2<S, TZ, TYB>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_align128(smem_raw);
    const f2 *ring = reinterpret_cast<const f2 *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Tl::R * Tl::SLOT_BYTES);
    constexpr int SLOT = Tl::SLOT_BYTES / 8;
    constexpr int NK = 2 * S + TZ;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::LZ;
    const int zend = min(z0 + Tl::LZ, g.nz);
    const int nsuper = (zend - z0 + TZ - 1) / TZ;
    const int nplanes = nsuper * TZ + 2 * S;
    const bool leader = (tx == 0 && ty == 0);
    const int bx = x0 + g.H - S - ox;
    const int by = y0 + g.H - S;
    constexpr uint32_t tx_bytes = (uint32_t)Tl::PLANE * 8u;

    if (leader) {
        prefetch_tensormap(&map_gn2);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {  // plane j holds interior z = z0 - S + j
        const int slot = j % Tl::R;
        const int zp = z0 - S + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
        tma_load_3d(base + slot * Tl::SLOT_BYTES, &map_gn2, bx, by, zp, &bars[slot]);
    };
    if (leader)
        for (int j = 0; j < Tl::R && j < nplanes; ++j) issue(j);

    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    const int toff = (ty + S) * Tl::BX + (tx + S + ox);
    const float half = 0.5f;

    for (int s = 0; s < nsuper; ++s) {
        const int j0 = s * TZ;
        for (int j = j0; j < j0 + NK; ++j)
            if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
                mbar_drain(bars, Tl::R, j, min(j0 + Tl::R, nplanes));
                return;
            }
        if (active) {
            // the epilogue's global loads are issued before the shell sum so their latency hides behind it
            float na[TZ], gr[TZ], old[TZ][3];
            long long idx[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const int z = min(z0 + j0 + t, zend - 1);
                idx[t] = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
                na[t] = npad_a[pidx(g, x, y, z)];
                gr[t] = g_ab[idx[t]];
#pragma unroll
                for (int c = 0; c < 3; ++c) old[t][c] = accumulate ? Cout[(long long)c * g.N + idx[t]] : 0.f;
            }
            const f2 *sb[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) sb[k] = ring + ((j0 + k) % Tl::R) * SLOT + toff;
            f2 acc[TZ][3];
#pragma unroll
            for (int t = 0; t < TZ; ++t)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[t][c] = 0ull;
            // centre column (0, 0, +-S): e^ = (0, 0, 1) for ez = +S
#pragma unroll
            for (int t = 0; t < TZ; ++t) acc[t][2] = f2add(acc[t][2], f2sub(sb[t + 2 * S][0], sb[t][0]));
            all_columns2<S, TZ, TYB>(sb, acc, std::make_integer_sequence<int, ColTable<S>::count>{});
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                if (z0 + j0 + t < zend) {
                    const float pre = coef * na[t];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 v = f2unpack(acc[t][c]);  // (sum over n_b, sum over g n_b)
                        Cout[(long long)c * g.N + idx[t]] = old[t][c] + pre * (half * gr[t] * v.x + half * v.y);
                        if (Pout) Pout[(long long)c * g.N + idx[t]] = v.x;
                    }
                }
            }
        }
        __syncthreads();
        if (leader) {
            fence_proxy_async_smem();
            for (int j = j0 + Tl::R; j < j0 + Tl::R + TZ && j < nplanes; ++j) issue(j);
        }
    }
}

// ---------------------------------------------------------------------------
// y-blocked variant (FP32, pair diameters 4 to 6): each thread produces two output rows (y, y + 1)
// and TZ outputs along z.  The half shell is walked column by column with ex fixed and ey ascending.
// Output row y takes the "+" row y + ey and the "-" row y - ey of column (ex, ey); output row y + 1
// takes y + 1 + ey and y + 1 - ey.  The "+" row y + 1 + ey is also the next column's "+" row of output y,
// and the "-" row y - ey the next column's "-" row of output y + 1, so each column step loads one new
// "+" row and one new "-" row (the planes both columns need) and keeps the other two in registers:
// about half the shared loads per output of the one-row walk, with the same +-e pairing.
// ---------------------------------------------------------------------------
template <int S, int TZ>
__host__ __device__ constexpr bool y_plus_needs(unsigned m, int k) {  // plane k = t + ez + S read by some t
    for (int t = 0; t < TZ; ++t) {
        int ez = k - t - S;
        if (ez >= -S && ez <= S && ((m >> (ez + S)) & 1u)) return true;
    }
    return false;
}
template <int S, int TZ>
__host__ __device__ constexpr bool y_minus_needs(unsigned m, int k) {  // plane k = t - ez + S
    for (int t = 0; t < TZ; ++t) {
        int ez = t + S - k;
        if (ez >= -S && ez <= S && ((m >> (ez + S)) & 1u)) return true;
    }
    return false;
}

template <int S, int TZ, int TYT, int EX, int EY>
__device__ __forceinline__ void y_column(const f2 *const *sb, f2 *Pc, f2 *Mc, f2 (*acc)[TZ][3]) {
    using Tl = ShellTileY<S, TZ, TYT>;
    constexpr int NK = 2 * S + TZ;
    constexpr unsigned m = col_mask(S, EX, EY);
    constexpr int hi = col_eymax(S, EX);
    constexpr unsigned mn = EY < hi ? col_mask(S, EX, EY + 1) : 0u;
    constexpr int offP = (EY + 1) * Tl::BX + EX;  // "+" row EY + 1 (x + ex)
    constexpr int offM = -EY * Tl::BX - EX;       // "-" row -EY (x - ex)
    f2 Pn[NK], Mn[NK];
    [&]<int... K>(std::integer_sequence<int, K...>) {
        (
            [&] {
                if constexpr (y_plus_needs<S, TZ>(m | mn, K)) Pn[K] = sb[K][offP];
                if constexpr (y_minus_needs<S, TZ>(m | mn, K)) Mn[K] = sb[K][offM];
            }(),
            ...);
    }(std::make_integer_sequence<int, NK>{});
    // row y: "+" row EY carried in Pc, "-" row -EY loaded now; row y + 1: "+" row EY + 1 loaded now, "-" row
    // 1 - EY carried in Mc
    [&]<int... J>(std::integer_sequence<int, J...>) {
        (
            [&] {
                // points in order of ez, the TZ outputs of one point side by side
                constexpr int t = J % TZ;
                constexpr int ez = J / TZ - S;
                if constexpr ((m >> (ez + S)) & 1u) {
                    constexpr double len = ct_sqrt((double)(EX * EX + EY * EY + ez * ez));
                    const f2 d0 = f2sub(Pc[t + ez + S], Mn[t - ez + S]);
                    const f2 d1 = f2sub(Pn[t + ez + S], Mc[t - ez + S]);
                    if constexpr (EX != 0) {
                        const f2 u = f2splat((float)(EX / len));
                        acc[0][t][0] = f2fma(u, d0, acc[0][t][0]);
                        acc[1][t][0] = f2fma(u, d1, acc[1][t][0]);
                    }
                    if constexpr (EY != 0) {
                        const f2 u = f2splat((float)(EY / len));
                        acc[0][t][1] = f2fma(u, d0, acc[0][t][1]);
                        acc[1][t][1] = f2fma(u, d1, acc[1][t][1]);
                    }
                    if constexpr (ez != 0) {
                        const f2 u = f2splat((float)(ez / len));
                        acc[0][t][2] = f2fma(u, d0, acc[0][t][2]);
                        acc[1][t][2] = f2fma(u, d1, acc[1][t][2]);
                    }
                }
            }(),
            ...);
    }(std::make_integer_sequence<int, TZ *(2 * S + 1)>{});
    // the next column's row y takes this "+" row EY + 1, its row y + 1 this "-" row -EY
    [&]<int... K>(std::integer_sequence<int, K...>) {
        (
            [&] {
                if constexpr (y_plus_needs<S, TZ>(m | mn, K)) Pc[K] = Pn[K];
                if constexpr (y_minus_needs<S, TZ>(m | mn, K)) Mc[K] = Mn[K];
            }(),
            ...);
    }(std::make_integer_sequence<int, NK>{});
}

template <int S, int TZ, int TYT, int EX>
__device__ __forceinline__ void y_chain(const f2 *const *sb, f2 (*acc)[TZ][3]) {
    using Tl = ShellTileY<S, TZ, TYT>;
    constexpr int NK = 2 * S + TZ;
    constexpr int hi = col_eymax(S, EX);
    constexpr int lo = EX == 0 ? 1 : -hi;
    if constexpr (hi >= 0 && lo <= hi) {
        constexpr unsigned m0 = col_mask(S, EX, lo);
        f2 Pc[NK], Mc[NK];
        // the first column: row y's "+" row lo, row y + 1's "-" row 1 - lo
        [&]<int... K>(std::integer_sequence<int, K...>) {
            (
                [&] {
                    if constexpr (y_plus_needs<S, TZ>(m0, K)) Pc[K] = sb[K][lo * Tl::BX + EX];
                    if constexpr (y_minus_needs<S, TZ>(m0, K)) Mc[K] = sb[K][(1 - lo) * Tl::BX - EX];
                }(),
                ...);
        }(std::make_integer_sequence<int, NK>{});
        [&]<int... I>(std::integer_sequence<int, I...>) {
            (y_column<S, TZ, TYT, EX, lo + I>(sb, Pc, Mc, acc), ...);
        }(std::make_integer_sequence<int, hi - lo + 1>{});
    }
}

template <int S, int TZ, int TYT, int... EX>
__device__ __forceinline__ void y_all(const f2 *const *sb, f2 (*acc)[TZ][3], std::integer_sequence<int, EX...>) {
    (y_chain<S, TZ, TYT, EX>(sb, acc), ...);
}

template <int S, int TZ, int TYT>
__global__ void __launch_bounds__(32 * TYT, 1)
    k_shell_force_yb(const __grid_constant__ CUtensorMap map_gn2, Grid g, int ox, const float *__restrict__ npad_a,
                     const float *__restrict__ g_ab, float *__restrict__ Cout, float *__restrict__ Pout, float coef,
                     int accumulate, int *err) {
    using Tl = ShellTileY<S, TZ, TYT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_align128(smem_raw);
    const f2 *ring = reinterpret_cast<const f2 *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Tl::R * Tl::SLOT_BYTES);
    constexpr int SLOT = Tl::SLOT_BYTES / 8;
    constexpr int NK = 2 * S + TZ;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::LZ;
    const int zend = min(z0 + Tl::LZ, g.nz);
    const int nsuper = (zend - z0 + TZ - 1) / TZ;
    const int nplanes = nsuper * TZ + 2 * S;
    const bool leader = (tx == 0 && ty == 0);
    const int bx = x0 + g.H - S - ox;
    const int by = y0 + g.H - S;
    constexpr uint32_t tx_bytes = (uint32_t)Tl::PLANE * 8u;

    if (leader) {
        prefetch_tensormap(&map_gn2);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {  // plane j holds interior z = z0 - S + j
        const int slot = j % Tl::R;
        const int zp = z0 - S + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
        tma_load_3d(base + slot * Tl::SLOT_BYTES, &map_gn2, bx, by, zp, &bars[slot]);
    };
    if (leader)
        for (int j = 0; j < Tl::R && j < nplanes; ++j) issue(j);

    const int x = x0 + tx;
    const int yb = y0 + 2 * ty;  // this thread's rows yb and yb + 1
    const int toff = (2 * ty + S) * Tl::BX + (tx + S + ox);
    const float half = 0.5f;

    for (int s = 0; s < nsuper; ++s) {
        const int j0 = s * TZ;
        for (int j = j0; j < j0 + NK; ++j)
            if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
                mbar_drain(bars, Tl::R, j, min(j0 + Tl::R, nplanes));
                return;
            }
        if (x < g.nx && yb < g.ny) {
            // the epilogue's global loads are issued before the shell sum so their latency hides behind it
            float pre[2][TZ], gr[2][TZ], old[2][TZ][3];
            long long idx[2][TZ];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    const int y = min(yb + r, g.ny - 1);
                    const int z = min(z0 + j0 + t, zend - 1);
                    idx[r][t] = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
                    pre[r][t] = coef * npad_a[pidx(g, x, y, z)];
                    gr[r][t] = g_ab[idx[r][t]];
#pragma unroll
                    for (int c = 0; c < 3; ++c) old[r][t][c] = accumulate ? Cout[(long long)c * g.N + idx[r][t]] : 0.f;
                }
            const f2 *sb[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) sb[k] = ring + ((j0 + k) % Tl::R) * SLOT + toff;
            f2 acc[2][TZ][3];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int t = 0; t < TZ; ++t)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[r][t][c] = 0ull;
            // centre column (0, 0, +-S): e^ = (0, 0, 1) for ez = +S
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int t = 0; t < TZ; ++t)
                    acc[r][t][2] = f2add(acc[r][t][2], f2sub(sb[t + 2 * S][r * Tl::BX], sb[t][r * Tl::BX]));
            y_all<S, TZ, TYT>(sb, acc, std::make_integer_sequence<int, S + 1>{});
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (yb + r >= g.ny) continue;
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    if (z0 + j0 + t >= zend) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 v = f2unpack(acc[r][t][c]);  // (sum over n_b, sum over g n_b)
                        Cout[(long long)c * g.N + idx[r][t]] =
                            old[r][t][c] + pre[r][t] * (half * gr[r][t] * v.x + half * v.y);
                        if (Pout) Pout[(long long)c * g.N + idx[r][t]] = v.x;
                    }
                }
            }
        }
        __syncthreads();
        if (leader) {
            fence_proxy_async_smem();
            for (int j = j0 + Tl::R; j < j0 + Tl::R + TZ && j < nplanes; ++j) issue(j);
        }
    }
}

template <int S, int TZ, int TYT>
cudaError_t launch_yb(const ShellLaunch &L, cudaStream_t st) {
    using Tl = ShellTileY<S, TZ, TYT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_shell_force_yb<S, TZ, TYT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const Grid &g = *L.grid;
    dim3 block(Tl::TX, Tl::TYT, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int ox = ((g.H - S) % Tl::A + Tl::A) % Tl::A;
    k_shell_force_yb<S, TZ, TYT><<<grid, block, Tl::SMEM, st>>>(*L.map_gn, g, ox, (const float *)L.npad_a,
                                                          (const float *)L.g_ab, (float *)L.Cout, (float *)L.Pout,
                                                          (float)L.coef, L.accumulate, L.err);
    return cudaGetLastError();
}

template <int S, int TZ, int TYB>
cudaError_t launch_zb(const ShellLaunch &L, cudaStream_t st) {
    using Tl = ShellTileZ2<S, TZ, TYB>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_shell_force_zb<S, TZ, TYB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const Grid &g = *L.grid;
    dim3 block(Tl::TX, Tl::TY, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int ox = ((g.H - S) % Tl::A + Tl::A) % Tl::A;
    k_shell_force_zb<S, TZ, TYB><<<grid, block, Tl::SMEM, st>>>(*L.map_gn, g, ox, (const float *)L.npad_a,
                                                              (const float *)L.g_ab, (float *)L.Cout,
                                                              (float *)L.Pout, (float)L.coef, L.accumulate, L.err);
    return cudaGetLastError();
}

template <typename T, int S>
cudaError_t launch_one(const ShellLaunch &L, cudaStream_t st) {
    using Tl = ShellTile<T, S>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_shell_force<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const Grid &g = *L.grid;
    dim3 block(Tl::TX, Tl::TY, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int A = Tl::A;
    const int ox = ((g.H - S) % A + A) % A;
    k_shell_force<T, S><<<grid, block, Tl::SMEM, st>>>(*L.map_n, *L.map_gn, g, ox, (const T *)L.npad_a,
                                                       (const T *)L.g_ab, (T *)L.Cout, (T *)L.Pout, (T)L.coef,
                                                       L.accumulate, L.err);
    return cudaGetLastError();
}

}  // namespace lbe
