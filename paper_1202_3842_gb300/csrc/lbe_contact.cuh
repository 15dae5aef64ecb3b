// K2: contact values (Appendix: g_ab evaluated at contact, a functional of the
// densities).  Per node:
//   n-bar_b = (1/|B_b|) sum_{|d| <= sigma_b/2} n_b(r + d)      (ball average)
//   xi_k    = (pi/6) sum_b sigma_b^k n-bar_b,  k = 2, 3
//   g_ab    = 1/(1-xi3) + 3 s xi2/(1-xi3)^2 + 2 s^2 xi2^2/(1-xi3)^3,
//             s = sigma_a sigma_b/(sigma_a + sigma_b)   (Boublik-Mansoori-
//             Carnahan-Starling-Leland contact value)
// Outputs: g_ab [M][M][N] and the padded product g_ab * n_b [M][M][P] (with
// its periodic images) that the shell-force kernel streams, stored for FP32 as
// the interleaved pair (n_b, g_ab n_b) [M][M][P] of float2; optionally xi2 and
// xi3 [2][N] (kept for the discrete adjoint).
//
// MODE 1 is the transpose of the ball average for the discrete adjoint: the
// same TMA ring and ball rows sum a padded field per species over the ball,
// and the kernel adds the sums to ln [M][N] (zero on solid nodes, whose
// density is fixed).  The ball is symmetric, so its transpose is the same sum.
//
// Data path: the padded densities of all species are streamed plane by plane
// (z-marching) into a shared-memory ring by TMA; each thread owns one (x, y)
// column of a 32 x 8 tile and sums the ball rows (dy, dz, half-width a) from
// shared memory (an unrolled, predicated loop over the widest row: per-row
// prefix sums and an exact-width switch were both measured slower).
#pragma once
#include <utility>

#include "lbe_device.cuh"
#include "lbe_launch.h"

namespace lbe {

template <typename T, int M, int RB>
struct ContactTile {
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int TX = 32;
    static constexpr int TY = 8;
    static constexpr int BX = ((TX + 2 * RB + A - 1) + A - 1) / A * A;
    static constexpr int BY = TY + 2 * RB;
    static constexpr int R = 2 * RB + 2;
    static constexpr int PLANE = BX * BY;
    static constexpr int PLANE_BYTES = ((PLANE * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int SLOT_BYTES = M * PLANE_BYTES;
    static constexpr int SMEM = R * SLOT_BYTES + 256 + 128;
    static constexpr int LZ = 8;
};

// Ball sum of one species with a compile-time ball |d|^2 <= SQ/4 (SQ = sigma^2 of an integer diameter),
// walked in the order of the runtime rows (dz, dy, dx ascending), so the sum is the same bit for bit.
template <typename T, int RB, int BX, int SQ>
__device__ __forceinline__ T ball_sum_ct(const T *const *sb, int boff) {
    constexpr int W = 2 * RB + 1;
    T acc = 0;
    [&]<int... K>(std::integer_sequence<int, K...>) {
        (
            [&] {
                constexpr int dz = K / (W * W) - RB;
                constexpr int dy = (K / W) % W - RB;
                constexpr int dx = K % W - RB;
                if constexpr (4 * (dx * dx + dy * dy + dz * dz) <= SQ) acc += sb[dz + RB][boff + dy * BX + dx];
            }(),
            ...);
    }(std::make_integer_sequence<int, W * W * W>{});
    return acc;
}

struct ContactMaps {
    CUtensorMap m[MAXS];
};

template <typename T, int M, int RB, int MODE, int SQ0 = 0, int SQ1 = 0>
__global__ void __launch_bounds__(256)
    k_contact_tma(const __grid_constant__ ContactMaps maps, Grid g, int ox, ContactParams cp, BallRows br,
                  T *__restrict__ gab, T *__restrict__ gnpad, T *__restrict__ xi_out,
                  const uint32_t *__restrict__ mask, T *__restrict__ ln, int *err) {
    using Tl = ContactTile<T, M, RB>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_align128(smem_raw);
    const T *ring = reinterpret_cast<const T *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Tl::R * Tl::SLOT_BYTES);
    constexpr int SLOT = Tl::SLOT_BYTES / (int)sizeof(T);
    constexpr int PL = Tl::PLANE_BYTES / (int)sizeof(T);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::LZ;
    const int zend = min(z0 + Tl::LZ, g.nz);
    const int nout = zend - z0;
    const int nplanes = nout + 2 * RB;
    const bool leader = (tx == 0 && ty == 0);
    const int bx = x0 + g.H - RB - ox;
    const int by = y0 + g.H - RB;
    constexpr uint32_t tx_bytes = (uint32_t)M * Tl::PLANE * (uint32_t)sizeof(T);

    if (leader) {
        for (int b = 0; b < M; ++b) prefetch_tensormap(&maps.m[b]);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {
        const int slot = j % Tl::R;
        unsigned char *dst = base + slot * Tl::SLOT_BYTES;
        const int zp = z0 - RB + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
#pragma unroll
        for (int b = 0; b < M; ++b) tma_load_3d(dst + b * Tl::PLANE_BYTES, &maps.m[b], bx, by, zp, &bars[slot]);
    };
    if (leader)
        for (int j = 0; j < 2 * RB + 1 && j < nplanes; ++j) issue(j);
    for (int j = 0; j < 2 * RB; ++j)
        if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
            mbar_drain(bars, Tl::R, j, min(2 * RB + 1, nplanes));
            return;
        }

    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    const int toff = (ty + RB) * Tl::BX + (tx + RB + ox);

    for (int iz = 0; iz < nout; ++iz) {
        if (leader && iz + 2 * RB + 1 < nplanes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(iz + 2 * RB + 1);
        }
        const int jn = iz + 2 * RB;
        if (!mbar_wait_bounded(&bars[jn % Tl::R], (jn / Tl::R) & 1, err)) {
            mbar_drain(bars, Tl::R, jn, min(iz + 2 * RB + 2, nplanes));
            return;
        }
        if (active) {
            T xi2 = 0, xi3 = 0, nloc[M];
            const T *sb[2 * RB + 1];
#pragma unroll
            for (int k = 0; k <= 2 * RB; ++k) sb[k] = ring + ((iz + k) % Tl::R) * SLOT + toff;
#pragma unroll
            for (int b = 0; b < M; ++b) {
                T acc = 0;
                if constexpr (SQ0 > 0) {  // balls known at compile time (common diameters): exact loads
                    acc = b == 0 ? ball_sum_ct<T, RB, Tl::BX, SQ0>(sb, 0)
                                 : ball_sum_ct<T, RB, Tl::BX, (SQ1 > 0 ? SQ1 : SQ0)>(sb, b * PL);
                } else {
#pragma unroll
                    for (int dz = -RB; dz <= RB; ++dz) {
                        const T *pz = sb[dz + RB] + b * PL;
                        const int k0 = br.first[b][dz + 4], k1 = br.first[b][dz + 5];
                        for (int k = k0; k < k1; ++k) {
                            const int a = br.a[b][k];
                            const T *row = pz + br.dy[b][k] * Tl::BX;
#pragma unroll
                            for (int dx = -RB; dx <= RB; ++dx)
                                if (dx >= -a && dx <= a) acc += row[dx];
                        }
                    }
                }
                if constexpr (MODE == 1) {
                    // transpose of the ball average: add the ball sum of this species' field to ln
                    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (z0 + iz));
                    T *o = ln + (long long)b * g.N + i;
                    *o = (mask[i] & 1u) ? (T)0 : *o + acc;
                } else {
                    const T nbar = acc / (T)br.count[b];
                    xi2 += (T)cp.xi2c[b] * nbar;
                    xi3 += (T)cp.xi3c[b] * nbar;
                    nloc[b] = sb[RB][b * PL];
                }
            }
            if constexpr (MODE == 0) {
            const T i1 = (T)1 / ((T)1 - xi3);
            if (!(xi3 < (T)1)) atomicOr(err, ERR_PACKING);
            const int z = z0 + iz;
            const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
            if (xi_out) {
                xi_out[i] = xi2;
                xi_out[g.N + i] = xi3;
            }
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) {
                    const T s = (T)cp.s_ab[a][b];
                    const T gv = i1 + (T)3 * s * xi2 * i1 * i1 + (T)2 * s * s * xi2 * xi2 * i1 * i1 * i1;
                    if (!isfinite(gv)) atomicOr(err, ERR_PACKING);
                    gab[(long long)(a * M + b) * g.N + i] = gv;
                    if constexpr (sizeof(T) == 4) {  // FP32: the interleaved pair (n_b, g_ab n_b)
                        write_padded<float2>(g, reinterpret_cast<float2 *>(gnpad) + (long long)(a * M + b) * g.P,
                                             x, y, z, make_float2(nloc[b], gv * nloc[b]));
                    } else {
                        write_padded<T>(g, gnpad + (long long)(a * M + b) * g.P, x, y, z, gv * nloc[b]);
                    }
                }
            }  // MODE == 0
        }
        __syncthreads();
    }
}

template <typename T, int M, int RB, int MODE, int SQ0 = 0, int SQ1 = 0>
cudaError_t launch_ct(const ContactLaunch &L, cudaStream_t st) {
    using Tl = ContactTile<T, M, RB>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_contact_tma<T, M, RB, MODE, SQ0, SQ1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const Grid &g = *L.grid;
    ContactMaps maps;
    for (int b = 0; b < M; ++b) maps.m[b] = L.maps[b];
    dim3 block(Tl::TX, Tl::TY, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int ox = ((g.H - RB) % Tl::A + Tl::A) % Tl::A;
    k_contact_tma<T, M, RB, MODE, SQ0, SQ1><<<grid, block, Tl::SMEM, st>>>(maps, g, ox, *L.cp, *L.br, (T *)L.gab,
                                                                (T *)L.gnpad, (T *)L.xi, L.mask, (T *)L.ln, L.err);
    return cudaGetLastError();
}

// sigma^2 of species b when sigma is an integer (0 otherwise)
inline int sigma_sq(const ContactParams &cp, int b) {
    const double s = cp.sigma[b];
    const double r = (double)(long long)(s + 0.5);
    return (s == r && r > 0.0 && r <= 8.0) ? (int)(r * r) : 0;
}

template <typename T, int M, int MODE>
cudaError_t dispatch_rb(const ContactLaunch &L, cudaStream_t st) {
    // compile-time balls for the common diameters: sigma 4/6 mixtures, sigma 6 and sigma 3
    if constexpr (M == 2) {
        if (L.RB == 3 && sigma_sq(*L.cp, 0) == 16 && sigma_sq(*L.cp, 1) == 36)
            return launch_ct<T, 2, 3, MODE, 16, 36>(L, st);
    }
    if constexpr (M == 1) {
        if (L.RB == 3 && sigma_sq(*L.cp, 0) == 36) return launch_ct<T, 1, 3, MODE, 36>(L, st);
        if (L.RB == 1 && sigma_sq(*L.cp, 0) == 9) return launch_ct<T, 1, 1, MODE, 9>(L, st);
    }
    switch (L.RB) {
        case 0: return launch_ct<T, M, 0, MODE>(L, st);
        case 1: return launch_ct<T, M, 1, MODE>(L, st);
        case 2: return launch_ct<T, M, 2, MODE>(L, st);
        case 3: return launch_ct<T, M, 3, MODE>(L, st);
        case 4: return launch_ct<T, M, 4, MODE>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int MODE>
cudaError_t dispatch_m(const ContactLaunch &L, cudaStream_t st) {
    switch (L.cp->M) {
        case 1: return dispatch_rb<T, 1, MODE>(L, st);
        case 2: return dispatch_rb<T, 2, MODE>(L, st);
        case 3: return dispatch_rb<T, 3, MODE>(L, st);
        case 4: return dispatch_rb<T, 4, MODE>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbe
