// Shell force of one ordered pair (a, b) transposed (discrete adjoint of K3),
// from shared-memory tiles.  Included by the translation units that
// instantiate it.
//
// Forward (Appendix, hard-sphere C^{alpha,mf}, with the pair-symmetric contact
// value of the endpoints):
//   C^a(r) += coef n_a(r) [ g(r)/2 P(r) + Q(r)/2 ],
//   P = sum_e e^ n_b(r+e),  Q = sum_e e^ (g n_b)(r+e),  g = g_ab.
// With Lambda = coef n_a lC^a / 2 (lC^a the adjoint of C^a), and because the
// shell is symmetric with e^(-e) = -e^(e):
//   TQ(s) = sum_e e^.Lambda(s+e),   TP(s) = sum_e e^.(g Lambda)(s+e),
//   ln_b(s) += -TP(s) - g(s) TQ(s),
//   lg(s)   += -n_b(s) TQ(s) + Lambda(s).P(s),
//   ln_a(s) += (g P + Q)(s).lC^a(s) coef/2  (summed over b: C^a(s).lC^a(s)/n_a(s)).
// The node-local terms are added by the prep kernel (lbe_adjoint.cu).  TQ and
// TP are divergences: component c of each needs only Lambda_c and (g Lambda)_c.
// One launch handles one component CC: the two padded fields Lambda_CC and
// (g Lambda)_CC are streamed plane by plane into the same shared-memory ring as
// the forward kernel (TMA boxes, bounded mbarrier waits), each thread produces
// TZ outputs along z, and the half shell is walked as column pairs with the
// compile-time offsets and unit-vector components of the forward kernel.  In
// FP32 the prep kernel writes the two fields interleaved, (Lambda_CC,
// (g Lambda)_CC) as one 8-byte element, and the sums run as packed f32x2
// arithmetic (k_adj_shell_tile2), like the forward kernel.
#pragma once
#include <utility>

#include "lbe_shell_kernels.cuh"

namespace lbe {

// e_CC of the point (ex, ey, ez)
template <int CC>
__host__ __device__ constexpr int comp(int ex, int ey, int ez) {
    return CC == 0 ? ex : (CC == 1 ? ey : ez);
}

// plane offset k (relative to the first output) is read by some output t for component CC
template <int S, int TZ, int CC>
__host__ __device__ constexpr bool adj_col_needs(int ex, int ey, unsigned mask, int k) {
    for (int t = 0; t < TZ; ++t) {
        const int ez = k - t;
        if (ez >= -S && ez <= S && ((mask >> (ez + S)) & 1u) && comp<CC>(ex, ey, ez) != 0) return true;
    }
    return false;
}

template <typename T, int S, int TZ, int TYB, int CC, int I>
__device__ __forceinline__ void adj_column_pair(const T *const *sb, T *aq, T *ap) {
    using Tl = ShellTileZ<T, S, TZ, TYB>;
    constexpr int ex = ColTable<S>::cols.ex[I];
    constexpr int ey = ColTable<S>::cols.ey[I];
    constexpr unsigned mask = ColTable<S>::cols.mask[I];
    if constexpr (!((CC == 0 && ex == 0) || (CC == 1 && ey == 0))) {
        constexpr int offc = ey * Tl::BX + ex;
        constexpr int GN = Tl::PLANE_BYTES / (int)sizeof(T);
        constexpr int NK = 2 * S + TZ;
        T cq[NK], cp[NK], mq[NK], mp[NK];
        [&]<int... K>(std::integer_sequence<int, K...>) {
            (
                [&] {
                    if constexpr (adj_col_needs<S, TZ, CC>(ex, ey, mask, K - S)) {
                        const T *p = sb[K];
                        cq[K] = p[offc];
                        cp[K] = p[offc + GN];
                        mq[K] = p[-offc];
                        mp[K] = p[-offc + GN];
                    }
                }(),
                ...);
        }(std::make_integer_sequence<int, NK>{});
        [&]<int... J>(std::integer_sequence<int, J...>) {
            (
                [&] {
                    constexpr int t = J / (2 * S + 1);
                    constexpr int ez = J % (2 * S + 1) - S;
                    constexpr int ec = comp<CC>(ex, ey, ez);
                    if constexpr (((mask >> (ez + S)) & 1u) && ec != 0) {
                        constexpr double len = ct_sqrt((double)(ex * ex + ey * ey + ez * ez));
                        constexpr T u = (T)(ec / len);
                        aq[t] += u * (cq[t + ez + S] - mq[t - ez + S]);
                        ap[t] += u * (cp[t + ez + S] - mp[t - ez + S]);
                    }
                }(),
                ...);
        }(std::make_integer_sequence<int, TZ *(2 * S + 1)>{});
    }
}

template <typename T, int S, int TZ, int TYB, int CC, int... I>
__device__ __forceinline__ void adj_all_columns(const T *const *sb, T *aq, T *ap, std::integer_sequence<int, I...>) {
    (adj_column_pair<T, S, TZ, TYB, CC, I>(sb, aq, ap), ...);
}

template <typename T, int S, int TZ, int TYB, int CC>
__global__ void __launch_bounds__(32 * TYB, 1)
    k_adj_shell_tile(const __grid_constant__ CUtensorMap map_L, const __grid_constant__ CUtensorMap map_gL, Grid g,
                     int ox, const T *__restrict__ npad_b, const T *__restrict__ g_ab, T *__restrict__ ln_b,
                     T *__restrict__ lg_ab, int *err) {
    using Tl = ShellTileZ<T, S, TZ, TYB>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_align128(smem_raw);
    T *ring = reinterpret_cast<T *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Tl::R * Tl::SLOT_BYTES);
    constexpr int SLOT = Tl::SLOT_BYTES / (int)sizeof(T);
    constexpr int GN = Tl::PLANE_BYTES / (int)sizeof(T);
    constexpr int NK = 2 * S + TZ;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY, z0 = blockIdx.z * Tl::LZ;
    const int zend = min(z0 + Tl::LZ, g.nz);
    const int nsuper = (zend - z0 + TZ - 1) / TZ;
    const int nplanes = nsuper * TZ + 2 * S;
    const bool leader = (tx == 0 && ty == 0);
    const int bx = x0 + g.H - S - ox;
    const int by = y0 + g.H - S;
    constexpr uint32_t tx_bytes = 2u * Tl::PLANE * (uint32_t)sizeof(T);

    if (leader) {
        prefetch_tensormap(&map_L);
        prefetch_tensormap(&map_gL);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {  // plane j holds interior z = z0 - S + j
        const int slot = j % Tl::R;
        unsigned char *dst = base + slot * Tl::SLOT_BYTES;
        const int zp = z0 - S + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
        tma_load_3d(dst, &map_L, bx, by, zp, &bars[slot]);
        tma_load_3d(dst + Tl::PLANE_BYTES, &map_gL, bx, by, zp, &bars[slot]);
    };
    if (leader)
        for (int j = 0; j < Tl::R && j < nplanes; ++j) issue(j);

    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    const int toff = (ty + S) * Tl::BX + (tx + S + ox);

    for (int s = 0; s < nsuper; ++s) {
        const int j0 = s * TZ;
        for (int j = j0; j < j0 + NK; ++j)
            if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
                mbar_drain(bars, Tl::R, j, min(j0 + Tl::R, nplanes));
                return;
            }
        if (active) {
            T nb[TZ], gr[TZ], oln[TZ], olg[TZ];
            long long idx[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const int z = min(z0 + j0 + t, zend - 1);
                idx[t] = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
                nb[t] = npad_b[pidx(g, x, y, z)];
                gr[t] = g_ab[idx[t]];
                oln[t] = ln_b[idx[t]];
                olg[t] = lg_ab[idx[t]];
            }
            const T *sb[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) sb[k] = ring + ((j0 + k) % Tl::R) * SLOT + toff;
            T aq[TZ], ap[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                aq[t] = (T)0;
                ap[t] = (T)0;
            }
            if constexpr (CC == 2) {
                // centre column (0, 0, +-S): e^ = (0, 0, 1) for ez = +S
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    aq[t] += sb[t + 2 * S][0] - sb[t][0];
                    ap[t] += sb[t + 2 * S][GN] - sb[t][GN];
                }
            }
            adj_all_columns<T, S, TZ, TYB, CC>(sb, aq, ap, std::make_integer_sequence<int, ColTable<S>::count>{});
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                if (z0 + j0 + t < zend) {
                    ln_b[idx[t]] = oln[t] - ap[t] - gr[t] * aq[t];
                    lg_ab[idx[t]] = olg[t] - nb[t] * aq[t];
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

// FP32 variant on the interleaved field (Lambda_CC, (g Lambda)_CC): one 8-byte element per node (the
// forward kernel's tile, ShellTileZ2), both divergence sums as packed f32x2 arithmetic (x: TQ, y: TP).
template <int S, int TZ, int TYB, int CC, int I>
__device__ __forceinline__ void adj_column_pair2(const f2 *const *sb, f2 *acc) {
    using Tl = ShellTileZ2<S, TZ, TYB>;
    constexpr int ex = ColTable<S>::cols.ex[I];
    constexpr int ey = ColTable<S>::cols.ey[I];
    constexpr unsigned mask = ColTable<S>::cols.mask[I];
    if constexpr (!((CC == 0 && ex == 0) || (CC == 1 && ey == 0))) {
        constexpr int offc = ey * Tl::BX + ex;
        constexpr int NK = 2 * S + TZ;
        f2 cp[NK], cm[NK];
        [&]<int... K>(std::integer_sequence<int, K...>) {
            (
                [&] {
                    if constexpr (adj_col_needs<S, TZ, CC>(ex, ey, mask, K - S)) {
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
                    constexpr int ec = comp<CC>(ex, ey, ez);
                    if constexpr (((mask >> (ez + S)) & 1u) && ec != 0) {
                        constexpr double len = ct_sqrt((double)(ex * ex + ey * ey + ez * ez));
                        acc[t] = f2fma(f2splat((float)(ec / len)), f2sub(cp[t + ez + S], cm[t - ez + S]), acc[t]);
                    }
                }(),
                ...);
        }(std::make_integer_sequence<int, TZ *(2 * S + 1)>{});
    }
}

template <int S, int TZ, int TYB, int CC, int... I>
__device__ __forceinline__ void adj_all_columns2(const f2 *const *sb, f2 *acc, std::integer_sequence<int, I...>) {
    (adj_column_pair2<S, TZ, TYB, CC, I>(sb, acc), ...);
}

template <int S, int TZ, int TYB, int CC>
__global__ void __launch_bounds__(32 * TYB, 1)
    k_adj_shell_tile2(const __grid_constant__ CUtensorMap map_LG, Grid g, int ox, const float *__restrict__ npad_b,
                      const float *__restrict__ g_ab, float *__restrict__ ln_b, float *__restrict__ lg_ab,
                      int *err) {
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
        prefetch_tensormap(&map_LG);
        for (int r = 0; r < Tl::R; ++r) mbar_init(&bars[r], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int j) {  // plane j holds interior z = z0 - S + j
        const int slot = j % Tl::R;
        const int zp = z0 - S + j + g.H;
        mbar_arrive_expect_tx(&bars[slot], tx_bytes);
        tma_load_3d(base + slot * Tl::SLOT_BYTES, &map_LG, bx, by, zp, &bars[slot]);
    };
    if (leader)
        for (int j = 0; j < Tl::R && j < nplanes; ++j) issue(j);

    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    const int toff = (ty + S) * Tl::BX + (tx + S + ox);

    for (int s = 0; s < nsuper; ++s) {
        const int j0 = s * TZ;
        for (int j = j0; j < j0 + NK; ++j)
            if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) {
                mbar_drain(bars, Tl::R, j, min(j0 + Tl::R, nplanes));
                return;
            }
        if (active) {
            float nb[TZ], gr[TZ], oln[TZ], olg[TZ];
            long long idx[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const int z = min(z0 + j0 + t, zend - 1);
                idx[t] = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
                nb[t] = npad_b[pidx(g, x, y, z)];
                gr[t] = g_ab[idx[t]];
                oln[t] = ln_b[idx[t]];
                olg[t] = lg_ab[idx[t]];
            }
            const f2 *sb[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) sb[k] = ring + ((j0 + k) % Tl::R) * SLOT + toff;
            f2 acc[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) acc[t] = 0ull;
            if constexpr (CC == 2) {
                // centre column (0, 0, +-S): e^ = (0, 0, 1) for ez = +S
#pragma unroll
                for (int t = 0; t < TZ; ++t) acc[t] = f2add(acc[t], f2sub(sb[t + 2 * S][0], sb[t][0]));
            }
            adj_all_columns2<S, TZ, TYB, CC>(sb, acc, std::make_integer_sequence<int, ColTable<S>::count>{});
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                if (z0 + j0 + t < zend) {
                    const float2 v = f2unpack(acc[t]);  // (TQ_CC, TP_CC)
                    ln_b[idx[t]] = oln[t] - v.y - gr[t] * v.x;
                    lg_ab[idx[t]] = olg[t] - nb[t] * v.x;
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

template <int S, int TZ, int TYB, int CC>
cudaError_t launch_adj_tile2_cc(const AdjShellTile &L, cudaStream_t st) {
    using Tl = ShellTileZ2<S, TZ, TYB>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_shell_tile2<S, TZ, TYB, CC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const Grid &g = *L.grid;
    dim3 block(Tl::TX, Tl::TY, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int ox = ((g.H - S) % Tl::A + Tl::A) % Tl::A;
    k_adj_shell_tile2<S, TZ, TYB, CC><<<grid, block, Tl::SMEM, st>>>(
        L.maps_L[CC], g, ox, (const float *)L.npad_b, (const float *)L.g_ab, (float *)L.ln_b, (float *)L.lg_ab,
        L.err);
    return cudaGetLastError();
}

template <int S, int TZ, int TYB>
cudaError_t launch_adj_tile2(const AdjShellTile &L, cudaStream_t st) {
    cudaError_t e = launch_adj_tile2_cc<S, TZ, TYB, 0>(L, st);
    if (e != cudaSuccess) return e;
    e = launch_adj_tile2_cc<S, TZ, TYB, 1>(L, st);
    if (e != cudaSuccess) return e;
    return launch_adj_tile2_cc<S, TZ, TYB, 2>(L, st);
}

// One launch of component CC; L.maps_L / L.maps_gL hold the three components' maps.
template <typename T, int S, int TZ, int TYB, int CC>
cudaError_t launch_adj_tile_cc(const AdjShellTile &L, cudaStream_t st) {
    using Tl = ShellTileZ<T, S, TZ, TYB>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_shell_tile<T, S, TZ, TYB, CC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Tl::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const Grid &g = *L.grid;
    dim3 block(Tl::TX, Tl::TY, 1);
    dim3 grid((g.nx + Tl::TX - 1) / Tl::TX, (g.ny + Tl::TY - 1) / Tl::TY, (g.nz + Tl::LZ - 1) / Tl::LZ);
    const int ox = ((g.H - S) % Tl::A + Tl::A) % Tl::A;
    k_adj_shell_tile<T, S, TZ, TYB, CC><<<grid, block, Tl::SMEM, st>>>(
        L.maps_L[CC], L.maps_gL[CC], g, ox, (const T *)L.npad_b, (const T *)L.g_ab, (T *)L.ln_b, (T *)L.lg_ab,
        L.err);
    return cudaGetLastError();
}

template <typename T, int S, int TZ, int TYB>
cudaError_t launch_adj_tile(const AdjShellTile &L, cudaStream_t st) {
    cudaError_t e = launch_adj_tile_cc<T, S, TZ, TYB, 0>(L, st);
    if (e != cudaSuccess) return e;
    e = launch_adj_tile_cc<T, S, TZ, TYB, 1>(L, st);
    if (e != cudaSuccess) return e;
    return launch_adj_tile_cc<T, S, TZ, TYB, 2>(L, st);
}

}  // namespace lbe
