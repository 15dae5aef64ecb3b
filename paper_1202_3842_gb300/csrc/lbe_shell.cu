// K3: mean-field Enskog force of one ordered species pair (a, b) (Appendix,
// hard-sphere C^{alpha,mf}):
//   C^a(r) (+)= -kT sigma_ab^2 w_ab n_a(r) sum_{e in K_ab} e^ (g_ab(r) + g_ab(r+e))/2 n_b(r+e)
//            =  coef * n_a(r) * [ g_ab(r)/2 * sum e^ n_b(r+e) + 1/2 * sum e^ (g_ab n_b)(r+e) ]
// with coef = -kT sigma_ab^2 w_ab.  Both sums run over the half shell as
// e^ [a(r+e) - a(r-e)].
//
// Data path: the padded density n_b and the padded product g_ab*n_b are
// streamed plane by plane (z-marching) into a shared-memory ring by TMA
// (cp.async.bulk.tensor, one 2-D box of (32 + 2S) x (TY + 2S) per field and
// plane, completion on an mbarrier per ring slot).  Each thread owns one
// (x, y) column of the 32 x TY tile and produces one output per plane; the
// shell offsets are compile-time immediates.
#include <cstdio>
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
                  T *__restrict__ Cout, T coef, int accumulate, int *err) {
    using Tl = ShellTile<T, S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
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
        if (!mbar_wait_bounded(&bars[j % Tl::R], (j / Tl::R) & 1, err)) return;

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
        if (!mbar_wait_bounded(&bars[jn % Tl::R], (jn / Tl::R) & 1, err)) return;
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
            }
        }
        __syncthreads();
    }
}

template <typename T, int S>
static cudaError_t launch_one(const ShellLaunch &L, cudaStream_t st) {
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
                                                       (const T *)L.g_ab, (T *)L.Cout, (T)L.coef, L.accumulate,
                                                       L.err);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch(int S, const ShellLaunch &L, cudaStream_t st) {
    switch (S) {
        case 1: return launch_one<T, 1>(L, st);
        case 2: return launch_one<T, 2>(L, st);
        case 3: return launch_one<T, 3>(L, st);
        case 4: return launch_one<T, 4>(L, st);
        case 5: return launch_one<T, 5>(L, st);
        case 6: return launch_one<T, 6>(L, st);
        case 7: return launch_one<T, 7>(L, st);
        default: break;
    }
    if constexpr (sizeof(T) == 4) {
        if (S == 8) return launch_one<T, 8>(L, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_shell_force(bool fp64, int S, const ShellLaunch &L, cudaStream_t st) {
    return fp64 ? dispatch<double>(S, L, st) : dispatch<float>(S, L, st);
}

bool shell_supported(bool fp64, int S) { return S >= 1 && S <= (fp64 ? 7 : 8); }

void shell_box(bool fp64, int S, int *bx, int *by) {
#define LBE_BOX(T, s)                    \
    case s:                              \
        *bx = ShellTile<T, s>::BX;       \
        *by = ShellTile<T, s>::BY;       \
        return;
    if (fp64) {
        switch (S) { LBE_BOX(double, 1) LBE_BOX(double, 2) LBE_BOX(double, 3) LBE_BOX(double, 4)
                     LBE_BOX(double, 5) LBE_BOX(double, 6) LBE_BOX(double, 7) default: break; }
    } else {
        switch (S) { LBE_BOX(float, 1) LBE_BOX(float, 2) LBE_BOX(float, 3) LBE_BOX(float, 4)
                     LBE_BOX(float, 5) LBE_BOX(float, 6) LBE_BOX(float, 7) LBE_BOX(float, 8) default: break; }
    }
#undef LBE_BOX
    *bx = 0;
    *by = 0;
}

// Half-shell listing used by the kernels (for the integer-work parity check).
int half_shell_host(int S, int *e, int cap) {
    int c = 0;
    for (int z = -S; z <= S; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z) && positive_half(x, y, z)) {
                    if (c < cap) {
                        e[3 * c] = x;
                        e[3 * c + 1] = y;
                        e[3 * c + 2] = z;
                    }
                    ++c;
                }
    return c;
}

}  // namespace lbe
