// Compile-time contact shells and the tile geometry of the shell-force kernel.
#pragma once

#include <utility>

// FP32 shell tiles for pair diameters 4 to 6 (the common ones); the defaults are the fastest of measured
// sweeps, and a build may set others to measure them.  Z-blocked kernel: LBE_SHELL_TZ outputs per thread
// along z on LBE_SHELL_TY thread rows.
#ifndef LBE_SHELL_TZ
#define LBE_SHELL_TZ 6
#endif
#ifndef LBE_SHELL_TY
#define LBE_SHELL_TY 12
#endif
// Y-blocked kernel, the one these diameters run when LBE_SHELL_YB is 1: two output rows per thread,
// LBE_SHELL_YTZ outputs along z, LBE_SHELL_YTY thread rows.
#ifndef LBE_SHELL_YB
#define LBE_SHELL_YB 1
#endif
#ifndef LBE_SHELL_YTZ
#define LBE_SHELL_YTZ 3
#endif
#ifndef LBE_SHELL_YTY
#define LBE_SHELL_YTY 8
#endif

namespace lbe {

// Contact shell of integer diameter S (Appendix, hard-sphere C^{alpha,mf}: the
// integral over unit vectors k^ at distance sigma becomes a sum over the lattice
// vectors e with S - 1/2 <= |e| < S + 1/2, i.e. S^2 - S + 1 <= |e|^2 <= S^2 + S).
// Only one vector of each +-e pair is listed ("half shell"): the kernel sums
// e^ [a(r+e) - a(r-e)], which is exact because the shell is symmetric.
__host__ __device__ constexpr bool in_shell(int S, int x, int y, int z) {
    int r2 = x * x + y * y + z * z;
    return r2 >= S * S - S + 1 && r2 <= S * S + S;
}
__host__ __device__ constexpr bool positive_half(int x, int y, int z) {
    return z > 0 || (z == 0 && (y > 0 || (y == 0 && x > 0)));
}
__host__ __device__ constexpr int half_shell_count(int S) {
    int c = 0;
    for (int z = -S; z <= S; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z) && positive_half(x, y, z)) ++c;
    return c;
}

template <int K>
struct HalfShell {
    int e[K > 0 ? K : 1][3];
};

template <int S>
__host__ __device__ constexpr HalfShell<half_shell_count(S)> make_half_shell() {
    HalfShell<half_shell_count(S)> h{};
    int c = 0;
    for (int z = -S; z <= S; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z) && positive_half(x, y, z)) {
                    h.e[c][0] = x;
                    h.e[c][1] = y;
                    h.e[c][2] = z;
                    ++c;
                }
    return h;
}

// sqrt of a positive integer at compile time: Newton's method started above
// the root, stopped when an iterate no longer decreases; the result is within
// one unit in the last place of the true root.
__host__ __device__ constexpr double ct_sqrt(double v) {
    double x = v > 1.0 ? v : 1.0;
    for (int i = 0; i < 200; ++i) {
        double nx = 0.5 * (x + v / x);
        if (!(nx < x)) break;
        x = nx;
    }
    return x;
}

// Tile of the shell kernel: 32 x TY outputs per z-plane, marching LZ planes in z.
template <typename T, int S>
struct ShellTile {
    static constexpr int A = 16 / (int)sizeof(T);  // TMA x-alignment in elements
    static constexpr int TX = 32;
    static constexpr int TY = (sizeof(T) == 8 && S >= 5) ? 4 : 8;
    static constexpr int BX = ((TX + 2 * S + A - 1) + A - 1) / A * A;  // box width incl. alignment slack
    static constexpr int BY = TY + 2 * S;
    static constexpr int R = 2 * S + 2;  // ring slots: 2S+1 planes in use + 1 in flight
    static constexpr int PLANE = BX * BY;  // elements of one field plane
    static constexpr int PLANE_BYTES = ((PLANE * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int SLOT_BYTES = 2 * PLANE_BYTES;  // density plane + g*n plane
    static constexpr int SMEM = R * SLOT_BYTES + 256 /*barriers*/ + 128 /*alignment*/;
    static constexpr int LZ = 16;
};

// Column organisation of the half shell for the z-blocked kernel: column
// pairs (ex, ey) / (-ex, -ey) with ex > 0 or (ex == 0, ey > 0); mask bit
// (ez + S) is set when (ex, ey, ez) lies in the shell.  The centre column
// (0, 0) holds ez = +-S only and is handled on its own.
__host__ __device__ constexpr int column_count(int S) {
    int c = 0;
    for (int y = -S; y <= S; ++y)
        for (int x = 0; x <= S; ++x) {
            if (!(x > 0 || y > 0)) continue;
            bool any = false;
            for (int z = -S; z <= S; ++z) any = any || in_shell(S, x, y, z);
            if (any) ++c;
        }
    return c;
}

template <int K>
struct Columns {
    int ex[K], ey[K];
    unsigned mask[K];
};

template <int S>
__host__ __device__ constexpr Columns<column_count(S)> make_columns() {
    Columns<column_count(S)> t{};
    int c = 0;
    for (int y = -S; y <= S; ++y)
        for (int x = 0; x <= S; ++x) {
            if (!(x > 0 || y > 0)) continue;
            unsigned m = 0;
            for (int z = -S; z <= S; ++z)
                if (in_shell(S, x, y, z)) m |= 1u << (z + S);
            if (m) {
                t.ex[c] = x;
                t.ey[c] = y;
                t.mask[c] = m;
                ++c;
            }
        }
    return t;
}

// Tile of the z-blocked shell kernel: 32 x TYB threads, TZ outputs per thread
// along z; the ring holds the 2S + TZ planes in use plus TZ in flight.
template <typename T, int S, int TZ, int TYB = 16>
struct ShellTileZ {
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int TX = 32;
    static constexpr int TY = TYB;
    static constexpr int BX = ((TX + 2 * S + A - 1) + A - 1) / A * A;
    static constexpr int BY = TY + 2 * S;
    static constexpr int R = 2 * S + 2 * TZ;
    static constexpr int PLANE = BX * BY;
    static constexpr int PLANE_BYTES = ((PLANE * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int SLOT_BYTES = 2 * PLANE_BYTES;
    static constexpr int SMEM = R * SLOT_BYTES + 256 + 128;
    static constexpr int LZ = TZ == 3 ? 18 : 16;  // planes per CTA, a multiple of TZ
};

// Tile of the FP32 z-blocked forward kernel on the interleaved field: one
// 8-byte element (n_b, g_ab n_b) per node, so one shared load fetches both
// values of a stencil point and the two sums run as packed f32x2 arithmetic.
// TMA sees 8-byte elements: the x coordinate must be even (A = 2).
template <int S, int TZ, int TYB = 16>
struct ShellTileZ2 {
    static constexpr int A = 2;
    static constexpr int TX = 32;
    static constexpr int TY = TYB;
    static constexpr int BX = ((TX + 2 * S + A - 1) + A - 1) / A * A;
    static constexpr int BY = TY + 2 * S;
    static constexpr int R = 2 * S + 2 * TZ;
    static constexpr int PLANE = BX * BY;  // 8-byte elements of one plane
    static constexpr int PLANE_BYTES = ((PLANE * 8) + 127) / 128 * 128;
    static constexpr int SLOT_BYTES = PLANE_BYTES;
    static constexpr int SMEM = R * SLOT_BYTES + 256 + 128;
    static constexpr int LZ = (16 + TZ - 1) / TZ * TZ;  // planes per CTA, a multiple of TZ
};

// Tile of the FP32 y-blocked forward kernel (k_shell_force_yb): 32 x TYT threads, each with two output
// rows (y, y + 1) and TZ outputs along z, so a plane of the tile holds 32 x 2TYT outputs.  The ring holds
// the 2S + TZ planes in use plus up to TZ in flight, as many of those as fit in 227 KB of shared memory.
template <int S, int TZ, int TYT_ = 8>
struct ShellTileY {
    static constexpr int A = 2;
    static constexpr int TX = 32;
    static constexpr int TYT = TYT_;     // thread rows
    static constexpr int TY = 2 * TYT;   // output rows
    static constexpr int BX = ((TX + 2 * S + A - 1) + A - 1) / A * A;
    static constexpr int BY = TY + 2 * S;
    static constexpr int PLANE = BX * BY;
    static constexpr int PLANE_BYTES = ((PLANE * 8) + 127) / 128 * 128;
    static constexpr int SLOT_BYTES = PLANE_BYTES;
    static constexpr int NK = 2 * S + TZ;
    static constexpr int RFIT = (227 * 1024 - 256 - 128) / SLOT_BYTES;
    static constexpr int R = RFIT < NK + TZ ? RFIT : NK + TZ;
    static_assert(R >= NK, "the planes one step reads do not fit in shared memory");
    static constexpr int SMEM = R * SLOT_BYTES + 256 + 128;
    static constexpr int LZ = (16 + TZ - 1) / TZ * TZ;
};

// Column bits of the shell: bit (ez + S) of col_mask(S, ex, ey) is set when (ex, ey, ez) is in the shell.
__host__ __device__ constexpr unsigned col_mask(int S, int ex, int ey) {
    unsigned m = 0;
    for (int z = -S; z <= S; ++z)
        if (in_shell(S, ex, ey, z)) m |= 1u << (z + S);
    return m;
}
// Largest |ey| with a nonempty column at ex (-1 if none).
__host__ __device__ constexpr int col_eymax(int S, int ex) {
    int r = -1;
    for (int y = 0; y <= S; ++y)
        if (col_mask(S, ex, y)) r = y;
    return r;
}

}  // namespace lbe
