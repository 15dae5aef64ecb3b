// Node-level helpers shared by the forward and adjoint kernels: population
// offsets, neighbour offsets with periodic wrap, the pull of one streamed
// population (mid-point bounce-back on blocked links), c_p . v.
#pragma once
#include <utility>

#include "lbe_device.cuh"

namespace lbe {

__device__ __forceinline__ long long pop_off(int a, int fg, int p, long long N) {
    return ((long long)(a * 2 + fg) * Q + p) * N;
}

// Lattices hold fewer than 2^31 nodes (checked at creation), so 32-bit
// division suffices.
__device__ __forceinline__ void node_xyz(const Grid &g, long long i, int &x, int &y, int &z) {
    const unsigned ii = (unsigned)i, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned r = ii / nx;
    x = (int)(ii - r * nx);
    const unsigned q = r / ny;
    y = (int)(r - q * ny);
    z = (int)q;
}

// Linear offsets to the six neighbours with periodic wrap (a closed axis wraps
// too; such links are masked, so the wrapped address is never used).  Lattices
// hold fewer than 2^31 nodes, so an offset, and the sum of three that reaches
// another node, fits in 32 bits (six registers fewer than 64-bit offsets).
struct NbrOff {
    int xm, xp, ym, yp, zm, zp;
};
__device__ __forceinline__ NbrOff nbr_offsets(const Grid &g, int x, int y, int z) {
    NbrOff o;
    const int sx = 1, sy = g.nx, sz = g.nx * g.ny;
    o.xm = (x > 0) ? -sx : (g.nx - 1) * sx;
    o.xp = (x < g.nx - 1) ? sx : -(g.nx - 1) * sx;
    o.ym = (y > 0) ? -sy : (g.ny - 1) * sy;
    o.yp = (y < g.ny - 1) ? sy : -(g.ny - 1) * sy;
    o.zm = (z > 0) ? -sz : (g.nz - 1) * sz;
    o.zp = (z < g.nz - 1) ? sz : -(g.nz - 1) * sz;
    return o;
}
// Offset of the source node r - c_p.
template <int P>
__device__ __forceinline__ long long src_off(const NbrOff &o) {
    int d = 0;
    if constexpr (cx(P) == 1) d += o.xm;
    if constexpr (cx(P) == -1) d += o.xp;
    if constexpr (cy(P) == 1) d += o.ym;
    if constexpr (cy(P) == -1) d += o.yp;
    if constexpr (cz(P) == 1) d += o.zm;
    if constexpr (cz(P) == -1) d += o.zp;
    return d;
}

template <typename S, typename T, int P, bool SOLID = true>
__device__ __forceinline__ T pull(const S *__restrict__ fg_base, long long N, long long i, const NbrOff &o,
                                  uint32_t m, T n0) {
    // fg_base points at population 0 of this species' f (or g) block
    const T wn0 = (T)wq(P) * n0;
    if constexpr (SOLID) {
        const long long off = (m & (1u << P)) ? (long long)opp(P) * N + i : (long long)P * N + i + src_off<P>(o);
        return Store<S, T>::load(fg_base + off, wn0);
    } else {
        return Store<S, T>::load(fg_base + (long long)P * N + i + src_off<P>(o), wn0);
    }
}

// The same pull, returning the deviation f - w_p n0 of the pulled population (see Store).
template <typename S, typename T, int P, bool SOLID = true>
__device__ __forceinline__ T pull_dev(const S *__restrict__ fg_base, long long N, long long i, const NbrOff &o,
                                      uint32_t m, T n0) {
    const T wn0 = (T)wq(P) * n0;
    if constexpr (SOLID) {
        const long long off = (m & (1u << P)) ? (long long)opp(P) * N + i : (long long)P * N + i + src_off<P>(o);
        return Store<S, T>::load_dev(fg_base + off, wn0);
    } else {
        return Store<S, T>::load_dev(fg_base + (long long)P * N + i + src_off<P>(o), wn0);
    }
}

template <typename T, int P>
__device__ __forceinline__ T cdot(const T *v) {
    T r = (T)0;
    if constexpr (cx(P) == 1) r += v[0];
    if constexpr (cx(P) == -1) r -= v[0];
    if constexpr (cy(P) == 1) r += v[1];
    if constexpr (cy(P) == -1) r -= v[1];
    if constexpr (cz(P) == 1) r += v[2];
    if constexpr (cz(P) == -1) r -= v[2];
    return r;
}

__device__ __forceinline__ int plane_index(const Grid &g, int axis, int x, int y, int z) {
    return axis == 0 ? y + g.ny * z : (axis == 1 ? x + g.nx * z : x + g.nx * y);
}

}  // namespace lbe
