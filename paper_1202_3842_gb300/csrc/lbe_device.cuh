// Device-side building blocks of the D3Q19 Lattice Boltzmann-Enskog kernels:
// lattice tables, population storage formats, padded halo layout, bounded
// mbarrier waits and TMA copies.  sm_103a only.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbe {

constexpr int Q = 19;
constexpr int MAXS = 4;

// D3Q19 velocities in the order of the public ABI: rest; +x,-x,+y,-y,+z,-z;
// then the 12 edge links with each opposite pair adjacent.
__host__ __device__ constexpr int cx(int p) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[p];
}
__host__ __device__ constexpr int cy(int p) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[p];
}
__host__ __device__ constexpr int cz(int p) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[p];
}
__host__ __device__ constexpr int opp(int p) { return p == 0 ? 0 : ((p & 1) ? p + 1 : p - 1); }
// Gauss-Hermite weights: 1/3 (rest), 1/18 (axis), 1/36 (edge).
__host__ __device__ constexpr double wq(int p) {
    return p == 0 ? 1.0 / 3.0 : (p <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Error bits of the device error word.
enum : int {
    ERR_DENSITY = 1,   // negative or non-finite density
    ERR_PACKING = 2,   // xi3 >= 1 or non-finite contact value
    ERR_TMA_WAIT = 4,  // an mbarrier wait ran out of iterations
};

// ---------------------------------------------------------------------------
// Population storage.  S is the stored type, T the arithmetic type.  FP64
// stores the populations f themselves.  The other forms store them shifted by
// their rest value w_p n0 (n0 the species' mean density over the fluid nodes),
// so that the stored quantum is relative to the deviation, not to f: FP32
// stores d = f - w_p n0, the 16-bit forms s = f/(w_p n0) - 1.
//   load(p, wn0)                 -> f
//   store(p, f, wn0, iwn0)       <- f
//   load_dev(p, wn0)             -> d = f - w_p n0
//   store_dev(p, d, wn0, iwn0)   <- d
// with wn0 = w_p n0 and iwn0 = 1/(w_p n0).  The fused collision works on the
// deviations throughout, so its rounding is relative to them as well.
// ---------------------------------------------------------------------------
template <typename S, typename T>
struct Store;

template <>
struct Store<double, double> {
    static __device__ __forceinline__ double load(const double *p, double) { return __ldg(p); }
    static __device__ __forceinline__ void store(double *p, double v, double, double) { *p = v; }
    static __device__ __forceinline__ double load_dev(const double *p, double wn0) { return __ldg(p) - wn0; }
    static __device__ __forceinline__ void store_dev(double *p, double d, double wn0, double) { *p = d + wn0; }
    static constexpr bool shifted = false;
};
template <>
struct Store<float, float> {
    static __device__ __forceinline__ float load(const float *p, float wn0) { return __ldg(p) + wn0; }
    static __device__ __forceinline__ void store(float *p, float v, float wn0, float) { *p = v - wn0; }
    static __device__ __forceinline__ float load_dev(const float *p, float) { return __ldg(p); }
    static __device__ __forceinline__ void store_dev(float *p, float d, float, float) { *p = d; }
    static constexpr bool shifted = true;
};
template <>
struct Store<__nv_bfloat16, float> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p, float wn0) {
        return fmaf(wn0, __bfloat162float(__ldg(p)), wn0);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v, float, float iwn0) {
        *p = __float2bfloat16_rn(fmaf(v, iwn0, -1.0f));
    }
    static __device__ __forceinline__ float load_dev(const __nv_bfloat16 *p, float wn0) {
        return wn0 * __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void store_dev(__nv_bfloat16 *p, float d, float, float iwn0) {
        *p = __float2bfloat16_rn(d * iwn0);
    }
    static constexpr bool shifted = true;
};
template <>
struct Store<__half, float> {
    static __device__ __forceinline__ float load(const __half *p, float wn0) {
        return fmaf(wn0, __half2float(__ldg(p)), wn0);
    }
    static __device__ __forceinline__ void store(__half *p, float v, float, float iwn0) {
        *p = __float2half_rn(fmaf(v, iwn0, -1.0f));
    }
    static __device__ __forceinline__ float load_dev(const __half *p, float wn0) {
        return wn0 * __half2float(__ldg(p));
    }
    static __device__ __forceinline__ void store_dev(__half *p, float d, float, float iwn0) {
        *p = __float2half_rn(d * iwn0);
    }
    static constexpr bool shifted = true;
};

// ---------------------------------------------------------------------------
// Lattice geometry passed by value to every kernel.
// ---------------------------------------------------------------------------
struct Grid {
    int nx, ny, nz;
    int per[3];
    long long N;
    // padded halo layout of the stencil fields (density, g*n): H ghost layers
    // on every side, rows padded to px elements (a multiple of 8)
    int H, px, py, pz;
    long long P;  // px*py*pz
};

__host__ __device__ __forceinline__ long long pidx(const Grid &g, int x, int y, int z) {
    return (long long)(x + g.H) + (long long)g.px * ((long long)(y + g.H) + (long long)g.py * (z + g.H));
}

// Wrap a coordinate on a periodic axis; returns false when it leaves a closed axis.
__device__ __forceinline__ bool wrap(int &v, int n, int periodic) {
    if (v < 0 || v >= n) {
        if (!periodic) return false;
        v = ((v % n) + n) % n;
    }
    return true;
}

// Write value v of interior node (x,y,z) into the padded field, including all
// its periodic images inside the halo.  Ghost cells of closed axes stay zero.
template <typename T>
__device__ __forceinline__ void write_padded(const Grid &g, T *f, int x, int y, int z, T v) {
    int kx0 = 0, kx1 = 0, ky0 = 0, ky1 = 0, kz0 = 0, kz1 = 0;
    if (g.per[0]) { kx0 = -((x + g.H) / g.nx); kx1 = (g.nx + g.H - 1 - x) / g.nx; }
    if (g.per[1]) { ky0 = -((y + g.H) / g.ny); ky1 = (g.ny + g.H - 1 - y) / g.ny; }
    if (g.per[2]) { kz0 = -((z + g.H) / g.nz); kz1 = (g.nz + g.H - 1 - z) / g.nz; }
    for (int kz = kz0; kz <= kz1; ++kz)
        for (int ky = ky0; ky <= ky1; ++ky)
            for (int kx = kx0; kx <= kx1; ++kx)
                f[pidx(g, x + kx * g.nx, y + ky * g.ny, z + kz * g.nz)] = v;
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (inline PTX).  Every wait is bounded: after the iteration
// limit the caller gets `false`, records ERR_TMA_WAIT and leaves its loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// First 128-byte aligned byte of the dynamic shared memory `raw`.  The offset is added to the pointer
// itself (not through an integer round trip), so every pointer derived from the result stays a
// shared-memory pointer to the compiler and reads through it compile to shared-memory loads.
__device__ __forceinline__ unsigned char *smem_align128(unsigned char *raw) {
    return raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity to complete: at most `polls` try_wait polls (the
// kernels use the default, 2^24) and at most WAIT_NS of wall time, whichever ends first; then
// ERR_TMA_WAIT is recorded and the caller gets false.  The time bound keeps a launch whose copies do
// not complete (a box that delivers fewer bytes than its barrier expects, say) from waiting out the
// polls of every CTA in turn.
constexpr long long WAIT_POLLS = 1ll << 24;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  long long polls = WAIT_POLLS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (long long it = 1; it < polls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && globaltimer_ns() - t0 > WAIT_NS) break;
    }
    atomicOr(err, ERR_TMA_WAIT);
    return false;
}

// After a wait gave up: wait again, with a bound, for the copies this CTA issued into planes [j, jend)
// of its ring of R slots (plane j in slot j % R, phase j / R), so that none of them lands in shared
// memory after the CTA has exited.  Each plane gets at most 2^20 polls or 0.1 s on %globaltimer; the
// error bit is already set.  Kept out of line: it runs only on the failure path.
constexpr long long DRAIN_POLLS = 1ll << 20;
constexpr unsigned long long DRAIN_NS = 100000000ull;
static __device__ __noinline__ void mbar_drain(uint64_t *bars, int R, int j, int jend) {
    for (; j < jend; ++j) {
        uint64_t *b = bars + (j % R);
        const uint32_t parity = (uint32_t)(j / R) & 1u;
        const unsigned long long t0 = globaltimer_ns();
        for (long long it = 0; it < DRAIN_POLLS; ++it) {
            if (mbar_try_wait(b, parity)) break;
            if ((it & 255) == 255 && globaltimer_ns() - t0 > DRAIN_NS) break;
        }
    }
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 3-D tiled TMA load of one box into shared memory; completion is signalled on bar.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace lbe
