// Species masses of the current state without any device allocation.
//
// For callers that must not allocate device memory at the moment they ask
// for the totals: code that runs with the device memory pool fully reserved
// by another framework, loops that cannot take the latency or the
// synchronisation of an allocation, and callers that keep a fixed,
// pre-declared device-memory footprint.  lbe_get_totals needs FP64 scratch
// fields of the lattice's size (allocated on its first use); this entry point
// instead fuses the pulled zeroth moment with a per-block FP64 partial sum and
// keeps the block partials in one file-scope device array.
//
// The array (g_mass_scratch) holds LBE_NOALLOC_MAX_BLOCKS partials for each of
// up to four species plus the four results: 4 * 4096 + 4 doubles (about
// 128 KiB).  It is part of the library image, so every GPU that loads the
// library keeps it until the process exits.  Every call shares it: a call
// overwrites all the partials it reads (nothing has to start at zero), the
// last call's contents stay behind, and calls that overlap on the GPU (two
// streams or two host threads at once) race on it.
#include <mutex>
#include <string>

#include "../../include/lbe.h"
#include "lbe_device.cuh"

namespace lbe {

constexpr int NOALLOC_MAX_BLOCKS = 4096;   // partial sums per species
constexpr int NOALLOC_NODES_PER_BLOCK = 4096;  // 256 threads x 16 nodes
constexpr int NOALLOC_THREADS = 256;

static __device__ __align__(256) double g_mass_scratch[MAXS * NOALLOC_MAX_BLOCKS + MAXS];

// Pulled density of species a at node i (the streamed zeroth moment; 0 on solid nodes).
template <typename S, typename T>
__device__ __forceinline__ T pulled_density(int nx, int ny, int nz, long long N, const S *__restrict__ pop,
                                            const uint32_t *__restrict__ mask, int a, T n0, long long i) {
    const uint32_t m = mask[i];
    if (m & 1u) return (T)0;
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    const long long sy = nx, sz = (long long)nx * ny;
    const long long xm = (x > 0) ? -1 : (nx - 1), xp = (x < nx - 1) ? 1 : -(nx - 1);
    const long long ym = (y > 0) ? -sy : (ny - 1) * sy, yp = (y < ny - 1) ? sy : -(ny - 1) * sy;
    const long long zm = (z > 0) ? -sz : (nz - 1) * sz, zp = (z < nz - 1) ? sz : -(nz - 1) * sz;
    const S *fb = pop + (long long)(a * 2) * Q * N;
    T n = (T)0;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        long long d = 0;
        d += cx(p) == 1 ? xm : (cx(p) == -1 ? xp : 0);
        d += cy(p) == 1 ? ym : (cy(p) == -1 ? yp : 0);
        d += cz(p) == 1 ? zm : (cz(p) == -1 ? zp : 0);
        const long long off = (m & (1u << p)) ? (long long)opp(p) * N + i : (long long)p * N + i + d;
        n += Store<S, T>::load(fb + off, (T)wq(p) * n0);
    }
    return n;
}

template <typename S, typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_mass_partials(int nx, int ny, int nz, long long N, const S *__restrict__ pop, const uint32_t *__restrict__ mask,
                    int M, double n00, double n01, double n02, double n03, double *__restrict__ scratch) {
    __shared__ double sh[NOALLOC_THREADS / 32];
    const double n0s[4] = {n00, n01, n02, n03};
    const long long b0 = (long long)blockIdx.x * NOALLOC_NODES_PER_BLOCK;
    for (int a = 0; a < M; ++a) {
        double s = 0.0;
        for (int k = threadIdx.x; k < NOALLOC_NODES_PER_BLOCK; k += NOALLOC_THREADS) {
            const long long i = b0 + k;
            if (i < N) s += (double)pulled_density<S, T>(nx, ny, nz, N, pop, mask, a, (T)n0s[a], i);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NOALLOC_THREADS / 32; ++w) t += sh[w];
            scratch[a * NOALLOC_MAX_BLOCKS + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_mass_final(int M, int nblocks, double *__restrict__ scratch) {
    __shared__ double sh[32];
    for (int a = 0; a < M; ++a) {
        double s = 0.0;
        for (int k = threadIdx.x; k < nblocks; k += 1024) s += scratch[a * NOALLOC_MAX_BLOCKS + k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 32; ++w) t += sh[w];
            scratch[MAXS * NOALLOC_MAX_BLOCKS + a] = t;
        }
        __syncthreads();
    }
}

// Device address of g_mass_scratch, looked up once per device (with that
// device current) on the first call made on it.
static std::mutex g_scratch_mutex;
static double *g_scratch_ptr[256];

cudaError_t noalloc_scratch(int device, double **out) {
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

cudaError_t launch_mass_noalloc(int prec, int nx, int ny, int nz, const void *pop, const uint32_t *mask, int M,
                                const double *n0, double *scratch, int nblocks, cudaStream_t st) {
    const long long N = (long long)nx * ny * nz;
    const double a0 = n0[0], a1 = M > 1 ? n0[1] : 0.0, a2 = M > 2 ? n0[2] : 0.0, a3 = M > 3 ? n0[3] : 0.0;
    switch (prec) {
        case LBE_FP64:
            k_mass_partials<double, double><<<nblocks, NOALLOC_THREADS, 0, st>>>(
                nx, ny, nz, N, (const double *)pop, mask, M, a0, a1, a2, a3, scratch);
            break;
        case LBE_FP32:
            k_mass_partials<float, float><<<nblocks, NOALLOC_THREADS, 0, st>>>(
                nx, ny, nz, N, (const float *)pop, mask, M, a0, a1, a2, a3, scratch);
            break;
        case LBE_BF16_SHIFTED:
            k_mass_partials<__nv_bfloat16, float><<<nblocks, NOALLOC_THREADS, 0, st>>>(
                nx, ny, nz, N, (const __nv_bfloat16 *)pop, mask, M, a0, a1, a2, a3, scratch);
            break;
        case LBE_FP16_SHIFTED:
            k_mass_partials<__half, float><<<nblocks, NOALLOC_THREADS, 0, st>>>(
                nx, ny, nz, N, (const __half *)pop, mask, M, a0, a1, a2, a3, scratch);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, 1024, 0, st>>>(M, nblocks, scratch);
    return cudaGetLastError();
}

long long noalloc_max_nodes() { return (long long)NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK; }
int noalloc_blocks(long long N) { return (int)((N + NOALLOC_NODES_PER_BLOCK - 1) / NOALLOC_NODES_PER_BLOCK); }
size_t noalloc_result_offset() { return (size_t)MAXS * NOALLOC_MAX_BLOCKS; }

}  // namespace lbe
