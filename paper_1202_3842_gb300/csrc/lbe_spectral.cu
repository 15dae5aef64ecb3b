// K3 by fast Fourier transforms: the spectral form of the mean-field shell force.
//
// The shell sums of one ordered pair (a, b) (Appendix, hard-sphere C^{alpha,mf})
//   P(r) = sum_{e in K_S} e^ n_b(r + e),   Q(r) = sum_{e in K_S} e^ (g_ab n_b)(r + e),
// are correlations of the densities with the fixed odd kernel K_S(e) = e / |e|.  On a grid that
// equals the lattice along periodic axes and carries at least S zero planes beyond the lattice along
// closed axes (the zero ghosts of a closed axis), a correlation is a circular convolution with
// kappa(x) = K_S(-x mod L), so
//   P^(k) = kappa^(k) n^(k),   kappa^(k) = i t(k),
// t real because kappa is real and odd.  The three components of t are tabulated once per shell by
// transforming kappa itself.  The ball averages of the contact values (n-bar_b, the mean of n_b over
// |d| <= sigma_b / 2) are convolutions with a real, even kernel, whose transform is real and is
// tabulated the same way.  One force stage (after K1) then runs
//   1. k_spec_embed_n: n_b into the zero-padded grid, one batched forward transform;
//   2. k_spec_ball_mul and one batched inverse transform: n-bar_b;
//   3. k_spec_contact: xi_2, xi_3 and the BMCSL g_ab of every node as in the direct contact kernel,
//      and g_ab n_b of every pair into the grid; one batched forward transform of those;
//   4. k_spec_multiply: the P spectra of every pair and component, and per species the Q spectra
//      summed with coef_ab / 2 (the inverse transform is linear), scaled by 1 / (L0 L1 L2);
//   5. one batched inverse transform of the 3 pairs + 3 M spectra;
//   6. k_spec_combine: C^a(r) = n_a(r) [ sum_b coef_ab / 2 g_ab(r) P_ab(r) + Qsum_a(r) ], the
//      arithmetic of the direct kernel regrouped (and P itself when the adjoint keeps it).
// The transforms are cuFFT's (a library FFT, like a library GEMM), loaded at run time from
// libcufft.so.12 so that the library still needs only libcuda to load; without it the spectral
// method reports LBE_ERR_UNSUPPORTED.
#include <cufft.h>
#include <dlfcn.h>

#include <mutex>
#include <type_traits>
#include <string>

#include "lbe_device.cuh"
#include "lbe_launch.h"

namespace lbe {

namespace {

struct CufftApi {
    decltype(&cufftCreate) create;
    decltype(&cufftDestroy) destroy;
    decltype(&cufftSetAutoAllocation) set_auto;
    decltype(&cufftMakePlanMany) make_many;
    decltype(&cufftSetWorkArea) set_work;
    decltype(&cufftSetStream) set_stream;
    decltype(&cufftExecR2C) r2c;
    decltype(&cufftExecC2R) c2r;
    decltype(&cufftExecD2Z) d2z;
    decltype(&cufftExecZ2D) z2d;
};

const CufftApi *cufft_api(std::string *why) {
    static std::mutex mu;
    static int state = 0;  // 0: not tried, 1: loaded, -1: missing
    static CufftApi api{};
    static std::string reason;
    std::lock_guard<std::mutex> lock(mu);
    if (state == 0) {
        void *h = nullptr;
        for (const char *name : {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"}) {
            h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
            if (h) break;
        }
        if (!h) {
            state = -1;
            reason = "cuFFT (libcufft.so.12) could not be loaded";
        } else {
            bool ok = true;
            auto get = [&](auto &fp, const char *sym) {
                fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(dlsym(h, sym));
                if (!fp) ok = false;
            };
            get(api.create, "cufftCreate");
            get(api.destroy, "cufftDestroy");
            get(api.set_auto, "cufftSetAutoAllocation");
            get(api.make_many, "cufftMakePlanMany");
            get(api.set_work, "cufftSetWorkArea");
            get(api.set_stream, "cufftSetStream");
            get(api.r2c, "cufftExecR2C");
            get(api.c2r, "cufftExecC2R");
            get(api.d2z, "cufftExecD2Z");
            get(api.z2d, "cufftExecZ2D");
            state = ok ? 1 : -1;
            if (!ok) reason = "libcufft.so.12 lacks a needed entry point";
        }
    }
    if (state < 0) {
        if (why) *why = reason;
        return nullptr;
    }
    return &api;
}

}  // namespace

struct SpectralShell {
    const CufftApi *api = nullptr;
    bool fp64 = false;
    int L[3] = {0, 0, 0};
    long long Nr = 0, Nc = 0;
    // 0: forward of the M densities; 1: inverse of the 3 pairs + 3 M force spectra; 2: forward of three
    // table fields; 3: forward of the pairs' g n; 4: inverse of the M ball averages
    static constexpr int NPLAN = 5;
    cufftHandle plan[NPLAN] = {0, 0, 0, 0, 0};
    bool made[NPLAN] = {false, false, false, false, false};
};

bool spectral_available(std::string *why) { return cufft_api(why) != nullptr; }

void spectral_destroy(SpectralShell *s) {
    if (!s) return;
    for (int k = 0; k < SpectralShell::NPLAN; ++k)
        if (s->made[k]) s->api->destroy(s->plan[k]);
    delete s;
}

int spectral_create(SpectralShell **out, bool fp64, const int L[3], int M, int npairs, int ninv, size_t *work_bytes,
                    std::string *why) {
    const int batch[SpectralShell::NPLAN] = {M, ninv, 3, npairs, M};
    const bool forward[SpectralShell::NPLAN] = {true, false, true, true, false};
    return spectral_create_plans(out, fp64, L, SpectralShell::NPLAN, batch, forward, work_bytes, why);
}

int spectral_create_plans(SpectralShell **out, bool fp64, const int L[3], int nplans, const int *batch,
                          const bool *forward, size_t *work_bytes, std::string *why) {
    *out = nullptr;
    if (nplans < 1 || nplans > SpectralShell::NPLAN) return -1;
    const CufftApi *api = cufft_api(why);
    if (!api) return -1;
    SpectralShell *s = new SpectralShell();
    s->api = api;
    s->fp64 = fp64;
    for (int k = 0; k < 3; ++k) s->L[k] = L[k];
    s->Nr = (long long)L[0] * L[1] * L[2];
    s->Nc = (long long)(L[0] / 2 + 1) * L[1] * L[2];
    int n[3] = {L[2], L[1], L[0]};  // row-major: x is the fastest (and the halved) dimension
    const cufftType fwd = fp64 ? CUFFT_D2Z : CUFFT_R2C, inv = fp64 ? CUFFT_Z2D : CUFFT_C2R;
    size_t wmax = 0;
    for (int k = 0; k < nplans; ++k) {
        cufftResult r = api->create(&s->plan[k]);
        if (r != CUFFT_SUCCESS) {
            if (why) *why = "cufftCreate failed (" + std::to_string((int)r) + ")";
            spectral_destroy(s);
            return -1;
        }
        s->made[k] = true;
        api->set_auto(s->plan[k], 0);
        size_t ws = 0;
        r = api->make_many(s->plan[k], 3, n, nullptr, 1, 0, nullptr, 1, 0, forward[k] ? fwd : inv, batch[k], &ws);
        if (r != CUFFT_SUCCESS) {
            if (why) *why = "cufftMakePlanMany failed (" + std::to_string((int)r) + ")";
            spectral_destroy(s);
            return -1;
        }
        wmax = ws > wmax ? ws : wmax;
    }
    *work_bytes = wmax;
    *out = s;
    return 0;
}

int spectral_bind(SpectralShell *s, void *work, cudaStream_t st) {
    for (int k = 0; k < SpectralShell::NPLAN; ++k) {
        if (!s->made[k]) continue;
        if (s->api->set_work(s->plan[k], work) != CUFFT_SUCCESS) return -1;
        if (s->api->set_stream(s->plan[k], st) != CUFFT_SUCCESS) return -1;
    }
    return 0;
}

// which: 0 the densities, 2 three table fields, 3 the pairs' g n; real -> half spectrum
int spectral_forward(SpectralShell *s, int which, void *R, void *Z) {
    cufftResult r = s->fp64 ? s->api->d2z(s->plan[which], (double *)R, (cufftDoubleComplex *)Z)
                            : s->api->r2c(s->plan[which], (float *)R, (cufftComplex *)Z);
    return r == CUFFT_SUCCESS ? 0 : (int)r;
}

// which: 1 the force spectra, 4 the ball averages; half spectrum -> real, unnormalised (the multiply
// kernels apply 1/(L0 L1 L2)); overwrites W
int spectral_inverse(SpectralShell *s, int which, void *W, void *R) {
    cufftResult r = s->fp64 ? s->api->z2d(s->plan[which], (cufftDoubleComplex *)W, (double *)R)
                            : s->api->c2r(s->plan[which], (cufftComplex *)W, (float *)R);
    return r == CUFFT_SUCCESS ? 0 : (int)r;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
    using type = float2;
};
template <>
struct Cplx<double> {
    using type = double2;
};

// kappa_c(-e mod L) += e_c / |e| for every shell point (aliases on a short periodic axis add up)
template <typename T>
__global__ void k_spec_scatter(T *R3, long long Nr, int L0, int L1, int L2, const int *e, const double *u, int ne) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ne) return;
    const int x = ((-e[3 * j] % L0) + L0) % L0;
    const int y = ((-e[3 * j + 1] % L1) + L1) % L1;
    const int z = ((-e[3 * j + 2] % L2) + L2) % L2;
    const long long idx = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    for (int c = 0; c < 3; ++c) atomicAdd(&R3[(long long)c * Nr + idx], (T)u[3 * j + c]);
}

template <typename T>
__global__ void k_spec_imag(const typename Cplx<T>::type *Z3, T *tab3, long long Nc) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nc) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) tab3[(long long)c * Nc + k] = Z3[(long long)c * Nc + k].y;
}

template <typename T>
__global__ void k_spec_real(const typename Cplx<T>::type *Z, T *tab, long long Nc) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < Nc) tab[k] = Z[k].x;
}

// one thread per grid point of a row: x = threadIdx + blockIdx.x * blockDim, y = blockIdx.y, z = blockIdx.z
template <typename T>
__global__ void k_spec_embed_n(Grid g, int L0, int L1, long long Nr, int M, const T *__restrict__ npad,
                               T *__restrict__ R) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L0) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long idx = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    const bool in = x < g.nx && y < g.ny && z < g.nz;
    const long long pi = in ? pidx(g, x, y, z) : 0;
    for (int b = 0; b < M; ++b) R[(long long)b * Nr + idx] = in ? npad[(long long)b * g.P + pi] : (T)0;
}

// W[b] = n^_b B^_b scale: the spectrum of the ball average (B^ real: the ball kernel is even)
template <typename T>
__global__ void k_spec_ball_mul(const typename Cplx<T>::type *__restrict__ Z, const T *__restrict__ btab,
                                typename Cplx<T>::type *__restrict__ W, long long Nc, int M, T scale) {
    using C2 = typename Cplx<T>::type;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nc) return;
    for (int b = 0; b < M; ++b) {
        const T w = btab[(long long)b * Nc + k] * scale;
        const C2 z = Z[(long long)b * Nc + k];
        C2 o;
        o.x = w * z.x;
        o.y = w * z.y;
        W[(long long)b * Nc + k] = o;
    }
}

// Contact values from the ball averages nbar [M][Nr] (grid layout), the arithmetic of the direct
// contact kernel: xi_k = sum_b xi_k-coefficient_b nbar_b, g_ab = BMCSL(xi2, xi3; s_ab).  Writes
// g_ab [M][M][N], optionally xi2, xi3 [2][N], and g_{a_q b_q} n_{b_q} of every pair q into the grid
// fields G [npairs][Nr] (zero outside the lattice).  Row kernel over the grid.
template <typename T, int M>
__global__ void k_spec_contact(Grid g, int L0, int L1, long long Nr, ContactParams cp, SpecPairs sp,
                               const T *__restrict__ npad, const T *__restrict__ nbar, T *__restrict__ gab,
                               T *__restrict__ xi_out, T *__restrict__ G, int *err) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L0) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long idx = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    if (!(x < g.nx && y < g.ny && z < g.nz)) {
        for (int q = 0; q < sp.npairs; ++q) G[(long long)q * Nr + idx] = (T)0;
        return;
    }
    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    const long long pi = pidx(g, x, y, z);
    T xi2 = 0, xi3 = 0, nl[M];
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const T nb = nbar[(long long)b * Nr + idx];
        xi2 += (T)cp.xi2c[b] * nb;
        xi3 += (T)cp.xi3c[b] * nb;
        nl[b] = npad[(long long)b * g.P + pi];
    }
    const T i1 = (T)1 / ((T)1 - xi3);
    if (!(xi3 < (T)1)) atomicOr(err, ERR_PACKING);
    if (xi_out) {
        xi_out[i] = xi2;
        xi_out[g.N + i] = xi3;
    }
    T gv[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const T s = (T)cp.s_ab[a][b];
            gv[a][b] = i1 + (T)3 * s * xi2 * i1 * i1 + (T)2 * s * s * xi2 * xi2 * i1 * i1 * i1;
            if (!isfinite(gv[a][b])) atomicOr(err, ERR_PACKING);
            gab[(long long)(a * M + b) * g.N + i] = gv[a][b];
        }
    for (int q = 0; q < sp.npairs; ++q) {
        T v = 0;
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b)
                if (sp.a[q] == a && sp.b[q] == b) v = gv[a][b] * nl[b];
        G[(long long)q * Nr + idx] = v;
    }
}

// W[3q + c] = i t_{S_q,c} n^_{b_q} scale ;  W[3 pairs + 3a + c] = sum_{q: a_q = a} coef_q / 2 i t_{S_q,c} G^_q scale
template <typename T>
__global__ void k_spec_multiply(const typename Cplx<T>::type *__restrict__ Z, const T *__restrict__ tab,
                                typename Cplx<T>::type *__restrict__ W, long long Nc, SpecPairs sp, T scale) {
    using C2 = typename Cplx<T>::type;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nc) return;
    for (int c = 0; c < 3; ++c) {
        T qr[MAXS], qi[MAXS];
        for (int a = 0; a < sp.M; ++a) qr[a] = qi[a] = (T)0;
        for (int q = 0; q < sp.npairs; ++q) {
            const T t = tab[((long long)sp.s[q] * 3 + c) * Nc + k] * scale;
            const C2 nb = Z[(long long)sp.b[q] * Nc + k];
            C2 o;
            o.x = -t * nb.y;
            o.y = t * nb.x;
            W[((long long)3 * q + c) * Nc + k] = o;
            const C2 gq = Z[(long long)(sp.M + q) * Nc + k];
            const T w = (T)sp.half_coef[q] * t;
            const int a = sp.a[q];
            qr[a] -= w * gq.y;
            qi[a] += w * gq.x;
        }
        for (int a = 0; a < sp.M; ++a) {
            C2 o;
            o.x = qr[a];
            o.y = qi[a];
            W[((long long)3 * sp.npairs + 3 * a + c) * Nc + k] = o;
        }
    }
}

// one thread per lattice node of a row: x = threadIdx + blockIdx.x * blockDim, y = blockIdx.y, z = blockIdx.z
template <typename T>
__global__ void k_spec_combine(Grid g, int L0, int L1, long long Nr, const T *__restrict__ R, const T *__restrict__ npad,
                               const T *__restrict__ gab, SpecPairs sp, T *__restrict__ Cout, T *__restrict__ Pout) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    const long long ri = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    const long long pi = pidx(g, x, y, z);
    for (int a = 0; a < sp.M; ++a) {
        const T na = npad[(long long)a * g.P + pi];
        for (int c = 0; c < 3; ++c) {
            T v = R[((long long)3 * sp.npairs + 3 * a + c) * Nr + ri];
            for (int q = 0; q < sp.npairs; ++q) {
                if (sp.a[q] != a) continue;
                const T Pq = R[((long long)3 * q + c) * Nr + ri];
                v += (T)sp.half_coef[q] * gab[(long long)(a * sp.M + sp.b[q]) * g.N + i] * Pq;
            }
            Cout[((long long)a * 3 + c) * g.N + i] = na * v;
        }
    }
    if (Pout)
        for (int q = 0; q < sp.npairs; ++q)
            for (int c = 0; c < 3; ++c)
                Pout[((long long)q * 3 + c) * g.N + i] = R[((long long)3 * q + c) * Nr + ri];
}

// The multiply and combine kernels for M = 1 or 2 species with all M^2 pairs present, in the order
// q = a M + b: every loop has compile-time bounds, so the sums stay in registers.
template <typename T, int M>
__global__ void k_spec_multiply_m(const typename Cplx<T>::type *__restrict__ Z, const T *__restrict__ tab,
                                  typename Cplx<T>::type *__restrict__ W, long long Nc, SpecPairs sp, T scale) {
    using C2 = typename Cplx<T>::type;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nc) return;
    C2 nh[M], gh[M * M];
#pragma unroll
    for (int b = 0; b < M; ++b) nh[b] = Z[(long long)b * Nc + k];
#pragma unroll
    for (int q = 0; q < M * M; ++q) gh[q] = Z[(long long)(M + q) * Nc + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T qr[M], qi[M];
#pragma unroll
        for (int a = 0; a < M; ++a) qr[a] = qi[a] = (T)0;
#pragma unroll
        for (int q = 0; q < M * M; ++q) {
            const T t = tab[((long long)sp.s[q] * 3 + c) * Nc + k] * scale;
            C2 o;
            o.x = -t * nh[q % M].y;
            o.y = t * nh[q % M].x;
            W[((long long)3 * q + c) * Nc + k] = o;
            const T w = (T)sp.half_coef[q] * t;
            qr[q / M] -= w * gh[q].y;
            qi[q / M] += w * gh[q].x;
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
            C2 o;
            o.x = qr[a];
            o.y = qi[a];
            W[((long long)3 * M * M + 3 * a + c) * Nc + k] = o;
        }
    }
}

template <typename T, int M>
__global__ void k_spec_combine_m(Grid g, int L0, int L1, long long Nr, const T *__restrict__ R,
                                 const T *__restrict__ npad, const T *__restrict__ gab, SpecPairs sp,
                                 T *__restrict__ Cout, T *__restrict__ Pout) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    const long long ri = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    const long long pi = pidx(g, x, y, z);
    T na[M], gq[M * M], P[M * M][3], Qs[M][3];
#pragma unroll
    for (int a = 0; a < M; ++a) na[a] = npad[(long long)a * g.P + pi];
#pragma unroll
    for (int q = 0; q < M * M; ++q) gq[q] = gab[(long long)q * g.N + i];
#pragma unroll
    for (int q = 0; q < M * M; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) P[q][c] = R[((long long)3 * q + c) * Nr + ri];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) Qs[a][c] = R[((long long)3 * M * M + 3 * a + c) * Nr + ri];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v = Qs[a][c];
#pragma unroll
            for (int b = 0; b < M; ++b) v += (T)sp.half_coef[a * M + b] * gq[a * M + b] * P[a * M + b][c];
            Cout[((long long)a * 3 + c) * g.N + i] = na[a] * v;
        }
    if (Pout)
#pragma unroll
        for (int q = 0; q < M * M; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) Pout[((long long)q * 3 + c) * g.N + i] = P[q][c];
}

// ---------------------------------------------------------------------------
// K3 transposed in spectral form (discrete adjoint).  For the pair q = (a, b) with Lambda_q = coef_q
// lambda_a, lambda_a = n_a lC^a / 2 (lC^a the adjoint of C^a), the shell sums of the transpose,
//   TQ_q(s) = sum_e e^ . Lambda_q(s + e),   TP_q(s) = sum_e e^ . (g_q Lambda_q)(s + e),
// are correlations with the forward kernel, so their spectra are i t_c times those of the fields.
// lambda_a does not depend on b: its transform serves every pair of species a.  The TP of the pairs
// of one species b are summed in spectral space (they enter only ln_b):
//   ln_b(s) -= TP_b(s) + sum_{q: b_q = b} g_q(s) TQ_q(s),   lg_q(s) -= n_b(s) TQ_q(s).
// Grid fields: lambda [M][3], then g lambda [npairs][3] (real); spectra TQ [npairs], TP [M].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adjspec_embed(Grid g, int L0, int L1, long long Nr, SpecPairs sp, const T *__restrict__ npad,
                                const T *__restrict__ lC, const T *__restrict__ gab, T *__restrict__ R) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L0) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long idx = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    const bool in = x < g.nx && y < g.ny && z < g.nz;
    const long long i = in ? (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z) : 0;
    const long long pi = in ? pidx(g, x, y, z) : 0;
    for (int a = 0; a < sp.M; ++a) {
        const T h = in ? (T)0.5 * npad[(long long)a * g.P + pi] : (T)0;
        for (int c = 0; c < 3; ++c)
            R[((long long)a * 3 + c) * Nr + idx] = in ? h * lC[((long long)a * 3 + c) * g.N + i] : (T)0;
    }
    for (int q = 0; q < sp.npairs; ++q) {
        const int a = sp.a[q];
        const T gh = in ? gab[(long long)(a * sp.M + sp.b[q]) * g.N + i] * (T)0.5 * npad[(long long)a * g.P + pi]
                        : (T)0;
        for (int c = 0; c < 3; ++c)
            R[((long long)(3 * sp.M + 3 * q + c)) * Nr + idx] = in ? gh * lC[((long long)a * 3 + c) * g.N + i] : (T)0;
    }
}

// W[q] = coef_q sum_c i t_{s_q,c} lambda^_{a_q,c};  W[npairs + b] = sum_{q: b_q = b} coef_q sum_c i t (g lambda)^_{q,c}
template <typename T>
__global__ void k_adjspec_multiply(const typename Cplx<T>::type *__restrict__ Z, const T *__restrict__ tab,
                                   typename Cplx<T>::type *__restrict__ W, long long Nc, SpecPairs sp, T scale) {
    using C2 = typename Cplx<T>::type;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nc) return;
    for (int q = 0; q < sp.npairs; ++q) {
        T re = 0, im = 0;
        for (int c = 0; c < 3; ++c) {
            const T t = tab[((long long)sp.s[q] * 3 + c) * Nc + k];
            const C2 l = Z[((long long)sp.a[q] * 3 + c) * Nc + k];
            re -= t * l.y;
            im += t * l.x;
        }
        const T w = (T)(2.0 * sp.half_coef[q]) * scale;
        C2 o;
        o.x = w * re;
        o.y = w * im;
        W[(long long)q * Nc + k] = o;
    }
    for (int b = 0; b < sp.M; ++b) {
        T re = 0, im = 0;
        for (int q = 0; q < sp.npairs; ++q) {
            if (sp.b[q] != b) continue;
            const T w = (T)(2.0 * sp.half_coef[q]);
            for (int c = 0; c < 3; ++c) {
                const T t = w * tab[((long long)sp.s[q] * 3 + c) * Nc + k];
                const C2 l = Z[((long long)(3 * sp.M + 3 * q + c)) * Nc + k];
                re -= t * l.y;
                im += t * l.x;
            }
        }
        C2 o;
        o.x = scale * re;
        o.y = scale * im;
        W[(long long)(sp.npairs + b) * Nc + k] = o;
    }
}

// ln [M][N], lg [M][M][N] of the lattice; R holds TQ [npairs] then TP [M] on the grid
template <typename T>
__global__ void k_adjspec_combine(Grid g, int L0, int L1, long long Nr, SpecPairs sp, const T *__restrict__ R,
                                  const T *__restrict__ npad, const T *__restrict__ gab, T *__restrict__ ln,
                                  T *__restrict__ lg) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    const long long ri = (long long)x + (long long)L0 * ((long long)y + (long long)L1 * z);
    const long long pi = pidx(g, x, y, z);
    for (int b = 0; b < sp.M; ++b) {
        T d = R[(long long)(sp.npairs + b) * Nr + ri];
        for (int q = 0; q < sp.npairs; ++q) {
            if (sp.b[q] != b) continue;
            const long long gi = (long long)(sp.a[q] * sp.M + b) * g.N + i;
            const T tq = R[(long long)q * Nr + ri];
            d += gab[gi] * tq;
            lg[gi] -= npad[(long long)b * g.P + pi] * tq;
        }
        ln[(long long)b * g.N + i] -= d;
    }
}

// all M^2 pairs present in the order a M + b, M = 1 or 2
bool full_pairs(const SpecPairs &sp) {
    if (sp.M > 2 || sp.npairs != sp.M * sp.M) return false;
    for (int q = 0; q < sp.npairs; ++q)
        if (sp.a[q] != q / sp.M || sp.b[q] != q % sp.M) return false;
    return true;
}

namespace {
constexpr int SNT = 256;
constexpr int RNT = 128;  // threads along x of the row kernels (grid y and z: the rows)
unsigned blocks(long long n) { return (unsigned)((n + SNT - 1) / SNT); }
}  // namespace

cudaError_t launch_spec_table(bool fp64, void *R3, long long Nr, const int L[3], const int *e, const double *u, int ne,
                              cudaStream_t st) {
    if (ne <= 0) return cudaSuccess;
    if (fp64)
        k_spec_scatter<double><<<blocks(ne), SNT, 0, st>>>((double *)R3, Nr, L[0], L[1], L[2], e, u, ne);
    else
        k_spec_scatter<float><<<blocks(ne), SNT, 0, st>>>((float *)R3, Nr, L[0], L[1], L[2], e, u, ne);
    return cudaGetLastError();
}

cudaError_t launch_spec_imag(bool fp64, const void *Z3, void *tab3, long long Nc, cudaStream_t st) {
    if (fp64)
        k_spec_imag<double><<<blocks(Nc), SNT, 0, st>>>((const double2 *)Z3, (double *)tab3, Nc);
    else
        k_spec_imag<float><<<blocks(Nc), SNT, 0, st>>>((const float2 *)Z3, (float *)tab3, Nc);
    return cudaGetLastError();
}

cudaError_t launch_adjspec_embed(bool fp64, const Grid &g, const int L[3], long long Nr, const SpecPairs &sp,
                                 const void *npad, const void *lC, const void *gab, void *R, cudaStream_t st) {
    const dim3 grid((unsigned)((L[0] + RNT - 1) / RNT), (unsigned)L[1], (unsigned)L[2]);
    if (fp64)
        k_adjspec_embed<double><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, sp, (const double *)npad,
                                                      (const double *)lC, (const double *)gab, (double *)R);
    else
        k_adjspec_embed<float><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, sp, (const float *)npad, (const float *)lC,
                                                     (const float *)gab, (float *)R);
    return cudaGetLastError();
}

cudaError_t launch_adjspec_multiply(bool fp64, const void *Z, const void *tab, void *W, long long Nc,
                                    const SpecPairs &sp, double scale, cudaStream_t st) {
    if (fp64)
        k_adjspec_multiply<double><<<blocks(Nc), SNT, 0, st>>>((const double2 *)Z, (const double *)tab,
                                                               (double2 *)W, Nc, sp, scale);
    else
        k_adjspec_multiply<float><<<blocks(Nc), SNT, 0, st>>>((const float2 *)Z, (const float *)tab, (float2 *)W,
                                                              Nc, sp, (float)scale);
    return cudaGetLastError();
}

cudaError_t launch_adjspec_combine(bool fp64, const Grid &g, const int L[3], long long Nr, const SpecPairs &sp,
                                   const void *R, const void *npad, const void *gab, void *ln, void *lg,
                                   cudaStream_t st) {
    const dim3 grid((unsigned)((g.nx + RNT - 1) / RNT), (unsigned)g.ny, (unsigned)g.nz);
    if (fp64)
        k_adjspec_combine<double><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, sp, (const double *)R,
                                                        (const double *)npad, (const double *)gab, (double *)ln,
                                                        (double *)lg);
    else
        k_adjspec_combine<float><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, sp, (const float *)R, (const float *)npad,
                                                       (const float *)gab, (float *)ln, (float *)lg);
    return cudaGetLastError();
}

cudaError_t launch_spec_real(bool fp64, const void *Z, void *tab, long long Nc, cudaStream_t st) {
    if (fp64)
        k_spec_real<double><<<blocks(Nc), SNT, 0, st>>>((const double2 *)Z, (double *)tab, Nc);
    else
        k_spec_real<float><<<blocks(Nc), SNT, 0, st>>>((const float2 *)Z, (float *)tab, Nc);
    return cudaGetLastError();
}

cudaError_t launch_spec_embed_n(bool fp64, const Grid &g, const int L[3], long long Nr, int M, const void *npad,
                                void *R, cudaStream_t st) {
    const dim3 grid((unsigned)((L[0] + RNT - 1) / RNT), (unsigned)L[1], (unsigned)L[2]);
    if (fp64)
        k_spec_embed_n<double><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, M, (const double *)npad, (double *)R);
    else
        k_spec_embed_n<float><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, M, (const float *)npad, (float *)R);
    return cudaGetLastError();
}

cudaError_t launch_spec_ball_mul(bool fp64, const void *Z, const void *btab, void *W, long long Nc, int M,
                                 double scale, cudaStream_t st) {
    if (fp64)
        k_spec_ball_mul<double><<<blocks(Nc), SNT, 0, st>>>((const double2 *)Z, (const double *)btab, (double2 *)W,
                                                            Nc, M, scale);
    else
        k_spec_ball_mul<float><<<blocks(Nc), SNT, 0, st>>>((const float2 *)Z, (const float *)btab, (float2 *)W, Nc,
                                                           M, (float)scale);
    return cudaGetLastError();
}

cudaError_t launch_spec_contact(bool fp64, const Grid &g, const int L[3], long long Nr, const ContactParams &cp,
                                const SpecPairs &sp, const void *npad, const void *nbar, void *gab, void *xi, void *G,
                                int *err, cudaStream_t st) {
    const dim3 grid((unsigned)((L[0] + RNT - 1) / RNT), (unsigned)L[1], (unsigned)L[2]);
#define LBE_SPEC_CONTACT(TT, MM)                                                                              \
    k_spec_contact<TT, MM><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, cp, sp, (const TT *)npad, (const TT *)nbar, \
                                                 (TT *)gab, (TT *)xi, (TT *)G, err)
#define LBE_SPEC_CONTACT_M(TT)                   \
    switch (sp.M) {                              \
        case 1: LBE_SPEC_CONTACT(TT, 1); break;  \
        case 2: LBE_SPEC_CONTACT(TT, 2); break;  \
        case 3: LBE_SPEC_CONTACT(TT, 3); break;  \
        case 4: LBE_SPEC_CONTACT(TT, 4); break;  \
        default: return cudaErrorInvalidValue;   \
    }
    if (fp64) {
        LBE_SPEC_CONTACT_M(double);
    } else {
        LBE_SPEC_CONTACT_M(float);
    }
#undef LBE_SPEC_CONTACT_M
#undef LBE_SPEC_CONTACT
    return cudaGetLastError();
}

cudaError_t launch_spec_multiply(bool fp64, const void *Z, const void *tab, void *W, long long Nc, const SpecPairs &sp,
                                 double scale, cudaStream_t st) {
    if (full_pairs(sp)) {
#define LBE_SPEC_MUL(TT, C2, MM)                                                                           \
    k_spec_multiply_m<TT, MM><<<blocks(Nc), SNT, 0, st>>>((const C2 *)Z, (const TT *)tab, (C2 *)W, Nc, sp, \
                                                          (TT)scale)
        if (fp64) {
            if (sp.M == 1) LBE_SPEC_MUL(double, double2, 1); else LBE_SPEC_MUL(double, double2, 2);
        } else {
            if (sp.M == 1) LBE_SPEC_MUL(float, float2, 1); else LBE_SPEC_MUL(float, float2, 2);
        }
#undef LBE_SPEC_MUL
        return cudaGetLastError();
    }
    if (fp64)
        k_spec_multiply<double><<<blocks(Nc), SNT, 0, st>>>((const double2 *)Z, (const double *)tab, (double2 *)W,
                                                            Nc, sp, scale);
    else
        k_spec_multiply<float><<<blocks(Nc), SNT, 0, st>>>((const float2 *)Z, (const float *)tab, (float2 *)W, Nc,
                                                           sp, (float)scale);
    return cudaGetLastError();
}

cudaError_t launch_spec_combine(bool fp64, const Grid &g, const int L[3], long long Nr, const void *R,
                                const void *npad, const void *gab, const SpecPairs &sp, void *Cout, void *Pout,
                                cudaStream_t st) {
    const dim3 grid((unsigned)((g.nx + RNT - 1) / RNT), (unsigned)g.ny, (unsigned)g.nz);
    if (full_pairs(sp)) {
#define LBE_SPEC_COMB(TT, MM)                                                                               \
    k_spec_combine_m<TT, MM><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, (const TT *)R, (const TT *)npad,      \
                                                   (const TT *)gab, sp, (TT *)Cout, (TT *)Pout)
        if (fp64) {
            if (sp.M == 1) LBE_SPEC_COMB(double, 1); else LBE_SPEC_COMB(double, 2);
        } else {
            if (sp.M == 1) LBE_SPEC_COMB(float, 1); else LBE_SPEC_COMB(float, 2);
        }
#undef LBE_SPEC_COMB
        return cudaGetLastError();
    }
    if (fp64)
        k_spec_combine<double><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, (const double *)R, (const double *)npad,
                                                     (const double *)gab, sp, (double *)Cout, (double *)Pout);
    else
        k_spec_combine<float><<<grid, RNT, 0, st>>>(g, L[0], L[1], Nr, (const float *)R, (const float *)npad,
                                                    (const float *)gab, sp, (float *)Cout, (float *)Pout);
    return cudaGetLastError();
}

}  // namespace lbe
