// C ABI of the Lattice Boltzmann-Enskog library (include/lbe.h): context,
// device memory, set-up, the time-step driver and the getters.  All compute
// runs in the kernels of lbe_kernels.cu and lbe_shell.cu on the context stream.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbe.h"
#include "lbe_device.cuh"
#include "lbe_launch.h"
#include "lbe_shell.cuh"

using namespace lbe;

namespace lbe {
cudaError_t noalloc_scratch(int device, double **out);
cudaError_t launch_mass_noalloc(int prec, int nx, int ny, int nz, const void *pop, const uint32_t *mask, int M,
                                const double *n0, double *scratch, int nblocks, cudaStream_t st);
long long noalloc_max_nodes();
int noalloc_blocks(long long N);
size_t noalloc_result_offset();
}  // namespace lbe

namespace {

thread_local std::string t_last_error;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct PairShell {
    int a, b, S;
    double coef;  // -kT sigma_ab^2 w_ab
    CUtensorMap map_n, map_gn;
};

}  // namespace

#ifndef LBE_SHELL_STREAMS
#define LBE_SHELL_STREAMS 2
#endif

struct lbe_ctx {
    lbe_config cfg{};
    Prec prec = Prec::F32;
    Grid g{};
    int M = 1;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbe_allocator alloc{};
    bool have_alloc = false;

    // species
    double sigma[MAXS] = {0}, tau[MAXS] = {0}, gbody[MAXS][3] = {{0}};
    bool species_set[MAXS] = {false};
    double n0[MAXS] = {0};

    // host copies
    std::vector<uint8_t> solid_h;

    // device buffers
    Buf pop[2];
    int cur = 0;
    Buf solid, mask, V, phi, amp, F;
    Buf npad, gab, gnpad, C;
    Buf flux_buf, flux_acc, flux_last;
    Buf err;
    Buf scratch64;  // FP64 scratch for getters: n [M][N] + J [M][3][N] (+ more)
    Buf partial, red_out;
    Buf res_rec;             // densities recorded by lbe_get_residual [M][N] (FP64)
    long long res_t0 = -1;   // step count of the record, -1: none

    // derived state
    bool geom_dirty = true, force_dirty = true, fields_dirty = true;
    std::vector<PairShell> pairs;
    ContactParams cparams{};
    BallRows brows{};
    int RB = 0;
    CUtensorMap contact_maps[MAXS];
    bool solid_links = false;  // some link can be blocked: a solid node or a closed axis
    int H = 0;

    // K3 method (lbe_set_shell_method); the spectral method's cuFFT plans and buffers
    int shell_method = LBE_SHELL_AUTO;
    bool spectral = false;
    SpectralShell *spec = nullptr;
    int specL[3] = {0, 0, 0};
    long long specNr = 0, specNc = 0;
    int specNS = 0;  // shells with a spectrum; the ball spectra follow them in specTab
    SpecPairs specPairs{};
    Buf specR, specZ, specW, specTab, specWork;
    // viscous Enskog force (enable_visc): shell tables of the pairs, tilde velocities, effective force
    ViscPairs vp{};
    Buf veoff, vehat, vut, Feff;
    // the discrete adjoint's spectral shell transpose, kept between calls until the pairs change
    SpectralShell *aspec = nullptr;
    int aL[3] = {0, 0, 0};
    long long aNr = 0, aNc = 0;
    SpecPairs asp{};
    Buf aR, aZ, aW, aTab, aWork;

    long long steps = 0;
    long long flux_count = 0;
    int flux_axis = -1, flux_plane = -1;
    long long launches = 0;
    long long steps_since_check = 0;
    std::string last_error;

    // second stream of the shell stage: the pair launches of odd species run there (created on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[LBE_NUM_STAGES];
    double stage_ms[LBE_NUM_STAGES] = {0};
    long long stage_launches[LBE_NUM_STAGES] = {0};
};

namespace {

lbe_status fail(lbe_ctx *c, lbe_status s, const std::string &msg) {
    t_last_error = msg;
    if (c) c->last_error = msg;
    return s;
}

lbe_status cuda_fail(lbe_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, LBE_ERR_CUDA, m);
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
    } while (0)

#define LAUNCH(call, where)                              \
    do {                                                 \
        cudaError_t _e = (call);                         \
        c->launches += 1;                                \
        if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
    } while (0)

lbe_status dev_alloc(lbe_ctx *c, Buf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return LBE_OK;
    if (b.p) {
        if (c->have_alloc)
            c->alloc.free(b.p, b.bytes, c->stream, c->alloc.user);
        else
            cudaFreeAsync(b.p, c->stream);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    void *p = nullptr;
    if (c->have_alloc) {
        p = c->alloc.alloc(bytes, c->stream, c->alloc.user);
        if (!p) return fail(c, LBE_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LBE_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = bytes;
    return LBE_OK;
}

void dev_free(lbe_ctx *c, Buf &b) {
    if (!b.p) return;
    if (c->have_alloc)
        c->alloc.free(b.p, b.bytes, c->stream, c->alloc.user);
    else
        cudaFreeAsync(b.p, c->stream);
    b.p = nullptr;
    b.bytes = 0;
}

#define TRY(x)                          \
    do {                                \
        lbe_status _s = (x);            \
        if (_s != LBE_OK) return _s;    \
    } while (0)

size_t real_bytes(const lbe_ctx *c) { return prec_fp64(c->prec) ? 8 : 4; }

cudaEvent_t pool_event(lbe_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets the kernel launches of a stage (count of them) with events when timing is on.
struct StageTimer {
    lbe_ctx *c;
    int stage;
    int count;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(lbe_ctx *c_, int st, int n = 1) : c(c_), stage(st), count(n) {
        if (c->timing) {
            a = pool_event(c);
            b = pool_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~StageTimer() {
        if (c->timing && a && b) {
            cudaEventRecord(b, c->stream);
            c->ev_pending[stage].push_back({a, b});
            c->stage_launches[stage] += count;
        }
    }
};

// Fold the pending event pairs into the totals (synchronises the stream).
void fold_stage_times(lbe_ctx *c) {
    cudaStreamSynchronize(c->stream);
    for (int s = 0; s < LBE_NUM_STAGES; ++s) {
        for (auto &pr : c->ev_pending[s]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) c->stage_ms[s] += ms;
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->ev_pending[s].clear();
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map over a padded field of the compute type, or (pair = true, FP32) over the interleaved
// (n_b, g_ab n_b) field as 8-byte elements.
lbe_status make_map(lbe_ctx *c, CUtensorMap *map, void *base, int bx, int by, bool pair = false) {
    auto enc = get_encode();
    if (!enc) return fail(c, LBE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const bool f64 = prec_fp64(c->prec);
    const bool e8 = f64 || pair;
    const size_t es = e8 ? 8 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)c->g.px, (cuuint64_t)c->g.py, (cuuint64_t)c->g.pz};
    cuuint64_t strides[2] = {(cuuint64_t)c->g.px * es, (cuuint64_t)c->g.px * c->g.py * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                       : (pair ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
    CUresult r = enc(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, LBE_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return LBE_OK;
}

const double kPi = 3.14159265358979323846;
const double kKT = 1.0 / 3.0;

// Shell weight w_sigma = 4 pi sigma / sum_{e in K_sigma} |e| (so that a linear
// density reproduces the continuum k^ integral).
double shell_weight(int S) {
    double sum = 0.0;
    for (int z = -S; z <= S; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z)) sum += std::sqrt((double)(x * x + y * y + z * z));
    return 4.0 * kPi * S / sum;
}

bool integer_diameter(double s, int *S) {
    double r = std::nearbyint(s);
    if (std::fabs(s - r) > 1e-12) return false;
    *S = (int)r;
    return true;
}

// Smallest n' >= n whose prime factors are 2, 3, 5 and 7 (sizes cuFFT transforms well).
int fft_size(int n) {
    for (int m = n;; ++m) {
        int r = m;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

// The row kernels of the spectral form take y and z from the grid's second and third dimensions.
bool spectral_shape_ok(const lbe_ctx *c, int Smax) {
    const Grid &g = c->g;
    const int ly = g.per[1] ? g.ny : fft_size(g.ny + Smax), lz = g.per[2] ? g.nz : fft_size(g.nz + Smax);
    return ly <= 65535 && lz <= 65535;
}

int shell_count(int S) {
    int k = 0;
    for (int z = -S; z <= S; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z)) ++k;
    return k;
}

// Cost rule of LBE_SHELL_AUTO, from measurements on GB300 (512x128x128 two-species channel, pair
// diameters 4, 5, 5, 6; 256^3 one-species well, diameter 6).  The spectral form replaces the contact
// kernel and the shell stencil; the stencil costs a fixed time per node and shell point, the spectral
// form a fixed time per grid point and pair.  Counting the contact kernel's time on the direct side,
// the two break even at a mean shell of about 280 (well) to 323 (channel) points per pair in FP32,
// scaled by the lattice over the grid, and about 100 in FP64, where the stencil is bound by the FP64
// rate.  The constants lean to the stencil.
bool spectral_cheaper(const lbe_ctx *c, bool f64, double stencil_factor = 1.0) {
    long long pts = 0;
    int Smax = 0;
    for (const auto &ps : c->pairs) {
        pts += shell_count(ps.S);
        Smax = std::max(Smax, ps.S);
    }
    const Grid &g = c->g;
    const int n3[3] = {g.nx, g.ny, g.nz};
    double Nr = 1.0;
    for (int k = 0; k < 3; ++k) Nr *= g.per[k] ? n3[k] : fft_size(n3[k] + Smax);
    const double even = (f64 ? 110.0 : 320.0) / stencil_factor;
    return spectral_shape_ok(c, Smax) && (double)pts * (double)g.N > even * (double)c->pairs.size() * Nr;
}

// The pairs as the spectral kernels see them (shell index into the table of distinct shells), the
// distinct shells, and the grid: the lattice along periodic axes, at least Smax zero planes beyond it
// along closed axes.
void spectral_pairs(const lbe_ctx *c, SpecPairs *sp, std::vector<int> *shells, int L[3]) {
    *sp = SpecPairs{};
    shells->clear();
    int Smax = 0;
    sp->M = c->M;
    sp->npairs = (int)c->pairs.size();
    for (int q = 0; q < sp->npairs; ++q) {
        const PairShell &ps = c->pairs[q];
        Smax = std::max(Smax, ps.S);
        int s = 0;
        while (s < (int)shells->size() && (*shells)[s] != ps.S) ++s;
        if (s == (int)shells->size()) shells->push_back(ps.S);
        sp->a[q] = ps.a;
        sp->b[q] = ps.b;
        sp->s[q] = s;
        sp->half_coef[q] = 0.5 * ps.coef;
    }
    const Grid &g = c->g;
    const int n3[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; ++k) L[k] = g.per[k] ? n3[k] : fft_size(n3[k] + Smax);
}

// Spectra of the shell kernels, t_c = Im FFT(kappa_c) with kappa_c(-e mod L) = e_c / |e|, into tab
// [nS][3][Nc]; with balls, then the ball spectra Re FFT(beta_b), beta_b(-d mod L) = 1 / |B_b| on the ball
// rows of the contact kernel (even, so the spectrum is real), into tab [M][Nc] after them.  R and Z are
// scratch of three fields; `spec` has the three-field forward plan 2.
lbe_status spectral_tables(lbe_ctx *c, SpectralShell *spec, const int L[3], long long Nr, long long Nc,
                           const std::vector<int> &shells, bool balls, void *tab, void *R, void *Z) {
    const bool f64 = prec_fp64(c->prec);
    const size_t rb = real_bytes(c);
    const int M = c->M, nS = (int)shells.size();
    void *const specR = R, *const specZ = Z, *const specTab = tab;
    // shell spectra t_c = Im FFT(kappa_c), kappa_c(-e mod L) = e_c / |e|; ball spectra Re FFT(beta_b),
    // beta_b(-d mod L) = 1 / |B_b| on the ball rows of the contact kernel (even, so the spectrum is real)
    const int ntab = nS + (balls ? M : 0);
    std::vector<std::vector<int>> eh(ntab);
    std::vector<std::vector<double>> uh(ntab);
    std::vector<Buf> ed(ntab), ud(ntab);
    lbe_status st = LBE_OK;
    for (int s = 0; s < ntab && st == LBE_OK; ++s) {
        if (s < nS) {
            const int S = shells[s];
            for (int z = -S; z <= S; ++z)
                for (int y = -S; y <= S; ++y)
                    for (int x = -S; x <= S; ++x)
                        if (in_shell(S, x, y, z)) {
                            const double len = std::sqrt((double)(x * x + y * y + z * z));
                            eh[s].insert(eh[s].end(), {x, y, z});
                            uh[s].insert(uh[s].end(), {x / len, y / len, z / len});
                        }
        } else {
            const int b = s - nS;
            const BallRows &br = c->brows;
            const double w = 1.0 / br.count[b];
            for (int dz = -4; dz <= 4; ++dz)
                for (int k = br.first[b][dz + 4]; k < br.first[b][dz + 5]; ++k)
                    for (int dx = -br.a[b][k]; dx <= br.a[b][k]; ++dx) {
                        eh[s].insert(eh[s].end(), {dx, (int)br.dy[b][k], dz});
                        uh[s].insert(uh[s].end(), {w, 0.0, 0.0});
                    }
        }
        const int ne = (int)(eh[s].size() / 3);
        if ((st = dev_alloc(c, ed[s], sizeof(int) * eh[s].size())) != LBE_OK) break;
        if ((st = dev_alloc(c, ud[s], sizeof(double) * uh[s].size())) != LBE_OK) break;
        cudaError_t e = cudaMemcpyAsync(ed[s].p, eh[s].data(), sizeof(int) * eh[s].size(), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ud[s].p, uh[s].data(), sizeof(double) * uh[s].size(), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(specR, 0, rb * 3 * Nr, c->stream);
        if (e == cudaSuccess)
            e = launch_spec_table(f64, specR, Nr, L, (const int *)ed[s].p, (const double *)ud[s].p, ne, c->stream);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "spectral shell tables");
            break;
        }
        c->launches += 1;
        if (spectral_forward(spec, 2, specR, specZ) != 0) {
            st = fail(c, LBE_ERR_CUDA, "spectral shell tables: cuFFT forward transform failed");
            break;
        }
        if (s < nS)
            e = launch_spec_imag(f64, specZ, (char *)specTab + rb * 3 * (size_t)s * Nc, Nc, c->stream);
        else
            e = launch_spec_real(f64, specZ, (char *)specTab + rb * (size_t)(3 * nS + s - nS) * Nc, Nc,
                                 c->stream);
        c->launches += 1;
        if (e != cudaSuccess) st = cuda_fail(c, e, "spectral shell tables");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);  // the host lists must outlive their copies
    for (int s = 0; s < ntab; ++s) {
        dev_free(c, ed[s]);
        dev_free(c, ud[s]);
    }
    if (st != LBE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "spectral shell tables");
    return LBE_OK;
}

// Plans, buffers and shell and ball spectra of the spectral K2 + K3 (lbe_spectral.cu) for the current pairs.
lbe_status spectral_setup(lbe_ctx *c) {
    const bool f64 = prec_fp64(c->prec);
    const size_t rb = real_bytes(c);
    SpecPairs sp;
    std::vector<int> shells;
    int L[3];
    spectral_pairs(c, &sp, &shells, L);
    int Smax = 0;
    for (int S : shells) Smax = std::max(Smax, S);
    if (!spectral_shape_ok(c, Smax))
        return fail(c, LBE_ERR_UNSUPPORTED, "spectral shell force: an axis of the grid is longer than 65535");
    const int M = c->M, nfwd = M + sp.npairs, ninv = 3 * sp.npairs + 3 * M, nS = (int)shells.size();
    spectral_destroy(c->spec);
    c->spec = nullptr;
    std::string why;
    size_t ws = 0;
    if (spectral_create(&c->spec, f64, L, M, sp.npairs, ninv, &ws, &why) != 0)
        return fail(c, LBE_ERR_UNSUPPORTED, "spectral shell force: " + why);
    const long long Nr = (long long)L[0] * L[1] * L[2], Nc = (long long)(L[0] / 2 + 1) * L[1] * L[2];
    // real fields: the densities, the pairs' g n and the ball averages, later the ninv force fields
    TRY(dev_alloc(c, c->specR, rb * (size_t)std::max(ninv, std::max(nfwd + M, 3)) * Nr));
    TRY(dev_alloc(c, c->specZ, 2 * rb * (size_t)std::max(nfwd, 3) * Nc));
    TRY(dev_alloc(c, c->specW, 2 * rb * (size_t)ninv * Nc));
    // tables: t_c of every shell [nS][3][Nc], then the ball spectrum of every species [M][Nc]
    TRY(dev_alloc(c, c->specTab, rb * (size_t)(3 * nS + M) * Nc));
    TRY(dev_alloc(c, c->specWork, ws));
    if (spectral_bind(c->spec, c->specWork.p, c->stream) != 0)
        return fail(c, LBE_ERR_CUDA, "spectral shell force: binding the cuFFT work area failed");
    for (int k = 0; k < 3; ++k) c->specL[k] = L[k];
    c->specNr = Nr;
    c->specNc = Nc;
    c->specPairs = sp;
    c->specNS = nS;
    return spectral_tables(c, c->spec, L, Nr, Nc, shells, true, c->specTab.p, c->specR.p, c->specZ.p);
}

// K2 and K3 in spectral form: g_ab [M][M][N] (xi2, xi3 into xibase for the adjoint) and C [M][3][N]
// (P [npairs][3][N] into Pbase for the adjoint).  Real fields in specR: the densities [M], the pairs'
// g n [npairs], the ball averages [M]; then the force fields [ninv].
lbe_status spectral_force(lbe_ctx *c, void *Pbase, void *xibase) {
    const bool f64 = prec_fp64(c->prec);
    const size_t rb = real_bytes(c);
    const int M = c->M, np = c->specPairs.npairs;
    const long long Nr = c->specNr, Nc = c->specNc;
    char *R = (char *)c->specR.p, *Z = (char *)c->specZ.p, *W = (char *)c->specW.p;
    const double scale = 1.0 / (double)Nr;
    {
        StageTimer t(c, LBE_STAGE_CONTACT);
        LAUNCH(launch_spec_embed_n(f64, c->g, c->specL, Nr, M, c->npad.p, R, c->stream), "spectral embed");
        if (spectral_forward(c->spec, 0, R, Z) != 0)
            return fail(c, LBE_ERR_CUDA, "spectral contact values: cuFFT forward transform failed");
        LAUNCH(launch_spec_ball_mul(f64, Z, (const char *)c->specTab.p + rb * 3 * (size_t)c->specNS * Nc, W, Nc, M,
                                    scale, c->stream),
               "spectral ball average");
        char *nbar = R + rb * (size_t)(M + np) * Nr;
        if (spectral_inverse(c->spec, 4, W, nbar) != 0)
            return fail(c, LBE_ERR_CUDA, "spectral contact values: cuFFT inverse transform failed");
        LAUNCH(launch_spec_contact(f64, c->g, c->specL, Nr, c->cparams, c->specPairs, c->npad.p, nbar, c->gab.p,
                                   xibase, R + rb * (size_t)M * Nr, (int *)c->err.p, c->stream),
               "spectral contact values");
    }
    StageTimer t(c, LBE_STAGE_SHELL);
    if (spectral_forward(c->spec, 3, R + rb * (size_t)M * Nr, Z + 2 * rb * (size_t)M * Nc) != 0)
        return fail(c, LBE_ERR_CUDA, "spectral shell force: cuFFT forward transform failed");
    LAUNCH(launch_spec_multiply(f64, Z, c->specTab.p, W, Nc, c->specPairs, scale, c->stream), "spectral multiply");
    if (spectral_inverse(c->spec, 1, W, R) != 0)
        return fail(c, LBE_ERR_CUDA, "spectral shell force: cuFFT inverse transform failed");
    LAUNCH(launch_spec_combine(f64, c->g, c->specL, Nr, R, c->npad.p, c->gab.p, c->specPairs, c->C.p, Pbase,
                               c->stream),
           "spectral combine");
    return LBE_OK;
}

// Shell tables of the viscous force (the pairs' shells, offsets and unit vectors in FP64) and its
// fields: the tilde velocities and the effective force F + C^visc / n.
lbe_status visc_setup(lbe_ctx *c) {
    const size_t rb = real_bytes(c);
    const long long N = c->g.N;
    ViscPairs vp{};
    vp.M = c->M;
    vp.npairs = (int)c->pairs.size();
    std::vector<int> eo;
    std::vector<double> eh;
    for (int q = 0; q < vp.npairs; ++q) {
        const PairShell &ps = c->pairs[q];
        vp.a[q] = ps.a;
        vp.b[q] = ps.b;
        vp.first[q] = (int)(eo.size() / 3);
        const int S = ps.S;
        for (int z = -S; z <= S; ++z)
            for (int y = -S; y <= S; ++y)
                for (int x = -S; x <= S; ++x)
                    if (in_shell(S, x, y, z)) {
                        const double len = std::sqrt((double)(x * x + y * y + z * z));
                        eo.insert(eo.end(), {x, y, z});
                        eh.insert(eh.end(), {x / len, y / len, z / len});
                    }
        vp.count[q] = (int)(eo.size() / 3) - vp.first[q];
        vp.pre[q] = 2.0 * (double)S * (double)S * std::sqrt(kKT / kPi) * shell_weight(S);
    }
    c->vp = vp;
    TRY(dev_alloc(c, c->veoff, sizeof(int) * std::max<size_t>(eo.size(), 3)));
    TRY(dev_alloc(c, c->vehat, sizeof(double) * std::max<size_t>(eh.size(), 3)));
    TRY(dev_alloc(c, c->vut, rb * 3 * (size_t)c->M * N));
    TRY(dev_alloc(c, c->Feff, rb * 3 * (size_t)c->M * N));
    if (!eo.empty()) {
        CK(cudaMemcpyAsync(c->veoff.p, eo.data(), sizeof(int) * eo.size(), cudaMemcpyHostToDevice, c->stream),
           "copy viscous shell offsets");
        CK(cudaMemcpyAsync(c->vehat.p, eh.data(), sizeof(double) * eh.size(), cudaMemcpyHostToDevice, c->stream),
           "copy viscous shell vectors");
        CK(cudaStreamSynchronize(c->stream), "stream sync");  // the host tables die here
    }
    return LBE_OK;
}

// Set up everything that depends on the species, geometry and potentials:
// halo width, padded fields, tensor maps, ball tables, force field.
lbe_status prepare(lbe_ctx *c) {
    for (int a = 0; a < c->M; ++a)
        if (!c->species_set[a]) return fail(c, LBE_ERR_STATE, "species " + std::to_string(a) + " not set");
    const bool f64 = prec_fp64(c->prec);
    if (c->fields_dirty) {
        // pair shells
        c->pairs.clear();
        int H = 1;
        bool direct_ok = true;  // every pair diameter has a compiled direct stencil
        for (int a = 0; a < c->M; ++a)
            for (int b = 0; b < c->M; ++b) {
                double sab = 0.5 * (c->sigma[a] + c->sigma[b]);
                if (!(sab > 0.0)) continue;
                int S = 0;
                if (!integer_diameter(sab, &S) || S > 16)
                    return fail(c, LBE_ERR_UNSUPPORTED,
                                "pair diameter " + std::to_string(sab) + " is not an integer of at most 16");
                if (!shell_supported(f64, S)) direct_ok = false;
                PairShell ps{};
                ps.a = a;
                ps.b = b;
                ps.S = S;
                ps.coef = -kKT * sab * sab * shell_weight(S);
                c->pairs.push_back(ps);
                H = std::max(H, S);
            }
        // K3 method: the direct stencil, or the spectral form for FP64 (bound by the FP64 rate) and
        // for diameters without a compiled stencil
        c->spectral = false;
        if (!c->pairs.empty()) {
            if (c->shell_method == LBE_SHELL_DIRECT && !direct_ok)
                return fail(c, LBE_ERR_UNSUPPORTED,
                            "a pair diameter has no compiled direct shell stencil (the spectral method takes it)");
            c->spectral = c->shell_method == LBE_SHELL_SPECTRAL ||
                          (c->shell_method == LBE_SHELL_AUTO && (!direct_ok || spectral_cheaper(c, f64)));
        }
        // ball radii
        ContactParams cp{};
        cp.M = c->M;
        int RB = 0;
        for (int b = 0; b < c->M; ++b) {
            double R = 0.5 * c->sigma[b];
            int Ri = (int)std::floor(R);
            RB = std::max(RB, Ri);
            cp.sigma[b] = c->sigma[b];
            cp.xi2c[b] = kPi / 6.0 * c->sigma[b] * c->sigma[b];
            cp.xi3c[b] = kPi / 6.0 * c->sigma[b] * c->sigma[b] * c->sigma[b];
        }
        if (RB > 4) return fail(c, LBE_ERR_UNSUPPORTED, "ball radius sigma/2 above 4 lattice units");
        H = std::max(H, RB);
        c->RB = RB;
        c->H = H;
        Grid &g = c->g;
        g.H = H;
        g.px = (g.nx + 2 * H + 7) / 8 * 8;
        g.py = g.ny + 2 * H;
        g.pz = g.nz + 2 * H;
        g.P = (long long)g.px * g.py * g.pz;
        // averaging ball |d| <= sigma_b/2 as rows (dy, dz) of half-width a along x, grouped by dz
        BallRows br{};
        for (int b = 0; b < c->M; ++b) {
            const double R = 0.5 * c->sigma[b], R2 = R * R;
            const int Ri = (int)std::floor(R);
            int nr = 0, cnt = 0;
            for (int dz = -4; dz <= 4; ++dz) {
                br.first[b][dz + 4] = (short)nr;
                if (dz < -Ri || dz > Ri) continue;
                for (int dy = -Ri; dy <= Ri; ++dy) {
                    const double rem = R2 - (double)(dy * dy + dz * dz);
                    if (rem < 0.0) continue;
                    int a = 0;
                    while ((double)((a + 1) * (a + 1)) <= rem) ++a;
                    br.dy[b][nr] = (signed char)dy;
                    br.a[b][nr] = (signed char)a;
                    cnt += 2 * a + 1;
                    ++nr;
                }
            }
            br.first[b][9] = (short)nr;
            br.count[b] = cnt;
        }
        c->brows = br;
        for (int a = 0; a < c->M; ++a)
            for (int b = 0; b < c->M; ++b) {
                double sa = c->sigma[a], sb = c->sigma[b];
                cp.s_ab[a][b] = (sa + sb > 0.0) ? sa * sb / (sa + sb) : 0.0;
            }
        c->cparams = cp;
        const size_t rb = real_bytes(c);
        TRY(dev_alloc(c, c->npad, rb * c->M * g.P));
        // g_ab n_b of every ordered pair for the direct shell stencil: FP32 stores the interleaved pair
        // (n_b, g_ab n_b), 8 bytes per node (the spectral form keeps its own grid fields instead)
        const size_t gnb = (f64 ? rb : 2 * rb) * c->M * c->M * g.P;
        if (!c->spectral) TRY(dev_alloc(c, c->gnpad, gnb));
        TRY(dev_alloc(c, c->gab, rb * c->M * c->M * g.N));
        TRY(dev_alloc(c, c->C, rb * c->M * 3 * g.N));
        CK(cudaMemsetAsync(c->npad.p, 0, rb * c->M * g.P, c->stream), "memset npad");
        if (!c->spectral) CK(cudaMemsetAsync(c->gnpad.p, 0, gnb, c->stream), "memset gnpad");
        CK(cudaMemsetAsync(c->C.p, 0, rb * c->M * 3 * g.N, c->stream), "memset C");
        for (auto &ps : c->pairs) {
            if (c->spectral) break;
            char *nb = (char *)c->npad.p + rb * ps.b * g.P;
            char *gn = (char *)c->gnpad.p + (f64 ? rb : 2 * rb) * (ps.a * c->M + ps.b) * g.P;
            int bx = 0, by = 0;
            shell_box(f64, ps.S, &bx, &by);
            if (f64) TRY(make_map(c, &ps.map_n, nb, bx, by));
            TRY(make_map(c, &ps.map_gn, gn, bx, by, !f64));
        }
        {
            int bx = 0, by = 0;
            contact_box(f64, c->M, c->RB, &bx, &by);
            for (int b = 0; b < c->M; ++b)
                TRY(make_map(c, &c->contact_maps[b], (char *)c->npad.p + rb * b * g.P, bx, by));
        }
        spectral_destroy(c->aspec);  // the adjoint's transpose plans and tables follow the pairs
        c->aspec = nullptr;
        if (c->spectral) TRY(spectral_setup(c));
        if (c->cfg.enable_visc) TRY(visc_setup(c));
        c->fields_dirty = false;
    }
    if (c->force_dirty) {
        const size_t rb = real_bytes(c);
        TRY(dev_alloc(c, c->F, rb * c->M * 3 * c->g.N));
        for (int a = 0; a < c->M; ++a) {
            LAUNCH(launch_force_field(c->prec, c->g, (const double *)c->V.p + (long long)a * c->g.N,
                                      (const double *)c->phi.p, (const double *)c->amp.p, c->gbody[a],
                                      (char *)c->F.p + rb * 3 * a * c->g.N, c->stream),
                   "force field");
        }
        c->force_dirty = false;
    }
    return LBE_OK;
}

StepParams step_params(const lbe_ctx *c) {
    StepParams sp{};
    sp.M = c->M;
    sp.consistent = c->cfg.consistent_moments ? 1 : 0;
    sp.flux_axis = c->flux_plane >= 0 ? c->flux_axis : -1;
    sp.flux_plane = c->flux_plane;
    sp.scheme = c->cfg.scheme;
    const bool euler = c->cfg.scheme == LBE_SD_EU || c->cfg.scheme == LBE_DD_EU;
    for (int a = 0; a < c->M; ++a) {
        double omega = 1.0 / (c->tau[a] - 0.5);
        // omega_eff = 1/tau, also the Euler rate
        species_const_set(sp.sp[a], omega / (1.0 + 0.5 * omega), euler ? 1.0 : 1.0 / (1.0 + 0.5 * omega), c->n0[a]);
    }
    return sp;
}

// K1 -> K2 -> K3 for the populations pop (default: the current state); fills
// npad, gab, gnpad, C.  With Pbase, the shell kernels also store P of every
// pair into Pbase [npairs][3][N], and with xibase the contact kernel stores
// xi2, xi3 into xibase [2][N] (both for the adjoint).
lbe_status force_stage_core(lbe_ctx *c, const void *pop, void *Pbase, void *xibase) {
    const bool f64 = prec_fp64(c->prec);
    const size_t rb = real_bytes(c);
    if (!pop) pop = c->pop[c->cur].p;
    {
        StageTimer t(c, LBE_STAGE_DENSITY);
        LAUNCH(launch_density(c->prec, c->g, pop, (const uint32_t *)c->mask.p, c->solid_links, c->M, c->n0,
                              c->npad.p, (int *)c->err.p, c->stream),
               "density kernel");
    }
    if (c->pairs.empty()) return LBE_OK;  // ideal gas: C stays zero
    if (c->spectral) return spectral_force(c, Pbase, xibase);
    {
        StageTimer t(c, LBE_STAGE_CONTACT);
        ContactLaunch L{};
        L.grid = &c->g;
        L.maps = c->contact_maps;
        L.cp = &c->cparams;
        L.br = &c->brows;
        L.RB = c->RB;
        L.gab = c->gab.p;
        L.gnpad = c->gnpad.p;
        L.xi = xibase;
        L.err = (int *)c->err.p;
        LAUNCH(launch_contact_tma(f64, L, c->stream), "contact kernel");
    }
    // Two or more species: the pairs of odd species a run on a second stream beside those of even a. Each
    // species' C still takes its pairs in order on one stream, and the launches of the two streams fill
    // each other's last partial wave (one thread block per SM at a time).
    const bool two = LBE_SHELL_STREAMS == 2 && c->M >= 2;
    if (two && !c->side) {
        CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "create the shell stage's second stream");
        CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "create fork event");
        CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "create join event");
    }
    std::vector<int> first(c->M, 1);
    StageTimer shell_timer(c, LBE_STAGE_SHELL, (int)c->pairs.size());
    // joins the second stream back on an early return too, so that later work on the main stream
    // never runs beside a pair launch already queued there
    struct SideJoin {
        lbe_ctx *c;
        bool pending;
        ~SideJoin() {
            if (pending) {
                cudaEventRecord(c->ev_join, c->side);
                cudaStreamWaitEvent(c->stream, c->ev_join, 0);
            }
        }
    } side_join{c, false};
    if (two) {
        CK(cudaEventRecord(c->ev_fork, c->stream), "record fork");
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork the shell stage");
        side_join.pending = true;
    }
    for (size_t q = 0; q < c->pairs.size(); ++q) {
        const PairShell &ps = c->pairs[q];
        ShellLaunch L{};
        L.grid = &c->g;
        L.map_n = &ps.map_n;
        L.map_gn = &ps.map_gn;
        L.npad_a = (const char *)c->npad.p + rb * ps.a * c->g.P;
        L.g_ab = (const char *)c->gab.p + rb * (ps.a * c->M + ps.b) * c->g.N;
        L.Cout = (char *)c->C.p + rb * 3 * ps.a * c->g.N;
        L.Pout = Pbase ? (char *)Pbase + rb * 3 * q * c->g.N : nullptr;
        L.coef = ps.coef;
        L.accumulate = first[ps.a] ? 0 : 1;
        L.err = (int *)c->err.p;
        first[ps.a] = 0;
        LAUNCH(launch_shell_force(f64, ps.S, L, two && (ps.a & 1) ? c->side : c->stream), "shell force kernel");
    }
    if (two) {
        side_join.pending = false;
        CK(cudaEventRecord(c->ev_join, c->side), "record join");
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join the shell stage");
    }
    for (int a = 0; a < c->M; ++a)
        if (first[a]) CK(cudaMemsetAsync((char *)c->C.p + rb * 3 * a * c->g.N, 0, rb * 3 * c->g.N, c->stream),
                         "memset C");
    return LBE_OK;
}

// The force field the collide and the getters use: F, or F + C^visc / n with the viscous force on.
const void *force_field(const lbe_ctx *c) { return c->cfg.enable_visc && !c->pairs.empty() ? c->Feff.p : c->F.p; }

lbe_status force_stage(lbe_ctx *c, const void *pop = nullptr, void *Pbase = nullptr, void *xibase = nullptr) {
    if (!pop) pop = c->pop[c->cur].p;
    TRY(force_stage_core(c, pop, Pbase, xibase));
    if (c->cfg.enable_visc && !c->pairs.empty()) {
        StageTimer t(c, LBE_STAGE_SHELL);
        LAUNCH(launch_visc(c->prec, c->g, pop, (const uint32_t *)c->mask.p, c->npad.p, c->gab.p, c->F.p,
                           step_params(c), c->vp, (const int *)c->veoff.p, (const double *)c->vehat.p, c->vut.p,
                           c->Feff.p, c->stream),
               "viscous force");
        c->launches += 1;  // two kernels
    }
    return LBE_OK;
}

int plane_size(const lbe_ctx *c) {
    const Grid &g = c->g;
    return c->flux_axis == 0 ? g.ny * g.nz : (c->flux_axis == 1 ? g.nx * g.nz : g.nx * g.ny);
}

lbe_status check_error_word(lbe_ctx *c) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error word");
    CK(cudaStreamSynchronize(c->stream), "stream sync");
    if (e & ERR_TMA_WAIT)
        return fail(c, LBE_ERR_CUDA, "a bounded TMA wait gave up: the copy it waited for did not complete");
    if (e & ERR_DENSITY) return fail(c, LBE_ERR_DIVERGED, "negative or non-finite density");
    if (e & ERR_PACKING) return fail(c, LBE_ERR_DIVERGED, "local packing xi3 >= 1 or non-finite contact value");
    return LBE_OK;
}

lbe_status ready(lbe_ctx *c) {
    if (!c) return fail(nullptr, LBE_ERR_INVALID_ARG, "null context");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    return LBE_OK;
}

// n [M][N] and J [M][3][N] (FP64, device scratch) of the current state.
lbe_status state_moments(lbe_ctx *c, double **n, double **J) {
    TRY(prepare(c));
    TRY(force_stage(c));
    const long long N = c->g.N;
    TRY(dev_alloc(c, c->scratch64, sizeof(double) * ((size_t)c->M * 4 * N + 4 * N)));
    *n = (double *)c->scratch64.p;
    *J = *n + (long long)c->M * N;
    StepParams sp = step_params(c);
    if (sp.scheme == LBE_DD_TR) {
        LAUNCH(launch_moments(c->prec, c->g, c->pop[c->cur].p, (const uint32_t *)c->mask.p, c->C.p, force_field(c), sp, *n,
                              *J, c->stream),
               "moments kernel");
    } else {
        LAUNCH(launch_moments_ablation(c->prec, c->g, c->pop[c->cur].p, (const uint32_t *)c->mask.p, c->C.p, c->F.p,
                                       sp, *n, *J, c->stream),
               "ablation moments kernel");
    }
    return LBE_OK;
}

// One step of the current populations (K1-K3, K4 of the configured scheme, and K5 when psize > 0).
lbe_status step_once(lbe_ctx *c, const StepParams &sp, int psize) {
    TRY(force_stage(c));
    {
        StageTimer tm(c, LBE_STAGE_COLLIDE);
        if (sp.scheme == LBE_DD_TR) {
            LAUNCH(launch_collide(c->prec, c->g, c->pop[c->cur].p, c->pop[1 - c->cur].p, (const uint32_t *)c->mask.p,
                                  c->solid_links, c->C.p, force_field(c), sp, (double *)c->flux_buf.p, c->stream),
                   "collide kernel");
        } else {
            LAUNCH(launch_collide_ablation(c->prec, c->g, c->pop[c->cur].p, c->pop[1 - c->cur].p,
                                           (const uint32_t *)c->mask.p, c->solid_links, c->C.p, c->F.p, sp,
                                           (double *)c->flux_buf.p, c->stream),
                   "ablation collide kernel");
        }
    }
    c->cur = 1 - c->cur;
    if (psize > 0) {
        StageTimer tm(c, LBE_STAGE_FLUX);
        LAUNCH(launch_flux_reduce(c->M, psize, (const double *)c->flux_buf.p, (double *)c->flux_acc.p,
                                  (double *)c->flux_last.p, c->stream),
               "flux reduction");
        c->flux_count += 1;
    }
    c->steps += 1;
    return LBE_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------
extern "C" {

const char *lbe_status_string(lbe_status s) {
    switch (s) {
        case LBE_OK: return "ok";
        case LBE_ERR_INVALID_ARG: return "invalid argument";
        case LBE_ERR_UNSUPPORTED: return "unsupported";
        case LBE_ERR_OOM: return "out of device memory";
        case LBE_ERR_CUDA: return "CUDA error";
        case LBE_ERR_DIVERGED: return "diverged";
        case LBE_ERR_TIMEOUT: return "timeout";
        case LBE_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char *lbe_last_error(lbe_ctx *ctx) {
    (void)ctx;
    return t_last_error.c_str();
}

lbe_status lbe_create(const lbe_config *cfg, const lbe_allocator *allocator, void *cuda_stream, lbe_ctx **out) {
    lbe_ctx *c = nullptr;
    if (!cfg || !out) return fail(nullptr, LBE_ERR_INVALID_ARG, "null config or output pointer");
    *out = nullptr;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return fail(nullptr, LBE_ERR_INVALID_ARG, "lattice sizes must be >= 1");
    if ((long long)cfg->nx * cfg->ny * cfg->nz > (1ll << 31) - 1)
        return fail(nullptr, LBE_ERR_INVALID_ARG, "lattice larger than 2^31 - 1 nodes");
    if (cfg->nspecies < 1 || cfg->nspecies > MAXS) return fail(nullptr, LBE_ERR_INVALID_ARG, "nspecies must be 1..4");
    if (cfg->precision < LBE_FP64 || cfg->precision > LBE_FP16_SHIFTED)
        return fail(nullptr, LBE_ERR_INVALID_ARG, "unknown precision");
    if (cfg->scheme < LBE_DD_TR || cfg->scheme > LBE_DD_EU) return fail(nullptr, LBE_ERR_INVALID_ARG, "unknown scheme");
    if (cfg->scheme != LBE_DD_TR) {
        const Prec pr = cfg->precision == LBE_FP64 ? Prec::F64 : (cfg->precision == LBE_FP32 ? Prec::F32 : Prec::BF16);
        if (!ablation_supported(pr, cfg->nspecies))
            return fail(nullptr, LBE_ERR_UNSUPPORTED,
                        "the SD-TR, SD-EU and DD-EU ablations run on FP64 or FP32 populations with one or two species");
        if (cfg->consistent_moments)
            return fail(nullptr, LBE_ERR_INVALID_ARG, "consistent_moments applies to the DD-TR scheme only");
    }
    if (cfg->enable_visc && cfg->scheme != LBE_DD_TR)
        return fail(nullptr, LBE_ERR_UNSUPPORTED, "the viscous Enskog force belongs to the DD-TR scheme");
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(nullptr, LBE_ERR_INVALID_ARG, "allocator needs both alloc and free");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, LBE_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return fail(nullptr, LBE_ERR_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(nullptr, LBE_ERR_CUDA,
                    "this library is built for sm_103a only; device is sm_" + std::to_string(prop.major) +
                        std::to_string(prop.minor));

    c = new (std::nothrow) lbe_ctx();
    if (!c) return fail(nullptr, LBE_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->prec = (Prec)cfg->precision;
    c->device = dev;
    c->stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        c->alloc = *allocator;
        c->have_alloc = true;
    }
    c->M = cfg->nspecies;
    Grid &g = c->g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = cfg->nz;
    for (int k = 0; k < 3; ++k) g.per[k] = cfg->periodic[k] ? 1 : 0;
    g.N = (long long)g.nx * g.ny * g.nz;
    for (int a = 0; a < MAXS; ++a) c->tau[a] = 1.0;

    const size_t pb = (size_t)prec_bytes(c->prec) * c->M * 2 * Q * g.N;
    lbe_status s;
    if ((s = dev_alloc(c, c->pop[0], pb)) != LBE_OK || (s = dev_alloc(c, c->pop[1], pb)) != LBE_OK ||
        (s = dev_alloc(c, c->solid, g.N)) != LBE_OK || (s = dev_alloc(c, c->mask, 4 * g.N)) != LBE_OK ||
        (s = dev_alloc(c, c->V, 8 * c->M * g.N)) != LBE_OK || (s = dev_alloc(c, c->phi, 8 * g.N)) != LBE_OK ||
        (s = dev_alloc(c, c->amp, 8 * g.N)) != LBE_OK || (s = dev_alloc(c, c->err, 64)) != LBE_OK ||
        (s = dev_alloc(c, c->flux_acc, 8 * MAXS)) != LBE_OK || (s = dev_alloc(c, c->flux_last, 8 * MAXS)) != LBE_OK ||
        (s = dev_alloc(c, c->partial, 16 * 1024)) != LBE_OK || (s = dev_alloc(c, c->red_out, 64)) != LBE_OK) {
        lbe_destroy(c);
        return s;
    }
    cudaMemsetAsync(c->pop[0].p, 0, pb, c->stream);
    cudaMemsetAsync(c->pop[1].p, 0, pb, c->stream);
    cudaMemsetAsync(c->solid.p, 0, g.N, c->stream);
    cudaMemsetAsync(c->V.p, 0, 8 * c->M * g.N, c->stream);
    cudaMemsetAsync(c->phi.p, 0, 8 * g.N, c->stream);
    cudaMemsetAsync(c->amp.p, 0, 8 * g.N, c->stream);
    cudaMemsetAsync(c->err.p, 0, 64, c->stream);
    cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream);
    cudaMemsetAsync(c->flux_last.p, 0, 8 * MAXS, c->stream);
    c->solid_h.assign(g.N, 0);
    c->solid_links = !(g.per[0] && g.per[1] && g.per[2]);
    e = launch_link_mask(g, (const uint8_t *)c->solid.p, (uint32_t *)c->mask.p, c->stream);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "create");
        lbe_destroy(c);
        return LBE_ERR_CUDA;
    }
    *out = c;
    return LBE_OK;
}

void lbe_destroy(lbe_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    fold_stage_times(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
        cudaEventDestroy(c->ev_fork);
        cudaEventDestroy(c->ev_join);
    }
    Buf *all[] = {&c->pop[0], &c->pop[1], &c->solid, &c->mask, &c->V, &c->phi, &c->amp, &c->F,
                  &c->npad, &c->gab, &c->gnpad, &c->C, &c->flux_buf, &c->flux_acc,
                  &c->flux_last, &c->err, &c->scratch64, &c->partial, &c->red_out, &c->res_rec,
                  &c->specR, &c->specZ, &c->specW, &c->specTab, &c->specWork,
                  &c->aR, &c->aZ, &c->aW, &c->aTab, &c->aWork, &c->veoff, &c->vehat, &c->vut, &c->Feff};
    spectral_destroy(c->spec);
    c->spec = nullptr;
    spectral_destroy(c->aspec);
    c->aspec = nullptr;
    for (Buf *b : all) dev_free(c, *b);
    cudaStreamSynchronize(c->stream);
    delete c;
}

lbe_status lbe_set_shell_method(lbe_ctx *c, int method) {
    TRY(ready(c));
    if (method < LBE_SHELL_AUTO || method > LBE_SHELL_SPECTRAL)
        return fail(c, LBE_ERR_INVALID_ARG, "shell method must be LBE_SHELL_AUTO, _DIRECT or _SPECTRAL");
    if (method == LBE_SHELL_SPECTRAL) {
        std::string why;
        if (!spectral_available(&why)) return fail(c, LBE_ERR_UNSUPPORTED, why);
    }
    c->shell_method = method;
    c->fields_dirty = true;
    return LBE_OK;
}

lbe_status lbe_get_shell_method(lbe_ctx *c, int *method) {
    TRY(ready(c));
    if (!method) return fail(c, LBE_ERR_INVALID_ARG, "null method");
    TRY(prepare(c));
    *method = c->spectral ? LBE_SHELL_SPECTRAL : LBE_SHELL_DIRECT;
    return LBE_OK;
}

lbe_status lbe_set_geometry(lbe_ctx *c, const uint8_t *solid) {
    TRY(ready(c));
    if (!solid) return fail(c, LBE_ERR_INVALID_ARG, "null solid mask");
    const long long N = c->g.N;
    bool any = false;
    for (long long i = 0; i < N; ++i) {
        c->solid_h[i] = solid[i] ? 1 : 0;
        any = any || solid[i];
    }
    c->solid_links = any || !(c->g.per[0] && c->g.per[1] && c->g.per[2]);
    CK(cudaMemcpyAsync(c->solid.p, c->solid_h.data(), N, cudaMemcpyHostToDevice, c->stream), "copy solid");
    LAUNCH(launch_link_mask(c->g, (const uint8_t *)c->solid.p, (uint32_t *)c->mask.p, c->stream), "link mask");
    CK(cudaStreamSynchronize(c->stream), "stream sync");
    return LBE_OK;
}

lbe_status lbe_set_species(lbe_ctx *c, int s, double sigma, double mass, double tau) {
    TRY(ready(c));
    if (s < 0 || s >= c->M) return fail(c, LBE_ERR_INVALID_ARG, "species index out of range");
    if (!(sigma >= 0.0) || !std::isfinite(sigma)) return fail(c, LBE_ERR_INVALID_ARG, "sigma must be >= 0");
    if (mass != 1.0) return fail(c, LBE_ERR_UNSUPPORTED, "species share the common mass m = 1");
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBE_ERR_INVALID_ARG, "tau must be > 1/2");
    if (sigma > 16.0) return fail(c, LBE_ERR_UNSUPPORTED, "sigma above 16 lattice units");
    c->sigma[s] = sigma;
    c->tau[s] = tau;
    c->species_set[s] = true;
    c->fields_dirty = true;
    return LBE_OK;
}

lbe_status lbe_set_potential(lbe_ctx *c, int s, const double *V) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !V) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null potential");
    CK(cudaMemcpyAsync((double *)c->V.p + (long long)s * c->g.N, V, 8 * c->g.N, cudaMemcpyHostToDevice, c->stream),
       "copy potential");
    CK(cudaStreamSynchronize(c->stream), "stream sync");
    c->force_dirty = true;
    return LBE_OK;
}

lbe_status lbe_set_wall_potential(lbe_ctx *c, const double *phi, const double *amp) {
    TRY(ready(c));
    if (!phi || !amp) return fail(c, LBE_ERR_INVALID_ARG, "null wall potential array");
    CK(cudaMemcpyAsync(c->phi.p, phi, 8 * c->g.N, cudaMemcpyHostToDevice, c->stream), "copy phi");
    CK(cudaMemcpyAsync(c->amp.p, amp, 8 * c->g.N, cudaMemcpyHostToDevice, c->stream), "copy amp");
    CK(cudaStreamSynchronize(c->stream), "stream sync");
    c->force_dirty = true;
    return LBE_OK;
}

lbe_status lbe_set_body_force(lbe_ctx *c, int s, const double gb[3]) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !gb) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null force");
    for (int k = 0; k < 3; ++k) c->gbody[s][k] = gb[k];
    c->force_dirty = true;
    return LBE_OK;
}

static void reset_counters(lbe_ctx *c) {
    c->steps = 0;
    c->res_t0 = -1;
    c->flux_count = 0;
    cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream);
    cudaMemsetAsync(c->flux_last.p, 0, 8 * MAXS, c->stream);
}

lbe_status lbe_init_density(lbe_ctx *c, int s, const double *n) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !n) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null density");
    const long long N = c->g.N;
    double sum = 0.0;
    long long cnt = 0;
    for (long long i = 0; i < N; ++i) {
        if (!(n[i] >= 0.0) || !std::isfinite(n[i])) return fail(c, LBE_ERR_INVALID_ARG, "density must be finite and >= 0");
        if (!c->solid_h[i]) {
            sum += n[i];
            ++cnt;
        }
    }
    c->n0[s] = cnt > 0 ? sum / cnt : 0.0;
    if (c->prec == Prec::BF16 || c->prec == Prec::F16) {
        if (!(c->n0[s] > 0.0)) return fail(c, LBE_ERR_INVALID_ARG, "shifted storage needs a positive mean density");
    }
    Buf tmp;
    TRY(dev_alloc(c, tmp, 8 * N));
    cudaError_t e = cudaMemcpyAsync(tmp.p, n, 8 * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_rest_state(c->prec, c->g, (const uint32_t *)c->mask.p, (const double *)tmp.p, c->pop[c->cur].p, s,
                              c->n0[s], c->stream);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "init density");
    reset_counters(c);
    return LBE_OK;
}

lbe_status lbe_init_density_quasipressure(lbe_ctx *c, const double *n) {
    TRY(ready(c));
    if (!n) return fail(c, LBE_ERR_INVALID_ARG, "null density");
    for (int a = 0; a < c->M; ++a)
        if (!c->species_set[a]) return fail(c, LBE_ERR_STATE, "species " + std::to_string(a) + " not set");
    const long long N = c->g.N;
    const int M = c->M;
    std::vector<double> nh((size_t)M * N);
    for (int a = 0; a < M; ++a) {
        double sum = 0.0;
        long long cnt = 0;
        for (long long i = 0; i < N; ++i) {
            const double v = n[(long long)a * N + i];
            if (!(v >= 0.0) || !std::isfinite(v)) return fail(c, LBE_ERR_INVALID_ARG, "density must be finite and >= 0");
            nh[(size_t)a * N + i] = c->solid_h[i] ? 0.0 : v;
            if (!c->solid_h[i]) {
                sum += v;
                ++cnt;
            }
        }
        c->n0[a] = cnt > 0 ? sum / cnt : 0.0;
        if ((c->prec == Prec::BF16 || c->prec == Prec::F16) && !(c->n0[a] > 0.0))
            return fail(c, LBE_ERR_INVALID_ARG, "shifted storage needs a positive mean density");
    }
    Buf nd, pid;
    auto done = [&](lbe_status st) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, nd);
        dev_free(c, pid);
        return st;
    };
    lbe_status st = dev_alloc(c, nd, 8 * (size_t)M * N);
    if (st == LBE_OK) st = dev_alloc(c, pid, 8 * (size_t)M * N);
    if (st != LBE_OK) return done(st);
    cudaError_t e = cudaMemcpyAsync(nd.p, nh.data(), 8 * (size_t)M * N, cudaMemcpyHostToDevice, c->stream);
    // the rest state of n, its force stage (C^mf of n), then Pi and the rest state with g from Pi
    for (int a = 0; a < M && e == cudaSuccess; ++a, ++c->launches)
        e = launch_rest_state(c->prec, c->g, (const uint32_t *)c->mask.p, (const double *)nd.p + (long long)a * N,
                              c->pop[c->cur].p, a, c->n0[a], c->stream);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "init quasi-pressure"));
    if ((st = prepare(c)) != LBE_OK || (st = force_stage(c)) != LBE_OK) return done(st);
    e = launch_quasipressure(prec_fp64(c->prec), c->g, M, (const double *)nd.p, c->C.p, c->F.p, (double *)pid.p,
                             c->stream);
    c->launches += 4;
    for (int a = 0; a < M && e == cudaSuccess; ++a, ++c->launches)
        e = launch_rest_state(c->prec, c->g, (const uint32_t *)c->mask.p, (const double *)nd.p + (long long)a * N,
                              c->pop[c->cur].p, a, c->n0[a], c->stream, (const double *)pid.p + (long long)a * N);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return done(cuda_fail(c, e, "init quasi-pressure"));
    reset_counters(c);
    return done(LBE_OK);
}

lbe_status lbe_step(lbe_ctx *c, int nsteps) {
    TRY(ready(c));
    if (nsteps < 0) return fail(c, LBE_ERR_INVALID_ARG, "nsteps must be >= 0");
    TRY(prepare(c));
    StepParams sp = step_params(c);
    const int psize = c->flux_plane >= 0 ? plane_size(c) : 0;
    if (psize > 0) TRY(dev_alloc(c, c->flux_buf, 8 * (size_t)c->M * psize));
    for (int t = 0; t < nsteps; ++t) {
        TRY(step_once(c, sp, psize));
        c->steps_since_check += 1;
        if (c->cfg.check_every > 0 && c->steps_since_check >= c->cfg.check_every) {
            c->steps_since_check = 0;
            TRY(check_error_word(c));
        }
    }
    return LBE_OK;
}

lbe_status lbe_get_density(lbe_ctx *c, int s, double *out) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    double *n, *J;
    TRY(state_moments(c, &n, &J));
    CK(cudaMemcpyAsync(out, n + (long long)s * c->g.N, 8 * c->g.N, cudaMemcpyDeviceToHost, c->stream), "copy density");
    return check_error_word(c);
}

lbe_status lbe_get_momentum(lbe_ctx *c, int s, double *out) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    double *n, *J;
    TRY(state_moments(c, &n, &J));
    CK(cudaMemcpyAsync(out, J + (long long)s * 3 * c->g.N, 24 * c->g.N, cudaMemcpyDeviceToHost, c->stream),
       "copy momentum");
    return check_error_word(c);
}

lbe_status lbe_get_velocity(lbe_ctx *c, int s, double *out) {
    TRY(ready(c));
    if (s < -1 || s >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    const long long N = c->g.N;
    double *dn, *dJ;
    TRY(state_moments(c, &dn, &dJ));
    double *du = dJ + (long long)c->M * 3 * N;  // scratch holds n, J and 4 more fields
    LAUNCH(launch_velocity(c->M, N, s, dn, dJ, du, nullptr, c->stream), "velocity kernel");
    CK(cudaMemcpyAsync(out, du, 24 * N, cudaMemcpyDeviceToHost, c->stream), "copy velocity");
    return check_error_word(c);
}

lbe_status lbe_get_divergence(lbe_ctx *c, int s, double *out) {
    TRY(ready(c));
    if (s < -1 || s >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    const long long N = c->g.N;
    double *dn, *dJ;
    TRY(state_moments(c, &dn, &dJ));
    double *du = dJ + (long long)c->M * 3 * N;  // scratch holds n, J and 4 more fields
    double *dd = du + 3 * N;
    LAUNCH(launch_velocity(c->M, N, s, dn, dJ, du, nullptr, c->stream), "velocity kernel");
    LAUNCH(launch_divergence(c->g, du, dd, c->stream), "divergence kernel");
    CK(cudaMemcpyAsync(out, dd, 8 * N, cudaMemcpyDeviceToHost, c->stream), "copy divergence");
    return check_error_word(c);
}

lbe_status lbe_get_force(lbe_ctx *c, int s, double *out) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    TRY(prepare(c));
    TRY(force_stage(c));
    const long long N = c->g.N;
    TRY(dev_alloc(c, c->scratch64, sizeof(double) * (size_t)c->M * 4 * N));
    LAUNCH(launch_to_f64(prec_fp64(c->prec), (const char *)c->C.p + real_bytes(c) * 3 * s * N, 3 * N,
                         (double *)c->scratch64.p, c->stream),
           "convert force");
    CK(cudaMemcpyAsync(out, c->scratch64.p, 24 * N, cudaMemcpyDeviceToHost, c->stream), "copy force");
    return check_error_word(c);
}

lbe_status lbe_get_contact(lbe_ctx *c, int a, int b, double *out) {
    TRY(ready(c));
    if (a < 0 || a >= c->M || b < 0 || b >= c->M || !out) return fail(c, LBE_ERR_INVALID_ARG, "bad pair or null output");
    TRY(prepare(c));
    TRY(force_stage(c));
    const long long N = c->g.N;
    if (c->pairs.empty()) {
        for (long long i = 0; i < N; ++i) out[i] = 1.0;
        return check_error_word(c);
    }
    TRY(dev_alloc(c, c->scratch64, sizeof(double) * (size_t)c->M * 4 * N));
    LAUNCH(launch_to_f64(prec_fp64(c->prec), (const char *)c->gab.p + real_bytes(c) * (a * c->M + b) * N, N,
                         (double *)c->scratch64.p, c->stream),
           "convert contact");
    CK(cudaMemcpyAsync(out, c->scratch64.p, 8 * N, cudaMemcpyDeviceToHost, c->stream), "copy contact");
    return check_error_word(c);
}

lbe_status lbe_set_flux_plane(lbe_ctx *c, int axis, int plane) {
    TRY(ready(c));
    if (axis < 0 || axis > 2) return fail(c, LBE_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
    const int n = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
    if (plane >= n) return fail(c, LBE_ERR_INVALID_ARG, "plane index out of range");
    c->flux_axis = axis;
    c->flux_plane = plane < 0 ? -1 : plane;
    c->flux_count = 0;
    CK(cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream), "memset flux");
    CK(cudaMemsetAsync(c->flux_last.p, 0, 8 * MAXS, c->stream), "memset flux");
    return LBE_OK;
}

lbe_status lbe_reset_flux_average(lbe_ctx *c) {
    TRY(ready(c));
    c->flux_count = 0;
    CK(cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream), "memset flux");
    return LBE_OK;
}

lbe_status lbe_get_flux(lbe_ctx *c, int s, double *inst, double *avg) {
    TRY(ready(c));
    if (s < -1 || s >= c->M) return fail(c, LBE_ERR_INVALID_ARG, "bad species index");
    if (c->flux_plane < 0) return fail(c, LBE_ERR_STATE, "no flux plane set");
    double acc[MAXS], last[MAXS];
    CK(cudaMemcpyAsync(acc, c->flux_acc.p, 8 * MAXS, cudaMemcpyDeviceToHost, c->stream), "copy flux");
    CK(cudaMemcpyAsync(last, c->flux_last.p, 8 * MAXS, cudaMemcpyDeviceToHost, c->stream), "copy flux");
    TRY(check_error_word(c));
    double A = 0.0, L = 0.0;
    for (int a = 0; a < c->M; ++a)
        if (s < 0 || a == s) {
            A += acc[a];
            L += last[a];
        }
    if (inst) *inst = L;
    if (avg) *avg = c->flux_count > 0 ? A / (double)c->flux_count : 0.0;
    return LBE_OK;
}

lbe_status lbe_get_totals(lbe_ctx *c, double *mass, double *momentum, double *max_u) {
    TRY(ready(c));
    double *n, *J;
    TRY(state_moments(c, &n, &J));
    const long long N = c->g.N;
    double r[2];
    for (int a = 0; a < c->M && mass; ++a) {
        LAUNCH(launch_reduce(n + (long long)a * N, N, (double *)c->partial.p, 1024, (double *)c->red_out.p, c->stream),
               "reduce mass");
        CK(cudaMemcpyAsync(r, c->red_out.p, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
        mass[a] = r[0];
    }
    if (momentum) {
        for (int k = 0; k < 3; ++k) {
            double tot = 0.0;
            for (int a = 0; a < c->M; ++a) {
                LAUNCH(launch_reduce(J + ((long long)a * 3 + k) * N, N, (double *)c->partial.p, 1024,
                                     (double *)c->red_out.p, c->stream),
                       "reduce momentum");
                CK(cudaMemcpyAsync(r, c->red_out.p, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
                CK(cudaStreamSynchronize(c->stream), "sync");
                tot += r[0];
            }
            momentum[k] = tot;
        }
    }
    if (max_u) {
        double *sp = J + (long long)c->M * 3 * N;
        LAUNCH(launch_velocity(c->M, N, -1, n, J, nullptr, sp, c->stream), "speed kernel");
        LAUNCH(launch_reduce(sp, N, (double *)c->partial.p, 1024, (double *)c->red_out.p, c->stream), "reduce speed");
        CK(cudaMemcpyAsync(r, c->red_out.p, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
        *max_u = r[1];
    }
    return check_error_word(c);
}

lbe_status lbe_get_populations(lbe_ctx *c, int s, double *f, double *gq) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !f || !gq) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null output");
    const long long N = c->g.N;
    Buf tmp;
    TRY(dev_alloc(c, tmp, 2 * 8 * Q * N));
    double *df = (double *)tmp.p, *dg = df + Q * N;
    cudaError_t e = launch_stream_out(c->prec, c->g, (const uint32_t *)c->mask.p, c->pop[c->cur].p, s, c->n0[s], df,
                                      dg, c->stream);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, df, 8 * Q * N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gq, dg, 8 * Q * N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "get populations");
    return LBE_OK;
}

lbe_status lbe_set_populations(lbe_ctx *c, int s, const double *f, const double *gq) {
    TRY(ready(c));
    if (s < 0 || s >= c->M || !f || !gq) return fail(c, LBE_ERR_INVALID_ARG, "bad species index or null input");
    const long long N = c->g.N;
    if (c->prec == Prec::BF16 || c->prec == Prec::F16) {
        // reference density: fluid-node mean of the zeroth moment
        double sum = 0.0;
        long long cnt = 0;
        for (long long i = 0; i < N; ++i)
            if (!c->solid_h[i]) {
                double nn = 0.0;
                for (int p = 0; p < Q; ++p) nn += f[(long long)p * N + i];
                sum += nn;
                ++cnt;
            }
        c->n0[s] = cnt > 0 ? sum / cnt : 0.0;
        if (!(c->n0[s] > 0.0)) return fail(c, LBE_ERR_INVALID_ARG, "shifted storage needs a positive mean density");
    }
    Buf tmp;
    TRY(dev_alloc(c, tmp, 2 * 8 * Q * N));
    double *df = (double *)tmp.p, *dg = df + Q * N;
    cudaError_t e = cudaMemcpyAsync(df, f, 8 * Q * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dg, gq, 8 * Q * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_unstream(c->prec, c->g, (const uint32_t *)c->mask.p, df, dg, c->pop[c->cur].p, s, c->n0[s],
                            c->stream);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "set populations");
    reset_counters(c);
    return LBE_OK;
}

lbe_status lbe_get_step_count(lbe_ctx *c, long long *steps) {
    if (!c || !steps) return fail(c, LBE_ERR_INVALID_ARG, "null argument");
    *steps = c->steps;
    return LBE_OK;
}

namespace {
// Layout of a saved state: this header, then the populations as stored.
struct StateHeader {
    char magic[8];
    int32_t version, nx, ny, nz, M, prec, flux_axis, flux_plane;
    int64_t steps, flux_count;
    double n0[MAXS], flux_acc[MAXS], flux_last[MAXS];
    uint64_t pop_bytes;
};
const char kStateMagic[8] = {'L', 'B', 'E', 'S', 'T', 'A', 'T', 'E'};
}  // namespace

lbe_status lbe_save_state(lbe_ctx *c, void *host_buf, size_t *bytes) {
    TRY(ready(c));
    if (!bytes) return fail(c, LBE_ERR_INVALID_ARG, "null size pointer");
    const size_t pop_bytes = (size_t)prec_bytes(c->prec) * c->M * 2 * Q * c->g.N;
    const size_t total = sizeof(StateHeader) + pop_bytes;
    if (!host_buf) {
        *bytes = total;
        return LBE_OK;
    }
    if (*bytes < total) return fail(c, LBE_ERR_INVALID_ARG, "state buffer of " + std::to_string(*bytes) +
                                                             " bytes, the state needs " + std::to_string(total));
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = 1;
    h.nx = c->g.nx;
    h.ny = c->g.ny;
    h.nz = c->g.nz;
    h.M = c->M;
    h.prec = (int32_t)c->prec;
    h.flux_axis = c->flux_axis;
    h.flux_plane = c->flux_plane;
    h.steps = c->steps;
    h.flux_count = c->flux_count;
    for (int a = 0; a < MAXS; ++a) h.n0[a] = c->n0[a];
    h.pop_bytes = pop_bytes;
    CK(cudaMemcpyAsync(h.flux_acc, c->flux_acc.p, 8 * MAXS, cudaMemcpyDeviceToHost, c->stream), "copy flux");
    CK(cudaMemcpyAsync(h.flux_last, c->flux_last.p, 8 * MAXS, cudaMemcpyDeviceToHost, c->stream), "copy flux");
    CK(cudaMemcpyAsync((char *)host_buf + sizeof(StateHeader), c->pop[c->cur].p, pop_bytes, cudaMemcpyDeviceToHost,
                       c->stream),
       "copy populations");
    CK(cudaStreamSynchronize(c->stream), "sync");
    std::memcpy(host_buf, &h, sizeof(h));
    *bytes = total;
    return LBE_OK;
}

lbe_status lbe_load_state(lbe_ctx *c, const void *host_buf, size_t bytes) {
    TRY(ready(c));
    if (!host_buf || bytes < sizeof(StateHeader)) return fail(c, LBE_ERR_INVALID_ARG, "no state in the buffer");
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    const size_t pop_bytes = (size_t)prec_bytes(c->prec) * c->M * 2 * Q * c->g.N;
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1)
        return fail(c, LBE_ERR_INVALID_ARG, "the buffer does not hold a saved state");
    if (h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz || h.M != c->M || h.prec != (int32_t)c->prec ||
        h.pop_bytes != pop_bytes || bytes < sizeof(StateHeader) + pop_bytes)
        return fail(c, LBE_ERR_INVALID_ARG, "the saved state has another lattice size, species count or precision");
    if (h.flux_plane >= 0) {
        const int extent = h.flux_axis == 0 ? c->g.nx : (h.flux_axis == 1 ? c->g.ny : c->g.nz);
        if (h.flux_axis < 0 || h.flux_axis > 2 || h.flux_plane >= extent)
            return fail(c, LBE_ERR_INVALID_ARG, "the saved flux plane is out of range");
    }
    CK(cudaMemcpyAsync(c->pop[c->cur].p, (const char *)host_buf + sizeof(StateHeader), pop_bytes,
                       cudaMemcpyHostToDevice, c->stream),
       "copy populations");
    CK(cudaMemcpyAsync(c->flux_acc.p, h.flux_acc, 8 * MAXS, cudaMemcpyHostToDevice, c->stream), "copy flux");
    CK(cudaMemcpyAsync(c->flux_last.p, h.flux_last, 8 * MAXS, cudaMemcpyHostToDevice, c->stream), "copy flux");
    CK(cudaStreamSynchronize(c->stream), "sync");
    for (int a = 0; a < MAXS; ++a) c->n0[a] = h.n0[a];
    c->steps = h.steps;
    c->flux_count = h.flux_count;
    c->flux_axis = h.flux_axis;
    c->flux_plane = h.flux_plane;
    c->res_t0 = -1;
    if (c->flux_plane >= 0) TRY(dev_alloc(c, c->flux_buf, 8 * (size_t)c->M * plane_size(c)));
    return LBE_OK;
}

lbe_status lbe_get_residual(lbe_ctx *c, double *res) {
    TRY(ready(c));
    if (!res) return fail(c, LBE_ERR_INVALID_ARG, "null output");
    const long long N = c->g.N;
    double *n, *J;
    TRY(state_moments(c, &n, &J));
    TRY(dev_alloc(c, c->res_rec, 8 * (size_t)c->M * N));
    const bool have = c->res_t0 >= 0 && c->steps > c->res_t0;
    InvN0 inv{};
    for (int a = 0; a < c->M; ++a) {
        const double n0 = c->n0[a] > 0.0 ? c->n0[a] : 1.0;
        inv.v[a] = have ? 1.0 / ((double)(c->steps - c->res_t0) * n0) : 0.0;
    }
    double *out = J + (long long)c->M * 3 * N;  // free FP64 scratch of N values
    LAUNCH(launch_residual(c->M, N, inv, n, (double *)c->res_rec.p, out, c->stream), "residual kernel");
    double r[2] = {-1.0, -1.0};
    if (have) {
        LAUNCH(launch_reduce(out, N, (double *)c->partial.p, 1024, (double *)c->red_out.p, c->stream),
               "reduce residual");
        CK(cudaMemcpyAsync(r, c->red_out.p, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
    }
    TRY(check_error_word(c));
    *res = have ? r[1] : -1.0;
    c->res_t0 = c->steps;
    return LBE_OK;
}

lbe_status lbe_get_link_mask(lbe_ctx *c, uint32_t *out) {
    TRY(ready(c));
    if (!out) return fail(c, LBE_ERR_INVALID_ARG, "null output");
    CK(cudaMemcpyAsync(out, c->mask.p, 4 * c->g.N, cudaMemcpyDeviceToHost, c->stream), "copy mask");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return LBE_OK;
}

lbe_status lbe_shell(double sigma, int *e, int cap, int *count) {
    if (!count) return fail(nullptr, LBE_ERR_INVALID_ARG, "null count");
    int S = 0;
    if (!integer_diameter(sigma, &S) || S < 0 || S > 16)
        return fail(nullptr, LBE_ERR_UNSUPPORTED, "shells are tabulated for integer diameters 0..16");
    int k = 0;
    for (int z = -S; z <= S && S > 0; ++z)
        for (int y = -S; y <= S; ++y)
            for (int x = -S; x <= S; ++x)
                if (in_shell(S, x, y, z)) {
                    if (e && k < cap) {
                        e[3 * k] = x;
                        e[3 * k + 1] = y;
                        e[3 * k + 2] = z;
                    }
                    ++k;
                }
    *count = k;
    return LBE_OK;
}

lbe_status lbe_adjoint_flux_gradient(lbe_ctx *c, int T, int K, int axis, int plane, double *dPhi_damp,
                                     double dPhi_dg[3], double *Phi) {
    TRY(ready(c));
    if (T < 1 || K < 1) return fail(c, LBE_ERR_INVALID_ARG, "nsteps and ckpt_every must be >= 1");
    if (axis < 0 || axis > 2) return fail(c, LBE_ERR_INVALID_ARG, "axis must be 0, 1 or 2");
    const int extent = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
    if (plane < 0 || plane >= extent) return fail(c, LBE_ERR_INVALID_ARG, "plane index out of range");
    if (!(c->prec == Prec::F32 || c->prec == Prec::F64))
        return fail(c, LBE_ERR_UNSUPPORTED, "the adjoint runs on FP64 or FP32 populations only");
    if (c->cfg.scheme != LBE_DD_TR) return fail(c, LBE_ERR_UNSUPPORTED, "the adjoint is that of the DD-TR scheme");
    if (c->cfg.enable_visc)
        return fail(c, LBE_ERR_UNSUPPORTED, "the adjoint does not transpose the viscous Enskog force");
    TRY(prepare(c));
    const bool f64 = prec_fp64(c->prec);
    // K3 transposed: the stencil tiles, or the spectral form (the same sums as correlations with the
    // forward kernel).  The stencil transposes read a 2-vector per component and shell point, about 2.6
    // times the forward stencil's shared-memory work (measured on GB300), so the automatic choice
    // weighs the stencil side by that factor.
    bool adj_direct_ok = true;
    int adj_smax = 0;
    for (const auto &ps : c->pairs) {
        adj_direct_ok = adj_direct_ok && shell_supported(f64, ps.S);
        adj_smax = std::max(adj_smax, ps.S);
    }
    bool adj_spectral = false;
    if (!c->pairs.empty()) {
        std::string why;
        const bool can_spectral = spectral_available(&why) && spectral_shape_ok(c, adj_smax);
        if (c->shell_method == LBE_SHELL_SPECTRAL)
            adj_spectral = true;
        else if (c->shell_method == LBE_SHELL_AUTO)
            adj_spectral = can_spectral && (!adj_direct_ok || spectral_cheaper(c, f64, 2.6));
        if (adj_spectral && !can_spectral)
            return fail(c, LBE_ERR_UNSUPPORTED, "the spectral shell transpose is not available: " + why);
        if (!adj_spectral && !adj_direct_ok)
            return fail(c, LBE_ERR_UNSUPPORTED, "the shell transpose has no compiled stencil for pair diameter " +
                                                    std::to_string(adj_smax));
    }
    const size_t rb = real_bytes(c);
    const long long N = c->g.N, P = c->g.P;
    const int M = c->M;
    const size_t pop_bytes = (size_t)prec_bytes(c->prec) * M * 2 * Q * N;
    const int nseg = (T + K - 1) / K;
    const int kseg = std::min(K, T);
    const long long steps_before = c->steps;
    const int old_axis = c->flux_axis, old_plane = c->flux_plane;

    // Device memory: checkpoints ck[s] (state at step s*K), the states 1..K-1 of the segment being
    // reversed (seg[k]), and per segment step the fields of its force stage (slot[k]): npad [M][P],
    // gab [M][M][N], C [M][3][N], xi2 and xi3 [2][N], P [npairs][3][N].
    const int npairs = (int)c->pairs.size();
    const size_t sl_npad = 0, sl_gab = sl_npad + rb * M * P,
                 sl_C = sl_gab + rb * M * M * N, sl_xi = sl_C + rb * M * 3 * N, sl_P = sl_xi + rb * 2 * N,
                 slot_bytes = sl_P + rb * 3 * (size_t)std::max(npairs, 1) * N;
    std::vector<Buf> ck(nseg), seg(kseg), slot(kseg);
    Buf lYf[2], lYg[2], lnd[2], lC, lF, lg, Lpad, gLpad, lnbar, lmom, outA, red;
    auto release = [&]() {
        for (auto &b : ck) dev_free(c, b);
        for (auto &b : seg) dev_free(c, b);
        for (auto &b : slot) dev_free(c, b);
        Buf *all[] = {&lYf[0], &lYf[1], &lYg[0], &lYg[1], &lnd[0], &lnd[1], &lC, &lF, &lg, &Lpad, &gLpad,
                      &lnbar, &lmom, &outA, &red};
        for (Buf *b : all) dev_free(c, *b);
    };
    auto alloc = [&](Buf &b, size_t bytes, bool zero) -> lbe_status {
        lbe_status st = dev_alloc(c, b, bytes);
        if (st != LBE_OK) return st;
        if (zero && cudaMemsetAsync(b.p, 0, bytes, c->stream) != cudaSuccess)
            return fail(c, LBE_ERR_CUDA, "memset of an adjoint buffer failed");
        return LBE_OK;
    };
#define ATRY(x)                   \
    do {                          \
        lbe_status _s = (x);      \
        if (_s != LBE_OK) {       \
            release();            \
            return _s;            \
        }                         \
    } while (0)
    for (auto &b : ck) ATRY(alloc(b, pop_bytes, false));
    for (int k = 1; k < kseg; ++k) ATRY(alloc(seg[k], pop_bytes, false));
    for (auto &b : slot) ATRY(alloc(b, slot_bytes, false));
    for (int k = 0; k < 2; ++k) {
        ATRY(alloc(lYf[k], rb * M * Q * N, true));
        ATRY(alloc(lYg[k], rb * M * Q * N, true));
        ATRY(alloc(lnd[k], rb * M * N, true));
    }
    ATRY(alloc(lC, rb * M * 3 * N, true));
    ATRY(alloc(lF, rb * M * 3 * N, true));
    ATRY(alloc(lg, rb * M * M * N, true));
    if (!adj_spectral) {
        ATRY(alloc(Lpad, (f64 ? rb : 2 * rb) * 3 * P, true));  // FP32: interleaved (Lambda_c, g Lambda_c)
        if (f64) ATRY(alloc(gLpad, rb * 3 * P, true));
    }
    ATRY(alloc(lnbar, rb * M * P, true));
    ATRY(alloc(lmom, rb * M * 5 * N, false));
    ATRY(alloc(outA, 8 * N, false));
    ATRY(alloc(red, 8 * N, false));

    // tensor maps of the padded adjoint ball averages (box of the contact kernel)
    std::vector<CUtensorMap> ballmaps(MAXS);
    {
        int bx = 0, by = 0;
        contact_box(f64, M, c->RB, &bx, &by);
        for (int b = 0; b < M; ++b) ATRY(make_map(c, &ballmaps[b], (char *)lnbar.p + rb * b * P, bx, by));
    }
    // the spectral transpose: grid fields lambda [M][3] and g lambda [npairs][3], spectra TQ [npairs]
    // and TP [M] (lbe_spectral.cu); plans, buffers and shell spectra stay in the context
    if (adj_spectral && !c->aspec) {
        std::vector<int> shells;
        spectral_pairs(c, &c->asp, &shells, c->aL);
        const int nf = 3 * M + 3 * npairs, ni = npairs + M;
        const int batch[3] = {nf, ni, 3};
        const bool fwd[3] = {true, false, true};
        std::string why;
        size_t ws = 0;
        SpectralShell *sp_new = nullptr;
        if (spectral_create_plans(&sp_new, f64, c->aL, 3, batch, fwd, &ws, &why) != 0) {
            release();
            return fail(c, LBE_ERR_UNSUPPORTED, "spectral shell transpose: " + why);
        }
        c->aspec = sp_new;
        c->aNr = (long long)c->aL[0] * c->aL[1] * c->aL[2];
        c->aNc = (long long)(c->aL[0] / 2 + 1) * c->aL[1] * c->aL[2];
        lbe_status st = LBE_OK;
        if (st == LBE_OK) st = dev_alloc(c, c->aR, rb * (size_t)std::max(nf, 3) * c->aNr);
        if (st == LBE_OK) st = dev_alloc(c, c->aZ, 2 * rb * (size_t)std::max(nf, 3) * c->aNc);
        if (st == LBE_OK) st = dev_alloc(c, c->aW, 2 * rb * (size_t)ni * c->aNc);
        if (st == LBE_OK) st = dev_alloc(c, c->aTab, rb * 3 * shells.size() * c->aNc);
        if (st == LBE_OK) st = dev_alloc(c, c->aWork, ws);
        if (st == LBE_OK && spectral_bind(c->aspec, c->aWork.p, c->stream) != 0)
            st = fail(c, LBE_ERR_CUDA, "spectral shell transpose: binding the cuFFT work area failed");
        if (st == LBE_OK) st = spectral_tables(c, c->aspec, c->aL, c->aNr, c->aNc, shells, false, c->aTab.p,
                                               c->aR.p, c->aZ.p);
        if (st != LBE_OK) {
            spectral_destroy(c->aspec);
            c->aspec = nullptr;
            release();
            return st;
        }
    }
    SpectralShell *aspec = c->aspec;
    const int *aL = c->aL;
    const long long aNr = c->aNr, aNc = c->aNc;
    const SpecPairs &asp = c->asp;
    Buf &aR = c->aR, &aZ = c->aZ, &aW = c->aW, &aTab = c->aTab;
    // tensor maps of the padded Lambda_c and (g Lambda)_c with the box of each pair's shell
    std::vector<CUtensorMap> mapL(3 * npairs), mapgL(3 * npairs);
    for (int q = 0; q < npairs && !adj_spectral; ++q) {
        int bx = 0, by = 0;
        if (f64) {
            adj_shell_box(true, c->pairs[q].S, &bx, &by);
            for (int cc = 0; cc < 3; ++cc) {
                ATRY(make_map(c, &mapL[3 * q + cc], (char *)Lpad.p + rb * cc * P, bx, by));
                ATRY(make_map(c, &mapgL[3 * q + cc], (char *)gLpad.p + rb * cc * P, bx, by));
            }
        } else {
            adj_shell_box(false, c->pairs[q].S, &bx, &by);
            for (int cc = 0; cc < 3; ++cc)
                ATRY(make_map(c, &mapL[3 * q + cc], (char *)Lpad.p + 2 * rb * cc * P, bx, by, true));
        }
    }

    // forward sweep with checkpoints; the objective is the flux average of these T steps
    c->flux_axis = axis;
    c->flux_plane = plane;
    c->flux_count = 0;
    CK(cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream), "memset flux");
    StepParams sp = step_params(c);
    const int psize = plane_size(c);
    ATRY(dev_alloc(c, c->flux_buf, 8 * (size_t)M * psize));
    for (int s = 0; s < nseg; ++s) {
        CK(cudaMemcpyAsync(ck[s].p, c->pop[c->cur].p, pop_bytes, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
        const int nst = std::min(K, T - s * K);
        for (int k = 0; k < nst; ++k) ATRY(step_once(c, sp, psize));
    }
    double acc[MAXS];
    CK(cudaMemcpyAsync(acc, c->flux_acc.p, 8 * MAXS, cudaMemcpyDeviceToHost, c->stream), "copy flux");
    CK(cudaStreamSynchronize(c->stream), "sync");
    double phi_val = 0.0;
    for (int a = 0; a < M; ++a) phi_val += acc[a];
    phi_val /= (double)T;

    // reverse sweep
    AdjParams ap{};
    ap.M = M;
    ap.consistent = c->cfg.consistent_moments ? 1 : 0;
    ap.axis = axis;
    ap.plane = plane;
    ap.wobj = 1.0 / (double)T;
    for (int a = 0; a < M; ++a) ap.sp[a] = sp.sp[a];
    StepParams sp0 = sp;
    sp0.flux_axis = -1;
    int cl = 0;
    for (int s = nseg - 1; s >= 0; --s) {
        const int nst = std::min(K, T - s * K);
        auto state = [&](int k) -> void * { return k == 0 ? ck[s].p : seg[k].p; };
        // recompute the segment: the force stage of every state (kept in its slot) and the states
        for (int k = 0; k < nst; ++k) {
            char *sl = (char *)slot[k].p;
            ATRY(force_stage(c, state(k), npairs ? sl + sl_P : nullptr, npairs ? sl + sl_xi : nullptr));
            CK(cudaMemcpyAsync(sl + sl_npad, c->npad.p, rb * M * P, cudaMemcpyDeviceToDevice, c->stream), "keep npad");
            if (npairs)
                CK(cudaMemcpyAsync(sl + sl_gab, c->gab.p, rb * M * M * N, cudaMemcpyDeviceToDevice, c->stream),
                   "keep gab");
            CK(cudaMemcpyAsync(sl + sl_C, c->C.p, rb * M * 3 * N, cudaMemcpyDeviceToDevice, c->stream), "keep C");
            if (k + 1 < nst) {
                StageTimer tm(c, LBE_STAGE_COLLIDE);
                LAUNCH(launch_collide(c->prec, c->g, state(k), state(k + 1), (const uint32_t *)c->mask.p,
                                      c->solid_links, c->C.p, c->F.p, sp0, (double *)c->flux_buf.p, c->stream),
                       "collide kernel");
            }
        }
        for (int k = nst - 1; k >= 0; --k) {
            const char *sl = (const char *)slot[k].p;
            LAUNCH(launch_adj_collide(c->prec, c->g, state(k), (const uint32_t *)c->mask.p, sl + sl_C, c->F.p, ap,
                                      lYf[cl].p, lYg[cl].p, lnd[cl].p, lYf[1 - cl].p, lYg[1 - cl].p, lC.p, lF.p,
                                      lmom.p, c->stream),
                   "adjoint collide");
            if (M > 2) c->launches += 1;  // k_adj_collide + k_adj_write (one kernel for one or two species)
            CK(cudaMemsetAsync(lnd[1 - cl].p, 0, rb * M * N, c->stream), "memset");
            CK(cudaMemsetAsync(lg.p, 0, rb * M * M * N, c->stream), "memset");
            std::vector<int> own(M, 1);
            for (int q = 0; q < npairs; ++q) {
                const auto &ps = c->pairs[q];
                AdjShell L{};
                L.npad_a = sl + sl_npad + rb * ps.a * P;
                L.gab = sl + sl_gab + rb * (ps.a * M + ps.b) * N;
                L.lC_a = (const char *)lC.p + rb * 3 * ps.a * N;
                L.P = sl + sl_P + rb * 3 * q * N;
                L.C_a = sl + sl_C + rb * 3 * ps.a * N;
                L.Lpad = adj_spectral ? nullptr : Lpad.p;  // the spectral transpose forms Lambda itself
                L.gLpad = adj_spectral ? nullptr : gLpad.p;
                L.coef = ps.coef;
                L.own = own[ps.a];
                own[ps.a] = 0;
                L.ln_a = (char *)lnd[1 - cl].p + rb * ps.a * N;
                L.lg = (char *)lg.p + rb * (ps.a * M + ps.b) * N;
                LAUNCH(launch_adj_shell_prep(f64, c->g, L, c->stream), "adjoint shell prep");
                if (adj_spectral) continue;
                AdjShellTile LT{};
                LT.grid = &c->g;
                LT.maps_L = &mapL[3 * q];
                LT.maps_gL = &mapgL[3 * q];
                LT.npad_b = sl + sl_npad + rb * ps.b * P;
                LT.g_ab = L.gab;
                LT.ln_b = (char *)lnd[1 - cl].p + rb * ps.b * N;
                LT.lg_ab = L.lg;
                LT.err = (int *)c->err.p;
                LAUNCH(launch_adj_shell_tile(f64, ps.S, LT, c->stream), "adjoint shell");
                c->launches += 2;  // one launch per component
            }
            if (npairs && adj_spectral) {
                // the shell sums of the transpose for every pair at once (lbe_spectral.cu)
                LAUNCH(launch_adjspec_embed(f64, c->g, aL, aNr, asp, sl + sl_npad, lC.p, sl + sl_gab, aR.p, c->stream),
                       "adjoint spectral embed");
                if (spectral_forward(aspec, 0, aR.p, aZ.p) != 0) {
                    release();
                    return fail(c, LBE_ERR_CUDA, "spectral shell transpose: cuFFT forward transform failed");
                }
                LAUNCH(launch_adjspec_multiply(f64, aZ.p, aTab.p, aW.p, aNc, asp, 1.0 / (double)aNr, c->stream),
                       "adjoint spectral multiply");
                if (spectral_inverse(aspec, 1, aW.p, aR.p) != 0) {
                    release();
                    return fail(c, LBE_ERR_CUDA, "spectral shell transpose: cuFFT inverse transform failed");
                }
                LAUNCH(launch_adjspec_combine(f64, c->g, aL, aNr, asp, aR.p, sl + sl_npad, sl + sl_gab,
                                              lnd[1 - cl].p, lg.p, c->stream),
                       "adjoint spectral combine");
            }
            if (npairs) {
                LAUNCH(launch_adj_contact_prep(f64, c->g, c->cparams, c->brows, sl + sl_xi, lg.p, lnbar.p, c->stream),
                       "adjoint contact");
                ContactLaunch LB{};
                LB.grid = &c->g;
                LB.maps = ballmaps.data();
                LB.cp = &c->cparams;
                LB.br = &c->brows;
                LB.RB = c->RB;
                LB.mask = (const uint32_t *)c->mask.p;
                LB.ln = lnd[1 - cl].p;
                LB.err = (int *)c->err.p;
                LAUNCH(launch_adj_ball_tma(f64, LB, c->stream), "adjoint ball sum");
            }
            cl = 1 - cl;
        }
    }

    // dPhi/damp and dPhi/dg
    if (dPhi_damp) {
        LAUNCH(launch_adj_amp(f64, c->g, M, lF.p, (const double *)c->phi.p, (double *)outA.p, c->stream),
               "adjoint amplitude");
        CK(cudaMemcpyAsync(dPhi_damp, outA.p, 8 * N, cudaMemcpyDeviceToHost, c->stream), "copy gradient");
    }
    if (dPhi_dg) {
        for (int k = 0; k < 3; ++k) {
            double tot = 0.0, r2[2];
            for (int a = 0; a < M; ++a) {
                LAUNCH(launch_to_f64(f64, (const char *)lF.p + rb * (3 * a + k) * N, N, (double *)red.p, c->stream),
                       "convert");
                LAUNCH(launch_reduce((const double *)red.p, N, (double *)c->partial.p, 1024, (double *)c->red_out.p,
                                     c->stream),
                       "reduce");
                CK(cudaMemcpyAsync(r2, c->red_out.p, 16, cudaMemcpyDeviceToHost, c->stream), "copy");
                CK(cudaStreamSynchronize(c->stream), "sync");
                tot += r2[0];
            }
            dPhi_dg[k] = tot;
        }
    }
    if (Phi) *Phi = phi_val;
    // leave the state as it was
    CK(cudaMemcpyAsync(c->pop[c->cur].p, ck[0].p, pop_bytes, cudaMemcpyDeviceToDevice, c->stream), "restore state");
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->steps = steps_before;
    c->flux_axis = old_axis;
    c->flux_plane = old_plane;
    c->flux_count = 0;
    CK(cudaMemsetAsync(c->flux_acc.p, 0, 8 * MAXS, c->stream), "memset flux");
    release();
#undef ATRY
    return check_error_word(c);
}

lbe_status lbe_set_stage_timing(lbe_ctx *c, int on) {
    TRY(ready(c));
    fold_stage_times(c);
    c->timing = on != 0;
    for (int s = 0; s < LBE_NUM_STAGES; ++s) {
        c->stage_ms[s] = 0.0;
        c->stage_launches[s] = 0;
    }
    return LBE_OK;
}

lbe_status lbe_get_stage_times(lbe_ctx *c, double *ms, long long *launches) {
    TRY(ready(c));
    fold_stage_times(c);
    for (int s = 0; s < LBE_NUM_STAGES; ++s) {
        if (ms) ms[s] = c->stage_ms[s];
        if (launches) launches[s] = c->stage_launches[s];
    }
    return LBE_OK;
}

lbe_status lbe_get_mass_noalloc(lbe_ctx *c, double *mass) {
    TRY(ready(c));
    if (!mass) return fail(c, LBE_ERR_INVALID_ARG, "null output");
    const long long N = c->g.N;
    if (N > noalloc_max_nodes())
        return fail(c, LBE_ERR_UNSUPPORTED,
                    "lbe_get_mass_noalloc: lattice of " + std::to_string(N) + " nodes exceeds its maximum of " +
                        std::to_string(noalloc_max_nodes()) + " nodes");
    double *scratch = nullptr;
    CK(noalloc_scratch(c->device, &scratch), "lbe_get_mass_noalloc: device address of the scratch array");
    LAUNCH(launch_mass_noalloc((int)c->prec, c->g.nx, c->g.ny, c->g.nz, c->pop[c->cur].p,
                               (const uint32_t *)c->mask.p, c->M, c->n0, scratch, noalloc_blocks(N), c->stream),
           "lbe_get_mass_noalloc kernels");
    c->launches += 1;  // partial sums + final sum
    CK(cudaMemcpyAsync(mass, scratch + noalloc_result_offset(), sizeof(double) * c->M, cudaMemcpyDeviceToHost,
                       c->stream),
       "lbe_get_mass_noalloc: copy result");
    CK(cudaStreamSynchronize(c->stream), "lbe_get_mass_noalloc: stream sync");
    return LBE_OK;
}

lbe_status lbe_probe_wait_timeout(lbe_ctx *c, int polls) {
    TRY(ready(c));
    if (polls < 1 || (long long)polls > WAIT_POLLS)
        return fail(c, LBE_ERR_INVALID_ARG, "polls must be in [1, 2^24]");
    CK(launch_wait_probe((int *)c->err.p, (long long)polls, c->stream), "wait probe launch");
    c->launches += 1;
    return check_error_word(c);
}

lbe_status lbe_get_launch_count(lbe_ctx *c, long long *launches) {
    if (!c || !launches) return fail(c, LBE_ERR_INVALID_ARG, "null argument");
    *launches = c->launches;
    return LBE_OK;
}

}  // extern "C"
