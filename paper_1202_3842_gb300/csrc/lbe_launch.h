// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lbe_device.cuh"

namespace lbe {

// Storage of the populations: [M][2 (f, g)][19][N] elements of the storage type.
enum class Prec : int { F64 = 0, F32 = 1, BF16 = 2, F16 = 3 };

inline int prec_bytes(Prec p) { return p == Prec::F64 ? 8 : (p == Prec::F32 ? 4 : 2); }
inline bool prec_fp64(Prec p) { return p == Prec::F64; }

// Per-species constants of the collision, in FP64 and rounded once to FP32 on the host.  Kernels with
// 16-bit storage read the float copies (their store needs 1/n0, which a thread would otherwise divide
// in FP64, at GB300's low FP64 rate).  Kernels with FP32 storage convert the doubles themselves, which
// compiled to fewer spills at the collide's register cap.
struct SpeciesConst {
    double omega_eff;  // omega h / (1 + omega h / 2) = 1/tau
    double inv;        // h / (1 + omega h / 2)
    double n0;         // reference density of the shifted storage
    double in0;        // 1 / n0 (0 if n0 is 0)
    float omega_eff_f, inv_f, n0_f, in0_f;
};

inline void species_const_set(SpeciesConst &s, double omega_eff, double inv, double n0) {
    s.omega_eff = omega_eff;
    s.inv = inv;
    s.n0 = n0;
    s.in0 = n0 > 0.0 ? 1.0 / n0 : 0.0;
    s.omega_eff_f = (float)s.omega_eff;
    s.inv_f = (float)s.inv;
    s.n0_f = (float)s.n0;
    s.in0_f = (float)s.in0;
}

// Whether a kernel with storage type S and arithmetic type T reads the float copies, and the constants
// in T either way.
template <typename S, typename T>
inline constexpr bool sc_float = sizeof(T) == 4 && sizeof(S) == 2;
template <typename S, typename T>
__host__ __device__ __forceinline__ T sc_omega(const SpeciesConst &s) {
    if constexpr (sc_float<S, T>) return s.omega_eff_f; else return (T)s.omega_eff;
}
template <typename S, typename T>
__host__ __device__ __forceinline__ T sc_inv(const SpeciesConst &s) {
    if constexpr (sc_float<S, T>) return s.inv_f; else return (T)s.inv;
}
template <typename S, typename T>
__host__ __device__ __forceinline__ T sc_n0(const SpeciesConst &s) {
    if constexpr (sc_float<S, T>) return s.n0_f; else return (T)s.n0;
}
template <typename S, typename T>
__host__ __device__ __forceinline__ T sc_in0(const SpeciesConst &s) {
    if constexpr (sc_float<S, T>) return s.in0_f; else return s.n0 > 0.0 ? (T)(1.0 / s.n0) : (T)0;
}

struct StepParams {
    int M;
    int scheme;          // lbe_scheme: DD_TR (k_collide) or an ablation (k_collide_ablation)
    int consistent;      // moment recovery: 0 printed, 1 map-consistent
    int flux_axis;       // -1: no flux plane
    int flux_plane;
    SpeciesConst sp[MAXS];
};

struct ContactParams {
    int M;
    int npairs;
    double sigma[MAXS];
    double s_ab[MAXS][MAXS];   // sigma_a sigma_b / (sigma_a + sigma_b)
    double xi2c[MAXS];         // (pi/6) sigma_b^2
    double xi3c[MAXS];         // (pi/6) sigma_b^3
};

// Rows of the averaging ball |d| <= sigma_b/2 of every species: row k of
// species b covers d = (-a..a, dy, dz); rows are grouped by dz, the rows with
// dz = z being first[b][z + 4] .. first[b][z + 5] - 1.
struct BallRows {
    int count[MAXS];
    short first[MAXS][10];
    signed char dy[MAXS][81], a[MAXS][81];
};

struct ContactLaunch {
    const Grid *grid;
    const CUtensorMap *maps;  // one per species (padded density, box from contact_box)
    const ContactParams *cp;
    const BallRows *br;
    int RB;                   // largest ball half-width
    void *gab;
    void *gnpad;
    void *xi;                  // NULL, or [2][N]: xi2, xi3 (kept for the adjoint)
    const uint32_t *mask;      // adjoint ball sum only
    void *ln;                  // adjoint ball sum only: [M][N] accumulated
    int *err;
};

struct ShellLaunch {
    const Grid *grid;
    const CUtensorMap *map_n;
    const CUtensorMap *map_gn;
    const void *npad_a;
    const void *g_ab;
    void *Cout;
    void *Pout;  // NULL, or [3][N]: P = sum_e e^ n_b(r+e) of the pair (for the adjoint)
    double coef;
    int accumulate;
    int *err;
};

// Geometry
cudaError_t launch_link_mask(const Grid &g, const uint8_t *solid, uint32_t *mask, cudaStream_t st);
cudaError_t launch_wait_probe(int *err, long long polls, cudaStream_t st);
// Force field F^a = -grad_h (V^a + amp*phi) + g^a, stored as T [3][N].
cudaError_t launch_force_field(Prec p, const Grid &g, const double *V, const double *phi, const double *amp,
                               const double gbody[3], void *F, cudaStream_t st);
// Populations: [19][N] FP64 streamed form <-> storage (post-collision form) of species a.
cudaError_t launch_unstream(Prec p, const Grid &g, const uint32_t *mask, const double *f, const double *gq,
                            void *pop, int a, double n0, cudaStream_t st);
cudaError_t launch_stream_out(Prec p, const Grid &g, const uint32_t *mask, const void *pop, int a, double n0,
                              double *f, double *gq, cudaStream_t st);
// pi (optional): the g distribution at rest from Pi [N] instead of n
cudaError_t launch_rest_state(Prec p, const Grid &g, const uint32_t *mask, const double *n, void *pop, int a,
                              double n0, cudaStream_t st, const double *pi = nullptr);
// Quasi-pressure Pi^a = n^a - beta * path integral of C^{a,mf} + n^a F^a (lbe_quasipressure.cu):
// n [M][N] FP64, C and F [M][3][N] in the compute type; Pi [M][N] FP64.
cudaError_t launch_quasipressure(bool fp64, const Grid &g, int M, const double *n, const void *C, const void *F,
                                 double *Pi, cudaStream_t st);
// K1: density (pulled zeroth moment) of every species into the padded field.
// solid = false: no solid node and every axis periodic (the link mask is not read).
cudaError_t launch_density(Prec p, const Grid &g, const void *pop, const uint32_t *mask, bool solid, int M,
                           const double *n0, void *npad, int *err, cudaStream_t st);
// K2: ball averages, BMCSL contact values g_ab [M][M][N] and padded g_ab*n_b [M][M][P].
cudaError_t launch_contact_tma(bool fp64, const ContactLaunch &L, cudaStream_t st);
// Transposed ball average: L.maps over the padded adjoint fields lnbar; ln[b] += ball sum, 0 on solid nodes.
cudaError_t launch_adj_ball_tma(bool fp64, const ContactLaunch &L, cudaStream_t st);
void contact_box(bool fp64, int M, int RB, int *bx, int *by);
// K3: shell force of one ordered pair.
cudaError_t launch_shell_force(bool fp64, int S, const ShellLaunch &L, cudaStream_t st);
bool shell_supported(bool fp64, int S);
void shell_box(bool fp64, int S, int *bx, int *by);      // forward: FP32 boxes count 8-byte (n, g n) elements
void adj_shell_box(bool fp64, int S, int *bx, int *by);  // shell transpose: boxes of its own tiles
// K4: fused moments + DD-TR collision + pull streaming.
cudaError_t launch_collide(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask, bool solid,
                           const void *C, const void *F, const StepParams &sp, double *flux_buf,
                           cudaStream_t st);
// Scheme ablations SD-TR, SD-EU, DD-EU (lbe_ablation.cu): FP64/FP32 storage, one or two species.
bool ablation_supported(Prec p, int M);
cudaError_t launch_collide_ablation(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask,
                                    bool solid, const void *C, const void *F, const StepParams &sp,
                                    double *flux_buf, cudaStream_t st);
cudaError_t launch_moments_ablation(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *C,
                                    const void *F, const StepParams &sp, double *n, double *J, cudaStream_t st);
// K1 for one or two species, species-parallel lanes (lbe_collide_pair.cu).
cudaError_t launch_density_pair(Prec p, const Grid &g, const void *pop, const uint32_t *mask, bool solid, int M,
                                const double *n0, void *npad, int *err, cudaStream_t st);
// K4 for one or two species, species-parallel lanes (lbe_collide_pair.cu).
cudaError_t launch_collide_pair(Prec p, const Grid &g, const void *src, void *dst, const uint32_t *mask, bool solid,
                                const void *C, const void *F, const StepParams &sp, double *flux_buf,
                                cudaStream_t st);
// Moments of the current state (FP64 out): n [M][N], J [M][3][N].
cudaError_t launch_moments(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *C,
                           const void *F, const StepParams &sp, double *n, double *J, cudaStream_t st);
// K5: flux of the step: sum of the plane buffer [M][plane] into acc[M] (+=) and last[M] (=).
cudaError_t launch_flux_reduce(int M, int plane_size, const double *buf, double *acc, double *last,
                               cudaStream_t st);
// Deterministic FP64 reductions: out[0] = sum x[0..n), out[1] = max |x|.
cudaError_t launch_reduce(const double *x, long long n, double *partial, int npartial, double *out,
                          cudaStream_t st);
// u [3][N] = J/n summed over species s (all for s < 0); speed [N] = |u| (either may be NULL).
cudaError_t launch_velocity(int M, long long N, int s, const double *n, const double *J, double *u, double *speed,
                            cudaStream_t st);
// Steady-state residual: out[i] = max_a |n_a(i) - rec_a(i)| * inv.v[a]; rec <- n.
struct InvN0 {
    double v[MAXS];
};
cudaError_t launch_residual(int M, long long N, const InvN0 &inv, const double *n, double *rec, double *out,
                            cudaStream_t st);
// div u [N] of a velocity field u [3][N] (FP64), isotropic D3Q19 gradient, u = 0 outside closed axes.
cudaError_t launch_divergence(const Grid &g, const double *u, double *out, cudaStream_t st);
// Convert a compute-precision field to FP64.
cudaError_t launch_to_f64(bool fp64, const void *src, long long n, double *dst, cudaStream_t st);
// Copy the interior of a padded field to a dense FP64 array.
cudaError_t launch_unpad(bool fp64, const Grid &g, const void *pad, double *dst, cudaStream_t st);

// ---------------------------------------------------------------------------
// discrete adjoint (lbe_adjoint.cu)
// ---------------------------------------------------------------------------
struct AdjParams {
    int M;
    int consistent;
    int axis;     // flux plane
    int plane;
    double wobj;  // weight of one step's flux in the objective (1/T)
    SpeciesConst sp[MAXS];
};

// Node-local part of the shell transpose of pair (a, b) (k_adj_shell_prep).
struct AdjShell {
    const void *npad_a;  // padded n_a
    const void *gab;     // g_ab [N]
    const void *lC_a;    // adjoint of C^a [3][N]
    const void *P;       // P = sum_e e^ n_b(r+e) of the pair [3][N] (forward recomputation)
    const void *C_a;     // C^a [3][N] of the forward state
    void *Lpad, *gLpad;  // out: padded Lambda and g*Lambda [3][P]
    double coef;
    int own;    // add the own-node density term of species a (once per species)
    void *ln_a; // [N] density adjoint of species a (accumulated)
    void *lg;   // [N] contact-value adjoint of this pair (accumulated)
};

// Shell sums of the transpose of pair (a, b): three launches, one per component.
struct AdjShellTile {
    const Grid *grid;
    const CUtensorMap *maps_L;   // [3] padded Lambda_c, box of adj_shell_box(S)
    const CUtensorMap *maps_gL;  // [3] padded (g Lambda)_c
    const void *npad_b;
    const void *g_ab;
    void *ln_b;   // [N] density adjoint of species b (accumulated)
    void *lg_ab;  // [N] contact-value adjoint of the pair (accumulated)
    int *err;
};

cudaError_t launch_adj_collide(Prec p, const Grid &g, const void *post, const uint32_t *mask, const void *C,
                               const void *F, const AdjParams &ap, const void *lYf_in, const void *lYg_in,
                               const void *lnd_in, void *lYf_out, void *lYg_out, void *lC, void *lF,
                               void *lmom /* [M][5][N] scratch */, cudaStream_t st);
cudaError_t launch_adj_collide_pair(Prec p, const Grid &g, const void *post, const uint32_t *mask, const void *C,
                                   const void *F, const AdjParams &ap, const void *lYf_in, const void *lYg_in,
                                   const void *lnd_in, void *lYf_out, void *lYg_out, void *lC, void *lF,
                                   cudaStream_t st);
cudaError_t launch_adj_shell_prep(bool fp64, const Grid &g, const AdjShell &L, cudaStream_t st);
cudaError_t launch_adj_shell_tile(bool fp64, int S, const AdjShellTile &L, cudaStream_t st);
cudaError_t launch_adj_contact_prep(bool fp64, const Grid &g, const ContactParams &cp, const BallRows &br,
                                   const void *xi, const void *lg, void *lnbar, cudaStream_t st);
cudaError_t launch_adj_amp(bool fp64, const Grid &g, int M, const void *lF, const double *phi, double *out,
                           cudaStream_t st);

// Viscous Enskog force folded into an effective force field (lbe_visc.cu): shell points of every
// ordered pair in eoff [3 per point] / ehat [3 per point], pair q's run first[q] .. first[q] + count[q].
struct ViscPairs {
    int M, npairs;
    int a[MAXS * MAXS], b[MAXS * MAXS];
    int first[MAXS * MAXS], count[MAXS * MAXS];
    double pre[MAXS * MAXS];  // 2 sigma_ab^2 sqrt(k_B T / pi) w_ab (times n_a / n_a: C^visc / n_a)
};
// u~ [M][3][N] scratch; Feff [M][3][N] = F + C^visc / n
cudaError_t launch_visc(Prec p, const Grid &g, const void *pop, const uint32_t *mask, const void *npad,
                        const void *gab, const void *F, const StepParams &sp, const ViscPairs &vp, const int *eoff,
                        const double *ehat, void *ut, void *Feff, cudaStream_t st);

// K3 by fast Fourier transforms (lbe_spectral.cu).
struct SpecPairs {
    int M, npairs;
    int a[MAXS * MAXS], b[MAXS * MAXS];  // species of each ordered pair
    int s[MAXS * MAXS];                  // index of the pair's shell spectrum
    double half_coef[MAXS * MAXS];       // coef_ab / 2
};
struct SpectralShell;  // cuFFT plans of one lattice
bool spectral_available(std::string *why);
// Plans for the grid L (x fastest): forward of the M densities (0), inverse of ninv force spectra (1),
// forward of three table fields (2), forward of the npairs fields g n (3), inverse of the M ball
// averages (4).  Returns 0, or -1 with the reason in *why.
int spectral_create(SpectralShell **out, bool fp64, const int L[3], int M, int npairs, int ninv, size_t *work_bytes,
                    std::string *why);
// The same with any plan list: plan k transforms batch[k] fields, forward (real to half spectrum) or not.
int spectral_create_plans(SpectralShell **out, bool fp64, const int L[3], int nplans, const int *batch,
                          const bool *forward, size_t *work_bytes, std::string *why);
void spectral_destroy(SpectralShell *s);
int spectral_bind(SpectralShell *s, void *work, cudaStream_t st);
int spectral_forward(SpectralShell *s, int which /* 0, 2 or 3 */, void *R, void *Z);
int spectral_inverse(SpectralShell *s, int which /* 1 or 4 */, void *W, void *R);
cudaError_t launch_spec_table(bool fp64, void *R3, long long Nr, const int L[3], const int *e, const double *u, int ne,
                              cudaStream_t st);
cudaError_t launch_spec_imag(bool fp64, const void *Z3, void *tab3, long long Nc, cudaStream_t st);
cudaError_t launch_spec_real(bool fp64, const void *Z, void *tab, long long Nc, cudaStream_t st);
// K3 transposed in spectral form (discrete adjoint)
cudaError_t launch_adjspec_embed(bool fp64, const Grid &g, const int L[3], long long Nr, const SpecPairs &sp,
                                 const void *npad, const void *lC, const void *gab, void *R, cudaStream_t st);
cudaError_t launch_adjspec_multiply(bool fp64, const void *Z, const void *tab, void *W, long long Nc,
                                    const SpecPairs &sp, double scale, cudaStream_t st);
cudaError_t launch_adjspec_combine(bool fp64, const Grid &g, const int L[3], long long Nr, const SpecPairs &sp,
                                   const void *R, const void *npad, const void *gab, void *ln, void *lg,
                                   cudaStream_t st);
cudaError_t launch_spec_embed_n(bool fp64, const Grid &g, const int L[3], long long Nr, int M, const void *npad,
                                void *R, cudaStream_t st);
cudaError_t launch_spec_ball_mul(bool fp64, const void *Z, const void *btab, void *W, long long Nc, int M,
                                 double scale, cudaStream_t st);
cudaError_t launch_spec_contact(bool fp64, const Grid &g, const int L[3], long long Nr, const ContactParams &cp,
                                const SpecPairs &sp, const void *npad, const void *nbar, void *gab, void *xi, void *G,
                                int *err, cudaStream_t st);
cudaError_t launch_spec_multiply(bool fp64, const void *Z, const void *tab, void *W, long long Nc, const SpecPairs &sp,
                                 double scale, cudaStream_t st);
cudaError_t launch_spec_combine(bool fp64, const Grid &g, const int L[3], long long Nr, const void *R,
                                const void *npad, const void *gab, const SpecPairs &sp, void *Cout, void *Pout,
                                cudaStream_t st);

}  // namespace lbe
