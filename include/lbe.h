/*
 * lbe.h -- C ABI of the GB300 (sm_103a) stabilized Lattice Boltzmann-Enskog
 * hot path: the per-time-step two-distribution trapezoidal (DD-TR) update of a
 * hard-sphere fluid or mixture on a D3Q19 lattice.
 *
 * Method: S. Melchionna and U. Marini Bettolo Marconi, "Stabilized Lattice
 * Boltzmann-Enskog method for compressible flows and its application to one
 * and two-component fluids in nanochannels" (arXiv:1202.3842).  Section and
 * equation names below refer to that paper.
 *
 * Conventions (all functions):
 *   - Every function returns lbe_status; no C++ exception crosses the ABI and
 *     nothing aborts.  lbe_last_error() gives a text for the last failure on a
 *     context (thread-local copy, valid until the next call on that thread).
 *   - Lattice units: time step h = 1, spacing 1, mass 1, k_B T = v_T^2 = 1/3.
 *   - Scalar fields are flat arrays of N = nx*ny*nz values, x fastest:
 *     i = x + nx*(y + ny*z).  Vector fields are [3][N] (component-major).
 *     Population arrays are [19][N] in the D3Q19 order: rest; +x,-x,+y,-y,+z,-z;
 *     (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),(+1,0,-1),
 *     (-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 *   - Host arrays passed in are caller-owned, read during the call and not
 *     retained.  Host arrays passed out are caller-allocated and filled.
 *     All host floating-point data is double precision, whatever the storage
 *     precision on the device.
 *   - The context owns its device memory (through the allocator given at
 *     creation) and issues all work on the CUDA stream given at creation.
 *     lbe_step only enqueues work; getters synchronise that stream.
 *   - The CUDA kernels are the only compute path: there is no CPU fallback.
 *     Without a usable sm_103a device lbe_create returns LBE_ERR_CUDA.
 */
#ifndef LBE_H
#define LBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbe_ctx lbe_ctx;

typedef enum {
    LBE_OK = 0,
    LBE_ERR_INVALID_ARG = 1, /* bad pointer, index, size or parameter value */
    LBE_ERR_UNSUPPORTED = 2, /* valid request this build does not implement  */
    LBE_ERR_OOM = 3,         /* device allocation failed                     */
    LBE_ERR_CUDA = 4,        /* a CUDA runtime/driver call failed            */
    LBE_ERR_DIVERGED = 5,    /* device check found n < 0, a non-finite value,
                                or a packing xi3 >= 1                        */
    LBE_ERR_TIMEOUT = 6,     /* reserved: not returned by this library (a
                                device wait that gives up is LBE_ERR_CUDA)   */
    LBE_ERR_STATE = 7        /* call out of order (e.g. step before species) */
} lbe_status;

/* Storage precision of the populations.  FP64 and FP32 compute in the same
 * precision; the shifted 16-bit forms store s_p = (f_p - w_p n0)/(w_p n0) and
 * compute in FP32.  Mass, momentum and flux accumulators are FP64 always. */
typedef enum {
    LBE_FP64 = 0,
    LBE_FP32 = 1,
    LBE_BF16_SHIFTED = 2,
    LBE_FP16_SHIFTED = 3
} lbe_precision;

/* Collision scheme (Sec. "Results": single (SD) or double (DD) distribution,
 * Euler (EU) or trapezoidal (TR) integration).  LBE_DD_TR is the method; the
 * others are ablations for accuracy studies (FP64 or FP32 storage, one or two
 * species; LBE_ERR_UNSUPPORTED otherwise):
 *   LBE_SD_TR: f only, S_f with the whole force, J = J~ + (C^mf + nF)/2 from f~;
 *   LBE_SD_EU: f only, f* = f + (f_eq - f)/tau + S_f, J = sum c f;
 *   LBE_DD_EU: f and g with the Euler update, J = sum c g, Pi = sum g.
 * In the SD schemes g is not evolved; it holds a copy of f.  The adjoint
 * (lbe_adjoint_flux_gradient) is that of LBE_DD_TR only. */
typedef enum { LBE_DD_TR = 0, LBE_SD_TR = 1, LBE_SD_EU = 2, LBE_DD_EU = 3 } lbe_scheme;

/* Method of the mean-field shell force C^{alpha,mf} (Appendix; the sums over
 * the shell K_sigma of every species pair):
 *   LBE_SHELL_DIRECT: the stencil sum, pair diameters 1..8 (FP32 and 16-bit
 *     storage) or 1..7 (FP64);
 *   LBE_SHELL_SPECTRAL: the same sums as circular convolutions by fast
 *     Fourier transforms (cuFFT, loaded at run time) on a grid padded with
 *     zeros along closed axes, and the ball averages of the contact values
 *     likewise; any integer pair diameter up to the limit of the contact
 *     values (sigma_b / 2 <= 4);
 *   LBE_SHELL_AUTO (default): spectral for diameters without a compiled
 *     stencil, and where it is cheaper by a cost rule measured on GB300: the
 *     mean shell of the pairs above about 320 points (FP32 arithmetic) or 110
 *     points (FP64, where the stencil is bound by the FP64 rate), scaled by
 *     the padded grid over the lattice; direct otherwise.
 * Both give the sums of the definition up to rounding.  The discrete adjoint
 * (lbe_adjoint_flux_gradient) transposes the shell sums with the method this
 * call sets: the stencil (pair diameters with a compiled stencil), the
 * spectral form (any), or under LBE_SHELL_AUTO the spectral form unless the
 * shells are small (the stencil transpose costs about 2.6 times the forward
 * stencil, so the rule's break-even is divided by 2.6). */
typedef enum { LBE_SHELL_AUTO = 0, LBE_SHELL_DIRECT = 1, LBE_SHELL_SPECTRAL = 2 } lbe_shell_method;

/* Optional device allocator.  alloc returns device memory of at least `bytes`
 * usable on `stream` (NULL on failure); free releases it.  NULL allocator:
 * the library uses cudaMallocAsync/cudaFreeAsync on the context stream. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} lbe_allocator;

typedef struct {
    int nx, ny, nz;           /* lattice size, each >= 1                         */
    int periodic[3];          /* 1 = periodic axis; 0 = closed (outside = wall)  */
    int nspecies;             /* M, 1..4                                         */
    lbe_precision precision;
    lbe_scheme scheme;        /* LBE_DD_TR, or an ablation (see lbe_scheme)      */
    int enable_visc;          /* 1: add the viscous Enskog force C^{alpha,visc}
                                 (Appendix) of the tilde velocities J~/n, where
                                 the scheme adds n F (moment recovery, S_f, S_g);
                                 LBE_DD_TR only, no discrete adjoint.  0: off  */
    int consistent_moments;   /* 0 (default): moments as printed in Sec. "Hard
                                 sphere fluid mixture": J = J~ + (C^mf + nF)/2,
                                 Pi = Pi~ - C^mf.u^alpha/2.  1: the map
                                 g = g~ + Omega/2 applied to the printed S_g:
                                 J = J~ + nF/2, Pi = Pi~ + beta C^mf.u^alpha/2.
                                 LBE_DD_TR only (LBE_ERR_INVALID_ARG otherwise). */
    int check_every;          /* > 0: lbe_step checks the device error word every
                                 this many steps (one stream sync each); 0: only
                                 getters check                                   */
} lbe_config;

/* Create a context.  cfg is copied.  cuda_stream is a cudaStream_t (NULL = the
 * legacy default stream).  The current CUDA device at this call is the
 * device used for every later call.  *out receives the context. */
lbe_status lbe_create(const lbe_config *cfg, const lbe_allocator *allocator, void *cuda_stream, lbe_ctx **out);

/* Release all device memory of the context (after synchronising its stream). */
void lbe_destroy(lbe_ctx *ctx);

/* Solid mask (Sec. "Channel flow with a bottleneck": no-slip walls by mid-point
 * bounce-back of f and g).  solid[N]: nonzero = solid node.  Solid nodes carry
 * no fluid: their density is 0 and links into them bounce back. */
lbe_status lbe_set_geometry(lbe_ctx *ctx, const uint8_t *solid);

/* Species s (0-based): hard-sphere diameter sigma >= 0 in lattice units
 * (sigma = 0: ideal gas, C^mf = 0), mass (must be 1: the paper's common mass m),
 * relaxation time tau > 1/2 with omega h = 1/(tau - 1/2), i.e. the TR
 * relaxation factor omega h/(1 + omega h/2) equals 1/tau (Sec. "Ideal fluid").
 * The force stencil is tabulated at compile time for integer pair diameters
 * (sigma_a + sigma_b)/2 in 1..8 and pure ideal gas; other values return
 * LBE_ERR_UNSUPPORTED. */
lbe_status lbe_set_species(lbe_ctx *ctx, int s, double sigma, double mass, double tau);

/* External potential V^s[N] (lattice energy units; 1 k_B T = 1/3) of species s.
 * The force is F = -grad_h V (isotropic D3Q19 gradient; a neighbour outside a
 * closed axis contributes V(r)); Sec. "Ideal fluid", F = -grad U. */
lbe_status lbe_set_potential(lbe_ctx *ctx, int s, const double *V);

/* Wall potential a(r) phi(r), added to the potential of every species.
 * phi[N] is the shape, amp[N] the per-node amplitude (energy units). */
lbe_status lbe_set_wall_potential(lbe_ctx *ctx, const double *phi, const double *amp);

/* Uniform body force g[3] per unit mass on species s (Sec. "Channel flow"). */
lbe_status lbe_set_body_force(lbe_ctx *ctx, int s, const double g[3]);

/* Populations at rest with the quasi-pressure of Sec. "Stabilization" (the
 * equation for Pi^alpha): f~_p = w_p n^a and g~_p = w_p Pi^a on fluid nodes,
 *   Pi^a(r) = n^a(r) - beta * integral to r of (C^{a,mf} + n^a F^a) . dr',
 * C^{a,mf} the mean-field force of the densities n, F^a the force field of the
 * potentials set so far.  The integral is the trapezoidal rule along the
 * lattice path from the origin along x (y = z = 0), then y (z = 0), then z
 * (the paper leaves the path open; its constant never enters the evolution).
 * n is [M][N], every species at once (all must be set with lbe_set_species);
 * solid nodes are taken as n = 0.  Otherwise as lbe_init_density: sets the
 * reference densities, resets the step counter and the flux average. */
lbe_status lbe_init_density_quasipressure(lbe_ctx *ctx, const double *n);

/* Choose the method of the shell force (lbe_shell_method; takes effect at the
 * next step).  LBE_ERR_INVALID_ARG for another value; LBE_ERR_UNSUPPORTED for
 * LBE_SHELL_SPECTRAL when cuFFT cannot be loaded. */
lbe_status lbe_set_shell_method(lbe_ctx *ctx, int method);

/* The method the next step will use (LBE_SHELL_DIRECT or LBE_SHELL_SPECTRAL)
 * for the species set so far; sets up the derived fields as a step would. */
lbe_status lbe_get_shell_method(lbe_ctx *ctx, int *method);

/* Populations at rest: f~_p = g~_p = w_p n[i] on fluid nodes, 0 on solid nodes
 * (so Pi(0) = n(0)).  n[N] >= 0.  Also sets the reference density n0 of the
 * shifted 16-bit storage to the fluid-node mean of n, resets the step counter
 * and the flux average. */
lbe_status lbe_init_density(lbe_ctx *ctx, int s, const double *n);

/* Advance nsteps >= 0 DD-TR steps (Sec. "Hard sphere fluid mixture in a
 * potential well": moments, f_eq, g_eq, S_f, S_g, trapezoidal collision,
 * streaming).  Enqueues work and returns; see check_every. */
lbe_status lbe_step(lbe_ctx *ctx, int nsteps);

/* Density n^s of the current state, out[N] (synchronises). */
lbe_status lbe_get_density(lbe_ctx *ctx, int s, double *out);

/* Velocity of the current state, out[3][N]: u^s = J^s/n^s for s >= 0, the
 * barycentric u = sum J / sum n for s = -1; 0 where the density is 0. */
lbe_status lbe_get_velocity(lbe_ctx *ctx, int s, double *out);

/* Divergence of the velocity u^s (s = -1: the barycentric u) of the current
 * state, out[N]: div u = (1/c_s^2) sum_p w_p c_p . u(r + c_p), the isotropic
 * D3Q19 gradient, with u = 0 on solid nodes and outside closed axes.  The
 * paper's compressibility check in the bottleneck (Sec. "Channel flow with a
 * bottleneck": the steady flow should have div u = 0). */
lbe_status lbe_get_divergence(lbe_ctx *ctx, int s, double *out);

/* Momentum density J^s of the current state, out[3][N]. */
lbe_status lbe_get_momentum(lbe_ctx *ctx, int s, double *out);

/* Mean-field Enskog force C^{s,mf} of the current state, out[3][N]
 * (Appendix, hard-sphere C^{alpha,mf}). */
lbe_status lbe_get_force(lbe_ctx *ctx, int s, double *out);

/* Contact values g_ab of the current state, out[N], for species pair (a, b). */
lbe_status lbe_get_contact(lbe_ctx *ctx, int a, int b, double *out);

/* Choose the plane whose flux is accumulated every step: axis 0/1/2, plane
 * index along that axis.  Resets the time average.  plane < 0 disables. */
lbe_status lbe_set_flux_plane(lbe_ctx *ctx, int axis, int plane);

/* Flux through the configured plane: *instantaneous = sum over the plane's
 * fluid nodes of J^s_axis for the last step taken (s = -1: all species);
 * *time_avg = mean over the steps since the plane was set or reset.  Either
 * pointer may be NULL. */
lbe_status lbe_get_flux(lbe_ctx *ctx, int s, double *instantaneous, double *time_avg);

/* Restart the flux time average. */
lbe_status lbe_reset_flux_average(lbe_ctx *ctx);

/* Totals of the current state: mass[M] = sum n^s, momentum[3] = sum_s sum J^s,
 * *max_u = max over fluid nodes of |u| (barycentric).  FP64 accumulation.
 * Any pointer may be NULL. */
lbe_status lbe_get_totals(lbe_ctx *ctx, double *mass, double *momentum, double *max_u);

/* Streamed populations f~(r,t), g~(r,t) of species s as [19][N] doubles (read
 * or overwrite the state).  Setting them also resets the flux average. */
lbe_status lbe_get_populations(lbe_ctx *ctx, int s, double *f, double *g);
lbe_status lbe_set_populations(lbe_ctx *ctx, int s, const double *f, const double *g);

/* Number of steps taken since lbe_init_density / lbe_set_populations. */
lbe_status lbe_get_step_count(lbe_ctx *ctx, long long *steps);

/* Checkpoint and restart of the state: the populations in their storage
 * precision, the reference densities n0 of the shifted 16-bit storage, the
 * step count, the flux plane and its accumulators.  The lattice geometry,
 * species, potentials and body forces are not part of it; a context that loads
 * a state is given the same ones through their own calls.
 * lbe_save_state: with host_buf NULL, *bytes receives the size of the state;
 * otherwise host_buf (caller-owned, *bytes bytes) receives the state and
 * *bytes its size (LBE_ERR_INVALID_ARG if *bytes is too small).  Synchronises.
 * lbe_load_state: LBE_ERR_INVALID_ARG if the buffer does not hold a state of
 * this library with the context's lattice size, species count and precision;
 * the context is unchanged then.  A state saved and loaded continues
 * bit-identically to the run it was saved from. */
lbe_status lbe_save_state(lbe_ctx *ctx, void *host_buf, size_t *bytes);
lbe_status lbe_load_state(lbe_ctx *ctx, const void *host_buf, size_t bytes);

/* Steady-state residual (the criterion of a run to steady state):
 *   *res = max over species s and nodes r of |n^s(r,t) - n^s(r,t0)| / ((t - t0) n0^s),
 * t the current step count, t0 the step count at the previous call and n0^s the
 * reference density of species s (the fluid-node mean of its last
 * lbe_init_density; 1 if none was given).  Every call records the current
 * densities for the next one; the first call after lbe_create,
 * lbe_init_density, lbe_set_populations or lbe_load_state, and a call with
 * t = t0, only record them and return *res = -1.  FP64; synchronises. */
lbe_status lbe_get_residual(lbe_ctx *ctx, double *res);

/* Per-node blocked-link mask (bit p set: the population arriving along c_p
 * comes from a solid node or from outside a closed axis), out[N]. */
lbe_status lbe_get_link_mask(lbe_ctx *ctx, uint32_t *out);

/* Contact shell of diameter sigma used by the force kernels (integer lattice
 * vectors e with sigma - 1/2 <= |e| < sigma + 1/2).  Writes up to cap vectors
 * as [k][3] ints into e (may be NULL) and the count into *count. */
lbe_status lbe_shell(double sigma, int *e, int cap, int *count);

/* Discrete adjoint (reverse mode through the whole step: streaming, DD-TR
 * collision and moment recovery, mean-field shell force, contact values,
 * density) of the time-averaged flux through a plane,
 *   Phi = (1/T) sum_{t<T} sum_s sum_{plane fluid nodes} J^s_axis(t),
 * over the next T = nsteps steps from the current state.  Outputs:
 *   *Phi; dPhi_damp[N] = dPhi/da(r) for the wall-potential amplitude a(r)
 *   (V^s += a(r) phi(r) for every species, lbe_set_wall_potential);
 *   dPhi_dg[3] = dPhi/dg for a body force g added to every species.
 * Checkpoints every K = ckpt_every steps are kept and each segment is
 * recomputed in the reverse sweep, keeping the states of the segment and the
 * fields of their force stages (device memory: ceil(T/K) + K - 1 copies of the
 * populations, plus for each of the K steps M^2 + 3 M + 2 + 3 npairs words
 * per node and M words per node of the padded lattice).  FP64 and FP32 storage only
 * (LBE_ERR_UNSUPPORTED for the 16-bit forms).  The state of the context is left as it was before the call;
 * the flux time average is reset.  Any output pointer may be NULL. */
lbe_status lbe_adjoint_flux_gradient(lbe_ctx *ctx, int nsteps, int ckpt_every, int axis, int plane,
                                     double *dPhi_damp, double dPhi_dg[3], double *Phi);

/* Stage timing: CUDA events recorded on the context stream around every kernel
 * launch of lbe_step.  on != 0 enables it and clears the totals; 0 disables it. */
lbe_status lbe_set_stage_timing(lbe_ctx *ctx, int on);

/* Stages of one step, in launch order. */
#define LBE_NUM_STAGES 5
enum { LBE_STAGE_DENSITY = 0,  /* K1: pulled zeroth moment into the padded field */
       LBE_STAGE_CONTACT = 1,  /* K2: ball averages and contact values         */
       LBE_STAGE_SHELL = 2,    /* K3: mean-field shell force, one launch per pair */
       LBE_STAGE_COLLIDE = 3,  /* K4: moments + DD-TR collision + streaming     */
       LBE_STAGE_FLUX = 4 };   /* K5: plane flux reduction                      */

/* Device time in milliseconds ms[LBE_NUM_STAGES] and launch counts
 * launches[LBE_NUM_STAGES] accumulated since timing was enabled (synchronises;
 * either pointer may be NULL). */
lbe_status lbe_get_stage_times(lbe_ctx *ctx, double *ms, long long *launches);

/* Number of kernel launches this context has issued (all entry points). */
lbe_status lbe_get_launch_count(lbe_ctx *ctx, long long *launches);

/* Self-test of the device-side failure detector (no counterpart in the
 * paper).  Every wait of the TMA kernels on a copy is bounded: after 2^24
 * polls it sets a bit in the context's device error word and the kernel
 * returns, so a copy that never completes cannot hang the GPU, and the next
 * checking call reports LBE_ERR_CUDA.  This call launches one CTA that arms
 * an mbarrier for 16 bytes that no copy will deliver (none is issued, so
 * nothing is in flight) and waits on it with that same bounded wait, limited
 * to `polls` polls (1 .. 2^24).  It returns what a kernel whose wait gave up
 * makes every later checking call return: LBE_ERR_CUDA, with
 * lbe_last_error() naming the TMA wait.  The error word stays set, so the
 * context's state is no longer trusted; destroy it.  LBE_ERR_INVALID_ARG for
 * polls out of range.  Synchronises the context stream. */
lbe_status lbe_probe_wait_timeout(lbe_ctx *ctx, int polls);

/* Species masses mass[M] = sum over the lattice of n^s of the current state,
 * like the mass of lbe_get_totals, but without allocating any device memory.
 * The paper has no counterpart: this is a service for callers that must not
 * allocate at the time of the call (the device memory pool is fully reserved
 * by another framework, a loop cannot take the latency or synchronisation of
 * an allocation, or the process keeps a fixed device-memory footprint).
 * The block partial sums live in one file-scope device array of the library
 * (4 x 4096 + 4 doubles, about 128 KiB, held by every GPU that loads the
 * library until the process exits), so the lattice may have at most
 * 4096 x 4096 = 16777216 nodes; larger lattices return LBE_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address; make that
 * first call before any CUDA stream capture.  All calls share the array (each
 * call overwrites the parts it reads, the last call's contents stay behind);
 * calls that overlap on the GPU race on it.  Synchronises the context stream. */
lbe_status lbe_get_mass_noalloc(lbe_ctx *ctx, double *mass);

const char *lbe_status_string(lbe_status status);
const char *lbe_last_error(lbe_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBE_H */
