/*
 * FP64 CPU oracle of the stabilized Lattice Boltzmann-Enskog step
 * (Melchionna & Marini Bettolo Marconi, "Stabilized Lattice Boltzmann-Enskog
 * method for compressible flows and its application to one and two-component
 * fluids in nanochannels", arXiv:1202.3842).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition the CUDA library is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never does, and the two share no code, tables or headers.
 *
 * Everything is double precision, plain loops, one thread, summed in the order
 * the paper writes the sums.  Lattice units: h = 1, dx = 1, m = 1,
 * v_T^2 = c_s^2 = 1/3, so k_B T = 1/3 and beta = 3.  Lattice D3Q19.
 *
 * Layouts (all caller-owned, x fastest): a scalar field is [N] with
 * i = x + nx*(y + ny*z); a vector field is [3][N]; populations are [19][N];
 * per-species arrays stack species first.
 *
 * Readings of the paper that the text leaves open (each is listed with its
 * justification in the design notes of the repository):
 *   tau      : omega*h = 1/(tau - 1/2), so the TR relaxation factor
 *              omega h/(1 + omega h/2) equals 1/tau (Sec. "Ideal fluid").
 *   shell    : the contact-sphere integral over k-hat (Appendix, C^{alpha,mf})
 *              becomes a sum over K_sigma = {e in Z^3 : sigma-1/2 <= |e| < sigma+1/2}
 *              with unit vectors e/|e| and one weight w_sigma = 4 pi sigma / sum|e|.
 *   contact  : g_ab is the Boublik-Mansoori-Carnahan-Starling-Leland contact
 *              value of ball-averaged densities (ball radius sigma_b/2), averaged
 *              over the two ends of each shell vector (pair symmetric).
 *   outside  : density is zero on solid nodes and outside non-periodic axes.
 *   moments  : as printed (Sec. "Hard sphere fluid mixture"):
 *              J = J~ + (h/2)(C^mf + C^visc + nF), Pi = Pi~ - (h/2) C^mf . u^alpha.
 *              consistent_moments = 1 instead applies the map g = g~ + h Omega/2
 *              to the printed S_g: J = J~ + (h/2)(C^visc + nF),
 *              Pi = Pi~ + (h/2) beta C^mf . u^alpha (an ablation; it diverges
 *              on strongly compressed starts because the dropped d Pi/d n
 *              term of S_g is then not small).  consistent_moments = 2 adds
 *              that term (see dpi_dn_term): an exact, relaxation-time
 *              independent rest state, stable only at low packing.
 *   S_g      : the coefficient of H2 in the C^mf term is 4, as printed.
 *   schemes  : (Sec. "Results") DD-TR is the default; the ablations are
 *              SD-TR: one distribution f, S = S_f with the whole force, and the
 *                     TR moments J = J~ + (h/2)(C^mf + nF) from f~;
 *              SD-EU: one distribution, Euler update
 *                     f* = f + (1/tau)(f_eq - f) + h S_f with J = sum c f;
 *              DD-EU: both distributions with the Euler update and
 *                     J = sum c g, Pi = sum g.
 *              Euler and trapezoidal updates relax at the same rate 1/tau
 *              (omega_EU h = 1/tau).  In the SD schemes g is not evolved: it
 *              is kept equal to f.
 *   force    : F = -grad_h V + g with the isotropic D3Q19 gradient.
 *   init     : f~ = g~ = w_p n(r,0) on fluid nodes, zero on solid nodes.
 *   C^visc   : opt-in (or_set_visc): the viscous Enskog force of the Appendix
 *              on the lattice shell, taken at the tilde velocities J~/n and
 *              added where n F enters (J, S_f, S_g); off by default.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The per-node loops carry OR_PARALLEL_FOR.  The parity build (no -fopenmp)
 * ignores it and runs one thread; the timing build of the same source
 * (-fopenmp) spreads those loops over the host cores.  Every node's arithmetic
 * is the same either way, and the reductions (the plane flux) stay serial. */
#ifdef _OPENMP
#define OR_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PARALLEL_FOR
#endif

#define Q 19
#define MAXS 4

static const double PI = 3.14159265358979323846;
static const double CS2 = 1.0 / 3.0;   /* v_T^2 = c_s^2 */
static const double KT = 1.0 / 3.0;    /* k_B T = m v_T^2 with m = 1 */
static const double BETA = 3.0;        /* 1/(k_B T) */

/* ------------------------------------------------------------------------- */
/* D3Q19 quadrature (Sec. "Numerical solution", Gauss-Hermite nodes c_p and   */
/* weights w_p).  Order: rest, 6 axis links, 12 edge links; opposite links    */
/* are adjacent (p, p+1) for odd p.                                          */
/* ------------------------------------------------------------------------- */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight_of(int p) {
    int c2 = CV[p][0] * CV[p][0] + CV[p][1] * CV[p][1] + CV[p][2] * CV[p][2];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int p) {
    for (int q = 0; q < Q; ++q)
        if (CV[q][0] == -CV[p][0] && CV[q][1] == -CV[p][1] && CV[q][2] == -CV[p][2]) return q;
    return -1;
}

/* Hermite tensors at the nodes (Sec. "Ideal fluid"):
 * H1_p = c_p / v_T^2,  H2_p = (c_p c_p - v_T^2 I) / (2 v_T^4). */
static void hermite(int p, double H1[3], double H2[3][3]) {
    for (int i = 0; i < 3; ++i) {
        H1[i] = CV[p][i] / CS2;
        for (int j = 0; j < 3; ++j)
            H2[i][j] = (CV[p][i] * CV[p][j] - (i == j ? CS2 : 0.0)) / (2.0 * CS2 * CS2);
    }
}

int or_lattice(int *c, double *w, int *opp) {
    for (int p = 0; p < Q; ++p) {
        for (int i = 0; i < 3; ++i) c[3 * p + i] = CV[p][i];
        w[p] = weight_of(p);
        opp[p] = opposite(p);
    }
    return Q;
}

/* ------------------------------------------------------------------------- */
/* Grid                                                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n[3];
    int per[3];
} grid_t;

static long nsites(const grid_t *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

/* Linear index of (x,y,z) after periodic wrap; -1 outside a non-periodic axis. */
static long site(const grid_t *g, int x, int y, int z) {
    int r[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) {
        if (r[a] < 0 || r[a] >= g->n[a]) {
            if (!g->per[a]) return -1;
            r[a] = ((r[a] % g->n[a]) + g->n[a]) % g->n[a];
        }
    }
    return r[0] + (long)g->n[0] * (r[1] + (long)g->n[1] * r[2]);
}

static void coords(const grid_t *g, long i, int *x, int *y, int *z) {
    *x = (int)(i % g->n[0]);
    *y = (int)((i / g->n[0]) % g->n[1]);
    *z = (int)(i / ((long)g->n[0] * g->n[1]));
}

/* Density as the stencils see it: zero on solid nodes and outside. */
static double field_at(const grid_t *g, const uint8_t *solid, const double *f, int x, int y, int z) {
    long s = site(g, x, y, z);
    if (s < 0) return 0.0;
    if (solid && solid[s]) return 0.0;
    return f[s];
}

/* Bounce-back link mask (mid-point bounce-back, Sec. "Channel flow"):
 * bit p of mask[r] is set when the population arriving at fluid node r along
 * c_p would come from a solid node or from outside a non-periodic axis. */
void or_link_mask(int nx, int ny, int nz, const int *per, const uint8_t *solid, uint32_t *mask) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    for (long i = 0; i < N; ++i) {
        int x, y, z;
        coords(&g, i, &x, &y, &z);
        uint32_t m = 0;
        for (int p = 1; p < Q; ++p) {
            long s = site(&g, x - CV[p][0], y - CV[p][1], z - CV[p][2]);
            if (s < 0 || (solid && solid[s])) m |= (1u << p);
        }
        mask[i] = m;
    }
}

/* ------------------------------------------------------------------------- */
/* Shell and ball lists                                                      */
/* ------------------------------------------------------------------------- */

/* Contact shell K_sigma = {e : (sigma-1/2)^2 <= |e|^2 < (sigma+1/2)^2}, listed
 * with z outermost, then y, then x, each ascending.  Writes up to cap triples;
 * returns the count. */
int or_shell(double sigma, int *e, int cap) {
    if (!(sigma > 0.0)) return 0;
    double lo = sigma - 0.5, hi = sigma + 0.5;
    double lo2 = lo > 0.0 ? lo * lo : 0.0, hi2 = hi * hi;
    int R = (int)ceil(hi);
    int count = 0;
    for (int z = -R; z <= R; ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                double r2 = (double)(x * x + y * y + z * z);
                if (r2 >= lo2 && r2 < hi2) {
                    if (count < cap) {
                        e[3 * count] = x;
                        e[3 * count + 1] = y;
                        e[3 * count + 2] = z;
                    }
                    ++count;
                }
            }
    return count;
}

/* Quadrature weight of the shell: sum_K w |e| e^ e^ = (4 pi sigma / 3) I, so a
 * linear density reproduces the continuum integral of k^ n(r + sigma k^). */
double or_shell_weight(double sigma) {
    if (!(sigma > 0.0)) return 0.0;
    int cap = 4096;
    int *e = (int *)malloc(sizeof(int) * 3 * cap);
    int k = or_shell(sigma, e, cap);
    double sum = 0.0;
    for (int t = 0; t < k; ++t)
        sum += sqrt((double)(e[3 * t] * e[3 * t] + e[3 * t + 1] * e[3 * t + 1] + e[3 * t + 2] * e[3 * t + 2]));
    free(e);
    return 4.0 * PI * sigma / sum;
}

/* Averaging ball B_R = {d : |d|^2 <= R^2}, same listing order as the shell. */
int or_ball(double radius, int *d, int cap) {
    double r2max = radius * radius;
    int R = (int)floor(radius);
    int count = 0;
    for (int z = -R; z <= R; ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                if ((double)(x * x + y * y + z * z) <= r2max) {
                    if (count < cap) {
                        d[3 * count] = x;
                        d[3 * count + 1] = y;
                        d[3 * count + 2] = z;
                    }
                    ++count;
                }
            }
    return count;
}

/* ------------------------------------------------------------------------- */
/* Contact value (Appendix: g_ab evaluated at contact, functional of n)       */
/* ------------------------------------------------------------------------- */

/* Boublik / Mansoori-Carnahan-Starling-Leland contact value of a hard-sphere
 * mixture from xi2 = (pi/6) sum sigma^2 n, xi3 = (pi/6) sum sigma^3 n. */
double or_bmcsl(double sa, double sb, double xi2, double xi3) {
    double s = (sa + sb > 0.0) ? sa * sb / (sa + sb) : 0.0;
    double one = 1.0 - xi3;
    return 1.0 / one + 3.0 * s * xi2 / (one * one) + 2.0 * s * s * xi2 * xi2 / (one * one * one);
}

/* xi2 = (pi/6) sum_b sigma_b^2 nbar_b and xi3 = (pi/6) sum_b sigma_b^3 nbar_b of
 * every node [N], with nbar_b the average of n_b over the ball B_{sigma_b/2}
 * (zero density on solid nodes and outside non-periodic axes). */
static void contact_xi(const grid_t *g, const uint8_t *solid, int M, const double *sigma, const double *n,
                       double *xi2, double *xi3) {
    long N = nsites(g);
    int cap = 8192;
    int *ball = (int *)malloc(sizeof(int) * 3 * cap);
    double *nbar = (double *)calloc((size_t)M * N, sizeof(double));
    for (int b = 0; b < M; ++b) {
        int kb = or_ball(0.5 * sigma[b], ball, cap);
        OR_PARALLEL_FOR
        for (long i = 0; i < N; ++i) {
            int x, y, z;
            coords(g, i, &x, &y, &z);
            double acc = 0.0;
            for (int t = 0; t < kb; ++t)
                acc += field_at(g, solid, n + (long)b * N, x + ball[3 * t], y + ball[3 * t + 1], z + ball[3 * t + 2]);
            nbar[(long)b * N + i] = acc / kb;
        }
    }
    OR_PARALLEL_FOR
    for (long i = 0; i < N; ++i) {
        double s2 = 0.0, s3 = 0.0;
        for (int b = 0; b < M; ++b) {
            s2 += (PI / 6.0) * sigma[b] * sigma[b] * nbar[(long)b * N + i];
            s3 += (PI / 6.0) * sigma[b] * sigma[b] * sigma[b] * nbar[(long)b * N + i];
        }
        xi2[i] = s2;
        xi3[i] = s3;
    }
    free(nbar);
    free(ball);
}

/* g_ab(r) for every node and ordered pair: gpair[(a*M + b)*N + i].
 * n is [M][N]; the densities are ball-averaged over B_{sigma_b/2}. */
void or_contact_values(int nx, int ny, int nz, const int *per, const uint8_t *solid, int M,
                       const double *sigma, const double *n, double *gpair) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    double *xi2 = (double *)malloc(sizeof(double) * N);
    double *xi3 = (double *)malloc(sizeof(double) * N);
    contact_xi(&g, solid, M, sigma, n, xi2, xi3);
    OR_PARALLEL_FOR
    for (long i = 0; i < N; ++i)
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b)
                gpair[((long)a * M + b) * N + i] = or_bmcsl(sigma[a], sigma[b], xi2[i], xi3[i]);
    free(xi2);
    free(xi3);
}

/* ------------------------------------------------------------------------- */
/* Mean-field Enskog force (Appendix, hard-sphere C^{alpha,mf}):              */
/* C^a(r) = -kT n_a(r) sum_b sigma_ab^2 w_ab sum_{e in K_ab} e^ gbar n_b(r+e)  */
/* with gbar = (g_ab(r) + g_ab(r+e))/2 and sigma_ab = (sigma_a + sigma_b)/2.   */
/* C is [M][3][N].                                                           */
/* ------------------------------------------------------------------------- */
void or_shell_force(int nx, int ny, int nz, const int *per, const uint8_t *solid, int M,
                    const double *sigma, const double *n, const double *gpair, double *C) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    int cap = 16384;
    int *K = (int *)malloc(sizeof(int) * 3 * cap);
    for (long t = 0; t < (long)M * 3 * N; ++t) C[t] = 0.0;
    for (int a = 0; a < M; ++a) {
        for (int b = 0; b < M; ++b) {
            double sab = 0.5 * (sigma[a] + sigma[b]);
            if (!(sab > 0.0)) continue;
            int k = or_shell(sab, K, cap);
            double wab = or_shell_weight(sab);
            const double *gab = gpair + ((long)a * M + b) * N;
            const double *nb = n + (long)b * N;
            OR_PARALLEL_FOR
            for (long i = 0; i < N; ++i) {
                int x, y, z;
                coords(&g, i, &x, &y, &z);
                double sum[3] = {0.0, 0.0, 0.0};
                for (int t = 0; t < k; ++t) {
                    int ex = K[3 * t], ey = K[3 * t + 1], ez = K[3 * t + 2];
                    long s = site(&g, x + ex, y + ey, z + ez);
                    if (s < 0 || (solid && solid[s])) continue;
                    double len = sqrt((double)(ex * ex + ey * ey + ez * ez));
                    double gbar = 0.5 * (gab[i] + gab[s]);
                    sum[0] += (ex / len) * gbar * nb[s];
                    sum[1] += (ey / len) * gbar * nb[s];
                    sum[2] += (ez / len) * gbar * nb[s];
                }
                double na = (solid && solid[i]) ? 0.0 : n[(long)a * N + i];
                for (int c = 0; c < 3; ++c) C[((long)a * 3 + c) * N + i] += -KT * na * sab * sab * wab * sum[c];
            }
        }
    }
    free(K);
}

/* Viscous part of the Enskog force (Appendix, C^{alpha,visc}): for hard spheres
 *   C^{a,visc}(r) = n_a(r) sum_b 2 sigma_ab^2 sqrt(m k_B T / pi)
 *                   integral dk^ k^ g_ab n_b(r + sigma k^) k^.(u_b(r + sigma k^) - u_b(r)),
 * on the lattice with the shell K_sigma, unit vectors e/|e|, the shell weight
 * w_sigma and the endpoint-averaged contact value of the mean-field force.
 * Neighbours outside a non-periodic axis or on solid nodes carry n_b = 0.
 * u [M][3][N]; V [M][3][N]. */
void or_visc_force(int nx, int ny, int nz, const int *per, const uint8_t *solid, int M,
                   const double *sigma, const double *n, const double *u, const double *gpair, double *V) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    int cap = 16384;
    int *K = (int *)malloc(sizeof(int) * 3 * cap);
    for (long t = 0; t < (long)M * 3 * N; ++t) V[t] = 0.0;
    for (int a = 0; a < M; ++a) {
        for (int b = 0; b < M; ++b) {
            double sab = 0.5 * (sigma[a] + sigma[b]);
            if (!(sab > 0.0)) continue;
            int k = or_shell(sab, K, cap);
            double wab = or_shell_weight(sab);
            double pre = 2.0 * sab * sab * sqrt(KT / PI) * wab;
            const double *gab = gpair + ((long)a * M + b) * N;
            const double *nb = n + (long)b * N;
            const double *ub = u + (long)b * 3 * N;
            OR_PARALLEL_FOR
            for (long i = 0; i < N; ++i) {
                int x, y, z;
                coords(&g, i, &x, &y, &z);
                double sum[3] = {0.0, 0.0, 0.0};
                for (int t = 0; t < k; ++t) {
                    int ex = K[3 * t], ey = K[3 * t + 1], ez = K[3 * t + 2];
                    long s = site(&g, x + ex, y + ey, z + ez);
                    if (s < 0 || (solid && solid[s])) continue;
                    double len = sqrt((double)(ex * ex + ey * ey + ez * ez));
                    double e[3] = {ex / len, ey / len, ez / len};
                    double gbar = 0.5 * (gab[i] + gab[s]);
                    double edu = 0.0;
                    for (int c = 0; c < 3; ++c) edu += e[c] * (ub[(long)c * N + s] - ub[(long)c * N + i]);
                    for (int c = 0; c < 3; ++c) sum[c] += e[c] * gbar * nb[s] * edu;
                }
                double na = (solid && solid[i]) ? 0.0 : n[(long)a * N + i];
                for (int c = 0; c < 3; ++c) V[((long)a * 3 + c) * N + i] += na * pre * sum[c];
            }
        }
    }
    free(K);
}

/* External force from a potential (Sec. "Ideal fluid": F = -grad U) plus a
 * uniform body force g.  The gradient is the isotropic D3Q19 stencil
 * grad_h V(r) = (1/c_s^2) sum_p w_p c_p V(r + c_p); a neighbour outside a
 * non-periodic axis contributes V(r).  F is [3][N]. */
void or_force_field(int nx, int ny, int nz, const int *per, const double *V, const double *gbody, double *F) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    OR_PARALLEL_FOR
    for (long i = 0; i < N; ++i) {
        int x, y, z;
        coords(&g, i, &x, &y, &z);
        double grad[3] = {0.0, 0.0, 0.0};
        for (int p = 1; p < Q; ++p) {
            long s = site(&g, x + CV[p][0], y + CV[p][1], z + CV[p][2]);
            double v = (s < 0) ? (V ? V[i] : 0.0) : (V ? V[s] : 0.0);
            for (int c = 0; c < 3; ++c) grad[c] += weight_of(p) * CV[p][c] * v;
        }
        for (int c = 0; c < 3; ++c) F[(long)c * N + i] = -grad[c] / CS2 + (gbody ? gbody[c] : 0.0);
    }
}

/* Quasi-pressure of the second distribution (Sec. "Stabilization", equation
 * for Pi^alpha): Pi^a = n^a - beta * integral to r of (C^{a,mf} + n^a F^a).dr',
 * the integral by the trapezoidal rule along the lattice path from the origin:
 * along x at y = z = 0, then along y at z = 0, then along z (the paper leaves
 * the path open).  n [M][N] (taken as 0 on solid nodes), V [M][N] the full
 * potential of each species, gbody [M][3]; C^{a,mf} from the contact values
 * and shell sums of n.  Pi is [M][N]. */
void or_quasipressure(int nx, int ny, int nz, const int *per, const uint8_t *solid, int M, const double *sigma,
                      const double *n, const double *V, const double *gbody, double *Pi) {
    grid_t g = {{nx, ny, nz}, {per[0], per[1], per[2]}};
    long N = nsites(&g);
    double *nn = (double *)malloc(sizeof(double) * M * N);
    double *gp = (double *)malloc(sizeof(double) * M * M * N);
    double *C = (double *)malloc(sizeof(double) * M * 3 * N);
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    double *W = (double *)malloc(sizeof(double) * 3 * N);   /* C + n F of one species */
    double *I = (double *)malloc(sizeof(double) * N);
    for (long t = 0; t < (long)M * N; ++t) nn[t] = (solid && solid[t % N]) ? 0.0 : n[t];
    or_contact_values(nx, ny, nz, per, solid, M, sigma, nn, gp);
    or_shell_force(nx, ny, nz, per, solid, M, sigma, nn, gp, C);
    for (int a = 0; a < M; ++a) {
        const double *na = nn + (long)a * N;
        or_force_field(nx, ny, nz, per, V + (long)a * N, gbody + 3 * a, F);
        for (int c = 0; c < 3; ++c)
            for (long i = 0; i < N; ++i) W[(long)c * N + i] = C[((long)a * 3 + c) * N + i] + na[i] * F[(long)c * N + i];
        /* x at y = z = 0 */
        I[0] = 0.0;
        for (int x = 1; x < nx; ++x) {
            long i1 = site(&g, x, 0, 0), i0 = site(&g, x - 1, 0, 0);
            I[i1] = I[i0] + 0.5 * (W[i0] + W[i1]);
        }
        /* y at z = 0, for every x */
        for (int x = 0; x < nx; ++x)
            for (int y = 1; y < ny; ++y) {
                long i1 = site(&g, x, y, 0), i0 = site(&g, x, y - 1, 0);
                I[i1] = I[i0] + 0.5 * (W[N + i0] + W[N + i1]);
            }
        /* z, for every (x, y) */
        for (int x = 0; x < nx; ++x)
            for (int y = 0; y < ny; ++y)
                for (int z = 1; z < nz; ++z) {
                    long i1 = site(&g, x, y, z), i0 = site(&g, x, y, z - 1);
                    I[i1] = I[i0] + 0.5 * (W[2 * N + i0] + W[2 * N + i1]);
                }
        for (long i = 0; i < N; ++i) Pi[(long)a * N + i] = na[i] - BETA * I[i];
    }
    free(nn); free(gp); free(C); free(F); free(W); free(I);
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    grid_t g;
    long N;
    int M;
    double sigma[MAXS], tau[MAXS];
    double gbody[MAXS][3];
    int consistent_moments;  /* 0 printed, 1 map-consistent, 2 map-consistent with the d Pi/d n term */
    int visc;            /* 1: add C^{visc} of the tilde velocities to the force terms */
    int scheme;          /* 0 DD-TR, 1 SD-TR, 2 SD-EU, 3 DD-EU */
    uint8_t *solid;      /* [N] */
    double *V;           /* [M][N] external potential per species */
    double *phi, *amp;   /* [N] wall potential shape and amplitude (a*phi added to every species) */
    double *f, *gd;      /* [M][Q][N] streamed populations f~(r,t), g~(r,t) */
    double *fpost, *gpost;
    /* per-step work fields */
    double *n, *gpair, *Cmf, *F, *J, *Pi;
    double *Cvisc, *ut;  /* C^{visc} [M][3][N] and the tilde velocities J~/n [M][3][N] */
    double *sD;          /* [M][N] zeroth moment of the d Pi/d n term of S_g (consistent_moments = 2) */
    double *nh1, *nh2;   /* [M][N] densities of the two previous steps, for that term */
    int nhist;           /* how many of nh1, nh2 hold a density */
    int flux_axis, flux_plane;
    double flux_sum[MAXS];
    long flux_count;
    long steps;
} or_sim;

or_sim *or_create(int nx, int ny, int nz, int px, int py, int pz, int M) {
    if (M < 1 || M > MAXS || nx < 1 || ny < 1 || nz < 1) return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->g.n[0] = nx; s->g.n[1] = ny; s->g.n[2] = nz;
    s->g.per[0] = px; s->g.per[1] = py; s->g.per[2] = pz;
    s->N = nsites(&s->g);
    s->M = M;
    long N = s->N;
    for (int a = 0; a < M; ++a) { s->sigma[a] = 0.0; s->tau[a] = 1.0; }
    s->solid = (uint8_t *)calloc(N, 1);
    s->V = (double *)calloc((size_t)M * N, sizeof(double));
    s->phi = (double *)calloc(N, sizeof(double));
    s->amp = (double *)calloc(N, sizeof(double));
    s->f = (double *)calloc((size_t)M * Q * N, sizeof(double));
    s->gd = (double *)calloc((size_t)M * Q * N, sizeof(double));
    s->fpost = (double *)calloc((size_t)M * Q * N, sizeof(double));
    s->gpost = (double *)calloc((size_t)M * Q * N, sizeof(double));
    s->n = (double *)calloc((size_t)M * N, sizeof(double));
    s->gpair = (double *)calloc((size_t)M * M * N, sizeof(double));
    s->Cmf = (double *)calloc((size_t)M * 3 * N, sizeof(double));
    s->F = (double *)calloc((size_t)M * 3 * N, sizeof(double));
    s->J = (double *)calloc((size_t)M * 3 * N, sizeof(double));
    s->Pi = (double *)calloc((size_t)M * N, sizeof(double));
    s->Cvisc = (double *)calloc((size_t)M * 3 * N, sizeof(double));
    s->ut = (double *)calloc((size_t)M * 3 * N, sizeof(double));
    s->sD = (double *)calloc((size_t)M * N, sizeof(double));
    s->nh1 = (double *)calloc((size_t)M * N, sizeof(double));
    s->nh2 = (double *)calloc((size_t)M * N, sizeof(double));
    s->flux_axis = 0;
    s->flux_plane = -1;
    return s;
}

void or_destroy(or_sim *s) {
    if (!s) return;
    free(s->solid); free(s->V); free(s->phi); free(s->amp);
    free(s->f); free(s->gd); free(s->fpost); free(s->gpost);
    free(s->n); free(s->gpair); free(s->Cmf); free(s->F); free(s->J); free(s->Pi);
    free(s->Cvisc); free(s->ut);
    free(s->sD); free(s->nh1); free(s->nh2);
    free(s);
}

int or_set_solid(or_sim *s, const uint8_t *solid) {
    memcpy(s->solid, solid, (size_t)s->N);
    return 0;
}

int or_set_species(or_sim *s, int a, double sigma, double tau) {
    if (a < 0 || a >= s->M || !(tau > 0.5) || sigma < 0.0) return -1;
    s->sigma[a] = sigma;
    s->tau[a] = tau;
    return 0;
}

int or_set_potential(or_sim *s, int a, const double *V) {
    if (a < 0 || a >= s->M) return -1;
    memcpy(s->V + (long)a * s->N, V, sizeof(double) * s->N);
    return 0;
}

int or_set_wall_potential(or_sim *s, const double *phi, const double *amp) {
    memcpy(s->phi, phi, sizeof(double) * s->N);
    memcpy(s->amp, amp, sizeof(double) * s->N);
    return 0;
}

int or_set_body_force(or_sim *s, int a, const double *g3) {
    if (a < 0 || a >= s->M) return -1;
    for (int c = 0; c < 3; ++c) s->gbody[a][c] = g3[c];
    return 0;
}

int or_set_consistent_moments(or_sim *s, int on) {
    if (on < 0 || on > 2) return -1;
    s->consistent_moments = on;
    return 0;
}

enum { DD_TR = 0, SD_TR = 1, SD_EU = 2, DD_EU = 3 };

/* C^{visc} on (DD-TR only): it enters the moment recovery and both sources
 * beside n F (Sec. "Hard sphere fluid mixture": J, S_f, S_g). */
int or_set_visc(or_sim *s, int on) {
    if (on && s->scheme != 0) return -1;
    s->visc = on ? 1 : 0;
    return 0;
}

int or_set_scheme(or_sim *s, int scheme) {
    if (scheme < DD_TR || scheme > DD_EU || (s->visc && scheme != DD_TR)) return -1;
    s->scheme = scheme;
    return 0;
}

static int single_distribution(const or_sim *s) { return s->scheme == SD_TR || s->scheme == SD_EU; }
static int trapezoidal(const or_sim *s) { return s->scheme == DD_TR || s->scheme == SD_TR; }

int or_set_flux_plane(or_sim *s, int axis, int plane) {
    if (axis < 0 || axis > 2) return -1;
    s->flux_axis = axis;
    s->flux_plane = plane;
    for (int a = 0; a < MAXS; ++a) s->flux_sum[a] = 0.0;
    s->flux_count = 0;
    return 0;
}

/* Rest populations f~ = g~ = w_p n on fluid nodes, zero on solid nodes. */
int or_init_density(or_sim *s, int a, const double *n0) {
    if (a < 0 || a >= s->M) return -1;
    long N = s->N;
    s->nhist = 0;
    for (int p = 0; p < Q; ++p)
        for (long i = 0; i < N; ++i) {
            double v = s->solid[i] ? 0.0 : weight_of(p) * n0[i];
            s->f[((long)a * Q + p) * N + i] = v;
            s->gd[((long)a * Q + p) * N + i] = v;
        }
    return 0;
}

int or_set_populations(or_sim *s, int a, const double *f, const double *g) {
    if (a < 0 || a >= s->M) return -1;
    s->nhist = 0;
    memcpy(s->f + (long)a * Q * s->N, f, sizeof(double) * Q * s->N);
    memcpy(s->gd + (long)a * Q * s->N, g, sizeof(double) * Q * s->N);
    return 0;
}

int or_get_populations(or_sim *s, int a, double *f, double *g) {
    if (a < 0 || a >= s->M) return -1;
    memcpy(f, s->f + (long)a * Q * s->N, sizeof(double) * Q * s->N);
    memcpy(g, s->gd + (long)a * Q * s->N, sizeof(double) * Q * s->N);
    return 0;
}

/* Force field of every species: potential V^a plus the wall potential a*phi. */
static void compute_forces(or_sim *s) {
    long N = s->N;
    double *Vt = (double *)malloc(sizeof(double) * N);
    for (int a = 0; a < s->M; ++a) {
        for (long i = 0; i < N; ++i) Vt[i] = s->V[(long)a * N + i] + s->amp[i] * s->phi[i];
        or_force_field(s->g.n[0], s->g.n[1], s->g.n[2], s->g.per, Vt, s->gbody[a], s->F + (long)a * 3 * N);
    }
    free(Vt);
}

/* The d Pi/d n term of S_g (Sec. "Stabilization", evolution equation of g):
 *   -sum_b (d Pi^a/d n^b - delta_ab) (div(n^b u^b) - u . grad n^b) Gamma_0,
 * which the paper's discrete S_g drops.  With div(n^b u^b) = -d n^b/dt the
 * bracket is minus the material derivative D n^b = dn^b/dt + u . grad n^b, so
 * the term is  sum_b A_ab D n^b Gamma_0  with A_ab = d Pi^a/d n^b - delta_ab.
 * Readings (the paper leaves them open):
 *   - A_ab in the local limit of the quasi-pressure: grad(Pi^a - n^a) =
 *     -beta C^a, and the lattice shell force of a slowly varying density is
 *     C^a = -kT n^a sum_b (4 pi/3) s_ab^3 [g_ab grad n^b + n^b grad g_ab / 2]
 *     (s_ab the pair diameter; the linear-ramp identity of the shell weight and
 *     the endpoint average of g), so
 *       A_ab = n^a [(4 pi/3) s_ab^3 g_ab
 *                   + sum_c (2 pi/3) s_ac^3 n^c (d g_ac/d xi2 dxi2/dn^b + d g_ac/d xi3 dxi3/dn^b)],
 *     dxi_k/dn^b = (pi/6) sigma_b^k, the BMCSL derivatives at the node's xi;
 *   - the mixture equation prints n^b before (d Pi^a/d n^b - delta_ab); the
 *     one-component equation and the equation for D(Pi - n)/Dt it comes from
 *     have no such factor, so it is not applied;
 *   - D n^b over the step [t, t+1] the trapezoidal rule integrates: the
 *     increment n(t+1) - n(t) by second-order extrapolation of the last two,
 *     (3/2)(n(t) - n(t-1)) - (1/2)(n(t-1) - n(t-2)) (n(t) - n(t-1) after one
 *     step, 0 at the first), plus u . grad_h n^b with the isotropic D3Q19
 *     gradient (a solid or outside neighbour contributes n^b(r));
 *   - Gamma_0 projects onto w_p (its higher Hermite moments vanish), so the
 *     term adds w_p s^a to S_g and s^a to its zeroth moment.
 * Fills s->sD [M][N] and adds s^a/2 to Pi^a (the map g = g~ + h Omega/2). */
static void bmcsl_derivatives(double sa, double sb, double xi2, double xi3, double *g, double *d2, double *d3) {
    double s = (sa + sb > 0.0) ? sa * sb / (sa + sb) : 0.0;
    double o = 1.0 - xi3;
    *g = 1.0 / o + 3.0 * s * xi2 / (o * o) + 2.0 * s * s * xi2 * xi2 / (o * o * o);
    *d2 = 3.0 * s / (o * o) + 4.0 * s * s * xi2 / (o * o * o);
    *d3 = 1.0 / (o * o) + 6.0 * s * xi2 / (o * o * o) + 6.0 * s * s * xi2 * xi2 / (o * o * o * o);
}

static void dpi_dn_term(or_sim *s) {
    long N = s->N;
    int M = s->M;
    double *xi2 = (double *)malloc(sizeof(double) * N), *xi3 = (double *)malloc(sizeof(double) * N);
    contact_xi(&s->g, s->solid, M, s->sigma, s->n, xi2, xi3);
    OR_PARALLEL_FOR
    for (long i = 0; i < N; ++i) {
        for (int a = 0; a < M; ++a) s->sD[(long)a * N + i] = 0.0;
        if (s->solid[i]) continue;
        int x, y, z;
        coords(&s->g, i, &x, &y, &z);
        double ntot = 0.0, Jtot[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < M; ++a) {
            ntot += s->n[(long)a * N + i];
            for (int c = 0; c < 3; ++c) Jtot[c] += s->J[((long)a * 3 + c) * N + i];
        }
        double u[3];
        for (int c = 0; c < 3; ++c) u[c] = ntot > 0.0 ? Jtot[c] / ntot : 0.0;
        double Dn[MAXS];
        for (int b = 0; b < M; ++b) {
            const double *nb = s->n + (long)b * N;
            double grad[3] = {0.0, 0.0, 0.0};
            for (int p = 1; p < Q; ++p) {
                long q = site(&s->g, x + CV[p][0], y + CV[p][1], z + CV[p][2]);
                double v = (q < 0 || s->solid[q]) ? nb[i] : nb[q];
                for (int c = 0; c < 3; ++c) grad[c] += weight_of(p) * CV[p][c] * v;
            }
            long k = (long)b * N + i;
            double inc = 0.0;
            if (s->nhist >= 2)
                inc = 1.5 * (nb[i] - s->nh1[k]) - 0.5 * (s->nh1[k] - s->nh2[k]);
            else if (s->nhist == 1)
                inc = nb[i] - s->nh1[k];
            Dn[b] = inc + (u[0] * grad[0] + u[1] * grad[1] + u[2] * grad[2]) / CS2;
        }
        for (int a = 0; a < M; ++a) {
            double sum = 0.0;
            for (int b = 0; b < M; ++b) {
                double sab = 0.5 * (s->sigma[a] + s->sigma[b]);
                if (!(sab > 0.0)) continue;
                double gab, d2, d3;
                bmcsl_derivatives(s->sigma[a], s->sigma[b], xi2[i], xi3[i], &gab, &d2, &d3);
                double A = (4.0 * PI / 3.0) * sab * sab * sab * gab;
                for (int c = 0; c < M; ++c) {
                    double sac = 0.5 * (s->sigma[a] + s->sigma[c]);
                    if (!(sac > 0.0)) continue;
                    double gac, e2, e3;
                    bmcsl_derivatives(s->sigma[a], s->sigma[c], xi2[i], xi3[i], &gac, &e2, &e3);
                    double dg = (PI / 6.0) * (s->sigma[b] * s->sigma[b] * e2 +
                                              s->sigma[b] * s->sigma[b] * s->sigma[b] * e3);
                    A += (2.0 * PI / 3.0) * sac * sac * sac * s->n[(long)c * N + i] * dg;
                }
                sum += s->n[(long)a * N + i] * A * Dn[b];
            }
            s->sD[(long)a * N + i] = sum;
            s->Pi[(long)a * N + i] += 0.5 * sum;
        }
    }
    free(xi2);
    free(xi3);
}

/* Moments of the streamed populations and the physical moments (Sec. "Hard
 * sphere fluid mixture", moment equations): n = sum f~, Pi~ = sum g~,
 * J~ = sum c g~, then J and Pi by the reading stated in the header.  The SD
 * schemes take J~ from f~ and have no Pi (set to n); the EU schemes use the
 * plain moments.  Fills s->n, s->gpair, s->Cmf, s->F, s->J, s->Pi. */
static void compute_moments(or_sim *s) {
    long N = s->N;
    int M = s->M;
    compute_forces(s);
    for (int a = 0; a < M; ++a)
        OR_PARALLEL_FOR
        for (long i = 0; i < N; ++i) {
            double nn = 0.0;
            if (!s->solid[i])
                for (int p = 0; p < Q; ++p) nn += s->f[((long)a * Q + p) * N + i];
            s->n[(long)a * N + i] = nn;
        }
    or_contact_values(s->g.n[0], s->g.n[1], s->g.n[2], s->g.per, s->solid, M, s->sigma, s->n, s->gpair);
    or_shell_force(s->g.n[0], s->g.n[1], s->g.n[2], s->g.per, s->solid, M, s->sigma, s->n, s->gpair, s->Cmf);
    if (s->visc) {
        /* C^{visc} of the tilde moments (the collision functional taken at M~): u~ = J~/n */
        for (int a = 0; a < M; ++a)
            OR_PARALLEL_FOR
            for (long i = 0; i < N; ++i) {
                double Jt[3] = {0.0, 0.0, 0.0};
                double nn = s->n[(long)a * N + i];
                if (!s->solid[i])
                    for (int p = 0; p < Q; ++p)
                        for (int c = 0; c < 3; ++c) Jt[c] += CV[p][c] * s->gd[((long)a * Q + p) * N + i];
                for (int c = 0; c < 3; ++c) s->ut[((long)a * 3 + c) * N + i] = nn > 0.0 ? Jt[c] / nn : 0.0;
            }
        or_visc_force(s->g.n[0], s->g.n[1], s->g.n[2], s->g.per, s->solid, M, s->sigma, s->n, s->ut, s->gpair,
                      s->Cvisc);
    }
    for (int a = 0; a < M; ++a)
        OR_PARALLEL_FOR
        for (long i = 0; i < N; ++i) {
            double Pit = 0.0, Jt[3] = {0.0, 0.0, 0.0};
            const double *mom = single_distribution(s) ? s->f : s->gd;
            if (!s->solid[i])
                for (int p = 0; p < Q; ++p) {
                    double gv = mom[((long)a * Q + p) * N + i];
                    Pit += gv;
                    for (int c = 0; c < 3; ++c) Jt[c] += CV[p][c] * gv;
                }
            double nn = s->n[(long)a * N + i];
            double Cm[3], nF[3];
            for (int c = 0; c < 3; ++c) {
                Cm[c] = s->Cmf[((long)a * 3 + c) * N + i];
                /* n F, plus C^{visc} where it is on: the two enter every formula together */
                nF[c] = nn * s->F[((long)a * 3 + c) * N + i] + (s->visc ? s->Cvisc[((long)a * 3 + c) * N + i] : 0.0);
            }
            double J[3];
            for (int c = 0; c < 3; ++c) {
                if (s->scheme == DD_TR)
                    J[c] = s->consistent_moments ? Jt[c] + 0.5 * nF[c] : Jt[c] + 0.5 * (Cm[c] + nF[c]);
                else if (s->scheme == SD_TR)
                    J[c] = Jt[c] + 0.5 * (Cm[c] + nF[c]);
                else
                    J[c] = Jt[c];
            }
            double ua[3];
            for (int c = 0; c < 3; ++c) ua[c] = (nn > 0.0) ? J[c] / nn : 0.0;
            double Cu = Cm[0] * ua[0] + Cm[1] * ua[1] + Cm[2] * ua[2];
            double Pi;
            if (s->scheme == DD_TR)
                Pi = s->consistent_moments ? Pit + 0.5 * BETA * Cu : Pit - 0.5 * Cu;
            else if (s->scheme == DD_EU)
                Pi = Pit;
            else
                Pi = nn;
            if (s->solid[i]) {
                for (int c = 0; c < 3; ++c) J[c] = 0.0;
                Pi = 0.0;
            }
            for (int c = 0; c < 3; ++c) s->J[((long)a * 3 + c) * N + i] = J[c];
            s->Pi[(long)a * N + i] = Pi;
        }
    if (s->scheme == DD_TR && s->consistent_moments == 2)
        dpi_dn_term(s);
    else
        for (long t = 0; t < (long)M * N; ++t) s->sD[t] = 0.0;
}

/* One DD-TR step (Sec. "Hard sphere fluid mixture", trapezoidal two-distribution
 * update): collide f~ and g~ with the explicit TR kernel
 *   f~* = f~ + h [omega (f_eq - f~) + S_f] / (1 + omega h / 2)
 * (derived from f~ = f - h Omega/2 and f~(r + c h, t + h) = f~ + h Omega),
 * then stream with mid-point bounce-back.  The EU schemes collide with
 *   f* = f + (1/tau)(f_eq - f) + h S_f  (Sec. "Ideal fluid", Euler update);
 * the SD schemes collide f only and copy it to g. */
static void one_step(or_sim *s) {
    long N = s->N;
    int M = s->M;
    compute_moments(s);

    /* time-averaged flux through the configured plane, from the physical J */
    if (s->flux_plane >= 0) {
        for (int a = 0; a < M; ++a) {
            double sum = 0.0;
            for (long i = 0; i < N; ++i) {
                int r[3];
                coords(&s->g, i, &r[0], &r[1], &r[2]);
                if (r[s->flux_axis] == s->flux_plane && !s->solid[i])
                    sum += s->J[((long)a * 3 + s->flux_axis) * N + i];
            }
            s->flux_sum[a] += sum;
        }
        s->flux_count += 1;
    }

    OR_PARALLEL_FOR
    for (long i = 0; i < N; ++i) {
        if (s->solid[i]) {
            for (int a = 0; a < M; ++a)
                for (int p = 0; p < Q; ++p) {
                    s->fpost[((long)a * Q + p) * N + i] = 0.0;
                    s->gpost[((long)a * Q + p) * N + i] = 0.0;
                }
            continue;
        }
        /* barycentric velocity u = sum_a J^a / sum_a n^a */
        double ntot = 0.0, Jtot[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < M; ++a) {
            ntot += s->n[(long)a * N + i];
            for (int c = 0; c < 3; ++c) Jtot[c] += s->J[((long)a * 3 + c) * N + i];
        }
        double u[3];
        for (int c = 0; c < 3; ++c) u[c] = (ntot > 0.0) ? Jtot[c] / ntot : 0.0;

        for (int a = 0; a < M; ++a) {
            double nn = s->n[(long)a * N + i];
            double Pi = s->Pi[(long)a * N + i];
            double ua[3], Cm[3], nF[3];
            for (int c = 0; c < 3; ++c) {
                ua[c] = (nn > 0.0) ? s->J[((long)a * 3 + c) * N + i] / nn : 0.0;
                Cm[c] = s->Cmf[((long)a * 3 + c) * N + i];
                nF[c] = nn * s->F[((long)a * 3 + c) * N + i] + (s->visc ? s->Cvisc[((long)a * 3 + c) * N + i] : 0.0);
            }
            double omega = 1.0 / (s->tau[a] - 0.5); /* omega h, h = 1 (TR) */
            double omega_eu = 1.0 / s->tau[a];       /* omega h of the Euler update */
            for (int p = 0; p < Q; ++p) {
                double H1[3], H2[3][3];
                hermite(p, H1, H2);
                double wp = weight_of(p);
                /* f_eq and g_eq (Eqs. for f^{a,eq}, g^{a,eq}) */
                double t1 = 0.0, t2 = 0.0;
                for (int c = 0; c < 3; ++c) t1 += nn * ua[c] * H1[c];
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) t2 += nn * (2.0 * ua[c] * u[d] - u[c] * u[d]) * H2[c][d];
                double feq = wp * (nn + t1 + t2);
                double geq = wp * (Pi + t1 + t2);
                /* H2 . u^a */
                double H2u[3];
                for (int c = 0; c < 3; ++c) {
                    H2u[c] = 0.0;
                    for (int d = 0; d < 3; ++d) H2u[c] += H2[c][d] * ua[d];
                }
                /* S_f = w_p (C^mf + n F) . [H1 + 2 H2 . u^a] */
                double Sf = 0.0;
                for (int c = 0; c < 3; ++c) Sf += (Cm[c] + nF[c]) * (H1[c] + 2.0 * H2u[c]);
                Sf *= wp;
                /* S_g = w_p { C^mf . [u^a / v_T^2 + 4 H2 . u^a] + n F . [H1 + 2 H2 . u^a] + s^a },
                 * s^a the d Pi/d n term where it is on (zero otherwise) */
                double Sg = 0.0;
                for (int c = 0; c < 3; ++c)
                    Sg += Cm[c] * (ua[c] / CS2 + 4.0 * H2u[c]) + nF[c] * (H1[c] + 2.0 * H2u[c]);
                Sg += s->sD[(long)a * N + i];
                Sg *= wp;
                long k = ((long)a * Q + p) * N + i;
                double ft = s->f[k], gt = s->gd[k];
                if (trapezoidal(s)) {
                    s->fpost[k] = ft + (omega * (feq - ft) + Sf) / (1.0 + 0.5 * omega);
                    s->gpost[k] = gt + (omega * (geq - gt) + Sg) / (1.0 + 0.5 * omega);
                } else {
                    s->fpost[k] = ft + omega_eu * (feq - ft) + Sf;
                    s->gpost[k] = gt + omega_eu * (geq - gt) + Sg;
                }
                if (single_distribution(s)) s->gpost[k] = s->fpost[k];
            }
        }
    }

    /* densities of this step and the one before, for the d Pi/d n term */
    memcpy(s->nh2, s->nh1, sizeof(double) * M * N);
    memcpy(s->nh1, s->n, sizeof(double) * M * N);
    if (s->nhist < 2) s->nhist += 1;

    /* streaming f~(r, t+1) = f~*(r - c_p), mid-point bounce-back on blocked links */
    for (int a = 0; a < M; ++a)
        OR_PARALLEL_FOR
        for (long i = 0; i < N; ++i) {
            int x, y, z;
            coords(&s->g, i, &x, &y, &z);
            for (int p = 0; p < Q; ++p) {
                long k = ((long)a * Q + p) * N + i;
                if (s->solid[i]) {
                    s->f[k] = 0.0;
                    s->gd[k] = 0.0;
                    continue;
                }
                long src = site(&s->g, x - CV[p][0], y - CV[p][1], z - CV[p][2]);
                if (src < 0 || s->solid[src]) {
                    long kb = ((long)a * Q + opposite(p)) * N + i;
                    s->f[k] = s->fpost[kb];
                    s->gd[k] = s->gpost[kb];
                } else {
                    long ks = ((long)a * Q + p) * N + src;
                    s->f[k] = s->fpost[ks];
                    s->gd[k] = s->gpost[ks];
                }
            }
        }
    s->steps += 1;
}

int or_step(or_sim *s, int nsteps) {
    for (int t = 0; t < nsteps; ++t) one_step(s);
    return 0;
}

/* Observables of the current (streamed) state: n [M][N], physical J [M][3][N],
 * C^mf [M][3][N], Pi [M][N], F [M][3][N], g_ab [M][M][N].  Any pointer may be NULL. */
int or_observe(or_sim *s, double *n, double *J, double *C, double *Pi, double *F, double *gpair) {
    compute_moments(s);
    long N = s->N;
    int M = s->M;
    if (n) memcpy(n, s->n, sizeof(double) * M * N);
    if (J) memcpy(J, s->J, sizeof(double) * M * 3 * N);
    if (C) memcpy(C, s->Cmf, sizeof(double) * M * 3 * N);
    if (Pi) memcpy(Pi, s->Pi, sizeof(double) * M * N);
    if (F) memcpy(F, s->F, sizeof(double) * M * 3 * N);
    if (gpair) memcpy(gpair, s->gpair, sizeof(double) * M * M * N);
    return 0;
}

/* Per-species running flux sum and the number of steps it holds. */
int or_get_flux(or_sim *s, double *flux_sum, long *count) {
    for (int a = 0; a < s->M; ++a) flux_sum[a] = s->flux_sum[a];
    *count = s->flux_count;
    return 0;
}

long or_steps_done(or_sim *s) { return s->steps; }
