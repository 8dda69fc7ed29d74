/*
 * FP64 CPU oracle for the implicit TDGL step of Sadovskyy, Koshelev, Phillips,
 * Karpeyev & Glatz, "Stable large-scale solver for Ginzburg-Landau equations
 * for superconductors" (arXiv:1409.8340).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links or calls this
 * file; it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark can compare the CUDA implementation against a plain, slow,
 * obviously correct restatement of the paper's discretisation.
 *
 * Every routine works site by site in the paper's own notation, in double
 * precision, with no blocking, fusion or reordering.  Loops over sites may run
 * in parallel (OpenMP); every reduction is a serial sum in index order.
 *
 * Grid: m = i + Nx*(j + Ny*k), x fastest (Sec. 3, discretisation of the
 * coordinates).  Complex arrays are interleaved (re, im) doubles.
 *
 * Field in the yz plane, large-lambda Landau gauge A = xbar [0, Bz, -By]
 * (Sec. 2.3, Eq. A_yz) with xbar = x - Lx/2, generalised potential
 * A~ = A - K xhat (Sec. 2.2), link variables U = exp(-i h A~) (Eq. link_variables).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { OR_PERIODIC = 0, OR_OPEN = 1 };

typedef struct {
    int32_t n[3];      /* Nx, Ny, Nz                                      */
    int32_t bc[3];     /* OR_PERIODIC or OR_OPEN per axis                  */
    double h[3];       /* hx, hy, hz                                      */
    double g;          /* anisotropy: z terms carry 1/g^2 (Sec. 2.1)       */
    double u;          /* relaxation constant u (Eq. GL_dimensionless)     */
    double beta;       /* coefficient of |psi|^2 psi (1 in the paper)      */
    double ht;         /* time step h_t (Eq. GL_numCN)                     */
    double By, Bz;     /* field components, yz plane (Eq. B_yz)            */
    double Jext;       /* applied current along x                          */
    const uint8_t *ins; /* insulating sites (Sec. 3.4 (ii)), u8[N]; NULL: none */
} or_grid;

static inline int64_t idx3(const or_grid *G, int i, int j, int k)
{
    return (int64_t)i + (int64_t)G->n[0] * ((int64_t)j + (int64_t)G->n[1] * (int64_t)k);
}

static inline int axis_active(const or_grid *G, int ax) { return G->n[ax] >= 2; }

/* Coefficient 1/h_a^2, with the 1/g^2 of the z axis (Eq. LaplUV_yz). */
static inline double axis_coef(const or_grid *G, int ax)
{
    double c = 1.0 / (G->h[ax] * G->h[ax]);
    if (ax == 2) c /= G->g * G->g;
    return c;
}

static double box_length(const or_grid *G, int ax)
{
    /* h = L/N (periodic) or L/(N-1) (open), Sec. 3 */
    return G->bc[ax] == OR_PERIODIC ? G->n[ax] * G->h[ax] : (G->n[ax] - 1) * G->h[ax];
}

/*
 * Forward link U_{ax}(i,j,k) from site (i,j,k) to its +ax neighbour.
 * theta != NULL: explicit link phases theta[ax*N + m] (gauge-test mode), times
 * exp(i hx K) on x links.  theta == NULL: Landau gauge of Eq. A_yz:
 *   U_x = exp(i hx K)                                 (A~_x = -K)
 *   U_y(i) = exp(-i hy Bz xbar_i)                     (A~_y = xbar Bz)
 *   U_z(i) = exp(+i hz By xbar_i)                     (A~_z = -xbar By)
 * and for periodic x the wrap link from i = Nx-1 to i = 0 carries conj(P_{j,k}),
 * P_{j,k} = exp(i(-j hy Lx Bz + k hz Lx By)) (Sec. 3.3.1, yz-field paragraph).
 */
static cplx link(const or_grid *G, const double *theta, double K, int ax, int i, int j, int k)
{
    if (theta) {
        int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
        cplx U = cexp(I * theta[ax * N + idx3(G, i, j, k)]);
        if (ax == 0) U *= cexp(I * G->h[0] * K);
        return U;
    }
    double Lx = box_length(G, 0);
    double xbar = i * G->h[0] - 0.5 * Lx;
    if (ax == 0) {
        cplx U = cexp(I * G->h[0] * K);
        if (G->bc[0] == OR_PERIODIC && i == G->n[0] - 1) {
            double phase = -j * G->h[1] * Lx * G->Bz + k * G->h[2] * Lx * G->By;
            U *= cexp(-I * phase);
        }
        return U;
    }
    if (ax == 1) return cexp(-I * G->h[1] * G->Bz * xbar);
    return cexp(I * G->h[2] * G->By * xbar);
}

static inline cplx load(const double *a, int64_t m) { return a[2 * m] + I * a[2 * m + 1]; }
static inline void store(double *a, int64_t m, cplx v) { a[2 * m] = creal(v); a[2 * m + 1] = cimag(v); }

static void step_index(const or_grid *G, int ax, int sgn, int c[3])
{
    c[ax] += sgn;
    if (c[ax] < 0) c[ax] += G->n[ax];
    if (c[ax] >= G->n[ax]) c[ax] -= G->n[ax];
}

/*
 * Insulating inclusions (Sec. 3.4 (ii)): no current crosses an internal edge
 * next to an insulating site.  Reading: a link that touches an insulating
 * site is removed from every link sum (the stencil of psi, its diagonal, the
 * Poisson operator and right-hand side, J_av, the energy); insulating sites
 * themselves hold psi = 0 and mu = 0.  Without insulating sites every factor
 * below is 1 and the operators are the plain ones.
 */
static inline int insulating(const or_grid *G, int i, int j, int k)
{
    return G->ins && G->ins[idx3(G, i, j, k)];
}

/* 1 if the link from (i,j,k) one step sgn along ax exists (inside the grid or
 * across a periodic wrap) and joins two conducting sites */
static double link_ok(const or_grid *G, int ax, int sgn, int i, int j, int k)
{
    int c[3] = {i, j, k};
    if (G->bc[ax] == OR_OPEN && ((sgn > 0 && c[ax] == G->n[ax] - 1) || (sgn < 0 && c[ax] == 0))) return 0.0;
    if (!G->ins) return 1.0;
    if (insulating(G, i, j, k)) return 0.0;
    step_index(G, ax, sgn, c);
    return insulating(G, c[0], c[1], c[2]) ? 0.0 : 1.0;
}

/*
 * Neighbour sum NS_m(psi) = sum over axes of c_a (U_a psi_{m+a} + U*_{a,m-a} psi_{m-a}),
 * where at an open face the missing neighbour is replaced by the Neumann ghost
 * (Sec. 3.3.2), which gives 2 c_a U psi_1 at index 0 and 2 c_a U* psi_{N-2}
 * at index N-1.  The gauge Laplacian of Eq. LaplUV_yz is NS_m - 2 S psi_m
 * with S = sum_a c_a.
 */
static cplx neighbour_sum(const or_grid *G, const double *theta, double K, const double *psi,
                          int i, int j, int k)
{
    cplx acc = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        if (!axis_active(G, ax)) continue;
        int c0[3] = {i, j, k};
        int idx = c0[ax];
        int n = G->n[ax];
        double c = axis_coef(G, ax);
        int cp[3] = {i, j, k}, cm[3] = {i, j, k};
        step_index(G, ax, +1, cp);
        step_index(G, ax, -1, cm);
        cplx fwd = link_ok(G, ax, +1, i, j, k) * link(G, theta, K, ax, i, j, k) * load(psi, idx3(G, cp[0], cp[1], cp[2]));
        cplx bwd = link_ok(G, ax, -1, i, j, k) * conj(link(G, theta, K, ax, cm[0], cm[1], cm[2])) *
                   load(psi, idx3(G, cm[0], cm[1], cm[2]));
        if (G->bc[ax] == OR_PERIODIC) {
            acc += c * (fwd + bwd);
        } else if (idx == 0) {
            acc += 2.0 * c * fwd;
        } else if (idx == n - 1) {
            acc += 2.0 * c * bwd;
        } else {
            acc += c * (fwd + bwd);
        }
    }
    return acc;
}

/* Diagonal weight of the gauge Laplacian at a site: sum over its links of c_a
 * (the ghost doubles the one link of an open face); 2S without insulators. */
static double diag_sum(const or_grid *G, int i, int j, int k)
{
    double acc = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        if (!axis_active(G, ax)) continue;
        int c0[3] = {i, j, k};
        double c = axis_coef(G, ax), f = link_ok(G, ax, +1, i, j, k), b = link_ok(G, ax, -1, i, j, k);
        if (G->bc[ax] == OR_PERIODIC) acc += c * (f + b);
        else if (c0[ax] == 0) acc += 2.0 * c * f;
        else if (c0[ax] == G->n[ax] - 1) acc += 2.0 * c * b;
        else acc += c * (f + b);
    }
    return acc;
}

static double sum_coef(const or_grid *G)
{
    double S = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        if (axis_active(G, ax)) S += axis_coef(G, ax);
    return S;
}

/* ------------------------------------------------------------------------ */
/* Public: link phase of the Landau gauge, for building gauge-test links.   */
/* theta_out[ax*N + m] = arg of the Landau link at K = 0 (unwrapped phase).  */
/* ------------------------------------------------------------------------ */
void or_landau_link_phases(const or_grid *G, double *theta_out)
{
    int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    double Lx = box_length(G, 0);
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                double xbar = i * G->h[0] - 0.5 * Lx;
                double tx = 0.0;
                if (G->bc[0] == OR_PERIODIC && i == G->n[0] - 1)
                    tx = -(-j * G->h[1] * Lx * G->Bz + k * G->h[2] * Lx * G->By);
                theta_out[m] = tx;
                theta_out[N + m] = -G->h[1] * G->Bz * xbar;
                theta_out[2 * N + m] = G->h[2] * G->By * xbar;
            }
}

/* ------------------------------------------------------------------------ */
/* Link phases of the other Landau gauge, field in the xz plane (Eq. B_xz,  */
/* Eq. A_xz: A = ybar [-Bz, 0, Bx], ybar = j hy - Ly/2), for the explicit-    */
/* link mode (K is added to the x links by link()):                          */
/*   U_x(j) = exp(i hx Bz ybar_j),  U_y = 1,  U_z(j) = exp(-i hz Bx ybar_j);  */
/* on a periodic y axis the wrap link from j = Ny-1 to j = 0 carries          */
/* conj(P_{i,k}), P_{i,k} = exp(i(i hx Ly Bz - k hz Ly Bx)) (Sec. 3.3.1,      */
/* xz-field paragraph: psi_{i,-1,k} = P_{i,k} psi_{i,Ny-1,k}).                */
/* ------------------------------------------------------------------------ */
void or_xz_link_phases(const or_grid *G, double Bx, double *theta_out)
{
    int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    double Ly = box_length(G, 1);
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                double ybar = j * G->h[1] - 0.5 * Ly;
                double ty = 0.0;
                if (G->bc[1] == OR_PERIODIC && j == G->n[1] - 1)
                    ty = -(i * G->h[0] * Ly * G->Bz - k * G->h[2] * Ly * Bx);
                theta_out[m] = G->h[0] * G->Bz * ybar;
                theta_out[N + m] = ty;
                theta_out[2 * N + m] = -G->h[2] * Bx * ybar;
            }
}

/* ------------------------------------------------------------------------ */
/* Init: diagonal M_mm and right-hand side b_m (Sec. 3.1, matrix M, Eq. b),  */
/* with psi_est = psi^- and no noise.                                       */
/*   M_mm = 1 + (ht/2)[beta|psi^-|^2 + 2S + i u mu - alpha]                  */
/*   b_m  = psi^- + (ht/2)[(alpha - i u mu) psi^- - beta|psi^-|^2 psi^-      */
/*                         + Lap_U psi^-]                                    */
/* ------------------------------------------------------------------------ */
void or_init(const or_grid *G, const double *theta, double K, const double *psi_prev,
             const double *mu, const double *alpha, double *b, double *D)
{
    double S = sum_coef(G);
    double ht2 = 0.5 * G->ht;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                if (insulating(G, i, j, k)) {   /* psi = 0: b = 0, M_mm = 1, no links */
                    store(D, m, 1.0);
                    store(b, m, 0.0);
                    continue;
                }
                cplx p = load(psi_prev, m);
                double a2 = creal(p) * creal(p) + cimag(p) * cimag(p);
                const double S2 = G->ins ? diag_sum(G, i, j, k) : 2.0 * S;
                cplx lap = neighbour_sum(G, theta, K, psi_prev, i, j, k) - S2 * p;
                cplx Dm = 1.0 + ht2 * (G->beta * a2 + S2 + I * G->u * mu[m] - alpha[m]);
                cplx bm = p + ht2 * ((alpha[m] - I * G->u * mu[m]) * p - G->beta * a2 * p + lap);
                store(D, m, Dm);
                store(b, m, bm);
            }
}

/* ------------------------------------------------------------------------ */
/* Thermal noise (Sec. 3.1.2): b_m gains (h_t/2) 2 zeta_m = h_t zeta_m with   */
/* zeta = zeta_max (v1 + i v2), v1 and v2 independent and uniform on [-1, 1), */
/* fresh for every site m and time step n.  The random numbers come from the  */
/* counter-based generator Philox4x32 with 10 rounds (Salmon, Moraes, Dror &  */
/* Shaw, SC'11), counter (m, n) and key = the seed: each 32-bit output x      */
/* gives v = (x >> 8) 2^-23 - 1, exact in single precision.                   */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    for (int q = 0; q < 4; ++q) out[q] = c[q];
}

void or_noise(const or_grid *G, double amp, uint64_t seed, int64_t step, double *b)
{
    const int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < N; ++m) {
        if (G->ins && G->ins[m]) continue;   /* insulating sites hold psi = 0 */
        const uint32_t ctr[4] = {(uint32_t)m, (uint32_t)((uint64_t)m >> 32), (uint32_t)step,
                                 (uint32_t)((uint64_t)step >> 32)};
        uint32_t x[4];
        or_philox4x32_10(ctr, key, x);
        const double v1 = ldexp((double)(x[0] >> 8), -23) - 1.0;
        const double v2 = ldexp((double)(x[1] >> 8), -23) - 1.0;
        b[2 * m] += amp * v1;
        b[2 * m + 1] += amp * v2;
    }
}

/* ------------------------------------------------------------------------ */
/* One Jacobi sweep (Eq. final) and the residual of its input iterate        */
/* (Eq. convergence): r^(l) = b - M psi^(l).                                 */
/* Off-diagonal entries of M are -(ht/2) times the neighbour coefficients.   */
/* Returns max_m |r_m|^2.                                                    */
/* ------------------------------------------------------------------------ */
double or_sweep(const or_grid *G, const double *theta, double K, const double *psi_in,
                const double *b, const double *D, double *psi_out)
{
    int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    double ht2 = 0.5 * G->ht;
    double *r2 = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                cplx offdiag = -ht2 * neighbour_sum(G, theta, K, psi_in, i, j, k); /* sum_{m'!=m} M psi */
                cplx Dm = load(D, m);
                cplx bm = load(b, m);
                cplx r = bm - (Dm * load(psi_in, m) + offdiag);
                store(psi_out, m, (bm - offdiag) / Dm);
                r2[m] = creal(r) * creal(r) + cimag(r) * cimag(r);
            }
    double mx = 0.0;
    for (int64_t m = 0; m < N; ++m)
        if (r2[m] > mx) mx = r2[m];
    free(r2);
    return mx;
}

/* Residual b - M psi for a given iterate (for tests). */
void or_residual(const or_grid *G, const double *theta, double K, const double *psi,
                 const double *b, const double *D, double *r_out)
{
    double ht2 = 0.5 * G->ht;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                cplx offdiag = -ht2 * neighbour_sum(G, theta, K, psi, i, j, k);
                store(r_out, m, load(b, m) - (load(D, m) * load(psi, m) + offdiag));
            }
}

/* ------------------------------------------------------------------------ */
/* Supercurrent mean along x (Sec. 3.1.1, J_av):                             */
/*   J_av = 1/(2 N hx) sum_m Im[psi*_m (U_x psi_{i+1} - U*_x psi_{i-1})]     */
/* Defined for periodic x (the paper's current formulation).                 */
/* ------------------------------------------------------------------------ */
double or_javg(const or_grid *G, const double *theta, double K, const double *psi)
{
    int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    double s = 0.0;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int c[3] = {i, j, k};
                int cp[3] = {i, j, k}, cm[3] = {i, j, k};
                step_index(G, 0, +1, cp);
                step_index(G, 0, -1, cm);
                cplx p = load(psi, idx3(G, c[0], c[1], c[2]));
                cplx fwd = link_ok(G, 0, +1, i, j, k) * link(G, theta, K, 0, i, j, k) *
                           load(psi, idx3(G, cp[0], cp[1], cp[2]));
                cplx bwd = link_ok(G, 0, -1, i, j, k) * conj(link(G, theta, K, 0, cm[0], cm[1], cm[2])) *
                           load(psi, idx3(G, cm[0], cm[1], cm[2]));
                s += cimag(conj(p) * (fwd - bwd));
            }
    return s / (2.0 * (double)N * G->h[0]);
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of the Poisson equation (Sec. 3.2, Eq. Poisson):          */
/*   f_m = sum_a c_a Im[psi*_m (U_a psi_{m+a} + U*_{a,m-a} psi_{m-a})]       */
/* i.e. Im[psi*_m NS_m(psi)], with the Neumann ghost at open faces.          */
/* ------------------------------------------------------------------------ */
void or_poisson_rhs(const or_grid *G, const double *theta, double K, const double *psi, double *f)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                f[m] = cimag(conj(load(psi, m)) * neighbour_sum(G, theta, K, psi, i, j, k));
            }
}

/* ------------------------------------------------------------------------ */
/* Discrete scalar Laplacian of Sec. 3.2 (left-hand side), with periodic     */
/* wrap or the Neumann ghost mu_{-1} = mu_1 at open faces.  For tests.       */
/* ------------------------------------------------------------------------ */
void or_laplacian_mu(const or_grid *G, const double *mu, double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                double acc = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    if (!axis_active(G, ax)) continue;
                    int c0[3] = {i, j, k};
                    int cp[3] = {i, j, k}, cm[3] = {i, j, k};
                    step_index(G, ax, +1, cp);
                    step_index(G, ax, -1, cm);
                    const double okp = link_ok(G, ax, +1, i, j, k), okm = link_ok(G, ax, -1, i, j, k);
                    double vp = okp * (mu[idx3(G, cp[0], cp[1], cp[2])] - mu[m]);
                    double vm = okm * (mu[idx3(G, cm[0], cm[1], cm[2])] - mu[m]);
                    if (G->bc[ax] == OR_OPEN) {
                        if (c0[ax] == 0) vm = vp;
                        if (c0[ax] == G->n[ax] - 1) vp = vm;
                    }
                    acc += axis_coef(G, ax) * (vp + vm);
                }
                out[m] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* Discrete free energy (the paper refers to F_GL, Sec. 2.1, but does not    */
/* write its discrete form).  Trapezoid weights w = product of 1/2 per open  */
/* face the site (or link) lies on, so that dF/dpsi*_m = w_m(-alpha psi +    */
/* beta|psi|^2 psi - Lap_U psi) dV exactly:                                  */
/*   F = dV { sum_m w_m[-alpha|psi|^2 + beta/2 |psi|^4]                      */
/*          + sum_links w_l c_a |U psi_{m+a} - psi_m|^2 }                    */
/* ------------------------------------------------------------------------ */
static double face_weight(const or_grid *G, int ax, int idx)
{
    if (G->bc[ax] == OR_OPEN && axis_active(G, ax) && (idx == 0 || idx == G->n[ax] - 1)) return 0.5;
    return 1.0;
}

double or_energy(const or_grid *G, const double *theta, double K, const double *psi, const double *alpha)
{
    double dV = 1.0;
    for (int ax = 0; ax < 3; ++ax)
        if (axis_active(G, ax)) dV *= G->h[ax];
    double F = 0.0;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int c[3] = {i, j, k};
                int64_t m = idx3(G, i, j, k);
                cplx p = load(psi, m);
                double a2 = creal(p) * creal(p) + cimag(p) * cimag(p);
                double w = face_weight(G, 0, i) * face_weight(G, 1, j) * face_weight(G, 2, k);
                F += w * (-alpha[m] * a2 + 0.5 * G->beta * a2 * a2);
                for (int ax = 0; ax < 3; ++ax) {
                    if (!axis_active(G, ax)) continue;
                    if (G->bc[ax] == OR_OPEN && c[ax] == G->n[ax] - 1) continue; /* no link beyond the face */
                    int cp[3] = {i, j, k};
                    step_index(G, ax, +1, cp);
                    double wl = 1.0;
                    for (int o = 0; o < 3; ++o)
                        if (o != ax) wl *= face_weight(G, o, c[o]);
                    cplx d = link(G, theta, K, ax, i, j, k) * load(psi, idx3(G, cp[0], cp[1], cp[2])) - p;
                    F += link_ok(G, ax, +1, i, j, k) * wl * axis_coef(G, ax) * (creal(d) * creal(d) + cimag(d) * cimag(d));
                }
            }
    return F * dV;
}

/* ------------------------------------------------------------------------ */
/* Vortex winding of xy plaquettes.  theta_ab = arg(psi*_a U_ab psi_b) in     */
/* (-pi, pi]; n_p = round((sum of the four theta + hx hy Bz) / 2 pi).        */
/* Writes per-plaquette integers (Nx*Ny*Nz, zero where no plaquette exists). */
/* Returns the signed total.                                                 */
/* ------------------------------------------------------------------------ */
int64_t or_winding(const or_grid *G, const double *theta, double K, const double *psi, int32_t *n_out)
{
    int nx = G->n[0], ny = G->n[1], nz = G->n[2];
    double flux = G->h[0] * G->h[1] * G->Bz;
    int64_t total = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t m = idx3(G, i, j, k);
                n_out[m] = 0;
                if (G->bc[0] == OR_OPEN && i == nx - 1) continue;
                if (G->bc[1] == OR_OPEN && j == ny - 1) continue;
                int a[3] = {i, j, k};
                int bb[3] = {i, j, k};
                step_index(G, 0, +1, bb);
                int d[3] = {i, j, k};
                step_index(G, 1, +1, d);
                int c[3] = {bb[0], bb[1], bb[2]};
                step_index(G, 1, +1, c);
                /* plaquettes with an insulating corner hold no winding */
                if (insulating(G, a[0], a[1], a[2]) || insulating(G, bb[0], bb[1], bb[2]) ||
                    insulating(G, c[0], c[1], c[2]) || insulating(G, d[0], d[1], d[2]))
                    continue;
                cplx pa = load(psi, idx3(G, a[0], a[1], a[2]));
                cplx pb = load(psi, idx3(G, bb[0], bb[1], bb[2]));
                cplx pc = load(psi, idx3(G, c[0], c[1], c[2]));
                cplx pd = load(psi, idx3(G, d[0], d[1], d[2]));
                double t_ab = carg(conj(pa) * link(G, theta, K, 0, a[0], a[1], a[2]) * pb);
                double t_bc = carg(conj(pb) * link(G, theta, K, 1, bb[0], bb[1], bb[2]) * pc);
                double t_cd = carg(conj(pc) * conj(link(G, theta, K, 0, d[0], d[1], d[2])) * pd);
                double t_da = carg(conj(pd) * conj(link(G, theta, K, 1, a[0], a[1], a[2])) * pa);
                double w = (t_ab + t_bc + t_cd + t_da + flux) / (2.0 * M_PI);
                int32_t np = (int32_t)floor(w + 0.5);
                n_out[m] = np;
                total += np;
            }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Inclusion pattern generator (Sec. 3.4).  Candidates are consumed in      */
/* order; a site at r = (i hx, j hy, k hz) is inside candidate n when        */
/*   q = d^T R diag(a^-2) R^T d <= 1,  d = r - c,                             */
/* with the minimum-image convention d -= L floor(d/L + 1/2) on periodic     */
/* axes.  R is the rotation of the unit quaternion (q0,q1,q2,q3).  A site is */
/* marked by the first candidate that contains it; candidates are added      */
/* until at least `target` sites are marked (target <= 0: use all).          */
/* alpha = alpha_in on marked sites, alpha_out elsewhere.                    */
/* Returns the number of candidates used; *marked receives the site count.   */
/* ------------------------------------------------------------------------ */
static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static double inside_q(const or_grid *G, const double *inc, int i, int j, int k)
{
    double r[3] = {i * G->h[0], j * G->h[1], k * G->h[2]};
    double d[3];
    for (int ax = 0; ax < 3; ++ax) {
        d[ax] = r[ax] - inc[ax];
        if (G->bc[ax] == OR_PERIODIC) {
            double L = G->n[ax] * G->h[ax];
            d[ax] -= L * floor(d[ax] / L + 0.5);
        }
    }
    double R[3][3];
    quat_to_rot(inc + 6, R);
    double q = 0.0;
    for (int a = 0; a < 3; ++a) {
        /* body-frame coordinate: column a of R dotted with d */
        double e = R[0][a] * d[0] + R[1][a] * d[1] + R[2][a] * d[2];
        double s = e / inc[3 + a];
        q += s * s;
    }
    return q;
}

int64_t or_pattern(const or_grid *G, const double *incl, int64_t n_incl, int64_t target,
                   double alpha_in, double alpha_out, double *alpha, int64_t *marked_out)
{
    int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    unsigned char *mark = (unsigned char *)calloc((size_t)N, 1);
    int64_t marked = 0, used = 0;
    for (int64_t n = 0; n < n_incl; ++n) {
        if (target > 0 && marked >= target) break;
        const double *inc = incl + 10 * n;
        double rmax = inc[3];
        if (inc[4] > rmax) rmax = inc[4];
        if (inc[5] > rmax) rmax = inc[5];
        int lo[3], hi[3];
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = (int)ceil((inc[ax] - rmax) / G->h[ax]);
            hi[ax] = (int)floor((inc[ax] + rmax) / G->h[ax]);
            if (G->bc[ax] == OR_OPEN) {
                if (lo[ax] < 0) lo[ax] = 0;
                if (hi[ax] > G->n[ax] - 1) hi[ax] = G->n[ax] - 1;
            } else if (hi[ax] - lo[ax] + 1 > G->n[ax]) {
                lo[ax] = 0;
                hi[ax] = G->n[ax] - 1;
            }
        }
        for (int kk = lo[2]; kk <= hi[2]; ++kk)
            for (int jj = lo[1]; jj <= hi[1]; ++jj)
                for (int ii = lo[0]; ii <= hi[0]; ++ii) {
                    int i = ((ii % G->n[0]) + G->n[0]) % G->n[0];
                    int j = ((jj % G->n[1]) + G->n[1]) % G->n[1];
                    int k = ((kk % G->n[2]) + G->n[2]) % G->n[2];
                    int64_t m = idx3(G, i, j, k);
                    if (mark[m]) continue;
                    if (inside_q(G, inc, i, j, k) <= 1.0) {
                        mark[m] = 1;
                        ++marked;
                    }
                }
        used = n + 1;
    }
    for (int64_t m = 0; m < N; ++m) alpha[m] = mark[m] ? alpha_in : alpha_out;
    free(mark);
    if (marked_out) *marked_out = marked;
    return used;
}

/* Plain inside test value q for one site and one inclusion (for tests). */
double or_inside_q(const or_grid *G, const double *inc, int i, int j, int k)
{
    return inside_q(G, inc, i, j, k);
}

/* ------------------------------------------------------------------------ */
/* Pattern generator, full form (Sec. 3.4): pinning landscapes built from     */
/* shapes (rectangles/cuboids, circles/spheres/ellipsoids, crosses, octants,  */
/* cylinders), lattices of a shape (square, triangular, honeycomb, kagome,    */
/* rectangular, hexagonal), a shape that claims its outside (a shaped         */
/* integration domain), and tessellations (checkerboard, Voronoi with the     */
/* Euclidean, absolute or maximum distance) as the background.               */
/*                                                                            */
/* A shape is 13 doubles: kind, flags, centre c[3], semi-axes a[3],           */
/* quaternion q[4] (body -> lab), value.  Site (i,j,k) sits at (i hx, j hy,   */
/* k hz); d = r - c with the minimum image on periodic axes; body coordinates */
/* e_a = sum_r R[r][a] d_r.  A site takes the value of the first shape (in    */
/* list order) that claims it; shapes are taken in order while fewer than     */
/* `target` sites are claimed (target <= 0: all).  Unclaimed sites take the   */
/* background.  flags bit 0: the shape claims its outside; bit 1: claimed     */
/* sites are insulating.                                                      */
/* ------------------------------------------------------------------------ */
enum { OR_ELLIPSOID = 0, OR_CUBOID = 1, OR_CYLINDER = 2, OR_CROSS = 3, OR_OCTANT = 4 };
enum { OR_INVERT = 1, OR_INSULATING = 2 };
enum { OR_BG_CONSTANT = 0, OR_BG_CHECKER = 1, OR_BG_VORONOI = 2 };
enum { OR_EUCLIDEAN = 0, OR_ABSOLUTE = 1, OR_MAXIMUM = 2 };
enum { OR_SQUARE = 0, OR_TRIANGULAR = 1, OR_HONEYCOMB = 2, OR_KAGOME = 3, OR_RECTANGULAR = 4, OR_HEXAGONAL = 5 };

static void min_image(const or_grid *G, const double *c, int i, int j, int k, double d[3])
{
    double r[3] = {i * G->h[0], j * G->h[1], k * G->h[2]};
    for (int ax = 0; ax < 3; ++ax) {
        d[ax] = r[ax] - c[ax];
        if (G->bc[ax] == OR_PERIODIC) {
            double L = G->n[ax] * G->h[ax];
            d[ax] -= L * floor(d[ax] / L + 0.5);
        }
    }
}

/* 1 if the shape contains site (i,j,k) (before the invert flag) */
int or_shape_contains(const or_grid *G, const double *sh, int i, int j, int k)
{
    const int kind = (int)sh[0];
    const double *c = sh + 2, *a = sh + 5, *q = sh + 8;
    double d[3], R[3][3], e[3];
    min_image(G, c, i, j, k, d);
    quat_to_rot(q, R);
    for (int b = 0; b < 3; ++b) e[b] = R[0][b] * d[0] + R[1][b] * d[1] + R[2][b] * d[2];
    double s0 = e[0] / a[0], s1 = e[1] / a[1], s2 = e[2] / a[2];
    switch (kind) {
    case OR_ELLIPSOID: return s0 * s0 + s1 * s1 + s2 * s2 <= 1.0;
    case OR_CUBOID: return fabs(e[0]) <= a[0] && fabs(e[1]) <= a[1] && fabs(e[2]) <= a[2];
    case OR_CYLINDER: return s0 * s0 + s1 * s1 <= 1.0 && fabs(e[2]) <= a[2];
    case OR_CROSS:
        return (fabs(e[0]) <= a[0] && fabs(e[1]) <= a[1] && fabs(e[2]) <= a[2]) ||
               (fabs(e[0]) <= a[1] && fabs(e[1]) <= a[0] && fabs(e[2]) <= a[2]);
    case OR_OCTANT: return e[0] >= 0.0 && e[1] >= 0.0 && e[2] >= 0.0 && s0 * s0 + s1 * s1 + s2 * s2 <= 1.0;
    default: return 0;
    }
}

/* Lattice (24 doubles: kind, n1, n2, n3, origin[3], spacing a b c, motif[13],  */
/* one pad) to shapes: point = origin + n1 a1 + n2 a2 + n3 a3 + basis_b, with   */
/* the motif centred at point + motif.c.  Order: n3, n2, n1, basis (fastest).   */
/* Triangular family: a1 = (a, 0, 0), a2 = (a/2, a sqrt(3)/2, 0); honeycomb     */
/* basis {0, (a1 + a2)/3}; kagome basis {0, a1/2, a2/2}.  2-D kinds stack n3    */
/* layers a3 = (0, 0, c); hexagonal = triangular layers, period c along z.      */
/* Returns the number of shapes (out may be NULL to count).                    */
int64_t or_lattice_shapes(const double *lat, double *out)
{
    const int kind = (int)lat[0];
    const int64_t n1 = (int64_t)lat[1], n2 = (int64_t)lat[2], n3 = (int64_t)lat[3];
    const double *o = lat + 4, *sp = lat + 7, *motif = lat + 10;
    const double a = sp[0], b = sp[1], cz = sp[2];
    const double s3h = sqrt(3.0) * 0.5;
    double a1[3] = {a, 0.0, 0.0}, a2[3] = {0.0, a, 0.0}, a3[3] = {0.0, 0.0, cz};
    double basis[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    int nb = 1;
    if (kind == OR_TRIANGULAR || kind == OR_HONEYCOMB || kind == OR_KAGOME || kind == OR_HEXAGONAL) {
        a2[0] = 0.5 * a;
        a2[1] = s3h * a;
    }
    if (kind == OR_RECTANGULAR) a2[1] = b;
    if (kind == OR_HONEYCOMB) {
        nb = 2;
        basis[1][0] = 0.5 * a;
        basis[1][1] = (s3h * a) / 3.0;
    }
    if (kind == OR_KAGOME) {
        nb = 3;
        basis[1][0] = 0.5 * a;
        basis[2][0] = 0.25 * a;
        basis[2][1] = 0.5 * (s3h * a);
    }
    int64_t n = 0;
    for (int64_t k3 = 0; k3 < n3; ++k3)
        for (int64_t k2 = 0; k2 < n2; ++k2)
            for (int64_t k1 = 0; k1 < n1; ++k1)
                for (int bb = 0; bb < nb; ++bb, ++n) {
                    if (!out) continue;
                    double *sh = out + 13 * n;
                    for (int t = 0; t < 13; ++t) sh[t] = motif[t];
                    for (int ax = 0; ax < 3; ++ax) {
                        double p = o[ax] + (double)k1 * a1[ax];
                        p = p + (double)k2 * a2[ax];
                        p = p + (double)k3 * a3[ax];
                        p = p + basis[bb][ax];
                        sh[2 + ax] = p + motif[2 + ax];
                    }
                }
    return n;
}

/* Background value at site (i,j,k). */
static double checker_value(const or_grid *G, const double *cell, const double *vals, double p_odd, uint64_t seed,
                            int i, int j, int k)
{
    const int ijk[3] = {i, j, k};
    int64_t ci[3], nc[3];
    for (int ax = 0; ax < 3; ++ax) {
        if (cell[ax] > 0.0) {
            ci[ax] = (int64_t)floor((ijk[ax] * G->h[ax]) / cell[ax]);
            nc[ax] = (int64_t)floor(((G->n[ax] - 1) * G->h[ax]) / cell[ax]) + 1;
        } else {
            ci[ax] = 0;
            nc[ax] = 1;
        }
    }
    if (p_odd < 0.0) return ((ci[0] + ci[1] + ci[2]) & 1) ? vals[1] : vals[0];
    /* random checkerboard: cell takes vals[1] with probability p_odd, drawn by       */
    /* Philox4x32-10 with counter (cell index, 0, 0x4B434548) and key = seed          */
    const uint64_t cidx = (uint64_t)(ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]));
    const uint32_t ctr[4] = {(uint32_t)cidx, (uint32_t)(cidx >> 32), 0u, 0x4B434548u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const double u = ldexp((double)(x[0] >> 8), -24);
    return (u < p_odd) ? vals[1] : vals[0];
}

/* Voronoi: the value of the nearest seed (x, y, z, value), minimum image on   */
/* periodic axes, distance Euclidean (compared squared), absolute or maximum;  */
/* equal distances go to the lower seed index.  Brute force over all seeds.    */
int64_t or_voronoi_owner(const or_grid *G, const double *seeds, int64_t n_seeds, int metric, int i, int j, int k)
{
    int64_t best = -1;
    double bd = 0.0;
    for (int64_t s = 0; s < n_seeds; ++s) {
        double d[3];
        min_image(G, seeds + 4 * s, i, j, k, d);
        double v;
        if (metric == OR_EUCLIDEAN) v = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        else if (metric == OR_ABSOLUTE) v = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
        else v = fmax(fmax(fabs(d[0]), fabs(d[1])), fabs(d[2]));
        if (best < 0 || v < bd) {
            best = s;
            bd = v;
        }
    }
    return best;
}

int64_t or_pattern_ex(const or_grid *G, const double *shapes, int64_t n_shapes, int64_t target, int bg_kind,
                      int bg_metric, double bg_value, const double *cell, const double *vals, double p_odd,
                      uint64_t seed, const double *seeds, int64_t n_seeds, double *alpha, uint8_t *insulating,
                      int64_t *marked_out)
{
    const int64_t N = (int64_t)G->n[0] * G->n[1] * G->n[2];
    int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t m = 0; m < N; ++m) owner[m] = -1;
    int64_t marked = 0, used = 0;
    for (int64_t n = 0; n < n_shapes; ++n) {
        if (target > 0 && marked >= target) break;
        const double *sh = shapes + 13 * n;
        const int inv = ((int)sh[1] & OR_INVERT) != 0;
        int64_t add = 0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : add)
        for (int k = 0; k < G->n[2]; ++k)
            for (int j = 0; j < G->n[1]; ++j)
                for (int i = 0; i < G->n[0]; ++i) {
                    int64_t m = idx3(G, i, j, k);
                    if (owner[m] >= 0) continue;
                    if (or_shape_contains(G, sh, i, j, k) != inv) {
                        owner[m] = n;
                        ++add;
                    }
                }
        marked += add;
        used = n + 1;
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int64_t m = idx3(G, i, j, k);
                if (owner[m] >= 0) {
                    alpha[m] = shapes[13 * owner[m] + 12];
                    if (insulating) insulating[m] = (((int)shapes[13 * owner[m] + 1]) & OR_INSULATING) ? 1 : 0;
                    continue;
                }
                if (insulating) insulating[m] = 0;
                if (bg_kind == OR_BG_CHECKER) alpha[m] = checker_value(G, cell, vals, p_odd, seed, i, j, k);
                else if (bg_kind == OR_BG_VORONOI && n_seeds > 0)
                    alpha[m] = seeds[4 * or_voronoi_owner(G, seeds, n_seeds, bg_metric, i, j, k) + 3];
                else alpha[m] = bg_value;
            }
    free(owner);
    if (marked_out) *marked_out = marked;
    return used;
}

/* Number of OpenMP threads the oracle's parallel loops use (for reporting). */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of the parallel loops (n >= 1); returns the new count. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Neighbour sum NS_m(psi) (complex) and its conjugate transpose, for the    */
/* adjoint of the step.  NS^H has entries conj(NS_{m',m}): the open-face      */
/* factor 2 moves from the face row to the row next to the face.             */
/* ------------------------------------------------------------------------ */
void or_ns(const or_grid *G, const double *theta, double K, const double *psi, double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i)
                store(out, idx3(G, i, j, k), neighbour_sum(G, theta, K, psi, i, j, k));
}

void or_ns_adj(const or_grid *G, const double *theta, double K, const double *lam, double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                int c0[3] = {i, j, k};
                cplx acc = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    if (!axis_active(G, ax)) continue;
                    int n = G->n[ax], idx = c0[ax];
                    double c = axis_coef(G, ax);
                    int cp[3] = {i, j, k}, cm[3] = {i, j, k};
                    step_index(G, ax, +1, cp);
                    step_index(G, ax, -1, cm);
                    int open = (G->bc[ax] == OR_OPEN);
                    /* row m+a holds U*_{a,m} lam_m as its backward term (times 2 if m+a is the
                       high open face); its conjugate transpose gives U_{a,m} lam_{m+a} here */
                    if (!open || idx < n - 1) {
                        double wgt = (open && idx + 1 == n - 1) ? 2.0 : 1.0;
                        acc += wgt * c * link(G, theta, K, ax, i, j, k) * load(lam, idx3(G, cp[0], cp[1], cp[2]));
                    }
                    /* row m-a holds U_{a,m-a} lam_m as its forward term (times 2 if m-a is the
                       low open face); its conjugate transpose gives conj(U_{a,m-a}) lam_{m-a} */
                    if (!open || idx > 0) {
                        double wgt = (open && idx - 1 == 0) ? 2.0 : 1.0;
                        acc += wgt * c * conj(link(G, theta, K, ax, cm[0], cm[1], cm[2])) *
                               load(lam, idx3(G, cm[0], cm[1], cm[2]));
                    }
                }
                store(out, idx3(G, i, j, k), acc);
            }
}
