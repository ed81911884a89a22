/*
 * Plain FP64 CPU oracle of the Weighted Density Lattice Boltzmann (WDLB) time
 * step of Marini Bettolo Marconi & Melchionna, "Weighted density Lattice
 * Boltzmann approach to fluids under confinement" (arXiv:1304.7880).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library: every table below is rebuilt here from its defining rule.
 *
 * Single thread, natural loop order (x fastest), double precision throughout,
 * no blocking, no fusion.  Each function names the passage it follows:
 *
 *   Sec. 2 (Model)            Eq. uno (kinetic equation), Eq. colonna (moments),
 *                             Eq. relaxationtime (BGK), Eq. eq:dufty2 and
 *                             Eq. dij (SMDB A-term), Eq. SMDB (evolution eq.),
 *                             Eq. extrapressure (the factor K of the A-term).
 *   Sec. 3 (Hard sphere)      smeared density nbar (Fischer-Methfessel),
 *                             Eq. campoc (field C), Eq. campod (field A),
 *                             F^mf / F^viscous split of C.
 *   Sec. 5 (Numerical results) D3Q19, isothermal; the five-step LB algorithm.
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   R1  g2 at contact of the homogeneous fluid: Carnahan-Starling (or PY, or 1).
 *   R2  g2(r, r+e) is evaluated at the mean of the smeared densities of the two
 *       ends (symmetric in the pair, hence exact momentum conservation).
 *   R3  nbar is the mean of n over the lattice ball |b|^2 <= (sigma/2)^2.
 *   R4  k-hat = e/|e|; the integral over k-hat is a sum over the lattice shell
 *       (sigma-1/2)^2 < |e|^2 <= (sigma+1/2)^2 with one uniform weight chosen so
 *       that sigma^2 * sum_e w khat_z e_z = 4 pi sigma^3 / 3 (the discrete
 *       virial coefficient then equals b = 2 pi sigma^3 / 3 exactly).
 *   R4c shell rule COMPACT (a quadrature of this library; the paper gives
 *       none): the union of two or three cubic orbits of the R4 shell, one
 *       weight per orbit, the weights fixed by three moment conditions,
 *         sigma^2 sum_e w_e khat_z e_z   = 4 pi sigma^3 / 3   (virial coefficient b)
 *         sum_e w_e khat_x^2 e_z^2       = 4 pi sigma^2 / 15  (continuum value of
 *                                          the collisional-viscosity moment)
 *         sum_e w_e khat_z^2 e_z^2       = 3 sum_e w_e khat_x^2 e_z^2  (isotropic
 *                                          fourth moment),
 *       every weight positive (> 1e-3 of the largest); of all such unions the
 *       one with the fewest vectors, then the smallest sum over its vectors of
 *       (|e|^2 - sigma^2)^2, then the first in orbit order (orbits ordered by
 *       |e|^2, then by their sorted components).
 *   R5  the SMDB source carries K times the traceless part of A in its second
 *       moment (K = 2 reproduces Eq. extrapressure).
 *   R6  lattice units a = dt = m = 1, k_B T = c_s^2 = 1/3.
 *   R7  "explicit trapezoidal rule": second-order forcing, u = (j + F/2)/n and
 *       a (1 - omega/2) prefactor on every source.  The fields take one
 *       velocity per node, v, on both ends of every pair (so C stays pairwise
 *       antisymmetric and momentum is conserved exactly).  v predicts the
 *       trapezoidal velocity u = j/n + g/2 + C/(2n), in which C depends on u
 *       itself, by a lagged linear-implicit step:
 *         (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev,
 *         H = kappa (beta/2) t_prev / 3,  t = sum_e w g2 n(r+e),
 *       with C_prev, t_prev, v_prev from the previous step (zero, zero and the
 *       initial velocity at the first step) and kappa = 2.  At a steady state
 *       v = u exactly.  beta t / 3 is the isotropic part of the local
 *       (diagonal) dependence of F^viscous on u(r); treating it implicitly
 *       keeps the collisional viscosity stable at liquid densities.
 *   R8  walls: nodes z = 0 and z = nz-1 are solid (n = 0 there, also beyond
 *       them); half-way bounce-back; x and y (and z without walls) periodic.
 *   R9  omega: constant 1/tau, or tau(r) - 1/2 scaled by
 *       n_ref g(n_ref) / (nbar(r) g(nbar(r))) (SMDB omega0 proportional to n g),
 *       n_ref the mean fluid density of the initial state unless given.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
static const double CS2 = 1.0 / 3.0;            /* R6 */
static const double KAPPA = 2.0;                /* R7 */

/* ---------------------------------------------------------------------- */
/* D3Q19 velocity set (Sec. 5): rest, six face and twelve edge neighbours.   */
/* ---------------------------------------------------------------------- */
static int C[Q][3];
static double W[Q];
static int OPP[Q];
static int d3q19_ready = 0;

static void build_d3q19(void)
{
    if (d3q19_ready) return;
    int q = 0;
    C[q][0] = C[q][1] = C[q][2] = 0; W[q] = 1.0 / 3.0; q++;
    for (int ax = 0; ax < 3; ax++)
        for (int s = -1; s <= 1; s += 2) {
            C[q][0] = C[q][1] = C[q][2] = 0;
            C[q][ax] = s; W[q] = 1.0 / 18.0; q++;
        }
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++)
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                    C[q][0] = C[q][1] = C[q][2] = 0;
                    C[q][a] = sa; C[q][b] = sb; W[q] = 1.0 / 36.0; q++;
                }
    for (int a = 0; a < Q; a++)
        for (int b = 0; b < Q; b++)
            if (C[a][0] == -C[b][0] && C[a][1] == -C[b][1] && C[a][2] == -C[b][2])
                OPP[a] = b;
    d3q19_ready = 1;
}

int wo_velocities(int *c_out, double *w_out)
{
    build_d3q19();
    for (int q = 0; q < Q; q++) {
        for (int d = 0; d < 3; d++) c_out[3 * q + d] = C[q][d];
        w_out[q] = W[q];
    }
    return Q;
}

/* ---------------------------------------------------------------------- */
/* Stencils (R3, R4).                                                       */
/* ---------------------------------------------------------------------- */
/* Ball of the smeared density (Sec. 3): all b with |b|^2 <= (sigma/2)^2.   */
int wo_ball(double sigma, int *b_out, int cap)
{
    int R = (int)floor(sigma / 2.0);
    double r2max = (sigma / 2.0) * (sigma / 2.0);
    int m = 0;
    for (int z = -R; z <= R; z++)
        for (int y = -R; y <= R; y++)
            for (int x = -R; x <= R; x++)
                if ((double)(x * x + y * y + z * z) <= r2max) {
                    if (b_out && m < cap) {
                        b_out[3 * m] = x; b_out[3 * m + 1] = y; b_out[3 * m + 2] = z;
                    }
                    m++;
                }
    return m;
}

/* Contact shell (Eq. campoc integrates over the sphere of radius sigma):   */
/* lattice vectors with (sigma-1/2)^2 < |e|^2 <= (sigma+1/2)^2, and the      */
/* uniform weight w of R4.                                                   */
int wo_shell(double sigma, int *e_out, int cap, double *w_out)
{
    int R = (int)floor(sigma + 0.5);
    double lo = (sigma - 0.5) * (sigma - 0.5), hi = (sigma + 0.5) * (sigma + 0.5);
    int m = 0;
    double mom = 0.0;                  /* sum_e e_z^2 / |e| */
    for (int z = -R; z <= R; z++)
        for (int y = -R; y <= R; y++)
            for (int x = -R; x <= R; x++) {
                double r2 = (double)(x * x + y * y + z * z);
                if (r2 > lo && r2 <= hi) {
                    if (e_out && m < cap) {
                        e_out[3 * m] = x; e_out[3 * m + 1] = y; e_out[3 * m + 2] = z;
                    }
                    mom += (double)(z * z) / sqrt(r2);
                    m++;
                }
            }
    if (w_out) *w_out = (4.0 * M_PI / 3.0) * sigma / mom;
    return m;
}

/* Compact contact shell (R4c).  Orbits of the cubic group: the distinct
 * sign changes and permutations of (a, b, c), 0 <= a <= b <= c.              */
#define WO_MAX_ORBITS 96

typedef struct {
    int a, b, c, r2, size;
    double m1;      /* sum over the orbit of khat_z e_z = e_z^2 / |e|              */
    double vc;      /* sum of khat_x^2 e_z^2 = e_x^2 e_z^2 / |e|^2                 */
    double an;      /* sum of khat_z^2 e_z^2 - 3 khat_x^2 e_z^2                     */
} wo_orbit;

static int orbit_members(int a, int b, int c, int out[48][3])
{
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int v[3] = {a, b, c};
    int m = 0;
    for (int p = 0; p < 6; p++)
        for (int sg = 0; sg < 8; sg++) {
            int e[3];
            for (int d = 0; d < 3; d++) e[d] = ((sg >> d) & 1) ? -v[perm[p][d]] : v[perm[p][d]];
            int dup = 0;
            for (int k = 0; k < m && !dup; k++)
                dup = out[k][0] == e[0] && out[k][1] == e[1] && out[k][2] == e[2];
            if (!dup) {
                out[m][0] = e[0]; out[m][1] = e[1]; out[m][2] = e[2];
                m++;
            }
        }
    return m;
}

static int orbit_less(const wo_orbit *p, const wo_orbit *q)
{
    if (p->r2 != q->r2) return p->r2 < q->r2;
    if (p->a != q->a) return p->a < q->a;
    if (p->b != q->b) return p->b < q->b;
    return p->c < q->c;
}

/* Weights of the orbits idx[0..k-1] (k = 2 or 3) solving the three moment
 * conditions of R4c: Cramer's rule for k = 3, the normal equations for k = 2
 * (then the residual of each condition must vanish).  Returns 1 with w[] if
 * the conditions hold and every weight is positive. */
static int compact_weights(const wo_orbit *o, const int *idx, int k, double sigma, double *w)
{
    double A[3][3], rhs[3] = {4.0 * M_PI * sigma / 3.0, 4.0 * M_PI * sigma * sigma / 15.0, 0.0};
    for (int j = 0; j < k; j++) {
        A[0][j] = o[idx[j]].m1;
        A[1][j] = o[idx[j]].vc;
        A[2][j] = o[idx[j]].an;
    }
    if (k == 3) {
        double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                   - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                   + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        double scale = 1.0;
        for (int j = 0; j < 3; j++)
            scale *= sqrt(A[0][j] * A[0][j] + A[1][j] * A[1][j] + A[2][j] * A[2][j]);
        if (fabs(det) <= 1e-12 * scale) return 0;
        for (int j = 0; j < 3; j++) {
            double M[3][3];
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) M[r][c] = (c == j) ? rhs[r] : A[r][c];
            double dj = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                      - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                      + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            w[j] = dj / det;
        }
    } else {
        double g00 = 0, g01 = 0, g11 = 0, b0 = 0, b1 = 0;
        for (int r = 0; r < 3; r++) {
            g00 += A[r][0] * A[r][0];
            g01 += A[r][0] * A[r][1];
            g11 += A[r][1] * A[r][1];
            b0 += A[r][0] * rhs[r];
            b1 += A[r][1] * rhs[r];
        }
        double det = g00 * g11 - g01 * g01;
        if (fabs(det) <= 1e-12 * g00 * g11) return 0;
        w[0] = (b0 * g11 - b1 * g01) / det;
        w[1] = (g00 * b1 - g01 * b0) / det;
    }
    double wmax = 0.0;
    for (int j = 0; j < k; j++) wmax = w[j] > wmax ? w[j] : wmax;
    for (int j = 0; j < k; j++)
        if (!(w[j] > 1e-3 * wmax)) return 0;
    for (int r = 0; r < 3; r++) {
        double lhs = 0.0, mag = fabs(rhs[r]);
        for (int j = 0; j < k; j++) {
            lhs += A[r][j] * w[j];
            mag += fabs(A[r][j] * w[j]);
        }
        if (fabs(lhs - rhs[r]) > 1e-9 * mag) return 0;
    }
    return 1;
}

/* The compact shell of R4c: its vectors and their weights.  Returns the
 * vector count, 0 if no union of two or three orbits satisfies R4c. */
int wo_shell_compact(double sigma, int *e_out, double *w_out, int cap)
{
    const int R = (int)floor(sigma + 0.5);
    const double lo = (sigma - 0.5) * (sigma - 0.5), hi = (sigma + 0.5) * (sigma + 0.5);
    wo_orbit o[WO_MAX_ORBITS];
    int no = 0;
    int mem[48][3];
    for (int c = 0; c <= R; c++)
        for (int b = 0; b <= c; b++)
            for (int a = 0; a <= b; a++) {
                int r2 = a * a + b * b + c * c;
                if (!((double)r2 > lo && (double)r2 <= hi) || no >= WO_MAX_ORBITS) continue;
                wo_orbit t = {a, b, c, r2, 0, 0.0, 0.0, 0.0};
                t.size = orbit_members(a, b, c, mem);
                for (int m = 0; m < t.size; m++) {
                    double ex = mem[m][0], ez = mem[m][2], len2 = (double)r2;
                    t.m1 += ez * ez / sqrt(len2);
                    t.vc += ex * ex * ez * ez / len2;
                    t.an += (ez * ez * ez * ez - 3.0 * ex * ex * ez * ez) / len2;
                }
                int pos = no++;                        /* insertion in orbit order */
                while (pos > 0 && orbit_less(&t, &o[pos - 1])) {
                    o[pos] = o[pos - 1];
                    pos--;
                }
                o[pos] = t;
            }
    int best[3] = {-1, -1, -1}, bestk = 0, bestn = 0;
    double bestw[3] = {0, 0, 0}, bests = 0.0;
    for (int k = 2; k <= 3; k++) {
        int idx[3];
        for (idx[0] = 0; idx[0] < no; idx[0]++)
            for (idx[1] = idx[0] + 1; idx[1] < no; idx[1]++)
                for (idx[2] = (k == 3 ? idx[1] + 1 : no); idx[2] <= (k == 3 ? no - 1 : no); idx[2]++) {
                    double w[3];
                    if (!compact_weights(o, idx, k, sigma, w)) continue;
                    int n = 0;
                    double spread = 0.0;
                    for (int j = 0; j < k; j++) {
                        double d = (double)o[idx[j]].r2 - sigma * sigma;
                        n += o[idx[j]].size;
                        spread += o[idx[j]].size * d * d;
                    }
                    if (bestk == 0 || n < bestn || (n == bestn && spread < bests - 1e-9 * (1.0 + bests))) {
                        bestk = k; bestn = n; bests = spread;
                        for (int j = 0; j < k; j++) { best[j] = idx[j]; bestw[j] = w[j]; }
                    }
                }
    }
    if (bestk == 0) return 0;
    int m = 0;
    for (int z = -R; z <= R; z++)
        for (int y = -R; y <= R; y++)
            for (int x = -R; x <= R; x++) {
                int v[3] = {abs(x), abs(y), abs(z)};
                for (int p = 0; p < 2; p++)             /* sort |components| */
                    for (int q = 0; q < 2 - p; q++)
                        if (v[q] > v[q + 1]) { int t = v[q]; v[q] = v[q + 1]; v[q + 1] = t; }
                for (int j = 0; j < bestk; j++) {
                    const wo_orbit *t = &o[best[j]];
                    if (v[0] == t->a && v[1] == t->b && v[2] == t->c) {
                        if (m < cap) {
                            if (e_out) { e_out[3 * m] = x; e_out[3 * m + 1] = y; e_out[3 * m + 2] = z; }
                            if (w_out) w_out[m] = bestw[j];
                        }
                        m++;
                    }
                }
            }
    return m;
}

/* ---------------------------------------------------------------------- */
/* Contact value of the homogeneous pair distribution (R1), chi = pi n s^3/6 */
/* ---------------------------------------------------------------------- */
double wo_closure(int closure, double chi)
{
    if (closure == 0) return (1.0 - 0.5 * chi) / ((1.0 - chi) * (1.0 - chi) * (1.0 - chi));
    if (closure == 1) return (1.0 + 0.5 * chi) / ((1.0 - chi) * (1.0 - chi));
    return 1.0;
}

/* ---------------------------------------------------------------------- */
/* State                                                                    */
/* ---------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz, walls;
    long N;
    double sigma, tau, g[3], k_cross, n_ref;
    double n_ref_opt;                  /* reference density asked for; 0: see wo_init */
    int closure, omega_mode, interactions;
    int nball, nshell;
    int *ball, *shell;
    double *wvec;                      /* weight of each shell vector (R4 or R4c) */
    int shell_rule;                    /* 0: R4 (full shell), 1: R4c (compact) */
    double *f, *fnew;                  /* [Q][N] */
    double *n, *j, *us;                /* n[N], j[3][N], field velocity v[3][N] */
    double *nbar;                      /* [N] */
    double *Cf, *A;                    /* C[3][N], A[6][N] of this step */
    double *Cprev;                     /* [3][N] */
    double *Tprev;                     /* t = sum_e w g2 n(r+e) of the previous step [N] */
    double *vprev;                     /* field velocity of the previous step [3][N] */
    double *Tcur;                      /* t of this step [N] */
    long steps;
    int unstable;
} wo_state;

static int is_wall(const wo_state *s, int z)
{
    return s->walls && (z == 0 || z == s->nz - 1);
}

/* Node index of (x+dx, y+dy, z+dz) with periodic x, y (and z without walls);
 * -1 if the point lies beyond a wall. */
static long neighbour(const wo_state *s, int x, int y, int z, int dx, int dy, int dz)
{
    int xx = ((x + dx) % s->nx + s->nx) % s->nx;
    int yy = ((y + dy) % s->ny + s->ny) % s->ny;
    int zz = z + dz;
    if (s->walls) {
        if (zz < 0 || zz >= s->nz) return -1;
    } else {
        zz = (zz % s->nz + s->nz) % s->nz;
    }
    return (long)xx + (long)s->nx * ((long)yy + (long)s->ny * (long)zz);
}

void wo_destroy(wo_state *s)
{
    if (!s) return;
    free(s->ball); free(s->shell); free(s->wvec); free(s->f); free(s->fnew); free(s->n); free(s->j);
    free(s->us); free(s->nbar); free(s->Cf); free(s->A); free(s->Cprev); free(s->Tprev); free(s->vprev); free(s->Tcur);
    free(s);
}

wo_state *wo_create(int nx, int ny, int nz, int walls, double sigma, double tau,
                    double gx, double gy, double gz, int closure, int omega_mode,
                    double k_cross, double n_ref, int interactions, int shell_rule)
{
    build_d3q19();
    if (nx < 1 || ny < 1 || nz < 1 || (walls && nz < 3) || sigma < 1.0 || tau <= 0.5)
        return NULL;
    if (shell_rule != 0 && (shell_rule != 1 || wo_shell_compact(sigma, NULL, NULL, 0) == 0))
        return NULL;
    wo_state *s = (wo_state *)calloc(1, sizeof(wo_state));
    s->nx = nx; s->ny = ny; s->nz = nz; s->walls = walls;
    s->N = (long)nx * ny * nz;
    s->sigma = sigma; s->tau = tau; s->g[0] = gx; s->g[1] = gy; s->g[2] = gz;
    s->closure = closure; s->omega_mode = omega_mode; s->k_cross = k_cross;
    s->n_ref = s->n_ref_opt = n_ref; s->interactions = interactions;
    s->nball = wo_ball(sigma, NULL, 0);
    s->ball = (int *)malloc(sizeof(int) * 3 * s->nball);
    wo_ball(sigma, s->ball, s->nball);
    s->shell_rule = shell_rule;
    if (shell_rule == 0) {
        double w;
        s->nshell = wo_shell(sigma, NULL, 0, &w);
        s->shell = (int *)malloc(sizeof(int) * 3 * s->nshell);
        s->wvec = (double *)malloc(sizeof(double) * s->nshell);
        wo_shell(sigma, s->shell, s->nshell, NULL);
        for (int m = 0; m < s->nshell; m++) s->wvec[m] = w;
    } else {
        s->nshell = wo_shell_compact(sigma, NULL, NULL, 0);
        s->shell = (int *)malloc(sizeof(int) * 3 * s->nshell);
        s->wvec = (double *)malloc(sizeof(double) * s->nshell);
        wo_shell_compact(sigma, s->shell, s->wvec, s->nshell);
    }
    long N = s->N;
    s->f = (double *)calloc((size_t)Q * N, sizeof(double));
    s->fnew = (double *)calloc((size_t)Q * N, sizeof(double));
    s->n = (double *)calloc(N, sizeof(double));
    s->j = (double *)calloc(3 * N, sizeof(double));
    s->us = (double *)calloc(3 * N, sizeof(double));
    s->nbar = (double *)calloc(N, sizeof(double));
    s->Cf = (double *)calloc(3 * N, sizeof(double));
    s->A = (double *)calloc(6 * N, sizeof(double));
    s->Cprev = (double *)calloc(3 * N, sizeof(double));
    s->Tprev = (double *)calloc(N, sizeof(double));
    s->vprev = (double *)calloc(3 * N, sizeof(double));
    s->Tcur = (double *)calloc(N, sizeof(double));
    return s;
}

/* Discrete local Maxwellian to second order in u (the D3Q19 projection of
 * n phi_M of Eq. relaxationtime, isothermal). */
static double feq(int q, double n, const double u[3])
{
    double cu = C[q][0] * u[0] + C[q][1] * u[1] + C[q][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[q] * n * (1.0 + cu / CS2 + 0.5 * cu * cu / (CS2 * CS2) - 0.5 * uu / CS2);
}

/* Step 1 of the algorithm of Sec. 5: populations from n and u. */
int wo_init(wo_state *s, const double *n0, const double *u0)
{
    long N = s->N;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                double u[3] = {u0[i], u0[N + i], u0[2 * N + i]};
                double n = is_wall(s, z) ? 0.0 : n0[i];
                if (is_wall(s, z)) u[0] = u[1] = u[2] = 0.0;
                for (int q = 0; q < Q; q++) s->f[q * N + i] = feq(q, n, u);
            }
    memset(s->Cprev, 0, sizeof(double) * 3 * N);
    memset(s->Tprev, 0, sizeof(double) * N);
    for (long i = 0; i < N; i++) {
        int z = (int)(i / ((long)s->nx * s->ny));
        for (int d = 0; d < 3; d++) s->vprev[d * N + i] = is_wall(s, z) ? 0.0 : u0[d * N + i];
    }
    /* R9's reference density, unless given: the mean density over the fluid
     * nodes of the initial state */
    if (s->n_ref_opt > 0.0) {
        s->n_ref = s->n_ref_opt;
    } else {
        double sum = 0.0;
        long fluid = 0;
        for (long i = 0; i < N; i++) {
            int z = (int)(i / ((long)s->nx * s->ny));
            if (is_wall(s, z)) continue;
            sum += n0[i];
            fluid++;
        }
        s->n_ref = sum / (double)fluid;
    }
    s->steps = 0;
    s->unstable = 0;
    return 0;
}

/* Step 4 of Sec. 5 / Eq. colonna: n = sum_q f_q, j = sum_q f_q c_q and the
 * field velocity v of R7.  Solid nodes carry n = 0, v = 0. */
static void moments(wo_state *s)
{
    long N = s->N;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                if (is_wall(s, z)) {
                    s->n[i] = 0.0;
                    for (int d = 0; d < 3; d++) { s->j[d * N + i] = 0.0; s->us[d * N + i] = 0.0; }
                    continue;
                }
                double n = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int q = 0; q < Q; q++) {
                    double fq = s->f[q * N + i];
                    n += fq;
                    for (int d = 0; d < 3; d++) j[d] += fq * C[q][d];
                }
                s->n[i] = n;
                double beta = 2.0 * s->sigma * s->sigma * sqrt(CS2 / M_PI);
                double h = 0.5 * beta * KAPPA;
                /* (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev, H = kappa beta t_prev / 6 */
                double H = h * s->Tprev[i] / 3.0;
                for (int a = 0; a < 3; a++) {
                    s->j[a * N + i] = j[a];
                    double rhs = (j[a] + 0.5 * (n * s->g[a] + s->Cprev[a * N + i])) / n + H * s->vprev[a * N + i];
                    s->us[a * N + i] = rhs / (1.0 + H);
                }
            }
}

/* Smeared density of Sec. 3 (R3): nbar(r) = mean over the ball of n(r+b). */
static void smeared_density(wo_state *s)
{
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                double sum = 0.0;
                for (int b = 0; b < s->nball; b++) {
                    long k = neighbour(s, x, y, z, s->ball[3 * b], s->ball[3 * b + 1], s->ball[3 * b + 2]);
                    if (k >= 0) sum += s->n[k];
                }
                s->nbar[i] = sum / s->nball;
            }
}

/* Step 2 of Sec. 5: the fields C (Eq. campoc, split as n (F^mf + F^viscous))
 * and A (Eq. campod) as sums over the contact shell (R2, R4), with
 * du = v(r+e) - v(r) (R7), plus t of R7 for the next step. */
static void shell_fields(wo_state *s)
{
    long N = s->N;
    double sig2 = s->sigma * s->sigma;
    double beta = 2.0 * sig2 * sqrt(CS2 / M_PI);
    double chi_of_n = M_PI * s->sigma * s->sigma * s->sigma / 6.0;
    memset(s->Cf, 0, sizeof(double) * 3 * N);
    memset(s->A, 0, sizeof(double) * 6 * N);
    memset(s->Tcur, 0, sizeof(double) * N);
    if (!s->interactions) return;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                if (is_wall(s, z)) continue;
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                double ni = s->n[i];
                double Fmf[3] = {0, 0, 0}, Fv[3] = {0, 0, 0}, S[3][3] = {{0}}, t = 0.0;
                for (int m = 0; m < s->nshell; m++) {
                    int ex = s->shell[3 * m], ey = s->shell[3 * m + 1], ez = s->shell[3 * m + 2];
                    long k = neighbour(s, x, y, z, ex, ey, ez);
                    if (k < 0 || is_wall(s, z + ez)) continue;
                    double len = sqrt((double)(ex * ex + ey * ey + ez * ez));
                    double kh[3] = {ex / len, ey / len, ez / len};
                    double chi = chi_of_n * 0.5 * (s->nbar[i] + s->nbar[k]);
                    if (chi >= 1.0) s->unstable = 1;
                    double wgn = s->wvec[m] * wo_closure(s->closure, chi) * s->n[k];
                    double du[3];
                    for (int d = 0; d < 3; d++) du[d] = s->us[d * N + k] - s->us[d * N + i];
                    double kdu = kh[0] * du[0] + kh[1] * du[1] + kh[2] * du[2];
                    for (int a = 0; a < 3; a++) {
                        Fmf[a] += -CS2 * sig2 * wgn * kh[a];
                        Fv[a] += beta * wgn * kh[a] * kdu;
                        for (int b = 0; b < 3; b++) S[a][b] += wgn * (kh[b] * du[a] + kh[a] * du[b]);
                    }
                    t += wgn;
                }
                for (int d = 0; d < 3; d++) s->Cf[d * N + i] = ni * (Fmf[d] + Fv[d]);
                double pa = -(CS2 / 5.0) * ni * sig2;
                s->A[0 * N + i] = pa * S[0][0];
                s->A[1 * N + i] = pa * S[1][1];
                s->A[2 * N + i] = pa * S[2][2];
                s->A[3 * N + i] = pa * S[0][1];
                s->A[4 * N + i] = pa * S[0][2];
                s->A[5 * N + i] = pa * S[1][2];
                s->Tcur[i] = t;
            }
}

/* Relaxation frequency (R9). */
static double omega_at(const wo_state *s, double nbar)
{
    if (s->omega_mode == 0) return 1.0 / s->tau;
    double chi_of_n = M_PI * s->sigma * s->sigma * s->sigma / 6.0;
    double ref = s->n_ref * wo_closure(s->closure, chi_of_n * s->n_ref);
    double loc = nbar * wo_closure(s->closure, chi_of_n * nbar);
    if (loc <= 0.0) return 0.0;
    double tau = 0.5 + (s->tau - 0.5) * ref / loc;
    if (tau < 0.5 + 1e-3) tau = 0.5 + 1e-3;
    return 1.0 / tau;
}

/* Step 3 of Sec. 5 at one node: BGK relaxation (Eq. relaxationtime) plus the
 * hydrodynamic projection with the total force F = n g + C (Eq. SMDB) and
 * the SMDB A-term (Eq. eq:dufty2, factor K of R5), integrated with the
 * second-order (trapezoidal) rule of R7.  fin/fout: Q values; A: xx, yy, zz,
 * xy, xz, yz (not yet made traceless). */
void wo_collide_node(const double *fin, const double *Fext, const double *A6,
                     double omega, double k_cross, double *fout)
{
    build_d3q19();
    double n = 0.0, j[3] = {0, 0, 0};
    for (int q = 0; q < Q; q++) {
        n += fin[q];
        for (int d = 0; d < 3; d++) j[d] += fin[q] * C[q][d];
    }
    double u[3];
    for (int d = 0; d < 3; d++) u[d] = (j[d] + 0.5 * Fext[d]) / n;
    double tr = A6[0] + A6[1] + A6[2];
    double At[3][3] = {{A6[0] - tr / 3.0, A6[3], A6[4]},
                       {A6[3], A6[1] - tr / 3.0, A6[5]},
                       {A6[4], A6[5], A6[2] - tr / 3.0}};
    for (int q = 0; q < Q; q++) {
        double cu = C[q][0] * u[0] + C[q][1] * u[1] + C[q][2] * u[2];
        double phi = 0.0;                 /* second-order Hermite force term */
        for (int d = 0; d < 3; d++)
            phi += ((C[q][d] - u[d]) / CS2 + cu * C[q][d] / (CS2 * CS2)) * Fext[d];
        phi *= W[q];
        double cac = 0.0;                 /* c . A~ . c */
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) cac += C[q][a] * At[a][b] * C[q][b];
        double sa = k_cross * W[q] / (2.0 * CS2 * CS2) * cac;
        fout[q] = fin[q] - omega * (fin[q] - feq(q, n, u)) + (1.0 - 0.5 * omega) * (phi + sa);
    }
}

/* Step 3 continued: streaming, f(r, t+1) = f*(r - c, t), with half-way
 * bounce-back f(r, t+1) = f*_{-c}(r, t) where r - c is solid (R8). */
static void collide_stream(wo_state *s)
{
    long N = s->N;
    double *fpost = s->fnew;             /* post-collision values, stored in place */
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                if (is_wall(s, z)) {
                    for (int q = 0; q < Q; q++) fpost[q * N + i] = 0.0;
                    continue;
                }
                double fin[Q], fout[Q], F[3], A6[6];
                for (int q = 0; q < Q; q++) fin[q] = s->f[q * N + i];
                for (int d = 0; d < 3; d++) F[d] = s->n[i] * s->g[d] + s->Cf[d * N + i];
                for (int c = 0; c < 6; c++) A6[c] = s->A[c * N + i];
                double om = omega_at(s, s->nbar[i]);
                wo_collide_node(fin, F, A6, om, s->interactions ? s->k_cross : 0.0, fout);
                for (int q = 0; q < Q; q++) fpost[q * N + i] = fout[q];
            }
    /* pull streaming into s->f */
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                for (int q = 0; q < Q; q++) {
                    if (is_wall(s, z)) { s->f[q * N + i] = 0.0; continue; }
                    long k = neighbour(s, x, y, z, -C[q][0], -C[q][1], -C[q][2]);
                    int kz = z - C[q][2];
                    if (k < 0 || is_wall(s, kz))
                        s->f[q * N + i] = fpost[OPP[q] * N + i];
                    else
                        s->f[q * N + i] = fpost[q * N + k];
                }
            }
}

/* The five-step algorithm of Sec. 5, repeated nsteps times. */
int wo_step(wo_state *s, long nsteps)
{
    long N = s->N;
    for (long t = 0; t < nsteps; t++) {
        moments(s);
        smeared_density(s);
        shell_fields(s);
        collide_stream(s);
        memcpy(s->Cprev, s->Cf, sizeof(double) * 3 * N);
        memcpy(s->Tprev, s->Tcur, sizeof(double) * N);
        memcpy(s->vprev, s->us, sizeof(double) * 3 * N);
        s->steps++;
    }
    return s->unstable ? 4 : 0;
}

/* n and the field velocity u* of the current populations. */
void wo_moments(wo_state *s, double *n_out, double *u_out)
{
    moments(s);
    long N = s->N;
    memcpy(n_out, s->n, sizeof(double) * N);
    memcpy(u_out, s->us, sizeof(double) * 3 * N);
}

/* nbar, C and A of the current populations (step 2 without stepping). */
void wo_fields(wo_state *s, double *nbar_out, double *C_out, double *A_out)
{
    long N = s->N;
    moments(s);
    smeared_density(s);
    shell_fields(s);
    if (nbar_out) memcpy(nbar_out, s->nbar, sizeof(double) * N);
    if (C_out) memcpy(C_out, s->Cf, sizeof(double) * 3 * N);
    if (A_out) memcpy(A_out, s->A, sizeof(double) * 6 * N);
}

/* Energy-equation fields of Sec. 3 on a prescribed temperature field T
 * (k_B T per node in lattice units, m = 1; solid nodes ignored), evaluated on
 * the current populations with the same quadrature (R4, R4c), contact values
 * (R2) and field velocity v (R7) as C and A:
 *   Q(r)   = T n sigma^2 sum_e w g2 n(r+e) [-khat.(v(r+e)-v(r))/2
 *                                           + sqrt(T/pi) (T(r+e)-T(r))/T]     (Eq. campob1)
 *   B_i(r) = -2 T n sigma^2 sum_e w khat_i g2 n(r+e) (T(r+e)-T(r))           (Eq. campos)
 *   F^T_i(r) = -(sigma^2/2) sum_e w khat_i g2 n(r+e) (T(r+e)-T(r))           (Eq. thermalforce)
 * with T, n, sigma^2 prefactors at r.  Sec. 5 evolves no temperature (the
 * paper's runs are isothermal); these are the fields of its energy equation
 * on a given T.  Outputs are zero on solid nodes. */
void wo_thermal_fields(wo_state *s, const double *T, double *Q_out, double *B_out, double *FT_out)
{
    long N = s->N;
    double sig2 = s->sigma * s->sigma;
    double chi_of_n = M_PI * s->sigma * s->sigma * s->sigma / 6.0;
    moments(s);
    smeared_density(s);
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long i = x + (long)s->nx * (y + (long)s->ny * z);
                double q = 0.0, b[3] = {0, 0, 0};
                if (!is_wall(s, z) && s->interactions) {
                    for (int m = 0; m < s->nshell; m++) {
                        int ex = s->shell[3 * m], ey = s->shell[3 * m + 1], ez = s->shell[3 * m + 2];
                        long k = neighbour(s, x, y, z, ex, ey, ez);
                        if (k < 0 || is_wall(s, z + ez)) continue;
                        double len = sqrt((double)(ex * ex + ey * ey + ez * ez));
                        double kh[3] = {ex / len, ey / len, ez / len};
                        double chi = chi_of_n * 0.5 * (s->nbar[i] + s->nbar[k]);
                        double wgn = s->wvec[m] * wo_closure(s->closure, chi) * s->n[k];
                        double dT = T[k] - T[i];
                        double kdu = 0.0;
                        for (int d = 0; d < 3; d++) kdu += kh[d] * (s->us[d * N + k] - s->us[d * N + i]);
                        q += wgn * (-0.5 * kdu + sqrt(T[i] / M_PI) * dT / T[i]);
                        for (int d = 0; d < 3; d++) b[d] += wgn * kh[d] * dT;
                    }
                }
                if (Q_out) Q_out[i] = is_wall(s, z) ? 0.0 : T[i] * s->n[i] * sig2 * q;
                for (int d = 0; d < 3; d++) {
                    if (B_out) B_out[d * N + i] = is_wall(s, z) ? 0.0 : -2.0 * T[i] * s->n[i] * sig2 * b[d];
                    if (FT_out) FT_out[d * N + i] = is_wall(s, z) ? 0.0 : -0.5 * sig2 * b[d];
                }
            }
}

void wo_get_populations(const wo_state *s, double *f_out)
{
    memcpy(f_out, s->f, sizeof(double) * Q * s->N);
}

void wo_set_populations(wo_state *s, const double *f_in)
{
    memcpy(s->f, f_in, sizeof(double) * Q * s->N);
}

void wo_get_cprev(const wo_state *s, double *c_out)
{
    memcpy(c_out, s->Cprev, sizeof(double) * 3 * s->N);
}

void wo_set_cprev(wo_state *s, const double *c_in)
{
    memcpy(s->Cprev, c_in, sizeof(double) * 3 * s->N);
}

long wo_steps(const wo_state *s) { return s->steps; }
int wo_unstable(const wo_state *s) { return s->unstable; }
