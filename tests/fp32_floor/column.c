/*
 * Column emulator of the FP32 GPU time step (test infrastructure: it pins the
 * analysis of the FP32 floor in driven slits; the library never uses it).
 *
 * It repeats the arithmetic of the FP32 tiled kernel on a 1 x 1 x nz slit
 * column (an x-y-uniform state: every shell and ball vector wraps onto the
 * column), written here in plain C: populations stored relative to the local
 * rest state w_q s(r) with s(r) the node's density one step earlier (Sec. 5
 * step 1 and the push of step 3), density and half packing fraction stored as
 * deviations from the reference, the moments and the field-velocity predictor
 * of reading R7 (Eq. colonna), the smeared density over the ball (Sec. 3), the
 * shell sums of Eq. campoc and Eq. campod over (+e, -e) pairs, and the
 * collision of Eq. SMDB with second-order forcing and the A-term.
 *
 * Precision: STORE (compile time, float or double) is the type of the stored
 * state and of the moments and smeared density.  Each fluid node then takes one
 * of these variants of the field and collision arithmetic:
 *   fc  pair weights, accumulators, forces and collision in float, with the
 *       in-plane momentum correction of the collision (the kernel in slits);
 *   ff  the same without the correction (the kernel's collision in periodic
 *       boxes);
 *   fd  pair weights, accumulators and forces in float, collision in double
 *       (the arithmetic the library's double-word collision carries out);
 *   df  pair weights, accumulators and forces in double, collision in float;
 *   dd  all of it in double.
 * Nodes within `band` layers of a wall take the variant `band_mode`, the rest
 * `inner_mode`.  `qd` picks the form of Q+ - Q- in the mean-field sum: sym (the
 * kernel's, odd under swapping the pair's ends bit for bit) or asym (the
 * earlier form, which rounds differently at the two ends).
 *
 *   column <nz> <n*> <sigma> <tau> <g_x> <steps> <band> <band_mode> <inner_mode> <qd>
 *
 * prints, per node z: n, v_x, v_z (the field velocity) after the steps, and on
 * stderr the x-momentum balance of the last step's fields: "xforce S D" with S
 * the column's sum of C_x (zero in exact arithmetic: the pair forces conserve
 * momentum) and D the sum of the driving force n g_x.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef STORE
#define STORE float
#endif
#define Q 19

static int C[Q][3];
static double W[Q];
static int OPP[Q];
static int NZ, NP, NB, BZ[64], PE[128][3];
static double SIG, TAU, GX, PK[128][3], WSH, NOFF, HOFF, CHIN, CHALF, BETA, HPRED, SIG2;
static STORE *f[2][Q], *nudn, *nuv[3], *hb, *cprev[3], *tprev;
static double *nscale;
static int cur = 0;
static int QD_ASYM = 0;
static double XF_INNER, XF_DRIVE;

/* D3Q19 in the library's order: rest, faces, edges (Sec. 5). */
static void d3q19(void)
{
    static const int v[Q][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                                {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int q = 0; q < Q; q++) {
        for (int d = 0; d < 3; d++) C[q][d] = v[q][d];
        W[q] = q == 0 ? 1.0 / 3 : (q <= 6 ? 1.0 / 18 : 1.0 / 36);
    }
    for (int a = 0; a < Q; a++)
        for (int b = 0; b < Q; b++)
            if (C[a][0] == -C[b][0] && C[a][1] == -C[b][1] && C[a][2] == -C[b][2]) OPP[a] = b;
}

/* Contact shell as (+e, -e) pairs, +e lexicographically positive (reading R4),
 * and the ball of the smeared density (reading R3, z components only). */
static void tables(void)
{
    int R = (int)floor(SIG + 0.5);
    double lo = (SIG - 0.5) * (SIG - 0.5), hi = (SIG + 0.5) * (SIG + 0.5), second = 0;
    NP = 0;
    for (int dx = 0; dx <= R; dx++)
        for (int dy = -R; dy <= R; dy++)
            for (int dz = -R; dz <= R; dz++) {
                int pos = dx > 0 || (dx == 0 && (dy > 0 || (dy == 0 && dz > 0)));
                double r2 = dx * dx + dy * dy + dz * dz;
                if (!pos || !(r2 > lo && r2 <= hi)) continue;
                double L = sqrt(r2);
                PE[NP][0] = dx; PE[NP][1] = dy; PE[NP][2] = dz;
                PK[NP][0] = (float)(dx / L); PK[NP][1] = (float)(dy / L); PK[NP][2] = (float)(dz / L);
                NP++;
                second += 2.0 * dz * dz / L;
            }
    WSH = (4 * M_PI / 3) * SIG / second;
    int Rb = (int)floor(SIG / 2);
    NB = 0;
    for (int dx = -Rb; dx <= Rb; dx++)
        for (int dy = -Rb; dy <= Rb; dy++)
            for (int dz = -Rb; dz <= Rb; dz++)
                if (4.0 * (dx * dx + dy * dy + dz * dz) <= SIG * SIG) BZ[NB++] = dz;
}

static int wall(int z) { return z == 0 || z == NZ - 1; }

/* Moments and the field-velocity predictor (Eq. colonna, reading R7). */
static void moments(void)
{
    for (int z = 0; z < NZ; z++) {
        if (wall(z)) {
            nudn[z] = (STORE)(-NOFF);
            for (int a = 0; a < 3; a++) nuv[a][z] = 0;
            continue;
        }
        STORE noff = (STORE)NOFF, dsc = (STORE)nscale[z], dl = 0, j[3] = {0, 0, 0};
        for (int q = 0; q < Q; q++) {
            STORE d = f[cur][q][z];
            dl += d;
            for (int a = 0; a < 3; a++)
                if (C[q][a]) j[a] += (STORE)C[q][a] * d;
        }
        STORE dn = dsc + dl, n = noff + dn, inv = (STORE)1 / n, H = (STORE)HPRED * tprev[z],
              den = (STORE)1 / ((STORE)1 + H);
        double g[3] = {GX, 0, 0};
        for (int a = 0; a < 3; a++)
            nuv[a][z] = ((j[a] + (STORE)0.5 * (n * (STORE)g[a] + cprev[a][z])) * inv + H * nuv[a][z]) * den;
        nudn[z] = dn;
    }
}

/* Smeared density as half packing fraction minus its reference (Sec. 3). */
static void ball(void)
{
    for (int z = 0; z < NZ; z++) {
        if (wall(z)) {
            hb[z] = (STORE)(-HOFF);
            continue;
        }
        STORE sum = 0;
        for (int b = 0; b < NB; b++) {
            int zz = z + BZ[b];
            sum += (zz < 0 || zz >= NZ) ? -(STORE)NOFF : nudn[zz];
        }
        hb[z] = (STORE)CHALF * sum;
    }
}

#define DEFINE_FETCH(NAME, TW)                                                     \
    static void NAME(int zz, TW *dn, TW *h, TW v[3])                               \
    {                                                                              \
        if (zz <= 0 || zz >= NZ - 1) {                                             \
            *dn = (TW)(-NOFF); *h = (TW)(-HOFF); v[0] = v[1] = v[2] = 0;           \
            return;                                                                \
        }                                                                          \
        *dn = (TW)nudn[zz]; *h = (TW)hb[zz];                                       \
        for (int a = 0; a < 3; a++) v[a] = (TW)nuv[a][zz];                         \
    }
DEFINE_FETCH(fetch_f, float)
DEFINE_FETCH(fetch_d, double)

#define CORR 0
#define TW float
#define TC float
#define FETCH fetch_f
static void node_ff(int z, int nxt, double *new_nscale)
{
#include "column_node.h"
}
#undef CORR
#define CORR 1
static void node_fc(int z, int nxt, double *new_nscale)
{
#include "column_node.h"
}
#undef CORR
#define CORR 0
#undef TC
#define TC double
static void node_fd(int z, int nxt, double *new_nscale)
{
#include "column_node.h"
}
#undef TC
#define TC float
#undef TW
#undef FETCH
#define TW double
#define FETCH fetch_d
static void node_df(int z, int nxt, double *new_nscale)
{
#include "column_node.h"
}
#undef TC
#define TC double
static void node_dd(int z, int nxt, double *new_nscale)
{
#include "column_node.h"
}
#undef TW
#undef TC
#undef FETCH
#undef CORR

typedef void (*node_fn)(int, int, double *);
static node_fn variant(const char *s)
{
    if (!strcmp(s, "ff")) return node_ff;
    if (!strcmp(s, "fc")) return node_fc;
    if (!strcmp(s, "fd")) return node_fd;
    if (!strcmp(s, "df")) return node_df;
    if (!strcmp(s, "dd")) return node_dd;
    fprintf(stderr, "mode must be fc, ff, fd, df or dd\n");
    exit(2);
}

int main(int argc, char **argv)
{
    if (argc != 11 || (strcmp(argv[10], "sym") && strcmp(argv[10], "asym"))) {
        fprintf(stderr, "column <nz> <n*> <sigma> <tau> <g_x> <steps> <band> <band_mode> <inner_mode> <sym|asym>\n");
        return 2;
    }
    QD_ASYM = !strcmp(argv[10], "asym");
    NZ = atoi(argv[1]);
    double nstar = atof(argv[2]);
    SIG = atof(argv[3]);
    TAU = atof(argv[4]);
    GX = atof(argv[5]);
    long steps = atol(argv[6]);
    int band = atoi(argv[7]);
    node_fn in_band = variant(argv[8]), inner = variant(argv[9]);
    d3q19();
    tables();
    for (int p = 0; p < 2; p++)
        for (int q = 0; q < Q; q++) f[p][q] = calloc(NZ, sizeof(STORE));
    nudn = calloc(NZ, sizeof(STORE));
    hb = calloc(NZ, sizeof(STORE));
    tprev = calloc(NZ, sizeof(STORE));
    for (int a = 0; a < 3; a++) {
        nuv[a] = calloc(NZ, sizeof(STORE));
        cprev[a] = calloc(NZ, sizeof(STORE));
    }
    nscale = calloc(NZ, sizeof(double));
    double *new_nscale = calloc(NZ, sizeof(double));
    /* a uniform fluid at rest: populations at the local equilibrium (zero deviation) */
    NOFF = nstar / (SIG * SIG * SIG);
    CHIN = M_PI * SIG * SIG * SIG / 6;
    HOFF = 0.5 * CHIN * NOFF;
    CHALF = CHIN / (2.0 * NB);
    SIG2 = SIG * SIG;
    BETA = 2 * SIG2 * sqrt((1.0 / 3) / M_PI);
    HPRED = 2.0 * BETA / 6.0;
    for (int z = 0; z < NZ; z++) nudn[z] = wall(z) ? (STORE)(-NOFF) : 0;
    for (long s = 0; s < steps; s++) {
        moments();
        ball();
        int nxt = cur ^ 1;
        for (int q = 0; q < Q; q++) memset(f[nxt][q], 0, NZ * sizeof(STORE));
        XF_INNER = XF_DRIVE = 0;
        for (int z = 1; z < NZ - 1; z++) (z <= band || z >= NZ - 1 - band ? in_band : inner)(z, nxt, new_nscale);
        for (int z = 1; z < NZ - 1; z++) nscale[z] = new_nscale[z];
        cur = nxt;
    }
    moments();
    fprintf(stderr, "xforce %.9g %.9g\n", XF_INNER, XF_DRIVE);
    for (int z = 0; z < NZ; z++) printf("%.17g %.17g %.17g\n", NOFF + (double)nudn[z], (double)nuv[0][z], (double)nuv[2][z]);
    return 0;
}
