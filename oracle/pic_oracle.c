/*
 * pic_oracle.c -- plain FP64 CPU oracle for the 3D PIC / FDTD-Drude time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the bench's CPU
 * baseline leg may load this library; the CUDA product path never does, and
 * the two share no code or headers.  It is written to be read against the
 * paper, not to be fast: one loop per update, full-size arrays everywhere,
 * particles handled one by one in input order.
 *
 * What it computes, per time step n -> n+1 (all FP64, SI units):
 *   1. H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n, forward differences on the
 *      Yee grid (vacuum magnetic update, Sec. II last paragraph), with the
 *      convolutional PML terms in the absorbing slabs.
 *   2. Each live electron: staggered trilinear gather of E^n and of
 *      B^n = mu0 (H^{n-1/2} + H^{n+1/2})/2 at x^n, relativistic Boris
 *      rotation u^{n-1/2} -> u^{n+1/2}, x^{n+1} = x^n + dt u/gamma.  An
 *      electron whose new position would lie within two cells of a
 *      non-periodic face or inside a cell with wp > 0 is frozen instead (its
 *      state is left unchanged and it never moves or deposits again).
 *   3. Charge-conserving current J_f^{n+1/2} from x^n -> x^{n+1}: Esirkepov
 *      decomposition with linear (cloud-in-cell) node shapes.
 *   4. Drude polarisation current first (Eq. 6, with E at level n):
 *        J^{n+1/2} = (2-g dt)/(2+g dt) J^{n-1/2} + 2 dt eps0 wp^2/(2+g dt) E^n
 *      then the Ampere update (Eq. 8, the two curl quotients subtracted):
 *        E^{n+1} = E^n + dt/(eps0 eps_inf) [curl H^{n+1/2} - J^{n+1/2} - J_f^{n+1/2}]
 *      (Sec. II: J is solved first and substituted into the E update; it is
 *      zero where wp is zero.)
 *   5. Probe DFT: F[p][c][f] += E_c^{n+1}(x_p) exp(+i 2 pi f (n+1) dt) dt.
 *
 * Grid and staggering (x fastest, arrays [nz][ny][nx], index (k*ny+j)*nx+i):
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Hx (i, j+1/2, k+1/2)  Hy (i+1/2, j, k+1/2)  Hz (i+1/2, j+1/2, k)
 * On a non-periodic axis the faces sit at node 0 and node n; tangential E on
 * them is held at zero (perfect conductor behind the absorbing layer), node n
 * lies outside the arrays and reads as zero.  Periodic axes wrap.
 *
 * Edge material (the paper gives wp per location, Sec. II): wp^2 on an E edge
 * is the mean of wp^2 over the four cells that share the edge (clamped at
 * non-periodic faces, wrapped on periodic ones); gamma is the wp^2-weighted
 * mean of gamma, eps_inf the plain mean.
 *
 * CPML (Roden-Gedney): depth rho (cells) into an absorbing face slab of L
 * cells, sigma = sigma_fac (m+1)/(eta0 d) (rho/L)^m, kappa = 1 +
 * (kappa_max-1)(rho/L)^m, alpha = alpha_max (1 - rho/L);
 * b = exp(-(sigma/kappa + alpha) dt/eps0), a = sigma (b-1)/(sigma kappa +
 * kappa^2 alpha); psi <- b psi + a dF, and the curl uses dF/kappa + psi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_CFL -2
#define ORC_ERR_OOM -3
#define ORC_ERR_STATE -5

enum { BC_CPML = 0, BC_PEC = 1, BC_PERIODIC = 2 };

typedef struct {
    int comp;                 /* 0,1,2 = Jx,Jy,Jz */
    long box[6];              /* i0,i1,j0,j1,k0,k1 (edge indices, half-open) */
    double amp, t0, tau, f0;  /* A/m^2, s, s, Hz */
} orc_source;

typedef struct {
    long n[3];
    double d[3];
    double dt, eps0, mu0;
    int bc[6];
    int cpml_L;
    double cpml_m, sigma_fac, kappa_max, alpha_max;
    int periodic[3];
    int has_cpml[3];

    uint8_t *mat;
    int nmat;
    double *mtab; /* [nmat][3] wp, gamma, eps_inf */

    double *E[3], *H[3], *Hold[3], *Jp[3], *Jf[3];
    double *psiE[3][3], *psiH[3][3]; /* [field comp][derivative axis] */
    double *kJ[3], *bJ[3], *cE[3];   /* per-edge Drude/Ampere coefficients */
    /* CPML profiles per axis at E positions (integer) and H positions (half) */
    double *bE[3], *aE[3], *ikE[3], *bH[3], *aH[3], *ikH[3];

    long np, npcap;
    double *px, *pu; /* [np][3] position (m), gamma*v (m/s) */
    uint8_t *pstat;
    double q, m;
    int deposit_on;

    int nsrc;
    orc_source src[16];

    int nprobe, nfreq;
    unsigned comp_mask;
    double *probe_xyz; /* [nprobe][3] */
    double *freq;      /* [nfreq] */
    double *F;         /* [nprobe][3][nfreq][2] */
    double *phase_c, *phase_s; /* scratch [nfreq] */

    long step;
} orc_sim;

static long cells(const orc_sim *o) { return o->n[0] * o->n[1] * o->n[2]; }
static long IDX(const orc_sim *o, long i, long j, long k) { return (k * o->n[1] + j) * o->n[0] + i; }

/* Index along axis a for a forward neighbour (i+1); returns -1 for "outside,
 * reads zero" on non-periodic axes. */
static long fwd(const orc_sim *o, int a, long i) {
    long n = o->n[a];
    if (i + 1 < n) return i + 1;
    return o->periodic[a] ? 0 : -1;
}
/* Backward neighbour (i-1): periodic wraps; never requested at i == 0 on a
 * non-periodic axis (those edges are held at zero). */
static long bwd(const orc_sim *o, int a, long i) {
    if (i > 0) return i - 1;
    return o->periodic[a] ? o->n[a] - 1 : 0;
}

static double *zalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* ---------------------------------------------------------------- CPML -- */
static void cpml_profile(const orc_sim *o, int a, double pos, double *b, double *aa, double *ik) {
    /* pos in cell units along axis a */
    double L = (double)o->cpml_L;
    double rho = 0.0;
    long n = o->n[a];
    if (o->has_cpml[a]) {
        if (o->bc[2 * a] == BC_CPML && pos < L) rho = L - pos;
        if (o->bc[2 * a + 1] == BC_CPML && pos > (double)n - L) {
            double r = pos - ((double)n - L);
            if (r > rho) rho = r;
        }
    }
    if (rho <= 0.0) { *b = 1.0; *aa = 0.0; *ik = 1.0; return; }
    double eta0 = sqrt(o->mu0 / o->eps0);
    double x = rho / L;
    double sigma = o->sigma_fac * (o->cpml_m + 1.0) / (eta0 * o->d[a]) * pow(x, o->cpml_m);
    double kappa = 1.0 + (o->kappa_max - 1.0) * pow(x, o->cpml_m);
    double alpha = o->alpha_max * (1.0 - x);
    double bb = exp(-(sigma / kappa + alpha) * o->dt / o->eps0);
    double den = sigma * kappa + kappa * kappa * alpha;
    *b = bb;
    *aa = (sigma > 0.0 && den > 0.0) ? sigma * (bb - 1.0) / den : 0.0;
    *ik = 1.0 / kappa;
}

/* ------------------------------------------------------ edge materials -- */
static long wrapc(const orc_sim *o, int a, long i) {
    long n = o->n[a];
    if (i < 0) return o->periodic[a] ? i + n : 0;
    if (i >= n) return o->periodic[a] ? i - n : n - 1;
    return i;
}

static void edge_coeffs(orc_sim *o) {
    for (int c = 0; c < 3; c++) {
        /* the two transverse axes of component c */
        int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        for (long k = 0; k < o->n[2]; k++)
            for (long j = 0; j < o->n[1]; j++)
                for (long i = 0; i < o->n[0]; i++) {
                    long p[3] = {i, j, k};
                    double sw = 0.0, swg = 0.0, se = 0.0;
                    for (int s1 = -1; s1 <= 0; s1++)
                        for (int s2 = -1; s2 <= 0; s2++) {
                            long q[3] = {p[0], p[1], p[2]};
                            q[a1] = wrapc(o, a1, p[a1] + s1);
                            q[a2] = wrapc(o, a2, p[a2] + s2);
                            int id = o->mat[IDX(o, q[0], q[1], q[2])];
                            double wp = o->mtab[3 * id], g = o->mtab[3 * id + 1], ei = o->mtab[3 * id + 2];
                            sw += wp * wp;
                            swg += wp * wp * g;
                            se += ei;
                        }
                    double wp2 = sw / 4.0;
                    double gam = sw > 0.0 ? swg / sw : 0.0;
                    double einf = se / 4.0;
                    double dt = o->dt;
                    long e = IDX(o, i, j, k);
                    o->kJ[c][e] = (2.0 - gam * dt) / (2.0 + gam * dt);
                    o->bJ[c][e] = 2.0 * dt * o->eps0 * wp2 / (2.0 + gam * dt);
                    o->cE[c][e] = dt / (o->eps0 * einf);
                }
    }
}

/* ------------------------------------------------------------- create -- */
void orc_destroy(orc_sim *o);

orc_sim *orc_create(const long *n, const double *d, double dt, double eps0, double mu0,
                    const int *bc, int cpml_L, double cpml_m, double sigma_fac,
                    double kappa_max, double alpha_max, const uint8_t *mat, int nmat,
                    const double *mtab, int *status) {
    *status = ORC_ERR_ARG;
    for (int a = 0; a < 3; a++) {
        if (n[a] < 1 || d[a] <= 0.0) return NULL;
        int lo = bc[2 * a], hi = bc[2 * a + 1];
        if ((lo == BC_PERIODIC) != (hi == BC_PERIODIC)) return NULL;
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return NULL;
        if ((lo == BC_CPML || hi == BC_CPML) && n[a] < 2 * cpml_L + 4) return NULL;
    }
    double wpmax = 0.0;
    for (int m = 0; m < nmat; m++) {
        if (mtab[3 * m] < 0.0 || mtab[3 * m + 1] < 0.0 || mtab[3 * m + 2] <= 0.0) return NULL;
        if (mtab[3 * m] > wpmax) wpmax = mtab[3 * m];
    }
    double c2 = 1.0 / (eps0 * mu0);
    double s = 0.0;
    for (int a = 0; a < 3; a++) s += 1.0 / (d[a] * d[a]);
    if (!(c2 * dt * dt * s + 0.25 * wpmax * wpmax * dt * dt < 1.0)) { *status = ORC_ERR_CFL; return NULL; }

    orc_sim *o = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!o) { *status = ORC_ERR_OOM; return NULL; }
    for (int a = 0; a < 3; a++) {
        o->n[a] = n[a];
        o->d[a] = d[a];
        o->periodic[a] = bc[2 * a] == BC_PERIODIC;
        o->has_cpml[a] = bc[2 * a] == BC_CPML || bc[2 * a + 1] == BC_CPML;
    }
    for (int f = 0; f < 6; f++) o->bc[f] = bc[f];
    o->dt = dt; o->eps0 = eps0; o->mu0 = mu0;
    o->cpml_L = cpml_L; o->cpml_m = cpml_m; o->sigma_fac = sigma_fac;
    o->kappa_max = kappa_max; o->alpha_max = alpha_max;
    o->deposit_on = 1;
    long N = cells(o);
    o->mat = (uint8_t *)malloc((size_t)N);
    o->nmat = nmat;
    o->mtab = zalloc(3 * nmat);
    for (long e = 0; e < N; e++) {
        if (mat[e] >= nmat) { orc_destroy(o); return NULL; }
        o->mat[e] = mat[e];
    }
    memcpy(o->mtab, mtab, sizeof(double) * 3 * nmat);
    for (int c = 0; c < 3; c++) {
        o->E[c] = zalloc(N); o->H[c] = zalloc(N); o->Hold[c] = zalloc(N);
        o->Jp[c] = zalloc(N); o->Jf[c] = zalloc(N);
        o->kJ[c] = zalloc(N); o->bJ[c] = zalloc(N); o->cE[c] = zalloc(N);
        for (int a = 0; a < 3; a++) { o->psiE[c][a] = zalloc(N); o->psiH[c][a] = zalloc(N); }
        if (!o->E[c] || !o->H[c] || !o->Hold[c] || !o->Jp[c] || !o->Jf[c] || !o->psiE[c][2]) {
            orc_destroy(o); *status = ORC_ERR_OOM; return NULL;
        }
    }
    for (int a = 0; a < 3; a++) {
        long na = o->n[a];
        o->bE[a] = zalloc(na); o->aE[a] = zalloc(na); o->ikE[a] = zalloc(na);
        o->bH[a] = zalloc(na); o->aH[a] = zalloc(na); o->ikH[a] = zalloc(na);
        for (long i = 0; i < na; i++) {
            cpml_profile(o, a, (double)i, &o->bE[a][i], &o->aE[a][i], &o->ikE[a][i]);
            cpml_profile(o, a, (double)i + 0.5, &o->bH[a][i], &o->aH[a][i], &o->ikH[a][i]);
        }
    }
    edge_coeffs(o);
    *status = ORC_OK;
    return o;
}

void orc_destroy(orc_sim *o) {
    if (!o) return;
    for (int c = 0; c < 3; c++) {
        free(o->E[c]); free(o->H[c]); free(o->Hold[c]); free(o->Jp[c]); free(o->Jf[c]);
        free(o->kJ[c]); free(o->bJ[c]); free(o->cE[c]);
        for (int a = 0; a < 3; a++) { free(o->psiE[c][a]); free(o->psiH[c][a]); }
    }
    for (int a = 0; a < 3; a++) {
        free(o->bE[a]); free(o->aE[a]); free(o->ikE[a]);
        free(o->bH[a]); free(o->aH[a]); free(o->ikH[a]);
    }
    free(o->mat); free(o->mtab); free(o->px); free(o->pu); free(o->pstat);
    free(o->probe_xyz); free(o->freq); free(o->F); free(o->phase_c); free(o->phase_s);
    free(o);
}

int orc_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* --------------------------------------------------------- field access -- */
static double *field_ptr(orc_sim *o, int which) {
    /* 0..2 E, 3..5 H, 6..8 Jp, 9..11 Jf */
    if (which < 0 || which > 11) return NULL;
    int c = which % 3;
    switch (which / 3) {
    case 0: return o->E[c];
    case 1: return o->H[c];
    case 2: return o->Jp[c];
    default: return o->Jf[c];
    }
}

int orc_get_field(orc_sim *o, int which, double *out) {
    double *p = field_ptr(o, which);
    if (!p) return ORC_ERR_ARG;
    memcpy(out, p, sizeof(double) * cells(o));
    return ORC_OK;
}

int orc_set_field(orc_sim *o, int which, const double *in) {
    double *p = field_ptr(o, which);
    if (!p || which >= 9) return ORC_ERR_ARG;
    memcpy(p, in, sizeof(double) * cells(o));
    return ORC_OK;
}

/* ------------------------------------------------------------ particles -- */
static int cell_is_metal(const orc_sim *o, const double *xi) {
    long c[3];
    for (int a = 0; a < 3; a++) {
        long f = (long)floor(xi[a]);
        if (o->periodic[a]) { f %= o->n[a]; if (f < 0) f += o->n[a]; }
        if (f < 0) f = 0;
        if (f >= o->n[a]) f = o->n[a] - 1;
        c[a] = f;
    }
    return o->mtab[3 * o->mat[IDX(o, c[0], c[1], c[2])]] > 0.0;
}

/* Position (cell units, periodic axes already wrapped) allowed for a live electron. */
static int position_allowed(const orc_sim *o, const double *xi) {
    for (int a = 0; a < 3; a++) {
        if (o->periodic[a]) continue;
        if (xi[a] < 2.0 || xi[a] >= (double)o->n[a] - 2.0) return 0;
    }
    return !cell_is_metal(o, xi);
}

int orc_add_particles(orc_sim *o, long np, const double *xyz, const double *u, double q, double m,
                      long *n_rejected) {
    if (np < 0 || m <= 0.0) return ORC_ERR_ARG;
    if (o->np > 0 && (q != o->q || m != o->m)) return ORC_ERR_ARG;
    long bad = 0;
    for (long p = 0; p < np; p++) {
        double xi[3];
        for (int a = 0; a < 3; a++) {
            xi[a] = xyz[3 * p + a] / o->d[a];
            if (o->periodic[a]) xi[a] -= floor(xi[a] / (double)o->n[a]) * (double)o->n[a];
        }
        if (!position_allowed(o, xi)) bad++;
    }
    if (n_rejected) *n_rejected = bad;
    if (bad) return ORC_ERR_ARG;
    long nn = o->np + np;
    o->px = (double *)realloc(o->px, sizeof(double) * 3 * (nn > 0 ? nn : 1));
    o->pu = (double *)realloc(o->pu, sizeof(double) * 3 * (nn > 0 ? nn : 1));
    o->pstat = (uint8_t *)realloc(o->pstat, (size_t)(nn > 0 ? nn : 1));
    for (long p = 0; p < np; p++) {
        for (int a = 0; a < 3; a++) {
            double x = xyz[3 * p + a];
            if (o->periodic[a]) {
                double L = o->n[a] * o->d[a];
                x -= floor(x / L) * L;
            }
            o->px[3 * (o->np + p) + a] = x;
            o->pu[3 * (o->np + p) + a] = u[3 * p + a];
        }
        o->pstat[o->np + p] = 0;
    }
    o->np = nn;
    o->q = q;
    o->m = m;
    return ORC_OK;
}

int orc_get_particles(orc_sim *o, double *xyz, double *u, uint8_t *status) {
    if (xyz) memcpy(xyz, o->px, sizeof(double) * 3 * o->np);
    if (u) memcpy(u, o->pu, sizeof(double) * 3 * o->np);
    if (status) memcpy(status, o->pstat, (size_t)o->np);
    return ORC_OK;
}

long orc_num_particles(orc_sim *o) { return o->np; }

void orc_set_deposit(orc_sim *o, int on) { o->deposit_on = on; }

/* Staggered trilinear interpolation of field f with stagger s (0 or 0.5 per
 * axis) at position xi (cell units). */
static double interp(const orc_sim *o, const double *f, const double *stag, const double *xi) {
    long base[3];
    double w1[3];
    for (int a = 0; a < 3; a++) {
        double sa = xi[a] - stag[a];
        double fl = floor(sa);
        base[a] = (long)fl;
        w1[a] = sa - fl;
    }
    double v = 0.0;
    for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++) {
                long i = wrapc(o, 0, base[0] + di), j = wrapc(o, 1, base[1] + dj), k = wrapc(o, 2, base[2] + dk);
                double w = (di ? w1[0] : 1.0 - w1[0]) * (dj ? w1[1] : 1.0 - w1[1]) * (dk ? w1[2] : 1.0 - w1[2]);
                v += w * f[IDX(o, i, j, k)];
            }
    return v;
}

static const double STAG_E[3][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
static const double STAG_H[3][3] = {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};

/* Relativistic Boris step (Boris 1970): u (gamma v, m/s) advanced by dt in
 * fields E (V/m) and B (T) for charge-to-mass ratio qm; c = light speed. */
void orc_boris(double *u, const double *E, const double *B, double qm, double dt, double c) {
    double h = 0.5 * qm * dt;
    double um[3], t[3], s[3], up[3], uq[3];
    for (int a = 0; a < 3; a++) um[a] = u[a] + h * E[a];
    double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) / (c * c));
    for (int a = 0; a < 3; a++) t[a] = h * B[a] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; a++) s[a] = 2.0 * t[a] / (1.0 + t2);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int a = 0; a < 3; a++) u[a] = uq[a] + h * E[a];
}

/* Linear node shape of a particle at local coordinate x on nodes 0..3. */
static void shape4(double x, double *S) {
    for (int m = 0; m < 4; m++) {
        double r = 1.0 - fabs(x - (double)m);
        S[m] = r > 0.0 ? r : 0.0;
    }
}

/* Esirkepov (Comput. Phys. Commun. 135 (2001) 144) current of one particle
 * of charge q moving xi0 -> xi1 (cell units, |xi1-xi0| < 1 per axis) during
 * dt, added into Jf.  Window: nodes floor(xi0)-1 .. floor(xi0)+2 per axis. */
static void esirkepov(orc_sim *o, const double *xi0, const double *xi1, double q) {
    long b[3];
    double S0[3][4], S1[3][4], dS[3][4];
    for (int a = 0; a < 3; a++) {
        b[a] = (long)floor(xi0[a]) - 1;
        shape4(xi0[a] - (double)b[a], S0[a]);
        shape4(xi1[a] - (double)b[a], S1[a]);
        for (int m = 0; m < 4; m++) dS[a][m] = S1[a][m] - S0[a][m];
    }
    for (int c = 0; c < 3; c++) {
        int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        double scale = -q / (o->dt * o->d[a1] * o->d[a2]);
        for (int m2 = 0; m2 < 4; m2++)
            for (int m1 = 0; m1 < 4; m1++) {
                double tr = S0[a1][m1] * S0[a2][m2] + 0.5 * dS[a1][m1] * S0[a2][m2] +
                            0.5 * S0[a1][m1] * dS[a2][m2] + dS[a1][m1] * dS[a2][m2] / 3.0;
                double acc = 0.0;
                for (int m0 = 0; m0 < 3; m0++) {
                    acc += dS[c][m0] * tr;
                    long p[3];
                    p[c] = b[c] + m0;
                    p[a1] = b[a1] + m1;
                    p[a2] = b[a2] + m2;
                    for (int a = 0; a < 3; a++) p[a] = wrapc(o, a, p[a]);
                    o->Jf[c][IDX(o, p[0], p[1], p[2])] += scale * acc;
                }
            }
    }
}

static void push_and_deposit(orc_sim *o) {
    double c = 1.0 / sqrt(o->eps0 * o->mu0);
    double qm = o->q / o->m;
    for (long p = 0; p < o->np; p++) {
        if (o->pstat[p]) continue;
        double xi0[3], E[3], B[3], u[3], xi1[3];
        for (int a = 0; a < 3; a++) { xi0[a] = o->px[3 * p + a] / o->d[a]; u[a] = o->pu[3 * p + a]; }
        for (int cc = 0; cc < 3; cc++) {
            E[cc] = interp(o, o->E[cc], STAG_E[cc], xi0);
            double h0 = interp(o, o->Hold[cc], STAG_H[cc], xi0);
            double h1 = interp(o, o->H[cc], STAG_H[cc], xi0);
            B[cc] = o->mu0 * 0.5 * (h0 + h1);
        }
        orc_boris(u, E, B, qm, o->dt, c);
        double g = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (c * c));
        double xw[3];
        for (int a = 0; a < 3; a++) {
            xi1[a] = xi0[a] + o->dt * u[a] / (g * o->d[a]);
            xw[a] = xi1[a];
            if (o->periodic[a]) xw[a] -= floor(xw[a] / (double)o->n[a]) * (double)o->n[a];
        }
        if (!position_allowed(o, xw)) { o->pstat[p] = 1; continue; }
        if (o->deposit_on) esirkepov(o, xi0, xi1, o->q);
        for (int a = 0; a < 3; a++) { o->px[3 * p + a] = xw[a] * o->d[a]; o->pu[3 * p + a] = u[a]; }
    }
}

/* -------------------------------------------------------------- sources -- */
int orc_add_source(orc_sim *o, int comp, const long *box, double amp, double t0, double tau, double f0) {
    if (o->nsrc >= 16 || comp < 0 || comp > 2 || tau <= 0.0) return ORC_ERR_ARG;
    orc_source *s = &o->src[o->nsrc++];
    s->comp = comp;
    for (int a = 0; a < 6; a++) s->box[a] = box[a];
    s->amp = amp; s->t0 = t0; s->tau = tau; s->f0 = f0;
    return ORC_OK;
}

/* Source waveform: a Gaussian-windowed sine for f0 > 0, the derivative of a
 * Gaussian (no DC part) for f0 == 0. */
static double source_value(const orc_source *s, double t) {
    double x = (t - s->t0) / s->tau;
    double g = exp(-x * x);
    if (s->f0 > 0.0) return s->amp * g * sin(2.0 * M_PI * s->f0 * (t - s->t0));
    return s->amp * (-2.0 * x) * g;
}

static void apply_sources(orc_sim *o) {
    double t = ((double)o->step + 0.5) * o->dt;
    for (int q = 0; q < o->nsrc; q++) {
        const orc_source *s = &o->src[q];
        double v = source_value(s, t);
        for (long k = s->box[4]; k < s->box[5]; k++)
            for (long j = s->box[2]; j < s->box[3]; j++)
                for (long i = s->box[0]; i < s->box[1]; i++)
                    o->Jf[s->comp][IDX(o, i, j, k)] += v;
    }
}

/* --------------------------------------------------------------- fields -- */
static void update_H(orc_sim *o) {
    const long nx = o->n[0], ny = o->n[1], nz = o->n[2];
    const double cH = o->dt / o->mu0;
    const double rx = 1.0 / o->d[0], ry = 1.0 / o->d[1], rz = 1.0 / o->d[2];
    double *Ex = o->E[0], *Ey = o->E[1], *Ez = o->E[2];
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; k++) {
        long kp = fwd(o, 2, k);
        for (long j = 0; j < ny; j++) {
            long jp = fwd(o, 1, j);
            for (long i = 0; i < nx; i++) {
                long ip = fwd(o, 0, i);
                long e = IDX(o, i, j, k);
                double ex = Ex[e], ey = Ey[e], ez = Ez[e];
                double ez_jp = jp < 0 ? 0.0 : Ez[IDX(o, i, jp, k)];
                double ey_kp = kp < 0 ? 0.0 : Ey[IDX(o, i, j, kp)];
                double ex_kp = kp < 0 ? 0.0 : Ex[IDX(o, i, j, kp)];
                double ez_ip = ip < 0 ? 0.0 : Ez[IDX(o, ip, j, k)];
                double ey_ip = ip < 0 ? 0.0 : Ey[IDX(o, ip, j, k)];
                double ex_jp = jp < 0 ? 0.0 : Ex[IDX(o, i, jp, k)];
                double dEz_dy = (ez_jp - ez) * ry, dEy_dz = (ey_kp - ey) * rz;
                double dEx_dz = (ex_kp - ex) * rz, dEz_dx = (ez_ip - ez) * rx;
                double dEy_dx = (ey_ip - ey) * rx, dEx_dy = (ex_jp - ex) * ry;
                double *pxy = &o->psiH[0][1][e], *pxz = &o->psiH[0][2][e];
                double *pyz = &o->psiH[1][2][e], *pyx = &o->psiH[1][0][e];
                double *pzx = &o->psiH[2][0][e], *pzy = &o->psiH[2][1][e];
                *pxy = o->bH[1][j] * *pxy + o->aH[1][j] * dEz_dy;
                *pxz = o->bH[2][k] * *pxz + o->aH[2][k] * dEy_dz;
                *pyz = o->bH[2][k] * *pyz + o->aH[2][k] * dEx_dz;
                *pyx = o->bH[0][i] * *pyx + o->aH[0][i] * dEz_dx;
                *pzx = o->bH[0][i] * *pzx + o->aH[0][i] * dEy_dx;
                *pzy = o->bH[1][j] * *pzy + o->aH[1][j] * dEx_dy;
                double cx = o->ikH[1][j] * dEz_dy + *pxy - o->ikH[2][k] * dEy_dz - *pxz;
                double cy = o->ikH[2][k] * dEx_dz + *pyz - o->ikH[0][i] * dEz_dx - *pyx;
                double cz = o->ikH[0][i] * dEy_dx + *pzx - o->ikH[1][j] * dEx_dy - *pzy;
                o->H[0][e] -= cH * cx;
                o->H[1][e] -= cH * cy;
                o->H[2][e] -= cH * cz;
            }
        }
    }
}

static void update_E(orc_sim *o) {
    const long nx = o->n[0], ny = o->n[1], nz = o->n[2];
    const double rx = 1.0 / o->d[0], ry = 1.0 / o->d[1], rz = 1.0 / o->d[2];
    double *Hx = o->H[0], *Hy = o->H[1], *Hz = o->H[2];
    const int npx = !o->periodic[0], npy = !o->periodic[1], npz = !o->periodic[2];
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; k++) {
        long km = bwd(o, 2, k);
        for (long j = 0; j < ny; j++) {
            long jm = bwd(o, 1, j);
            for (long i = 0; i < nx; i++) {
                long im = bwd(o, 0, i);
                long e = IDX(o, i, j, k);
                /* Ex (i+1/2, j, k): tangential on y and z faces */
                if (!((npy && j == 0) || (npz && k == 0))) {
                    double dHz_dy = (Hz[e] - Hz[IDX(o, i, jm, k)]) * ry;
                    double dHy_dz = (Hy[e] - Hy[IDX(o, i, j, km)]) * rz;
                    double *py = &o->psiE[0][1][e], *pz = &o->psiE[0][2][e];
                    *py = o->bE[1][j] * *py + o->aE[1][j] * dHz_dy;
                    *pz = o->bE[2][k] * *pz + o->aE[2][k] * dHy_dz;
                    double curl = o->ikE[1][j] * dHz_dy + *py - o->ikE[2][k] * dHy_dz - *pz;
                    o->Jp[0][e] = o->kJ[0][e] * o->Jp[0][e] + o->bJ[0][e] * o->E[0][e];
                    o->E[0][e] += o->cE[0][e] * (curl - o->Jp[0][e] - o->Jf[0][e]);
                }
                /* Ey (i, j+1/2, k) */
                if (!((npx && i == 0) || (npz && k == 0))) {
                    double dHx_dz = (Hx[e] - Hx[IDX(o, i, j, km)]) * rz;
                    double dHz_dx = (Hz[e] - Hz[IDX(o, im, j, k)]) * rx;
                    double *pz = &o->psiE[1][2][e], *px = &o->psiE[1][0][e];
                    *pz = o->bE[2][k] * *pz + o->aE[2][k] * dHx_dz;
                    *px = o->bE[0][i] * *px + o->aE[0][i] * dHz_dx;
                    double curl = o->ikE[2][k] * dHx_dz + *pz - o->ikE[0][i] * dHz_dx - *px;
                    o->Jp[1][e] = o->kJ[1][e] * o->Jp[1][e] + o->bJ[1][e] * o->E[1][e];
                    o->E[1][e] += o->cE[1][e] * (curl - o->Jp[1][e] - o->Jf[1][e]);
                }
                /* Ez (i, j, k+1/2) */
                if (!((npx && i == 0) || (npy && j == 0))) {
                    double dHy_dx = (Hy[e] - Hy[IDX(o, im, j, k)]) * rx;
                    double dHx_dy = (Hx[e] - Hx[IDX(o, i, jm, k)]) * ry;
                    double *px = &o->psiE[2][0][e], *py = &o->psiE[2][1][e];
                    *px = o->bE[0][i] * *px + o->aE[0][i] * dHy_dx;
                    *py = o->bE[1][j] * *py + o->aE[1][j] * dHx_dy;
                    double curl = o->ikE[0][i] * dHy_dx + *px - o->ikE[1][j] * dHx_dy - *py;
                    o->Jp[2][e] = o->kJ[2][e] * o->Jp[2][e] + o->bJ[2][e] * o->E[2][e];
                    o->E[2][e] += o->cE[2][e] * (curl - o->Jp[2][e] - o->Jf[2][e]);
                }
            }
        }
    }
}

/* --------------------------------------------------------------- probes -- */
int orc_probe_dft(orc_sim *o, int np, const double *xyz, unsigned comp_mask, int nf, const double *freq) {
    if (np < 0 || nf < 0 || (comp_mask & ~7u)) return ORC_ERR_ARG;
    for (int p = 0; p < np; p++)
        for (int a = 0; a < 3; a++) {
            double xi = xyz[3 * p + a] / o->d[a];
            if (!o->periodic[a] && (xi < 1.0 || xi >= (double)o->n[a] - 1.0)) return ORC_ERR_ARG;
        }
    free(o->probe_xyz); free(o->freq); free(o->F); free(o->phase_c); free(o->phase_s);
    o->nprobe = np; o->nfreq = nf; o->comp_mask = comp_mask;
    o->probe_xyz = zalloc(3 * np);
    memcpy(o->probe_xyz, xyz, sizeof(double) * 3 * np);
    o->freq = zalloc(nf);
    memcpy(o->freq, freq, sizeof(double) * nf);
    o->F = zalloc((long)np * 3 * nf * 2);
    o->phase_c = zalloc(nf);
    o->phase_s = zalloc(nf);
    return ORC_OK;
}

static void probe_accumulate(orc_sim *o) {
    if (o->nprobe == 0) return;
    double t = (double)(o->step + 1) * o->dt;
    for (int f = 0; f < o->nfreq; f++) {
        double th = 2.0 * M_PI * o->freq[f] * t;
        o->phase_c[f] = cos(th);
        o->phase_s[f] = sin(th);
    }
    for (int p = 0; p < o->nprobe; p++) {
        double xi[3];
        for (int a = 0; a < 3; a++) xi[a] = o->probe_xyz[3 * p + a] / o->d[a];
        for (int c = 0; c < 3; c++) {
            if (!(o->comp_mask & (1u << c))) continue;
            double v = interp(o, o->E[c], STAG_E[c], xi) * o->dt;
            double *F = o->F + ((long)p * 3 + c) * o->nfreq * 2;
            for (int f = 0; f < o->nfreq; f++) {
                F[2 * f] += v * o->phase_c[f];
                F[2 * f + 1] += v * o->phase_s[f];
            }
        }
    }
}

int orc_probe_read(orc_sim *o, double *out) {
    if (o->nprobe == 0) return ORC_ERR_STATE;
    memcpy(out, o->F, sizeof(double) * (long)o->nprobe * 3 * o->nfreq * 2);
    return ORC_OK;
}

/* ----------------------------------------------------------------- step -- */
int orc_step(orc_sim *o, long nsteps) {
    if (nsteps < 0) return ORC_ERR_ARG;
    long N = cells(o);
    for (long s = 0; s < nsteps; s++) {
        for (int c = 0; c < 3; c++) memcpy(o->Hold[c], o->H[c], sizeof(double) * N);
        update_H(o);
        for (int c = 0; c < 3; c++) memset(o->Jf[c], 0, sizeof(double) * N);
        push_and_deposit(o);
        apply_sources(o);
        update_E(o);
        probe_accumulate(o);
        o->step++;
    }
    return ORC_OK;
}

long orc_get_step(orc_sim *o) { return o->step; }

/* Edge coefficients, for inspection by tests: which 0..2 = kJ, bJ, cE. */
int orc_get_coeff(orc_sim *o, int which, int comp, double *out) {
    if (comp < 0 || comp > 2 || which < 0 || which > 2) return ORC_ERR_ARG;
    double *src = which == 0 ? o->kJ[comp] : which == 1 ? o->bJ[comp] : o->cE[comp];
    memcpy(out, src, sizeof(double) * cells(o));
    return ORC_OK;
}
