/*
 * FP64 CPU oracle for the per-timestep hot path of the two-component Shan-Chen D3Q19 lattice Boltzmann
 * method coupled to triangulated capsule membranes (Wouters, Aouane, Krueger, Harting, arXiv:1904.11386).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA path: naive array-of-structures layout f[node][19], two
 * lattices, push streaming, double precision everywhere, no blocking or fusion beyond what the equations
 * state.  Every function names the passage of the paper it follows.
 *
 * Parity status (what pins each function; the pins live in tests/test_oracle_*.py):
 *   fluid collide/stream (Eq. 1-5, Sec. II.A)        mass conservation, Poiseuille order, Couette sign
 *   Shan-Chen force (Eq. 13, Sec. II.D)             Laplace law gamma = 0.0388 (Sec. III), flat interface
 *   Skalak / volume forces (Eq. 6-8, Sec. II.B)      finite-difference gradients, net force/torque, rest shape
 *   Helfrich-Meyer bending (Eq. 9-10, Sec. II.B)     Gauss-Bonnet, mixed-area partition, spheroid curvatures,
 *                                                    energy-descent cosine
 *   2-point immersed boundary (not in the paper)     adjoint identity, partition of unity, linear exactness
 *   particle-particle repulsion (Eq. 26, Sec. III.E) brute-force pair sum, Newton's third law
 *   bounce-back coupling, wetting, fresh nodes (Sec. II.C-E): see the second part of this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------------------------- */
/* D3Q19 velocity set and weights (Eq. 3).  Ordering: rest, +-x, +-y, +-z, then the 12 diagonals, each    */
/* direction followed by its opposite.                                                                    */
/* ---------------------------------------------------------------------------------------------------- */
static const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W[19] = {1.0 / 3,
                             1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

#define CS2 (1.0 / 3.0)
#define OWNER_WALL 0xFFFF

int o_d3q19(int* cx, int* cy, int* cz, double* w, int* opp) {
    for (int i = 0; i < 19; i++) {
        cx[i] = CX[i]; cy[i] = CY[i]; cz[i] = CZ[i]; w[i] = W[i]; opp[i] = OPP(i);
    }
    return 19;
}

int o_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void o_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------------------------------- */
/* Problem description                                                                                   */
/* ---------------------------------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int walls;              /* 1: wall planes z=0 and z=nz-1, else periodic in z */
    double u_lo[3], u_hi[3];/* wall velocities */
    double tau, G;
    int psi_kind;           /* 0: 1-exp(-rho), 1: rho */
    double g[3];            /* body acceleration: force density rho^c g on component c */
    int coupling;           /* 0: bounce-back (paper), 1: 2-point immersed boundary, 2: no capsules */
    double rho_maj, rho_min, C0;
    int mass_correction;
    double pp_eps, pp_d0;
    int wall_kind;          /* 0: walls moving at u_lo / u_hi (half-way bounce-back, Eq. 11); 1: resting walls and
                               on-site velocity boundaries u_lo / u_hi on the planes z = 1 and z = nz-2 */
} o_params;

typedef struct {
    int nv, nt;
    double kS, C, kB, kV, mass, colour;
} o_mesh_params;

typedef struct {
    o_params p;
    long N;
    double* f;              /* [2][N][19] */
    double* fn;             /* [2][N][19] */
    double* rho;            /* [2][N] */
    double* psi;            /* [2][N] pseudo-potential of rho */
    double* u;              /* [3][N] velocity incl. half force, last collision */
    double* Fibm;           /* [3][N] spread force density */
    double* Fsc;            /* [2][3][N] Shan-Chen force of the last step (diagnostic) */
    uint16_t* owner;        /* [N]: 0 bulk fluid, k+1 inside capsule k, OWNER_WALL for wall nodes */
    uint16_t* owner_old;
    /* capsules */
    int nm;
    o_mesh_params* mp;
    double* ecol;           /* [T] colour of each element (NULL: the capsule's colour on every element) */
    int* voff;              /* vertex offset per capsule (nm+1) */
    int* toff;              /* triangle offset per capsule (nm+1) */
    int* tri;               /* global vertex ids [T][3] */
    double* X;              /* [V][3] */
    double* Vel;            /* [V][3] */
    double* F;              /* [V][3] total node force of the last step */
    double* refX;           /* [V][3] reference shape */
    double* V0;             /* reference volume per capsule */
    /* bounce-back coupling state (second part) */
    double* emom_now;       /* [T][3] momentum handed to elements in the current step */
    double* emom_prev;      /* [T][3] previous step (two-step smoothing) */
    double* epend;          /* [T][3] momenta applied without smoothing (SC reactions, fresh nodes) */
    double M0[2];
    double Vsys;
    long n_fresh_total, n_fresh_fallback;
    /* boundary table rebuilt after each classification: node -> row, row -> crossed element per direction */
    int* brow;              /* [N] row of a boundary node, -1 otherwise */
    int* belem;             /* [rows][19] crossed element of each cut membrane link, -1 if not cut */
    long nb, nb_cap;
    long n_elem_fallback;
    double* blink;          /* [rows][19][6] per cut link: exchanged momentum (0..2), SC reaction (3..5) */
    long step;
} osim;

static inline long IDX(const osim* s, int x, int y, int z) {
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}
static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static inline int is_wall_z(const osim* s, int z) { return s->p.walls && (z == 0 || z == s->p.nz - 1); }

/* velocity of the wall plane z (zero for resting walls next to on-site velocity planes) */
static double wall_u(const osim* s, int z, int k) {
    if (s->p.wall_kind == 1) return 0.0;
    return z == 0 ? s->p.u_lo[k] : s->p.u_hi[k];
}

/* neighbour of (x,y,z) along direction i; returns -1 if it leaves a non-periodic z range */
static long nbr(const osim* s, int x, int y, int z, int i, int* zz_out) {
    int xx = wrap(x + CX[i], s->p.nx), yy = wrap(y + CY[i], s->p.ny), zz = z + CZ[i];
    if (s->p.walls) {
        if (zz < 0 || zz >= s->p.nz) return -1;
    } else {
        zz = wrap(zz, s->p.nz);
    }
    if (zz_out) *zz_out = zz;
    return IDX(s, xx, yy, zz);
}

/* ---------------------------------------------------------------------------------------------------- */
/* Equilibrium (Eq. 2) and pseudo-potential (Sec. II.D, below Eq. 13: psi = 1 - exp(-rho/rho0), rho0 = 1)              */
/* ---------------------------------------------------------------------------------------------------- */
static double feq(int i, double rho, const double u[3]) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

static double psi_of(const osim* s, double rho) {
    return s->p.psi_kind == 1 ? rho : 1.0 - exp(-rho);
}

double o_feq(int i, double rho, double ux, double uy, double uz) {
    double u[3] = {ux, uy, uz};
    return feq(i, rho, u);
}

/* ---------------------------------------------------------------------------------------------------- */
/* Creation / state access                                                                              */
/* ---------------------------------------------------------------------------------------------------- */
osim* o_create(const o_params* p, int nm, const o_mesh_params* mp, const int* tri_local,
               const double* refX, const double* initX) {
    osim* s = (osim*)calloc(1, sizeof(osim));
    s->p = *p;
    long N = (long)p->nx * p->ny * p->nz;
    s->N = N;
    s->f = (double*)calloc((size_t)2 * N * 19, sizeof(double));
    s->fn = (double*)calloc((size_t)2 * N * 19, sizeof(double));
    s->rho = (double*)calloc((size_t)2 * N, sizeof(double));
    s->psi = (double*)calloc((size_t)2 * N, sizeof(double));
    s->u = (double*)calloc((size_t)3 * N, sizeof(double));
    s->Fibm = (double*)calloc((size_t)3 * N, sizeof(double));
    s->Fsc = (double*)calloc((size_t)6 * N, sizeof(double));
    s->owner = (uint16_t*)calloc((size_t)N, sizeof(uint16_t));
    s->owner_old = (uint16_t*)calloc((size_t)N, sizeof(uint16_t));
    for (int z = 0; z < p->nz; z++)
        if (is_wall_z(s, z))
            for (int y = 0; y < p->ny; y++)
                for (int x = 0; x < p->nx; x++) s->owner[IDX(s, x, y, z)] = OWNER_WALL;
    memcpy(s->owner_old, s->owner, (size_t)N * sizeof(uint16_t));
    s->nm = nm;
    s->mp = (o_mesh_params*)calloc((size_t)(nm > 0 ? nm : 1), sizeof(o_mesh_params));
    s->voff = (int*)calloc((size_t)nm + 1, sizeof(int));
    s->toff = (int*)calloc((size_t)nm + 1, sizeof(int));
    for (int m = 0; m < nm; m++) {
        s->mp[m] = mp[m];
        s->voff[m + 1] = s->voff[m] + mp[m].nv;
        s->toff[m + 1] = s->toff[m] + mp[m].nt;
    }
    int NV = s->voff[nm], NT = s->toff[nm];
    s->tri = (int*)calloc((size_t)3 * (NT > 0 ? NT : 1), sizeof(int));
    s->X = (double*)calloc((size_t)3 * (NV > 0 ? NV : 1), sizeof(double));
    s->Vel = (double*)calloc((size_t)3 * (NV > 0 ? NV : 1), sizeof(double));
    s->F = (double*)calloc((size_t)3 * (NV > 0 ? NV : 1), sizeof(double));
    s->refX = (double*)calloc((size_t)3 * (NV > 0 ? NV : 1), sizeof(double));
    s->V0 = (double*)calloc((size_t)(nm > 0 ? nm : 1), sizeof(double));
    s->emom_now = (double*)calloc((size_t)3 * (NT > 0 ? NT : 1), sizeof(double));
    s->emom_prev = (double*)calloc((size_t)3 * (NT > 0 ? NT : 1), sizeof(double));
    s->epend = (double*)calloc((size_t)3 * (NT > 0 ? NT : 1), sizeof(double));
    for (int m = 0; m < nm; m++)
        for (int t = 0; t < mp[m].nt; t++)
            for (int k = 0; k < 3; k++)
                s->tri[3 * (s->toff[m] + t) + k] = tri_local[3 * (s->toff[m] + t) + k] + s->voff[m];
    if (NV > 0) {
        memcpy(s->refX, refX, (size_t)3 * NV * sizeof(double));
        memcpy(s->X, initX, (size_t)3 * NV * sizeof(double));
    }
    return s;
}

void o_destroy(osim* s) {
    if (!s) return;
    free(s->f); free(s->fn); free(s->rho); free(s->psi); free(s->u); free(s->Fibm); free(s->Fsc);
    free(s->owner); free(s->owner_old); free(s->mp); free(s->voff); free(s->toff); free(s->tri);
    free(s->X); free(s->Vel); free(s->F); free(s->refX); free(s->V0);
    free(s->emom_now); free(s->emom_prev); free(s->epend); free(s->brow); free(s->belem); free(s->blink);
    free(s->ecol);
    free(s);
}

/* Colour of each element (Sec. V: an individually coloured particle surface, a Janus particle), T values in the
   global triangle order; NULL restores the capsules' uniform colours. */
void o_set_elem_colour(osim* s, const double* col) {
    free(s->ecol);
    s->ecol = NULL;
    if (!col || s->nm == 0) return;
    const int T = s->toff[s->nm];
    s->ecol = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    memcpy(s->ecol, col, sizeof(double) * (size_t)T);
}

/* populations f = f_eq(rho^c, u) on every node (wall nodes included; they are never used as fluid) */
static void onsite_velocity(osim* s);

/* Initial state: f = f_eq(rho, u) at every node; with on-site velocity planes the state satisfies their
   boundary condition from the start (the populations they would receive from the walls are reconstructed, as
   after every streaming step). */
void o_set_state(osim* s, const double* rhoA, const double* rhoB, const double* u /* [3][N] or NULL */) {
    for (long n = 0; n < s->N; n++) {
        double uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[n]; uu[1] = u[s->N + n]; uu[2] = u[2 * s->N + n]; }
        for (int i = 0; i < 19; i++) {
            s->f[(0 * s->N + n) * 19 + i] = feq(i, rhoA[n], uu);
            s->f[(1 * s->N + n) * 19 + i] = feq(i, rhoB[n], uu);
        }
        s->rho[n] = rhoA[n];
        s->rho[s->N + n] = rhoB[n];
    }
    if (s->p.walls && s->p.wall_kind == 1) onsite_velocity(s);
}

void o_get_f(const osim* s, double* out) { memcpy(out, s->f, sizeof(double) * 2 * 19 * s->N); }
void o_set_f(osim* s, const double* in) { memcpy(s->f, in, sizeof(double) * 2 * 19 * s->N); }

/* rho^c = sum_i f_i^c (Eq. 4, rho0 = 1) for every non-wall node */
static void compute_rho(osim* s) {
    long N = s->N;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        for (int c = 0; c < 2; c++) {
            double r = 0;
            if (s->owner[n] != OWNER_WALL)
                for (int i = 0; i < 19; i++) r += s->f[(c * N + n) * 19 + i];
            s->rho[c * N + n] = r;
            s->psi[c * N + n] = psi_of(s, r);
        }
    }
}

/* densities and barycentric velocity of the current state (Eq. 4-5 without the half force):
   rho^c = sum_i f_i^c, u = sum_c sum_i f_i^c c_i / sum_c rho^c; wall nodes report 0 */
void o_get_fields(osim* s, double* rhoA, double* rhoB, double* u) {
    compute_rho(s);
    long N = s->N;
    for (long n = 0; n < N; n++) {
        if (rhoA) rhoA[n] = s->rho[n];
        if (rhoB) rhoB[n] = s->rho[N + n];
        if (!u) continue;
        double j[3] = {0, 0, 0};
        double rt = s->rho[n] + s->rho[N + n];
        if (s->owner[n] != OWNER_WALL && rt > 0)
            for (int c = 0; c < 2; c++)
                for (int i = 0; i < 19; i++) {
                    double fi = s->f[(c * N + n) * 19 + i];
                    j[0] += fi * CX[i]; j[1] += fi * CY[i]; j[2] += fi * CZ[i];
                }
        for (int k = 0; k < 3; k++) u[k * N + n] = rt > 0 ? j[k] / rt : 0.0;
    }
}

void o_get_fsc(const osim* s, double* out) { memcpy(out, s->Fsc, sizeof(double) * 6 * s->N); }

double o_mass(osim* s, int c) {
    compute_rho(s);
    double m = 0;
    for (long n = 0; n < s->N; n++)
        if (s->owner[n] != OWNER_WALL) m += s->rho[c * s->N + n];
    return m;
}

/* total fluid momentum sum_c sum_n sum_i f c (no half force) */
void o_momentum(const osim* s, double* out3) {
    double m[3] = {0, 0, 0};
    for (long n = 0; n < s->N; n++) {
        if (s->owner[n] == OWNER_WALL) continue;
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < 19; i++) {
                double fi = s->f[(c * s->N + n) * 19 + i];
                m[0] += fi * CX[i]; m[1] += fi * CY[i]; m[2] += fi * CZ[i];
            }
    }
    out3[0] = m[0]; out3[1] = m[1]; out3[2] = m[2];
}

void o_get_vertices(const osim* s, double* X, double* V, double* F) {
    int NV = s->voff[s->nm];
    if (X) memcpy(X, s->X, sizeof(double) * 3 * NV);
    if (V) memcpy(V, s->Vel, sizeof(double) * 3 * NV);
    if (F) memcpy(F, s->F, sizeof(double) * 3 * NV);
}

void o_set_vertices(osim* s, const double* X, const double* V) {
    int NV = s->voff[s->nm];
    if (X) memcpy(s->X, X, sizeof(double) * 3 * NV);
    if (V) memcpy(s->Vel, V, sizeof(double) * 3 * NV);
}

void o_get_owner(const osim* s, uint16_t* out) { memcpy(out, s->owner, sizeof(uint16_t) * s->N); }

/* ---------------------------------------------------------------------------------------------------- */
/* Membrane mechanics (Sec. II.B)                                                                        */
/* ---------------------------------------------------------------------------------------------------- */
static void sub3(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/*
 * Skalak strain energy (Eq. 6) on linear triangles, integrated over the reference (stress-free) area A0.
 * The invariants of the in-plane right Cauchy-Green tensor are frame-free:
 *   tr G = tr(g0^{-1} g),  det G = det g / det g0
 * with g, g0 the 2x2 metric tensors (Gram matrices) of the current and reference edge vectors
 * e1 = x2 - x1, e2 = x3 - x1.  I1 = tr G - 2 = lambda1^2 + lambda2^2 - 2, I2 = det G - 1.
 * Nodal forces are F = -dE/dx (Eq. 8), differentiated analytically through (g11, g12, g22).
 * F may be NULL (energy only).  Returns the energy.
 */
double o_skalak(int nv, int nt, const double* x, const int* tri, const double* ref, double kS, double C,
                double* F) {
    double E = 0;
    if (F) memset(F, 0, sizeof(double) * 3 * nv);
    for (int t = 0; t < nt; t++) {
        int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        double r1[3], r2[3], e1[3], e2[3];
        sub3(ref + 3 * b, ref + 3 * a, r1); sub3(ref + 3 * c, ref + 3 * a, r2);
        sub3(x + 3 * b, x + 3 * a, e1); sub3(x + 3 * c, x + 3 * a, e2);
        double P = dot3(r1, r1), Q = dot3(r1, r2), R = dot3(r2, r2);
        double det0 = P * R - Q * Q;
        double A0 = 0.5 * sqrt(det0);
        /* inverse of g0 = [[P,Q],[Q,R]] */
        double ia = R / det0, ib = -Q / det0, ic = P / det0;
        double p = dot3(e1, e1), q = dot3(e1, e2), r = dot3(e2, e2);
        double trG = ia * p + 2 * ib * q + ic * r;
        double detG = (p * r - q * q) / det0;
        double I1 = trG - 2.0, I2 = detG - 1.0;
        double pre = kS / 4.0 * A0;
        E += pre * (I1 * I1 + 2 * I1 - 2 * I2 + C * I2 * I2);
        if (!F) continue;
        double dW1 = pre * (2 * I1 + 2), dW2 = pre * (-2 + 2 * C * I2);
        double Wp = dW1 * ia + dW2 * r / det0;
        double Wq = dW1 * 2 * ib + dW2 * (-2 * q) / det0;
        double Wr = dW1 * ic + dW2 * p / det0;
        double g1[3], g2[3];        /* dE/de1, dE/de2 */
        for (int k = 0; k < 3; k++) {
            g1[k] = 2 * Wp * e1[k] + Wq * e2[k];
            g2[k] = Wq * e1[k] + 2 * Wr * e2[k];
        }
        for (int k = 0; k < 3; k++) {
            F[3 * b + k] -= g1[k];
            F[3 * c + k] -= g2[k];
            F[3 * a + k] += g1[k] + g2[k];
        }
    }
    return E;
}

/* enclosed volume V = sum_T x1 . (x2 x x3) / 6 for outward-oriented triangles */
double o_volume(int nv, int nt, const double* x, const int* tri) {
    (void)nv;
    double V = 0;
    for (int t = 0; t < nt; t++) {
        const double *a = x + 3 * tri[3 * t], *b = x + 3 * tri[3 * t + 1], *c = x + 3 * tri[3 * t + 2];
        double bc[3];
        cross3(b, c, bc);
        V += dot3(a, bc) / 6.0;
    }
    return V;
}

/* volume penalty (Eq. 7): E = kV/2 (V-V0)^2/V0, F_b = -kV (V-V0)/V0 dV/dx_b.  Adds into F.  Returns E. */
double o_volume_force(int nv, int nt, const double* x, const int* tri, double kV, double V0, double* F) {
    double V = o_volume(nv, nt, x, tri);
    double k = -kV * (V - V0) / V0;
    if (F)
        for (int t = 0; t < nt; t++) {
            int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
            const double *a = x + 3 * ia, *b = x + 3 * ib, *c = x + 3 * ic;
            double da[3], db[3], dc[3];
            cross3(b, c, da); cross3(c, a, db); cross3(a, b, dc);
            for (int q = 0; q < 3; q++) {
                F[3 * ia + q] += k * da[q] / 6.0;
                F[3 * ib + q] += k * db[q] / 6.0;
                F[3 * ic + q] += k * dc[q] / 6.0;
            }
        }
    return 0.5 * kV * (V - V0) * (V - V0) / V0;
}

/*
 * Helfrich bending (Eq. 9-10) with the discrete differential-geometry operators of Meyer et al.:
 *   A_i     mixed Voronoi area (obtuse triangles: half / quarter of the triangle area)
 *   K_i     = 1/(2 A_i) sum_j (cot a_ij + cot b_ij)(x_i - x_j)      mean-curvature normal (= 2 H n)
 *   n_i     area-weighted average of the outward face normals
 *   H_i     = K_i . n_i / 2        (H = 1/R > 0 on a sphere)
 *   KG_i    = (2 pi - sum of the angles at i) / A_i
 *   LH_i    = 1/(2 A_i) sum_j (cot a_ij + cot b_ij)(H_j - H_i)       Laplace-Beltrami of H
 *   F_i     = 2 kB [2 H (H^2 - KG) + LH] A_i n_i                      (force density x Voronoi area)
 * Optional outputs (NULL to skip): F (adds), H, KG, A, LH, n.  Returns the discrete energy
 * E = kB/2 sum_i (2 H_i)^2 A_i.
 */
double o_bending(int nv, int nt, const double* x, const int* tri, double kB, double* F, double* Hout,
                 double* KGout, double* Aout, double* LHout, double* nout) {
    double* A = (double*)calloc((size_t)nv, sizeof(double));
    double* Kv = (double*)calloc((size_t)3 * nv, sizeof(double));
    double* ang = (double*)calloc((size_t)nv, sizeof(double));
    double* nn = (double*)calloc((size_t)3 * nv, sizeof(double));
    double* H = (double*)calloc((size_t)nv, sizeof(double));
    double* LH = (double*)calloc((size_t)nv, sizeof(double));
    double* cotw = (double*)calloc((size_t)3 * nt, sizeof(double));   /* cot of the angle at vertex k of t */
    for (int t = 0; t < nt; t++) {
        int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        double th[3], e[3][3], l2[3];
        for (int k = 0; k < 3; k++) {
            /* edge opposite vertex k: from v[k+1] to v[k+2] */
            sub3(x + 3 * v[(k + 2) % 3], x + 3 * v[(k + 1) % 3], e[k]);
            l2[k] = dot3(e[k], e[k]);
        }
        double nrm[3], u1[3], u2[3];
        sub3(x + 3 * v[1], x + 3 * v[0], u1); sub3(x + 3 * v[2], x + 3 * v[0], u2);
        cross3(u1, u2, nrm);
        double area = 0.5 * norm3(nrm);
        for (int k = 0; k < 3; k++) {
            double a1[3], a2[3];
            sub3(x + 3 * v[(k + 1) % 3], x + 3 * v[k], a1);
            sub3(x + 3 * v[(k + 2) % 3], x + 3 * v[k], a2);
            double cs = dot3(a1, a2);
            double cr[3];
            cross3(a1, a2, cr);
            double sn = norm3(cr);
            th[k] = atan2(sn, cs);
            cotw[3 * t + k] = cs / sn;
        }
        int obtuse = -1;
        for (int k = 0; k < 3; k++) if (th[k] > M_PI / 2) obtuse = k;
        for (int k = 0; k < 3; k++) {
            int i = v[k];
            ang[i] += th[k];
            for (int q = 0; q < 3; q++) nn[3 * i + q] += nrm[q];   /* |nrm| = 2 area: area weighting */
            if (obtuse < 0) {
                /* Voronoi part: 1/8 (cot(angle at k+1) |edge k..k+2|^2 + cot(angle at k+2) |edge k..k+1|^2) */
                int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                A[i] += (cotw[3 * t + k1] * l2[k1] + cotw[3 * t + k2] * l2[k2]) / 8.0;
            } else if (obtuse == k) {
                A[i] += area / 2.0;
            } else {
                A[i] += area / 4.0;
            }
        }
        /* edge (v[k+1], v[k+2]) is opposite vertex k with weight cot(theta_k) */
        for (int k = 0; k < 3; k++) {
            int i = v[(k + 1) % 3], j = v[(k + 2) % 3];
            double w = cotw[3 * t + k];
            for (int q = 0; q < 3; q++) {
                Kv[3 * i + q] += w * (x[3 * i + q] - x[3 * j + q]);
                Kv[3 * j + q] += w * (x[3 * j + q] - x[3 * i + q]);
            }
        }
    }
    double E = 0;
    for (int i = 0; i < nv; i++) {
        double nl = norm3(nn + 3 * i);
        for (int q = 0; q < 3; q++) { nn[3 * i + q] /= nl; Kv[3 * i + q] /= (2.0 * A[i]); }
        H[i] = 0.5 * dot3(Kv + 3 * i, nn + 3 * i);
        E += 0.5 * kB * (2 * H[i]) * (2 * H[i]) * A[i];
    }
    for (int t = 0; t < nt; t++) {
        int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        for (int k = 0; k < 3; k++) {
            int i = v[(k + 1) % 3], j = v[(k + 2) % 3];
            double w = cotw[3 * t + k];
            LH[i] += w * (H[j] - H[i]);
            LH[j] += w * (H[i] - H[j]);
        }
    }
    for (int i = 0; i < nv; i++) {
        LH[i] /= (2.0 * A[i]);
        double KG = (2.0 * M_PI - ang[i]) / A[i];
        double fmag = 2.0 * kB * (2.0 * H[i] * (H[i] * H[i] - KG) + LH[i]) * A[i];
        if (F) for (int q = 0; q < 3; q++) F[3 * i + q] += fmag * nn[3 * i + q];
        if (Hout) Hout[i] = H[i];
        if (KGout) KGout[i] = KG;
        if (Aout) Aout[i] = A[i];
        if (LHout) LHout[i] = LH[i];
        if (nout) for (int q = 0; q < 3; q++) nout[3 * i + q] = nn[3 * i + q];
    }
    free(A); free(Kv); free(ang); free(nn); free(H); free(LH); free(cotw);
    return E;
}

/* ---------------------------------------------------------------------------------------------------- */
/* Particle-particle hard-core repulsion (Eq. 26, Sec. III.E): F = eps (d0 - d)^{3/2} along the separation for     */
/* boundary nodes of different capsules closer than d0.  Linked-cell search; minimum image in periodic     */
/* directions.  Adds into F.                                                                             */
/* ---------------------------------------------------------------------------------------------------- */
void o_pp_forces(int NV, const double* X, const int* cap_of, double eps, double d0, int nx, int ny, int nz,
                 int pz, double* F) {
    double L[3] = {nx, ny, nz};
    int per[3] = {1, 1, pz};
    int nc[3];
    for (int k = 0; k < 3; k++) { nc[k] = (int)floor(L[k] / d0); if (nc[k] < 1) nc[k] = 1; }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * ncell);
    int* next = (int*)malloc(sizeof(int) * (NV > 0 ? NV : 1));
    int* cell = (int*)malloc(sizeof(int) * 3 * (NV > 0 ? NV : 1));
    for (long c = 0; c < ncell; c++) head[c] = -1;
    for (int v = 0; v < NV; v++) {
        int cc[3];
        for (int k = 0; k < 3; k++) {
            double p = X[3 * v + k];
            if (per[k]) { p = fmod(p, L[k]); if (p < 0) p += L[k]; }
            int ci = (int)floor(p / (L[k] / nc[k]));
            if (ci < 0) ci = 0;
            if (ci >= nc[k]) ci = nc[k] - 1;
            cc[k] = ci;
        }
        cell[3 * v] = cc[0]; cell[3 * v + 1] = cc[1]; cell[3 * v + 2] = cc[2];
        long id = cc[0] + (long)nc[0] * (cc[1] + (long)nc[1] * cc[2]);
        next[v] = head[id];
        head[id] = v;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int v = 0; v < NV; v++) {
        double f[3] = {0, 0, 0};
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int cc[3] = {cell[3 * v] + dx, cell[3 * v + 1] + dy, cell[3 * v + 2] + dz};
                    int skip = 0;
                    for (int k = 0; k < 3; k++) {
                        if (cc[k] < 0 || cc[k] >= nc[k]) {
                            if (per[k]) cc[k] = wrap(cc[k], nc[k]); else skip = 1;
                        }
                    }
                    if (skip) continue;
                    /* avoid visiting the same cell twice when a periodic direction has < 3 cells */
                    int dup = 0;
                    int dd[3] = {dx, dy, dz};
                    for (int k = 0; k < 3; k++)
                        if (per[k] && nc[k] < 3 && dd[k] != 0) {
                            if (nc[k] == 1) dup = 1;
                            if (nc[k] == 2 && dd[k] == 1) dup = 1;
                        }
                    if (dup) continue;
                    long id = cc[0] + (long)nc[0] * (cc[1] + (long)nc[1] * cc[2]);
                    for (int w = head[id]; w >= 0; w = next[w]) {
                        if (cap_of[w] == cap_of[v]) continue;
                        double r[3];
                        for (int k = 0; k < 3; k++) {
                            r[k] = X[3 * v + k] - X[3 * w + k];
                            if (per[k]) r[k] -= L[k] * floor(r[k] / L[k] + 0.5);
                        }
                        double d = norm3(r);
                        if (d < d0 && d > 0) {
                            double m = eps * pow(d0 - d, 1.5) / d;
                            for (int k = 0; k < 3; k++) f[k] += m * r[k];
                        }
                    }
                }
        for (int k = 0; k < 3; k++) F[3 * v + k] += f[k];
    }
    free(head); free(next); free(cell);
}

/* ---------------------------------------------------------------------------------------------------- */
/* 2-point immersed boundary (Peskin's hat kernel phi2(r) = prod_k max(0, 1-|r_k|)).  Not part of the    */
/* paper, which couples by bounce-back; provided as the alternative coupling.                           */
/* ---------------------------------------------------------------------------------------------------- */
static void ibm_stencil(const osim* s, const double* Xb, long nodes[8], double w[8]) {
    int b[3];
    double fr[3];
    for (int k = 0; k < 3; k++) {
        double fl = floor(Xb[k]);
        b[k] = (int)fl;
        fr[k] = Xb[k] - fl;
    }
    int q = 0;
    for (int dz = 0; dz <= 1; dz++)
        for (int dy = 0; dy <= 1; dy++)
            for (int dx = 0; dx <= 1; dx++) {
                int xx = wrap(b[0] + dx, s->p.nx), yy = wrap(b[1] + dy, s->p.ny), zz = b[2] + dz;
                if (!s->p.walls) zz = wrap(zz, s->p.nz);
                double ww = (dx ? fr[0] : 1 - fr[0]) * (dy ? fr[1] : 1 - fr[1]) * (dz ? fr[2] : 1 - fr[2]);
                if (zz < 0 || zz >= s->p.nz) { nodes[q] = -1; w[q] = 0; }
                else { nodes[q] = IDX(s, xx, yy, zz); w[q] = ww; }
                q++;
            }
}

/* F_ibm(x) = sum_b phi2(x - X_b) F_b  (overwrites s->Fibm) */
void o_ibm_spread(osim* s, const double* Fb) {
    memset(s->Fibm, 0, sizeof(double) * 3 * s->N);
    int NV = s->voff[s->nm];
    for (int v = 0; v < NV; v++) {
        long nd[8];
        double w[8];
        ibm_stencil(s, s->X + 3 * v, nd, w);
        for (int q = 0; q < 8; q++) {
            if (nd[q] < 0 || s->owner[nd[q]] == OWNER_WALL) continue;
            for (int k = 0; k < 3; k++) s->Fibm[k * s->N + nd[q]] += w[q] * Fb[3 * v + k];
        }
    }
}

/* U_b = sum_x phi2(x - X_b) u(x); wall nodes contribute their wall velocity */
void o_ibm_interp(const osim* s, const double* ufield, double* Ub) {
    int NV = s->voff[s->nm];
    for (int v = 0; v < NV; v++) {
        long nd[8];
        double w[8];
        ibm_stencil(s, s->X + 3 * v, nd, w);
        double U[3] = {0, 0, 0};
        for (int q = 0; q < 8; q++) {
            if (nd[q] < 0) continue;
            for (int k = 0; k < 3; k++) {
                double uk;
                if (s->owner[nd[q]] == OWNER_WALL) {
                    int z = (int)(nd[q] / ((long)s->p.nx * s->p.ny));
                    uk = wall_u(s, z, k);
                } else {
                    uk = ufield[k * s->N + nd[q]];
                }
                U[k] += w[q] * uk;
            }
        }
        for (int k = 0; k < 3; k++) Ub[3 * v + k] = U[k];
    }
}

/* exposed for pins: spread arbitrary Fb into out[3][N]; interpolate arbitrary field */
void o_ibm_spread_field(osim* s, const double* Fb, double* out) {
    o_ibm_spread(s, Fb);
    memcpy(out, s->Fibm, sizeof(double) * 3 * s->N);
}

/* ---------------------------------------------------------------------------------------------------- */
/* Elastic + repulsive node forces for all capsules                                                     */
/* ---------------------------------------------------------------------------------------------------- */
void o_membrane_forces(osim* s, double* Fout) {
    int NV = s->voff[s->nm];
    memset(Fout, 0, sizeof(double) * 3 * NV);
    for (int m = 0; m < s->nm; m++) {
        int v0 = s->voff[m], nv = s->mp[m].nv, nt = s->mp[m].nt;
        int* tl = (int*)malloc(sizeof(int) * 3 * nt);
        for (int t = 0; t < 3 * nt; t++) tl[t] = s->tri[3 * s->toff[m] + t] - v0;
        double* Fl = (double*)calloc((size_t)3 * nv, sizeof(double));
        o_skalak(nv, nt, s->X + 3 * v0, tl, s->refX + 3 * v0, s->mp[m].kS, s->mp[m].C, Fl);
        o_volume_force(nv, nt, s->X + 3 * v0, tl, s->mp[m].kV, s->V0[m], Fl);
        if (s->mp[m].kB != 0.0)
            o_bending(nv, nt, s->X + 3 * v0, tl, s->mp[m].kB, Fl, NULL, NULL, NULL, NULL, NULL);
        for (int q = 0; q < 3 * nv; q++) Fout[3 * v0 + q] += Fl[q];
        free(Fl);
        free(tl);
    }
    if (s->nm > 1 && s->p.pp_eps != 0.0) {
        int* cap_of = (int*)malloc(sizeof(int) * NV);
        for (int m = 0; m < s->nm; m++)
            for (int v = s->voff[m]; v < s->voff[m + 1]; v++) cap_of[v] = m;
        o_pp_forces(NV, s->X, cap_of, s->p.pp_eps, s->p.pp_d0, s->p.nx, s->p.ny, s->p.nz, !s->p.walls, Fout);
        free(cap_of);
    }
}

/* capsule volume (FP64) and centre of mass (vertex average) */
void o_capsule_diag(const osim* s, int m, double* vol, double* com3) {
    int v0 = s->voff[m], nv = s->mp[m].nv, nt = s->mp[m].nt;
    int* tl = (int*)malloc(sizeof(int) * 3 * nt);
    for (int t = 0; t < 3 * nt; t++) tl[t] = s->tri[3 * s->toff[m] + t] - v0;
    if (vol) *vol = o_volume(nv, nt, s->X + 3 * v0, tl);
    if (com3) {
        double c[3] = {0, 0, 0};
        for (int v = 0; v < nv; v++)
            for (int k = 0; k < 3; k++) c[k] += s->X[3 * (v0 + v) + k];
        for (int k = 0; k < 3; k++) com3[k] = c[k] / nv;
    }
    free(tl);
}

/* ---------------------------------------------------------------------------------------------------- */
/* Fluid: Shan-Chen force (Eq. 13), forcing by equilibrium-velocity shift (Sec. II.A), BGK collision      */
/* (Eq. 1), push streaming with half-way bounce-back (Eq. 11) on wall links and on membrane-cut links.    */
/* ---------------------------------------------------------------------------------------------------- */

/* On-site velocity boundaries (Zou and He, in the D3Q19 form of Hecht and Harting; Sec. III.A and III.C use
   them to impose the shear): on the fluid planes next to the walls (z = 1 with U = u_lo, z = nz-2 with
   U = u_hi) the populations that arrived from the wall are replaced, component by component, so that the
   node's velocity is U.  With n the inward normal (+z at the bottom, -z at the top): rho = (sum of the
   populations with c.n = 0 + 2 x those with c.n < 0) / (1 - U.n); each unknown f_i (c_i.n > 0) is
   f_opp(i) + 6 w_i rho c_i.U - c_i,t . N_t, with the tangential correction
   N_t = 1/2 sum_{c.n = 0} f c_t - rho U_t / 3, which makes sum_i f_i c_i = rho U exactly. */
static void onsite_velocity(osim* s) {
    const long N = s->N;
    for (int side = 0; side < 2; side++) {
        const int z = side == 0 ? 1 : s->p.nz - 2;
        const int nrm = side == 0 ? 1 : -1;
        const double* U = side == 0 ? s->p.u_lo : s->p.u_hi;
        for (int y = 0; y < s->p.ny; y++)
            for (int x = 0; x < s->p.nx; x++) {
                const long n = IDX(s, x, y, z);
                if (s->owner[n] == OWNER_WALL) continue;
                for (int c = 0; c < 2; c++) {
                    double* f = s->f + (c * N + n) * 19;
                    double s0 = 0, sin = 0, tx = 0, ty = 0;
                    for (int i = 0; i < 19; i++) {
                        if (CZ[i] == 0) {
                            s0 += f[i];
                            tx += f[i] * CX[i];
                            ty += f[i] * CY[i];
                        } else if (CZ[i] == -nrm) {
                            sin += f[i];
                        }
                    }
                    const double rho = (s0 + 2.0 * sin) / (1.0 - nrm * U[2]);
                    const double Nx = 0.5 * tx - rho * U[0] / 3.0, Ny = 0.5 * ty - rho * U[1] / 3.0;
                    for (int i = 0; i < 19; i++)
                        if (CZ[i] == nrm)
                            f[i] = f[OPP(i)] + 6.0 * W[i] * rho * (CX[i] * U[0] + CY[i] * U[1] + CZ[i] * U[2]) -
                                   (CX[i] * Nx + CY[i] * Ny);
                }
            }
    }
}

/* virtual density seen across a wall link: mean of rho over the fluid neighbours of the wall node */
static double wall_virtual_rho(const osim* s, long wn, int c) {
    int z = (int)(wn / ((long)s->p.nx * s->p.ny));
    int rem = (int)(wn % ((long)s->p.nx * s->p.ny));
    int y = rem / s->p.nx, x = rem % s->p.nx;
    double sum = 0;
    int cnt = 0;
    for (int k = 1; k < 19; k++) {
        long m = nbr(s, x, y, z, k, NULL);
        if (m < 0 || s->owner[m] == OWNER_WALL) continue;
        sum += s->rho[c * s->N + m];
        cnt++;
    }
    return cnt ? sum / cnt : 0.0;
}

/* hooks implemented in the bounce-back part */
static double bb_virtual_psi(osim* s, long n, int x, int y, int z, int i, long m, int c_other,
                             double* react_elem_out, int* elem_out);
static void bb_link(osim* s, long n, int x, int y, int z, int i, long m, int c, double fstar, double rho_c);

/* one collide + stream of both components; F_ibm is used when coupling == 1 */
static void fluid_step(osim* s) {
    const long N = s->N;
    const double tau = s->p.tau, G = s->p.G;
    compute_rho(s);
    memset(s->fn, 0, sizeof(double) * 2 * 19 * N);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        if (s->owner[n] == OWNER_WALL) continue;
        int z = (int)(n / ((long)s->p.nx * s->p.ny));
        int rem = (int)(n % ((long)s->p.nx * s->p.ny));
        int y = rem / s->p.nx, x = rem % s->p.nx;
        double rho[2] = {s->rho[n], s->rho[N + n]};
        double j[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < 19; i++) {
                double fi = s->f[(c * N + n) * 19 + i];
                j[c][0] += fi * CX[i]; j[c][1] += fi * CY[i]; j[c][2] += fi * CZ[i];
            }
        /* Shan-Chen force (Eq. 13) on component c from the other component c' (G^{AB} = G^{BA} = G) */
        double Fc[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int c = 0; c < 2; c++) {
            int co = 1 - c;
            double acc[3] = {0, 0, 0};
            for (int i = 1; i < 19; i++) {
                int zz;
                long m = nbr(s, x, y, z, i, &zz);
                double psin;
                if (m < 0) {
                    psin = 0.0;               /* cannot happen: wall planes bound z */
                } else if (s->owner[m] == OWNER_WALL) {
                    psin = psi_of(s, wall_virtual_rho(s, m, co));
                } else if (s->owner[m] != s->owner[n]) {
                    psin = bb_virtual_psi(s, n, x, y, z, i, m, co, NULL, NULL);
                } else {
                    psin = s->psi[co * N + m];
                }
                acc[0] += W[i] * psin * CX[i]; acc[1] += W[i] * psin * CY[i]; acc[2] += W[i] * psin * CZ[i];
            }
            double pc = s->psi[c * N + n];
            for (int k = 0; k < 3; k++) Fc[c][k] = -pc * G * acc[k];
            for (int k = 0; k < 3; k++) s->Fsc[(c * 3 + k) * N + n] = Fc[c][k];
        }
        double rt = rho[0] + rho[1];
        double Ftot[3] = {0, 0, 0};
        for (int c = 0; c < 2; c++)
            for (int k = 0; k < 3; k++) {
                Fc[c][k] += rho[c] * s->p.g[k];
                if (s->p.coupling == 1 && rt > 0) Fc[c][k] += rho[c] / rt * s->Fibm[k * N + n];
                Ftot[k] += Fc[c][k];
            }
        double up[3];
        for (int k = 0; k < 3; k++) up[k] = rt > 0 ? (j[0][k] + j[1][k]) / rt : 0.0;
        for (int k = 0; k < 3; k++) s->u[k * N + n] = rt > 0 ? (j[0][k] + j[1][k] + 0.5 * Ftot[k]) / rt : 0.0;
        for (int c = 0; c < 2; c++) {
            double ueq[3];
            for (int k = 0; k < 3; k++) ueq[k] = up[k] + (rho[c] > 0 ? tau * Fc[c][k] / rho[c] : 0.0);
            for (int i = 0; i < 19; i++) {
                double fi = s->f[(c * N + n) * 19 + i];
                double fs = fi - (fi - feq(i, rho[c], ueq)) / tau;
                int zz;
                long m = nbr(s, x, y, z, i, &zz);
                if (i == 0) {
                    s->fn[(c * N + n) * 19] = fs;
                } else if (s->owner[m] == OWNER_WALL) {
                    /* half-way bounce-back on a moving wall (Eq. 11, v0 = wall velocity); c_i points into the
                       wall, the population returns to n in the opposite direction */
                    double cu = CX[i] * wall_u(s, zz, 0) + CY[i] * wall_u(s, zz, 1) + CZ[i] * wall_u(s, zz, 2);
                    s->fn[(c * N + n) * 19 + OPP(i)] = fs - 2.0 * W[i] * rho[c] * cu / CS2;
                } else if (s->owner[m] != s->owner[n]) {
                    bb_link(s, n, x, y, z, i, m, c, fs, rho[c]);
                } else {
                    s->fn[(c * N + m) * 19 + i] = fs;
                }
            }
        }
    }
    double* t = s->f; s->f = s->fn; s->fn = t;
    if (s->p.walls && s->p.wall_kind == 1) onsite_velocity(s);
}

/* ---------------------------------------------------------------------------------------------------- */
/* One time step                                                                                         */
/* ---------------------------------------------------------------------------------------------------- */
static void bb_prepare(osim* s);
static void bb_before_fluid(osim* s);
static void bb_collect(osim* s);
static void bb_after_fluid(osim* s);

static void ibm_step(osim* s) {
    int NV = s->voff[s->nm];
    if (NV > 0) {
        o_membrane_forces(s, s->F);
        o_ibm_spread(s, s->F);
    }
    fluid_step(s);
    if (NV > 0) {
        double* Ub = (double*)malloc(sizeof(double) * 3 * NV);
        o_ibm_interp(s, s->u, Ub);
        for (int q = 0; q < 3 * NV; q++) { s->X[q] += Ub[q]; s->Vel[q] = Ub[q]; }
        free(Ub);
    }
}

void o_init(osim* s) {
    for (int m = 0; m < s->nm; m++) {
        int v0 = s->voff[m], nv = s->mp[m].nv, nt = s->mp[m].nt;
        int* tl = (int*)malloc(sizeof(int) * 3 * nt);
        for (int t = 0; t < 3 * nt; t++) tl[t] = s->tri[3 * s->toff[m] + t] - v0;
        s->V0[m] = o_volume(nv, nt, s->refX + 3 * v0, tl);
        free(tl);
    }
    if (s->p.coupling == 0) bb_prepare(s);
}

void o_step(osim* s, int n) {
    for (int k = 0; k < n; k++) {
        if (s->p.coupling == 0) {
            bb_before_fluid(s);
            fluid_step(s);
            bb_collect(s);
            bb_after_fluid(s);
        } else {
            ibm_step(s);
        }
        s->step++;
    }
}

#include "scbb_oracle_bb.c"
