/*
 * FP64 CPU oracle of the coupled colour-gradient LBM / DEM method of
 * Naga, Zhang, Yang & Kusumaatmaja, "Modelling droplet-particle interactions
 * on solid surfaces by coupling the lattice Boltzmann and discrete element
 * methods" (arXiv 2505.10171).
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow, obviously-correct reference
 * the CUDA library is checked against.  Only tests/, the smoke check and the
 * CPU-baseline leg of bench.py load it.  It shares no code with the CUDA
 * path.  Every step follows the paper's section/equation named beside it, in
 * the paper's order, with dense matrix products where the paper writes them;
 * no fusion, blocking or reordering.
 *
 * Readings taken where the paper is silent or garbled are marked READING and
 * carry the same label as the list of readings kept with the design notes
 * (c1 ... c31).
 *
 * Parity pins: see tests/test_oracle_*.py.  Every function here is pinned by
 * at least one closed form, invariant or brute-force check.  The whole
 * coupled step has no single closed form; it is pinned through whole-step
 * behaviour: the exact Poiseuille profile between halfway walls, a uniform
 * flow over a moving wall that stays steady, component mass conservation of a
 * drop on a sliding wall, the Laplace law of a drop, the sessile contact
 * angle, the momentum balance between the fluid and a sphere, and the mass
 * bookkeeping of a sphere that covers and uncovers nodes.  The refill values
 * (one-hop, two-hop and ambient branches), the momentum-exchange torque (an
 * exact angular-momentum balance with a spinning sphere across the periodic
 * boundary) and the sphere branch of the wetting normal (the rotated
 * gradient's angle to the nearest sphere's normal) have pins of their own,
 * and so does the immersed fraction behind the buoyancy (reading c28): the
 * cap volume cut off by a flat interface, and a neutrally buoyant sphere
 * that keeps its place.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FLUID 0
#define WALL 1
#define PRESS 63 /* inlet/outlet face of a pressure boundary (Sec. V D); particles are 2 + p, p < 61 */

/* ---------------------------------------------------------------------- */
/* Sec. IV: D3Q19 velocity set (Krueger et al. 2016).  Weights follow from */
/* |c|^2: 1/3 (rest), 1/18 (axis), 1/36 (face diagonal).                   */
/* ---------------------------------------------------------------------- */
static const int OR_C[OR_Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double OR_W[OR_Q];
static int OR_OPP[OR_Q];
static double OR_M[OR_Q][OR_Q];
static double OR_MINV[OR_Q][OR_Q];
static int OR_SKIND[OR_Q]; /* 0: conserved, 1: omega, 2: omega' */
static int or_ready = 0;

/* READING c1: d'Humieres et al. (2002) moment basis, rows in the order the
 * relaxation matrix S of Sec. IV (MRT) lists them:
 * rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz,
 * mx, my, mz. Each row is a polynomial in c. */
static double moment_row(int k, const int *c)
{
    double cx = c[0], cy = c[1], cz = c[2];
    double c2 = cx * cx + cy * cy + cz * cz;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: return cx;
    case 4: return (5.0 * c2 - 9.0) * cx;
    case 5: return cy;
    case 6: return (5.0 * c2 - 9.0) * cy;
    case 7: return cz;
    case 8: return (5.0 * c2 - 9.0) * cz;
    case 9: return 3.0 * cx * cx - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);
    case 11: return cy * cy - cz * cz;
    case 12: return (3.0 * c2 - 5.0) * (cy * cy - cz * cz);
    case 13: return cx * cy;
    case 14: return cy * cz;
    case 15: return cx * cz;
    case 16: return (cy * cy - cz * cz) * cx;
    case 17: return (cz * cz - cx * cx) * cy;
    case 18: return (cx * cx - cy * cy) * cz;
    }
    return 0.0;
}

/* Gauss-Jordan inversion with partial pivoting (a library-style step). */
static void invert19(double A[OR_Q][OR_Q], double R[OR_Q][OR_Q])
{
    double a[OR_Q][2 * OR_Q];
    for (int i = 0; i < OR_Q; i++)
        for (int j = 0; j < 2 * OR_Q; j++)
            a[i][j] = j < OR_Q ? A[i][j] : (j - OR_Q == i ? 1.0 : 0.0);
    for (int col = 0; col < OR_Q; col++) {
        int piv = col;
        for (int r = col + 1; r < OR_Q; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 2 * OR_Q; j++) {
                double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
            }
        double d = a[col][col];
        for (int j = 0; j < 2 * OR_Q; j++) a[col][j] /= d;
        for (int r = 0; r < OR_Q; r++) {
            if (r == col) continue;
            double f = a[r][col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * OR_Q; j++) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < OR_Q; i++)
        for (int j = 0; j < OR_Q; j++) R[i][j] = a[i][OR_Q + j];
}

static void or_init_lattice(void)
{
    if (or_ready) return;
    for (int i = 0; i < OR_Q; i++) {
        int c2 = OR_C[i][0] * OR_C[i][0] + OR_C[i][1] * OR_C[i][1] + OR_C[i][2] * OR_C[i][2];
        OR_W[i] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < OR_Q; j++)
            if (OR_C[j][0] == -OR_C[i][0] && OR_C[j][1] == -OR_C[i][1] && OR_C[j][2] == -OR_C[i][2])
                OR_OPP[i] = j;
    }
    for (int k = 0; k < OR_Q; k++)
        for (int i = 0; i < OR_Q; i++) OR_M[k][i] = moment_row(k, OR_C[i]);
    invert19(OR_M, OR_MINV);
    /* Sec. IV: S = diag[0,w,w,0,w',0,w',0,w',w,w,w,w,w,w,w,w',w',w'] */
    static const int kind[OR_Q] = {0, 1, 1, 0, 2, 0, 2, 0, 2, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2};
    for (int k = 0; k < OR_Q; k++) OR_SKIND[k] = kind[k];
    or_ready = 1;
}

void or_lattice(int *c, double *w, int *opp)
{
    or_init_lattice();
    for (int i = 0; i < OR_Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = OR_C[i][a];
        w[i] = OR_W[i];
        opp[i] = OR_OPP[i];
    }
}

void or_mrt_matrices(double *M, double *Minv, double *S_pattern)
{
    or_init_lattice();
    for (int i = 0; i < OR_Q; i++) {
        for (int j = 0; j < OR_Q; j++) {
            M[i * OR_Q + j] = OR_M[i][j];
            Minv[i * OR_Q + j] = OR_MINV[i][j];
        }
        S_pattern[i] = OR_SKIND[i];
    }
}

/* ---------------------------------------------------------------------- */
/* simulation state                                                       */
/* ---------------------------------------------------------------------- */
typedef struct {
    double x[3], v[3], w[3], q[4];
    double R, Rc, m, I, theta;
    double Fp[3], Tp[3];          /* total force/torque of the last DEM step */
    double Feta[3], Teta[3];      /* hydrodynamic, Sec. V B                 */
    double Fsig[3], Tsig[3];      /* capillary, Sec. V F                    */
    double Fc[3], Tc[3];          /* contact, Sec. III                      */
    double sub, Fb[3];            /* immersed fraction, buoyancy (c28)      */
    int kin;                      /* prescribed (kinematic) motion          */
} or_part;

struct or_sim {
    or_params p;
    int nx, ny, nz;
    long N;
    double *fa, *fb;    /* post-collision state f^{a,b*}(x,t)   [19][N] */
    double *fas, *fbs;  /* post-streaming f^{a,b}(x,t+1)         [19][N] */
    double *phi, *grad, *nrm, *u;
    unsigned char *owner, *stat, *old_owner, *fresh;
    int np;
    or_part P[OR_MAXP];
    double xi_w[OR_MAXP][3], xir_w[OR_MAXP][3];
    double (*xi_p)[OR_MAXP][3], (*xir_p)[OR_MAXP][3];
    double diag[8];
    long steps;              /* time steps taken                            */
    double sp_f0[3];         /* body_force_a at creation (controller base)  */
    double sp_int[3];        /* controller integral of the velocity error   */
    double sp_u[3];          /* phase-a velocity at the last update          */
};

static inline int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}
static inline long lidx(const or_sim *s, int x, int y, int z)
{
    return ((long)z * s->ny + y) * s->nx + x;
}
static inline long nbr(const or_sim *s, int x, int y, int z, int dx, int dy, int dz)
{
    return lidx(s, wrapi(x + dx, s->nx), wrapi(y + dy, s->ny), wrapi(z + dz, s->nz));
}
/* minimum-image displacement on a periodic axis of n nodes */
static inline double minimg(double d, int n)
{
    return d - n * floor(d / n + 0.5);
}
static inline double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void cross3(const double *a, const double *b, double *r)
{
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    r[0] = t0; r[1] = t1; r[2] = t2;
}

/* Sec. V C, equilibrium: w_i rho [1 + c.u/cs2 + (c.u)^2/(2cs4) - u.u/(2cs2)] */
static void feq(double rho, const double *u, double *f)
{
    double uu = dot3(u, u);
    for (int i = 0; i < OR_Q; i++) {
        double cu = OR_C[i][0] * u[0] + OR_C[i][1] * u[1] + OR_C[i][2] * u[2];
        f[i] = OR_W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

or_sim *or_create(const or_params *p)
{
    or_init_lattice();
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    if (!s) return NULL;
    s->p = *p;
    for (int a = 0; a < 3; a++) s->sp_f0[a] = p->body_force_a[a];
    s->nx = p->nx; s->ny = p->ny; s->nz = p->nz;
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    s->fa = calloc((size_t)OR_Q * N, sizeof(double));
    s->fb = calloc((size_t)OR_Q * N, sizeof(double));
    s->fas = calloc((size_t)OR_Q * N, sizeof(double));
    s->fbs = calloc((size_t)OR_Q * N, sizeof(double));
    s->phi = calloc(N, sizeof(double));
    s->grad = calloc(3 * N, sizeof(double));
    s->nrm = calloc(3 * N, sizeof(double));
    s->u = calloc(3 * N, sizeof(double));
    s->owner = calloc(N, 1);
    s->stat = calloc(N, 1);
    s->old_owner = calloc(N, 1);
    s->fresh = calloc(N, 1);
    s->xi_p = calloc(OR_MAXP, sizeof(*s->xi_p));
    s->xir_p = calloc(OR_MAXP, sizeof(*s->xir_p));
    if (!s->fa || !s->fb || !s->fas || !s->fbs || !s->phi || !s->grad || !s->nrm || !s->u ||
        !s->owner || !s->stat || !s->old_owner || !s->fresh || !s->xi_p || !s->xir_p) {
        or_destroy(s);
        return NULL;
    }
    /* READING c15: the substrate is the node plane z=0; the halfway wall sits
     * at z=0.5 (and, the domain being periodic in z, at z=nz-0.5 on top). */
    if (p->wall_z0)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) s->stat[lidx(s, x, y, 0)] = 1;
    /* Sec. V D pressure boundaries: the node planes z=0 and z=nz-1 are the
     * outside of the inlet and outlet faces, which sit halfway, at z=0.5 and
     * z=nz-1.5; the domain is then not periodic in z for the fluid */
    if (p->pressure_z)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) s->stat[lidx(s, x, y, 0)] = s->stat[lidx(s, x, y, s->nz - 1)] = 2;
    for (long i = 0; i < N; i++) s->owner[i] = s->stat[i] == 2 ? PRESS : (s->stat[i] ? WALL : FLUID);
    return s;
}

void or_destroy(or_sim *s)
{
    if (!s) return;
    free(s->fa); free(s->fb); free(s->fas); free(s->fbs);
    free(s->phi); free(s->grad); free(s->nrm); free(s->u);
    free(s->owner); free(s->stat); free(s->old_owner); free(s->fresh);
    free(s->xi_p); free(s->xir_p);
    free(s);
}

static int solid_owner_of(const or_sim *s, int x, int y, int z)
{
    if (s->stat[lidx(s, x, y, z)] == 2) return PRESS;
    if (s->stat[lidx(s, x, y, z)]) return WALL;
    /* READING c15: node x is inside particle p iff |x - x_p|^2 < R_p^2 */
    for (int p = 0; p < s->np; p++) {
        const or_part *P = &s->P[p];
        double dx = minimg(x - P->x[0], s->nx);
        double dy = minimg(y - P->x[1], s->ny);
        double dz = minimg(z - P->x[2], s->nz);
        if (dx * dx + dy * dy + dz * dz < P->R * P->R) return 2 + p;
    }
    return FLUID;
}

int or_set_static_solid(or_sim *s, const unsigned char *mask)
{
    for (long i = 0; i < s->N; i++)
        if (s->stat[i] != 2) s->stat[i] = mask[i] ? 1 : 0;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++)
                s->owner[lidx(s, x, y, z)] = (unsigned char)solid_owner_of(s, x, y, z);
    return 0;
}

int or_init_fields(or_sim *s, const double *phi, const double *rho, const double *u)
{
    long N = s->N;
    double f[OR_Q];
    for (long n = 0; n < N; n++) {
        double uu[3] = {u ? u[n] : 0.0, u ? u[N + n] : 0.0, u ? u[2 * N + n] : 0.0};
        double r = rho ? rho[n] : s->p.rho0;
        double ra = 0.5 * r * (1.0 + phi[n]);
        double rb = 0.5 * r * (1.0 - phi[n]);
        feq(ra, uu, f);
        for (int i = 0; i < OR_Q; i++) s->fa[i * N + n] = f[i];
        feq(rb, uu, f);
        for (int i = 0; i < OR_Q; i++) s->fb[i * N + n] = f[i];
        for (int a = 0; a < 3; a++) s->u[a * N + n] = s->owner[n] == FLUID ? uu[a] : 0.0;
    }
    return 0;
}

int or_set_pops(or_sim *s, const double *fa, const double *fb)
{
    memcpy(s->fa, fa, sizeof(double) * OR_Q * s->N);
    memcpy(s->fb, fb, sizeof(double) * OR_Q * s->N);
    return 0;
}

int or_add_particle(or_sim *s, const double *x, const double *v, const double *w,
                    double R, double rho_p, double theta_deg, int kinematic)
{
    if (s->np >= OR_MAXP) return -1;
    or_part *P = &s->P[s->np];
    memset(P, 0, sizeof(*P));
    for (int a = 0; a < 3; a++) { P->x[a] = x[a]; P->v[a] = v[a]; P->w[a] = w[a]; }
    P->q[0] = 1.0;
    P->R = R;
    P->Rc = R + s->p.delta_R;                     /* Sec. V H */
    /* READING c25: m_p from the hydrodynamic radius, I_p of a solid sphere */
    P->m = rho_p * 4.0 / 3.0 * M_PI * R * R * R;
    P->I = 0.4 * P->m * R * R;
    P->theta = theta_deg * M_PI / 180.0;
    P->kin = kinematic;
    /* the first Verlet half-step uses the external force only */
    for (int a = 0; a < 3; a++) P->Fp[a] = s->p.g_particle[a];
    s->np++;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int xx = 0; xx < s->nx; xx++)
                s->owner[lidx(s, xx, y, z)] = (unsigned char)solid_owner_of(s, xx, y, z);
    return 0;
}

/* velocity of the solid that owns a node, at the point xw (Sec. V A) */
static void surface_velocity(const or_sim *s, int owner, const double *xw, double *uw, double *lever)
{
    if (owner == WALL) {
        for (int a = 0; a < 3; a++) { uw[a] = s->p.wall_velocity[a]; lever[a] = 0.0; }
        return;
    }
    const or_part *P = &s->P[owner - 2];
    double d[3] = {minimg(xw[0] - P->x[0], s->nx), minimg(xw[1] - P->x[1], s->ny),
                   minimg(xw[2] - P->x[2], s->nz)};
    double wx[3];
    cross3(P->w, d, wx);
    for (int a = 0; a < 3; a++) { uw[a] = P->v[a] + wx[a]; lever[a] = d[a]; }
}

/* Sec. IV harmonic-mean viscosity; READING c3: eta^{a,b} = rho0 nu^{a,b},
 * tau = eta/(rho cs2) + 1/2 with the local total density. */
double or_omega_of_phi(const or_params *p, double phi, double rho)
{
    double eta_a = p->rho0 * p->nu_a, eta_b = p->rho0 * p->nu_b;
    double inv_eta = (1.0 + phi) / (2.0 * eta_a) + (1.0 - phi) / (2.0 * eta_b);
    double eta = 1.0 / inv_eta;
    double tau = eta / (rho / 3.0) + 0.5;
    return 1.0 / tau;
}

/* Sec. IV: one node's collision (Eq. Collision step with the MRT operator
 * and Guo forcing in moment space), followed by the recolouring step.
 * fa, fb: post-streaming populations of the node; F_ext: force density;
 * nhat: unit colour-gradient direction (zero allowed). */
void or_collide_node(const double *fa, const double *fb, const double *F_ext,
                     const double *nhat, double omega, double omega_p, double beta,
                     double *fa_out, double *fb_out, double *u_out)
{
    or_init_lattice();
    double f[OR_Q], fe[OR_Q], Fb[OR_Q], m[OR_Q], me[OR_Q], mF[OR_Q], ms[OR_Q], fs[OR_Q];
    double ra = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < OR_Q; i++) {
        f[i] = fa[i] + fb[i];
        ra += fa[i];
        rb += fb[i];
        for (int a = 0; a < 3; a++) j[a] += OR_C[i][a] * f[i];
    }
    double rho = ra + rb;
    /* Sec. IV: rho_f u = sum_i c_i f_i + F/2 */
    double u[3];
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F_ext[a]) / rho;
    feq(rho, u, fe);
    /* Eq. force4: Fbar_i = w_i [c.F/cs2 + u_j F_k (c_j c_k - cs2 d_jk)/cs4] */
    double uF = dot3(u, F_ext);
    for (int i = 0; i < OR_Q; i++) {
        double cF = OR_C[i][0] * F_ext[0] + OR_C[i][1] * F_ext[1] + OR_C[i][2] * F_ext[2];
        double cu = OR_C[i][0] * u[0] + OR_C[i][1] * u[1] + OR_C[i][2] * u[2];
        Fb[i] = OR_W[i] * (3.0 * cF + 9.0 * (cu * cF) - 3.0 * uF);
    }
    for (int k = 0; k < OR_Q; k++) {
        m[k] = me[k] = mF[k] = 0.0;
        for (int i = 0; i < OR_Q; i++) {
            m[k] += OR_M[k][i] * f[i];
            me[k] += OR_M[k][i] * fe[i];
            mF[k] += OR_M[k][i] * Fb[i];
        }
    }
    /* f* = f - M^-1 S M (f - feq) + M^-1 (I - S/2) M Fbar */
    for (int k = 0; k < OR_Q; k++) {
        double sk = OR_SKIND[k] == 0 ? 0.0 : (OR_SKIND[k] == 1 ? omega : omega_p);
        ms[k] = m[k] - sk * (m[k] - me[k]) + (1.0 - 0.5 * sk) * mF[k];
    }
    for (int i = 0; i < OR_Q; i++) {
        fs[i] = 0.0;
        for (int k = 0; k < OR_Q; k++) fs[i] += OR_MINV[i][k] * ms[k];
    }
    /* Sec. IV recolouring (Latva-Kokko & Rothman).  READING c8: the
     * perturbation carries cos(phi_i) = c_i.n/|c_i| with n pointing towards
     * phi=+1, added to phase a; the rest direction gets none. */
    double ab = ra * rb / rho;
    for (int i = 0; i < OR_Q; i++) {
        double cn = 0.0;
        if (i != 0) {
            double cl = sqrt((double)(OR_C[i][0] * OR_C[i][0] + OR_C[i][1] * OR_C[i][1] +
                                      OR_C[i][2] * OR_C[i][2]));
            cn = (OR_C[i][0] * nhat[0] + OR_C[i][1] * nhat[1] + OR_C[i][2] * nhat[2]) / cl;
        }
        double pert = beta * ab * OR_W[i] * cn;
        fa_out[i] = ra / rho * fs[i] + pert;
        fb_out[i] = rb / rho * fs[i] - pert;
    }
    if (u_out)
        for (int a = 0; a < 3; a++) u_out[a] = u[a];
}

/* Sec. V E, geometric wetting condition (Xu 2017, Akai 2018).
 * READING c11: n* = -grad(phi)/|grad(phi)| points out of the phi=+1 phase,
 * theta is measured inside phase a, n_s points out of the solid.  Of the two
 * candidates n_+, n_- the one closer to n* is taken; the gradient keeps its
 * magnitude and takes the direction -n_chosen. */
void or_wetting_rotate(double *g, const double *ns, double theta)
{
    double gm = sqrt(dot3(g, g));
    if (gm == 0.0) return;
    double nst[3] = {-g[0] / gm, -g[1] / gm, -g[2] / gm};
    double ca = dot3(ns, nst);
    if (ca > 1.0) ca = 1.0;
    if (ca < -1.0) ca = -1.0;
    double alpha = acos(ca);
    double sa = sin(alpha), cal = cos(alpha);
    /* READING c11: where n* is parallel to n_s (sin alpha* -> 0) the plane of
     * rotation, i.e. the contact-line direction, is undefined and the formula
     * divides rounding noise by sin alpha*; below 1e-4 (0.006 deg) the gradient
     * is left as it is. */
    if (sa < 1e-4) return;
    double best[3], bestdot = -2.0;
    for (int sg = 0; sg < 2; sg++) {
        double th = sg == 0 ? theta : -theta;
        double a1 = cos(th) - sin(th) * cal / sa;
        double a2 = sin(th) / sa;
        double n[3] = {a1 * ns[0] + a2 * nst[0], a1 * ns[1] + a2 * nst[1], a1 * ns[2] + a2 * nst[2]};
        double d = dot3(n, nst);
        if (d > bestdot) {
            bestdot = d;
            for (int a = 0; a < 3; a++) best[a] = n[a];
        }
    }
    for (int a = 0; a < 3; a++) g[a] = -gm * best[a];
}

/* outward solid normal and contact angle for a fluid node next to a solid.
 * READING c12: a particle normal (x - x_p)/|x - x_p| when any neighbour
 * belongs to a particle (the nearest particle surface if several), otherwise
 * the substrate normal -sum_i w_i c_i [x+c_i is substrate], normalised. */
static int solid_normal(const or_sim *s, int x, int y, int z, double *ns, double *theta)
{
    int best_p = -1;
    double best_d = 0.0;
    double ws[3] = {0.0, 0.0, 0.0};
    int any = 0;
    for (int i = 1; i < OR_Q; i++) {
        long id = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
        int o = s->owner[id];
        if (o == FLUID || o == PRESS) continue; /* a pressure face carries no contact angle */
        any = 1;
        if (o == WALL) {
            for (int a = 0; a < 3; a++) ws[a] -= OR_W[i] * OR_C[i][a];
        } else {
            const or_part *P = &s->P[o - 2];
            double dx = minimg(x - P->x[0], s->nx), dy = minimg(y - P->x[1], s->ny),
                   dz = minimg(z - P->x[2], s->nz);
            double dist = sqrt(dx * dx + dy * dy + dz * dz) - P->R;
            if (best_p < 0 || dist < best_d || (dist == best_d && o - 2 < best_p)) {
                best_p = o - 2;
                best_d = dist;
            }
        }
    }
    if (!any) return 0;
    if (best_p >= 0) {
        const or_part *P = &s->P[best_p];
        double d[3] = {minimg(x - P->x[0], s->nx), minimg(y - P->x[1], s->ny), minimg(z - P->x[2], s->nz)};
        double dl = sqrt(dot3(d, d));
        for (int a = 0; a < 3; a++) ns[a] = d[a] / dl;
        *theta = P->theta;
        return 1;
    }
    double wl = sqrt(dot3(ws, ws));
    if (wl == 0.0) return 0;
    for (int a = 0; a < 3; a++) ns[a] = ws[a] / wl;
    *theta = s->p.theta_wall_deg * M_PI / 180.0;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* Sec. V F: capillary force on particle p from the Lagrangian surface     */
/* points.  READING c17/c18: dF = C sigma (1-phi^2) dA [n_s - (n.n_s) n],  */
/* points at alpha_j = (j+1/2) 2deg, varphi_k = k 2deg on r = R_p; phi and */
/* grad(phi) by trilinear interpolation over fluid corners only.           */
/* ---------------------------------------------------------------------- */
int or_capillary(const or_sim *s, int p, double *F, double *T)
{
    const or_part *P = &s->P[p];
    const double da = 2.0 * M_PI / 180.0, dv = 2.0 * M_PI / 180.0;
    const long N = s->N;
    double Fs[3] = {0, 0, 0}, Ts[3] = {0, 0, 0};
    int used = 0;
    for (int j = 0; j < 90; j++) {
        double al = (j + 0.5) * da;
        for (int k = 0; k < 180; k++) {
            double vp = k * dv;
            double ns[3] = {sin(al) * cos(vp), sin(al) * sin(vp), cos(al)};
            double xi[3] = {P->x[0] + P->R * ns[0], P->x[1] + P->R * ns[1], P->x[2] + P->R * ns[2]};
            double dA = P->R * P->R * sin(al) * da * dv;
            int b[3];
            double fr[3];
            for (int a = 0; a < 3; a++) {
                double fl = floor(xi[a]);
                b[a] = (int)fl;
                fr[a] = xi[a] - fl;
            }
            double ws = 0.0, ph = 0.0, g[3] = {0, 0, 0};
            for (int cz = 0; cz < 2; cz++)
                for (int cy = 0; cy < 2; cy++)
                    for (int cx = 0; cx < 2; cx++) {
                        long id = lidx(s, wrapi(b[0] + cx, s->nx), wrapi(b[1] + cy, s->ny),
                                       wrapi(b[2] + cz, s->nz));
                        if (s->owner[id] != FLUID) continue;
                        double wgt = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1]) *
                                     (cz ? fr[2] : 1.0 - fr[2]);
                        ws += wgt;
                        ph += wgt * s->phi[id];
                        for (int a = 0; a < 3; a++) g[a] += wgt * s->grad[a * N + id];
                    }
            if (ws <= 0.0) continue;
            ph /= ws;
            for (int a = 0; a < 3; a++) g[a] /= ws;
            if (fabs(ph) >= 1.0) continue; /* outside the diffuse interface */
            /* READING c6: interface normal n = g/sqrt(|g|^2 + eps^2); m is the
             * paper's (n x n_s) x n = (n.n) n_s - (n.n_s) n */
            double gr = sqrt(dot3(g, g) + s->p.grad_eps * s->p.grad_eps);
            double n[3] = {g[0] / gr, g[1] / gr, g[2] / gr};
            double nxs[3], mvec[3];
            cross3(n, ns, nxs);
            cross3(nxs, n, mvec);
            double coef = s->p.cap_norm * s->p.sigma * (1.0 - ph * ph) * dA;
            double dF[3] = {coef * mvec[0], coef * mvec[1], coef * mvec[2]};
            double r[3] = {P->R * ns[0], P->R * ns[1], P->R * ns[2]}, t[3];
            cross3(r, dF, t);
            for (int a = 0; a < 3; a++) { Fs[a] += dF[a]; Ts[a] += t[a]; }
            used++;
        }
    }
    for (int a = 0; a < 3; a++) { F[a] = Fs[a]; T[a] = Ts[a]; }
    return used;
}

/* ---------------------------------------------------------------------- */
/* READING c28 (Sec. VI A: the particle's effective weight drops by the    */
/* buoyancy of the drop once it enters it; no mechanism given).  Phase-a   */
/* share of the sphere surface: s = (1+phi)/2 clipped to [0,1] at the      */
/* capillary force's surface points, phi trilinear over fluid corners,     */
/* area-weighted over the points that have a fluid corner: a = sum s dA /  */
/* sum dA.  By Archimedes' hat-box theorem a spherical zone's area is      */
/* proportional to its height, so a flat interface at height h = (2a-1) R  */
/* above the centre cuts off the volume fraction v = (1+t)^2 (2-t)/4,      */
/* t = h/R, below it.  Returns v (0 when no point has a fluid corner).     */
/* ---------------------------------------------------------------------- */
double or_immersed_fraction(const or_sim *s, int p)
{
    const or_part *P = &s->P[p];
    const double da = 2.0 * M_PI / 180.0, dv = 2.0 * M_PI / 180.0;
    double num = 0.0, den = 0.0;
    for (int j = 0; j < 90; j++) {
        double al = (j + 0.5) * da;
        for (int k = 0; k < 180; k++) {
            double vp = k * dv;
            double ns[3] = {sin(al) * cos(vp), sin(al) * sin(vp), cos(al)};
            double xi[3] = {P->x[0] + P->R * ns[0], P->x[1] + P->R * ns[1], P->x[2] + P->R * ns[2]};
            double dA = P->R * P->R * sin(al) * da * dv;
            int b[3];
            double fr[3];
            for (int a = 0; a < 3; a++) {
                double fl = floor(xi[a]);
                b[a] = (int)fl;
                fr[a] = xi[a] - fl;
            }
            double ws = 0.0, ph = 0.0;
            for (int cz = 0; cz < 2; cz++)
                for (int cy = 0; cy < 2; cy++)
                    for (int cx = 0; cx < 2; cx++) {
                        long id = lidx(s, wrapi(b[0] + cx, s->nx), wrapi(b[1] + cy, s->ny),
                                       wrapi(b[2] + cz, s->nz));
                        if (s->owner[id] != FLUID) continue;
                        double wgt = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1]) *
                                     (cz ? fr[2] : 1.0 - fr[2]);
                        ws += wgt;
                        ph += wgt * s->phi[id];
                    }
            if (ws <= 0.0) continue;
            double sa = 0.5 * (1.0 + ph / ws);
            if (sa < 0.0) sa = 0.0;
            if (sa > 1.0) sa = 1.0;
            num += sa * dA;
            den += dA;
        }
    }
    if (den <= 0.0) return 0.0;
    double t = 2.0 * (num / den) - 1.0;
    return (1.0 + t) * (1.0 + t) * (2.0 - t) / 4.0;
}

/* ---------------------------------------------------------------------- */
/* Sec. III: DEM contact (normal spring-dashpot, Luding sliding and       */
/* rolling friction) and Verlet integration.                              */
/* ---------------------------------------------------------------------- */

/* one friction spring (Sec. III B; READING c22: xi projected on the
 * current tangent plane).  Returns the (capped) force, updates xi. */
static void friction_spring(double *xi, const double *n, const double *vt, double k, double gam,
                            double FC, double *Fout)
{
    double xn = dot3(xi, n);
    for (int a = 0; a < 3; a++) xi[a] -= xn * n[a];
    double F0[3];
    for (int a = 0; a < 3; a++) F0[a] = -k * xi[a] - gam * vt[a];
    double F0m = sqrt(dot3(F0, F0));
    if (F0m <= FC) {
        for (int a = 0; a < 3; a++) { Fout[a] = F0[a]; xi[a] += vt[a]; }
    } else {
        for (int a = 0; a < 3; a++) Fout[a] = FC * F0[a] / F0m;
        for (int a = 0; a < 3; a++) xi[a] = k > 0.0 ? -(Fout[a] + gam * vt[a]) / k : 0.0;
    }
}

/* contact between particle i and partner j (j<0: substrate).
 * n: unit normal from partner to i; delta > 0 the overlap.
 * READING c19: F_n = [k_n delta - g_n (v_rel.n)] n;  READING c21: contact
 * point at X_i - (R_c,i - delta/2) n;  READING c23: rolling velocity
 * v_r = -a'(w_i - w_j) x n, rolling torque (X_C - X_i)-lever: -a' n x F_r. */
static void contact(or_sim *s, int i, int j, const double *xn, const double *vp, const double *wp,
                    const double *n, double delta, double *xi, double *xir)
{
    const or_params *pp = &s->p;
    or_part *Pi = &s->P[i];
    double bi[3], bj[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) bi[a] = -(Pi->Rc - 0.5 * delta) * n[a];
    double vi[3], t[3];
    cross3(&wp[3 * i], bi, t);
    for (int a = 0; a < 3; a++) vi[a] = vp[3 * i + a] + t[a];
    double vj[3];
    double ap;
    if (j >= 0) {
        or_part *Pj = &s->P[j];
        for (int a = 0; a < 3; a++) bj[a] = (Pj->Rc - 0.5 * delta) * n[a];
        cross3(&wp[3 * j], bj, t);
        for (int a = 0; a < 3; a++) vj[a] = vp[3 * j + a] + t[a];
        ap = Pi->Rc * Pj->Rc / (Pi->Rc + Pj->Rc);
    } else {
        for (int a = 0; a < 3; a++) vj[a] = pp->wall_velocity[a];
        ap = Pi->Rc;
    }
    (void)xn;
    double vrel[3];
    for (int a = 0; a < 3; a++) vrel[a] = vi[a] - vj[a];
    double vn = dot3(vrel, n);
    double Fnm = pp->kn * delta - pp->gn * vn;
    double Fn[3], vt[3];
    for (int a = 0; a < 3; a++) { Fn[a] = Fnm * n[a]; vt[a] = vrel[a] - vn * n[a]; }
    double Ft[3];
    friction_spring(xi, n, vt, pp->kt, pp->gt, pp->mu_s * fabs(Fnm), Ft);
    double wrel[3];
    for (int a = 0; a < 3; a++) wrel[a] = wp[3 * i + a] - (j >= 0 ? wp[3 * j + a] : 0.0);
    double vr[3];
    cross3(wrel, n, vr);
    for (int a = 0; a < 3; a++) vr[a] *= -ap;
    double Fr[3];
    friction_spring(xir, n, vr, pp->kr, pp->gr, pp->mu_r * fabs(Fnm), Fr);
    double Tt[3], Tr[3];
    cross3(bi, Ft, Tt);
    cross3(n, Fr, Tr);
    for (int a = 0; a < 3; a++) {
        Pi->Fc[a] += Fn[a] + Ft[a];
        Pi->Tc[a] += Tt[a] - ap * Tr[a];
    }
    if (j >= 0) {
        or_part *Pj = &s->P[j];
        double mFt[3] = {-Ft[0], -Ft[1], -Ft[2]}, Ttj[3];
        cross3(bj, mFt, Ttj);
        for (int a = 0; a < 3; a++) {
            Pj->Fc[a] -= Fn[a] + Ft[a];
            Pj->Tc[a] += Ttj[a] + ap * Tr[a];
        }
    }
}

static void quat_rotate(double *q, const double *w)
{
    double wm = sqrt(dot3(w, w));
    if (wm == 0.0) return;
    double h = 0.5 * wm;
    double dq[4] = {cos(h), sin(h) * w[0] / wm, sin(h) * w[1] / wm, sin(h) * w[2] / wm};
    double r[4];
    r[0] = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
    r[1] = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
    r[2] = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
    r[3] = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
    double l = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int a = 0; a < 4; a++) q[a] = r[a] / l;
}

/* READING c24: velocity Verlet, dt = 1.  Contact forces at step n+1 use the
 * new positions and the predicted velocities v_n + a_n; the fluid forces are
 * those of the LBM step just taken. */
static void dem_step(or_sim *s, int with_fluid)
{
    int np = s->np;
    double xn[3 * OR_MAXP], vp[3 * OR_MAXP], wp[3 * OR_MAXP];
    for (int p = 0; p < np; p++) {
        or_part *P = &s->P[p];
        for (int a = 0; a < 3; a++) {
            if (P->kin) {
                xn[3 * p + a] = P->x[a] + P->v[a];
                vp[3 * p + a] = P->v[a];
                wp[3 * p + a] = P->w[a];
            } else {
                double acc = P->Fp[a] / P->m, alp = P->Tp[a] / P->I;
                xn[3 * p + a] = P->x[a] + P->v[a] + 0.5 * acc;
                vp[3 * p + a] = P->v[a] + acc;
                wp[3 * p + a] = P->w[a] + alp;
            }
        }
        for (int a = 0; a < 3; a++) { P->Fc[a] = 0.0; P->Tc[a] = 0.0; }
    }
    /* particle-substrate contacts: delta = R_c - (z_p - z_s), z_s = 0.5 */
    for (int p = 0; p < np; p++) {
        double delta = s->P[p].Rc - (xn[3 * p + 2] - 0.5);
        if (s->p.wall_z0 && delta > 0.0) {
            double n[3] = {0.0, 0.0, 1.0};
            contact(s, p, -1, xn, vp, wp, n, delta, s->xi_w[p], s->xir_w[p]);
        } else {
            for (int a = 0; a < 3; a++) { s->xi_w[p][a] = 0.0; s->xir_w[p][a] = 0.0; }
        }
    }
    /* particle-particle contacts: delta_ij = R_i + R_j - |X_i - X_j| */
    for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
            double d[3] = {minimg(xn[3 * i] - xn[3 * j], s->nx), minimg(xn[3 * i + 1] - xn[3 * j + 1], s->ny),
                           minimg(xn[3 * i + 2] - xn[3 * j + 2], s->nz)};
            double dl = sqrt(dot3(d, d));
            double delta = s->P[i].Rc + s->P[j].Rc - dl;
            if (delta > 0.0 && dl > 0.0) {
                double n[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
                contact(s, i, j, xn, vp, wp, n, delta, s->xi_p[i][j], s->xir_p[i][j]);
            } else {
                for (int a = 0; a < 3; a++) { s->xi_p[i][j][a] = 0.0; s->xir_p[i][j][a] = 0.0; }
            }
        }
    for (int p = 0; p < np; p++) {
        or_part *P = &s->P[p];
        double F[3], T[3];
        for (int a = 0; a < 3; a++) {
            F[a] = P->Fc[a] + s->p.g_particle[a] + (with_fluid ? P->Feta[a] + P->Fsig[a] + P->Fb[a] : 0.0);
            T[a] = P->Tc[a] + (with_fluid ? P->Teta[a] + P->Tsig[a] : 0.0);
        }
        double wold[3] = {P->w[0], P->w[1], P->w[2]};
        if (!P->kin) {
            for (int a = 0; a < 3; a++) {
                P->v[a] += 0.5 * (P->Fp[a] + F[a]) / P->m;
                P->w[a] += 0.5 * (P->Tp[a] + T[a]) / P->I;
            }
        }
        double wm[3] = {0.5 * (wold[0] + P->w[0]), 0.5 * (wold[1] + P->w[1]), 0.5 * (wold[2] + P->w[2])};
        quat_rotate(P->q, wm);
        for (int a = 0; a < 3; a++) {
            /* periodic domain: positions kept in [0, n) */
            const int per = a == 0 ? s->nx : (a == 1 ? s->ny : s->nz);
            P->x[a] = xn[3 * p + a] - per * floor(xn[3 * p + a] / per);
            P->Fp[a] = F[a];
            P->Tp[a] = T[a];
        }
    }
}

int or_dem_only_step(or_sim *s, int n, double *traj)
{
    for (int t = 0; t < n; t++) {
        for (int p = 0; p < s->np; p++)
            for (int a = 0; a < 3; a++)
                s->P[p].Feta[a] = s->P[p].Teta[a] = s->P[p].Fsig[a] = s->P[p].Tsig[a] = 0.0;
        dem_step(s, 0);
        if (traj)
            for (int p = 0; p < s->np; p++) {
                double *o = traj + ((long)t * s->np + p) * 13;
                for (int a = 0; a < 3; a++) { o[a] = s->P[p].x[a]; o[3 + a] = s->P[p].v[a]; o[6 + a] = s->P[p].w[a]; }
                for (int a = 0; a < 4; a++) o[9 + a] = s->P[p].q[a];
            }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* one coupled time step (READING c26: the order of the flow chart of the */
/* coupled algorithm, Fig. 4, is taken as stream + bounce-back + momentum */
/* exchange, moments, gradient + wetting, curvature, force, MRT + Guo,     */
/* recolour, capillary force, DEM, refill)                                 */
/* ---------------------------------------------------------------------- */
static void step_once(or_sim *s)
{
    const long N = s->N;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const or_params *pp = &s->p;
    double bb_mass = 0.0;

    /* (1) Sec. IV streaming with Sec. V A halfway bounce-back.
     * READING c13: f_i(x_f) = f*_ibar(x_f) + 2 w_i rho^{a,b}(x_f) (c_i.u_w)/cs2,
     * c_i pointing from the wall into the fluid, rho^{a,b}(x_f) the density
     * at x_f before streaming; u_w taken at the link midpoint. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] != FLUID) continue;
                double ra = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
                int have_rho = 0;
                for (int i = 0; i < OR_Q; i++) {
                    long sid = nbr(s, x, y, z, -OR_C[i][0], -OR_C[i][1], -OR_C[i][2]);
                    int o = s->owner[sid];
                    if (o == FLUID) {
                        s->fas[i * N + id] = s->fa[i * N + sid];
                        s->fbs[i * N + id] = s->fb[i * N + sid];
                        continue;
                    }
                    if (!have_rho) {
                        for (int k = 0; k < OR_Q; k++) {
                            ra += s->fa[k * N + id];
                            rb += s->fb[k * N + id];
                            for (int a = 0; a < 3; a++) j[a] += OR_C[k][a] * (s->fa[k * N + id] + s->fb[k * N + id]);
                        }
                        have_rho = 1;
                    }
                    if (o == PRESS) {
                        /* Sec. V D anti-bounce-back (Krueger et al. 2016):
                         * f_in(x_b) = -f*_out(x_b)
                         *   + 2 w_i rho_w [1 + (c_i.u_w)^2/(2 cs^4) - u_w^2/(2 cs^2)],
                         * p_w = cs^2 rho_w.  READING: rho_w = rho_in on the face
                         * below the fluid (source plane z=0), rho_out above; u_w
                         * = j / rho and the colour split rho^{a,b}_w =
                         * rho_w rho^{a,b} / rho of x_b's own post-collision state. */
                        const double rw = OR_C[i][2] > 0 ? pp->rho_in : pp->rho_out;
                        const double rt = ra + rb;
                        const double uw[3] = {j[0] / rt, j[1] / rt, j[2] / rt};
                        const double cu = OR_C[i][0] * uw[0] + OR_C[i][1] * uw[1] + OR_C[i][2] * uw[2];
                        const double e = 1.0 + 4.5 * cu * cu - 1.5 * dot3(uw, uw);
                        int ib = OR_OPP[i];
                        s->fas[i * N + id] = -s->fa[ib * N + id] + 2.0 * OR_W[i] * rw * (ra / rt) * e;
                        s->fbs[i * N + id] = -s->fb[ib * N + id] + 2.0 * OR_W[i] * rw * (rb / rt) * e;
                        continue;
                    }
                    double xw[3] = {x - 0.5 * OR_C[i][0], y - 0.5 * OR_C[i][1], z - 0.5 * OR_C[i][2]};
                    double uw[3], lev[3];
                    surface_velocity(s, o, xw, uw, lev);
                    double cu = OR_C[i][0] * uw[0] + OR_C[i][1] * uw[1] + OR_C[i][2] * uw[2];
                    int ib = OR_OPP[i];
                    s->fas[i * N + id] = s->fa[ib * N + id] + 6.0 * OR_W[i] * ra * cu;
                    s->fbs[i * N + id] = s->fb[ib * N + id] + 6.0 * OR_W[i] * rb * cu;
                }
            }

    /* (2) Sec. V B momentum exchange (Wen 2014).  READING c14: per link the
     * force on the particle is (c_out - u_w) f_out - (c_in - u_w) f_in, with
     * f_out the population that left the fluid node towards the solid and
     * f_in the one bounced back, summed over both components; lever arm from
     * the particle centre to the link midpoint.  Serial, in node order. */
    for (int p = 0; p < s->np; p++)
        for (int a = 0; a < 3; a++) s->P[p].Feta[a] = s->P[p].Teta[a] = 0.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] != FLUID) continue;
                for (int i = 1; i < OR_Q; i++) {
                    long sid = nbr(s, x, y, z, -OR_C[i][0], -OR_C[i][1], -OR_C[i][2]);
                    int o = s->owner[sid];
                    if (o == FLUID) continue;
                    int ib = OR_OPP[i];
                    double fout = s->fa[ib * N + id] + s->fb[ib * N + id];
                    double fin = s->fas[i * N + id] + s->fbs[i * N + id];
                    bb_mass += fin - fout;
                    if (o == WALL || o == PRESS) continue;
                    or_part *P = &s->P[o - 2];
                    double xw[3] = {x - 0.5 * OR_C[i][0], y - 0.5 * OR_C[i][1], z - 0.5 * OR_C[i][2]};
                    double uw[3], lev[3];
                    surface_velocity(s, o, xw, uw, lev);
                    double dp[3], t[3];
                    for (int a = 0; a < 3; a++)
                        dp[a] = (OR_C[ib][a] - uw[a]) * fout - (OR_C[i][a] - uw[a]) * fin;
                    cross3(lev, dp, t);
                    for (int a = 0; a < 3; a++) { P->Feta[a] += dp[a]; P->Teta[a] += t[a]; }
                }
            }

    /* (3) Sec. IV order parameter phi = (rho^a - rho^b)/(rho^a + rho^b) */
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; id++) {
        if (s->owner[id] != FLUID) continue;
        double ra = 0.0, rb = 0.0;
        for (int i = 0; i < OR_Q; i++) { ra += s->fas[i * N + id]; rb += s->fbs[i * N + id]; }
        s->phi[id] = (ra - rb) / (ra + rb);
    }
    /* (4) READING c9: phi on solid nodes = w-weighted mean of fluid neighbours */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] == FLUID) continue;
                double sw = 0.0, sp = 0.0;
                for (int i = 1; i < OR_Q; i++) {
                    long nid = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
                    if (s->owner[nid] != FLUID) continue;
                    sw += OR_W[i];
                    sp += OR_W[i] * s->phi[nid];
                }
                s->phi[id] = sw > 0.0 ? sp / sw : 0.0;
            }
    /* (5) READING c5: grad phi = (1/cs2) sum_i w_i c_i phi(x + c_i); then the
     * Sec. V E wetting rotation at fluid nodes next to a solid inside the
     * diffuse interface (READING c10: |phi| < wet_phi_max = 0.99). */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] != FLUID) {
                    for (int a = 0; a < 3; a++) s->grad[a * N + id] = s->nrm[a * N + id] = 0.0;
                    continue;
                }
                double g[3] = {0, 0, 0};
                for (int i = 1; i < OR_Q; i++) {
                    long nid = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
                    for (int a = 0; a < 3; a++) g[a] += 3.0 * OR_W[i] * OR_C[i][a] * s->phi[nid];
                }
                if (fabs(s->phi[id]) < pp->wet_phi_max) {
                    double ns[3], th;
                    if (solid_normal(s, x, y, z, ns, &th)) or_wetting_rotate(g, ns, th);
                }
                for (int a = 0; a < 3; a++) s->grad[a * N + id] = g[a];
                double gr = sqrt(dot3(g, g) + pp->grad_eps * pp->grad_eps);
                for (int a = 0; a < 3; a++) s->nrm[a * N + id] = g[a] / gr;
            }
    /* (6) curvature, force, collision, recolouring.
     * READING c6: kappa = div(n) with the same stencil, n the interface normal
     * grad(phi)/|grad(phi)| taken in the regularised form
     * grad(phi)/sqrt(|grad(phi)|^2 + eps^2), continuous where grad(phi) vanishes
     * inside the diffuse interface; READING c7: a solid neighbour contributes
     * the node's own n.
     * Sec. IV CSF: F = -1/2 sigma kappa grad(phi); body forces weighted by the
     * local phase fractions (1 +- phi)/2 (Sec. II, Sec. VI A). */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] != FLUID) {
                    for (int a = 0; a < 3; a++) s->u[a * N + id] = 0.0;
                    continue;
                }
                double kap = 0.0;
                for (int i = 1; i < OR_Q; i++) {
                    long nid = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
                    long src = s->owner[nid] == FLUID ? nid : id;
                    double cn = 0.0;
                    for (int a = 0; a < 3; a++) cn += OR_C[i][a] * s->nrm[a * N + src];
                    kap += OR_W[i] * cn;
                }
                kap *= 3.0;
                double ph = s->phi[id];
                double F[3];
                for (int a = 0; a < 3; a++)
                    F[a] = -0.5 * pp->sigma * kap * s->grad[a * N + id] +
                           0.5 * (1.0 + ph) * pp->body_force_a[a] + 0.5 * (1.0 - ph) * pp->body_force_b[a];
                double fa[OR_Q], fb[OR_Q], fao[OR_Q], fbo[OR_Q], nh[3], uo[3];
                double rho = 0.0;
                for (int i = 0; i < OR_Q; i++) {
                    fa[i] = s->fas[i * N + id];
                    fb[i] = s->fbs[i * N + id];
                    rho += fa[i] + fb[i];
                }
                for (int a = 0; a < 3; a++) nh[a] = s->nrm[a * N + id];
                double om = or_omega_of_phi(pp, ph, rho);
                double omp = 8.0 * (2.0 - om) / (8.0 - om);
                or_collide_node(fa, fb, F, nh, om, omp, pp->beta, fao, fbo, uo);
                for (int i = 0; i < OR_Q; i++) {
                    s->fa[i * N + id] = fao[i];
                    s->fb[i * N + id] = fbo[i];
                }
                for (int a = 0; a < 3; a++) s->u[a * N + id] = uo[a];
            }
    /* (7) capillary force, Sec. V F */
    for (int p = 0; p < s->np; p++) or_capillary(s, p, s->P[p].Fsig, s->P[p].Tsig);
    /* (7b) buoyancy, READING c28: F_b = (4/3) pi R^3 v b_a (v reported only
     * where the buoyancy is on; with b_a = 0 both stay 0) */
    const int buoy_on = s->p.buoyancy_a[0] != 0.0 || s->p.buoyancy_a[1] != 0.0 || s->p.buoyancy_a[2] != 0.0;
    for (int p = 0; buoy_on && p < s->np; p++) {
        or_part *P = &s->P[p];
        P->sub = or_immersed_fraction(s, p);
        const double vol = 4.0 / 3.0 * M_PI * P->R * P->R * P->R;
        for (int a = 0; a < 3; a++) P->Fb[a] = vol * P->sub * s->p.buoyancy_a[a];
    }
    /* (8) DEM, Sec. III and Eqs. (Newton second law), (Newton - rotation) */
    if (s->np > 0) dem_step(s, 1);
    /* (9) geometry update and Sec. V C refilling (Caiazzo 2008).
     * READING c16: neighbours are the 18 moving directions, fluid and not
     * fresh; none -> the nodes two steps away along the same directions;
     * still none -> the ambient state (rho^a, rho^b) = (0, rho0). */
    double refill_mass = 0.0, cover_mass = 0.0;
    if (s->np > 0) {
        memcpy(s->old_owner, s->owner, N);
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    long id = lidx(s, x, y, z);
                    int o = solid_owner_of(s, x, y, z);
                    s->owner[id] = (unsigned char)o;
                    s->fresh[id] = (s->old_owner[id] >= 2 && o == FLUID);
                    if (s->old_owner[id] == FLUID && o != FLUID)
                        for (int i = 0; i < OR_Q; i++) cover_mass += s->fa[i * N + id] + s->fb[i * N + id];
                }
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    long id = lidx(s, x, y, z);
                    if (!s->fresh[id]) continue;
                    double ra = 0.0, rb = 0.0;
                    int nf = 0;
                    for (int hop = 1; hop <= 2 && nf == 0; hop++)
                        for (int i = 1; i < OR_Q; i++) {
                            long nid = nbr(s, x, y, z, hop * OR_C[i][0], hop * OR_C[i][1], hop * OR_C[i][2]);
                            if (s->owner[nid] != FLUID || s->fresh[nid]) continue;
                            for (int k = 0; k < OR_Q; k++) { ra += s->fa[k * N + nid]; rb += s->fb[k * N + nid]; }
                            nf++;
                        }
                    if (nf > 0) { ra /= nf; rb /= nf; }
                    else { ra = 0.0; rb = pp->rho0; }
                    const or_part *P = &s->P[s->old_owner[id] - 2];
                    double d[3] = {minimg(x - P->x[0], nx), minimg(y - P->x[1], ny), minimg(z - P->x[2], nz)};
                    double un[3];
                    cross3(P->w, d, un);
                    for (int a = 0; a < 3; a++) un[a] += P->v[a];
                    double f[OR_Q];
                    feq(ra, un, f);
                    for (int i = 0; i < OR_Q; i++) s->fa[i * N + id] = f[i];
                    feq(rb, un, f);
                    for (int i = 0; i < OR_Q; i++) s->fb[i * N + id] = f[i];
                    refill_mass += ra + rb;
                }
    }
    /* diagnostics of the post-collision state */
    double mass = 0.0, mom[3] = {0, 0, 0};
    for (long id = 0; id < N; id++) {
        if (s->owner[id] != FLUID) continue;
        for (int i = 0; i < OR_Q; i++) {
            double f = s->fa[i * N + id] + s->fb[i * N + id];
            mass += f;
            for (int a = 0; a < 3; a++) mom[a] += OR_C[i][a] * f;
        }
    }
    s->diag[0] = bb_mass;
    s->diag[1] = refill_mass;
    s->diag[2] = cover_mass;
    s->diag[3] = mass;
    for (int a = 0; a < 3; a++) s->diag[4 + a] = mom[a];
}

/* phi, grad(phi) (with the wetting rotation) and n evaluated from the
 * current post-collision state without streaming: steps (3)-(5) of a time
 * step applied to f* itself.  Used by the pin tests of the gradient, wetting
 * and capillary-force parts; leaves the populations untouched. */
int or_eval_interface(or_sim *s)
{
    const long N = s->N;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    for (long id = 0; id < N; id++) {
        if (s->owner[id] != FLUID) continue;
        double ra = 0.0, rb = 0.0;
        for (int i = 0; i < OR_Q; i++) { ra += s->fa[i * N + id]; rb += s->fb[i * N + id]; }
        s->phi[id] = (ra - rb) / (ra + rb);
    }
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                if (s->owner[id] == FLUID) continue;
                double sw = 0.0, sp = 0.0;
                for (int i = 1; i < OR_Q; i++) {
                    long nid = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
                    if (s->owner[nid] != FLUID) continue;
                    sw += OR_W[i];
                    sp += OR_W[i] * s->phi[nid];
                }
                s->phi[id] = sw > 0.0 ? sp / sw : 0.0;
            }
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long id = lidx(s, x, y, z);
                double g[3] = {0, 0, 0};
                if (s->owner[id] == FLUID) {
                    for (int i = 1; i < OR_Q; i++) {
                        long nid = nbr(s, x, y, z, OR_C[i][0], OR_C[i][1], OR_C[i][2]);
                        for (int a = 0; a < 3; a++) g[a] += 3.0 * OR_W[i] * OR_C[i][a] * s->phi[nid];
                    }
                    if (fabs(s->phi[id]) < s->p.wet_phi_max) {
                        double ns[3], th;
                        if (solid_normal(s, x, y, z, ns, &th)) or_wetting_rotate(g, ns, th);
                    }
                }
                double gr = sqrt(dot3(g, g) + s->p.grad_eps * s->p.grad_eps);
                for (int a = 0; a < 3; a++) {
                    s->grad[a * N + id] = g[a];
                    s->nrm[a * N + id] = g[a] / gr;
                }
            }
    return 0;
}

void or_get_phi(const or_sim *s, double *phi)
{
    memcpy(phi, s->phi, sizeof(double) * s->N);
}

/* READING c27: the drop is driven by the body force on phase a.
   Every `interval` steps the mass-weighted velocity of phase a over the fluid
   nodes of the current (post-collision) state,
       U_a = sum_x (rho^a / rho) j / sum_x rho^a,  j = sum_i c_i (f^a_i + f^b_i),
   is compared with the target, e = U_target - U_a, and each controlled
   component follows the PI law f_a = f0 + kp e + ki sum_k (e_k interval). */
static void speed_control(or_sim *s)
{
    const or_params *p = &s->p;
    double sa = 0.0, su[3] = {0.0, 0.0, 0.0};
    for (long id = 0; id < s->N; id++) {
        if (s->owner[id] != FLUID) continue;
        double ra = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < OR_Q; i++) {
            const double fa = s->fa[i * s->N + id], fb = s->fb[i * s->N + id];
            ra += fa;
            rb += fb;
            for (int a = 0; a < 3; a++) j[a] += OR_C[i][a] * (fa + fb);
        }
        const double w = ra / (ra + rb);
        for (int a = 0; a < 3; a++) su[a] += w * j[a];
        sa += ra;
    }
    double kp = p->drop_speed_kp, ki = p->drop_speed_ki;
    if (kp == 0.0 && ki == 0.0) {
        kp = p->rho0 / 1000.0;
        ki = kp / 5000.0;
    }
    const int iv = p->drop_speed_interval > 0 ? p->drop_speed_interval : 100;
    for (int a = 0; a < 3; a++) {
        s->sp_u[a] = sa > 0.0 ? su[a] / sa : 0.0;
        if (!(p->drop_speed_control & (1 << a))) continue;
        const double e = p->drop_speed_target[a] - s->sp_u[a];
        s->sp_int[a] += e * iv;
        s->p.body_force_a[a] = s->sp_f0[a] + kp * e + ki * s->sp_int[a];
    }
}

int or_step(or_sim *s, int n)
{
    for (int t = 0; t < n; t++) {
        step_once(s);
        s->steps++;
        const int iv = s->p.drop_speed_interval > 0 ? s->p.drop_speed_interval : 100;
        if (s->p.drop_speed_control && s->steps % iv == 0) speed_control(s);
    }
    return 0;
}

void or_get_speed_control(const or_sim *s, double *out)
{
    for (int a = 0; a < 3; a++) {
        out[a] = s->p.body_force_a[a];
        out[3 + a] = s->sp_u[a];
    }
}

void or_get_pops(const or_sim *s, double *fa, double *fb)
{
    for (int i = 0; i < OR_Q; i++)
        for (long id = 0; id < s->N; id++) {
            int fl = s->owner[id] == FLUID;
            fa[i * s->N + id] = fl ? s->fa[i * s->N + id] : 0.0;
            fb[i * s->N + id] = fl ? s->fb[i * s->N + id] : 0.0;
        }
}

void or_get_fields(const or_sim *s, double *rho_a, double *rho_b, double *phi, double *u)
{
    const long N = s->N;
    for (long id = 0; id < N; id++) {
        double ra = 0.0, rb = 0.0;
        if (s->owner[id] == FLUID)
            for (int i = 0; i < OR_Q; i++) { ra += s->fa[i * N + id]; rb += s->fb[i * N + id]; }
        if (rho_a) rho_a[id] = ra;
        if (rho_b) rho_b[id] = rb;
        if (phi) phi[id] = s->owner[id] == FLUID ? (ra - rb) / (ra + rb) : 0.0;
        if (u)
            for (int a = 0; a < 3; a++) u[a * N + id] = s->u[a * N + id];
    }
}

void or_get_grad(const or_sim *s, double *grad)
{
    memcpy(grad, s->grad, sizeof(double) * 3 * s->N);
}

void or_get_owner(const or_sim *s, unsigned char *owner)
{
    memcpy(owner, s->owner, s->N);
}

int or_num_particles(const or_sim *s) { return s->np; }

void or_get_particles(const or_sim *s, double *out)
{
    for (int p = 0; p < s->np; p++) {
        const or_part *P = &s->P[p];
        double *o = out + 36 * p;
        for (int a = 0; a < 3; a++) {
            o[a] = P->Feta[a]; o[3 + a] = P->Teta[a];
            o[6 + a] = P->Fsig[a]; o[9 + a] = P->Tsig[a];
            o[12 + a] = P->Fc[a]; o[15 + a] = P->Tc[a];
            o[18 + a] = P->x[a]; o[21 + a] = P->v[a]; o[24 + a] = P->w[a];
        }
        for (int a = 0; a < 4; a++) o[27 + a] = P->q[a];
        o[31] = P->m;
        o[32] = P->sub;
        for (int a = 0; a < 3; a++) o[33 + a] = P->Fb[a];
    }
}

void or_get_diag(const or_sim *s, double *out)
{
    for (int k = 0; k < 7; k++) out[k] = s->diag[k];
}
