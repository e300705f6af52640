/*
 * FP64 CPU oracle of the coupled colour-gradient LBM / DEM method
 * (Naga, Zhang, Yang, Kusumaatmaja, arXiv 2505.10171).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lbm_oracle.c are the plain,
 * slow reference against which the CUDA path is checked.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, table or constant with the CUDA library.
 *
 * Every array is z-major: index = (z*ny + y)*nx + x.  Populations are
 * [19][N] per component, in the velocity order of OR_C below.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_Q 19
#define OR_MAXP 61

typedef struct {
    int nx, ny, nz;
    int wall_z0;                 /* 1: node plane z=0 is solid substrate */
    double wall_velocity[3];     /* tangential substrate velocity         */
    double theta_wall_deg;       /* substrate contact angle (inside phase a) */
    double rho0;                 /* reference density                      */
    double nu_a, nu_b;           /* kinematic viscosities of phases a, b   */
    double sigma;                /* interfacial tension                    */
    double beta;                 /* recolouring segregation parameter      */
    double cap_norm;             /* capillary-force prefactor C (Sec. V F) */
    double body_force_a[3];      /* force density on phase a               */
    double body_force_b[3];      /* force density on phase b               */
    double kn, kt, kr;           /* DEM spring stiffnesses                 */
    double gn, gt, gr;           /* DEM damping constants                  */
    double mu_s, mu_r;           /* sliding / rolling friction coeffs      */
    double delta_R;              /* R_c - R_p                              */
    double g_particle[3];        /* external force on every particle       */
    double grad_eps;             /* eps of the normal g/sqrt(|g|^2+eps^2) */
    double wet_phi_max;          /* wetting applied where |phi| < this     */
    int drop_speed_control;      /* bit a set: PI control of body_force_a[a] */
    double drop_speed_target[3]; /* target mean velocity of phase a        */
    double drop_speed_kp, drop_speed_ki;  /* PI gains; both 0: rho0/1000, rho0/(1000*5000) */
    int drop_speed_interval;     /* steps between updates; 0: 100          */
    int pressure_z;              /* 1: node planes z=0 and z=nz-1 are pressure faces (Sec. V D) */
    double rho_in, rho_out;      /* density imposed on the face at z=0.5 / z=nz-1.5 */
    double buoyancy_a[3];        /* READING c28: force per unit particle volume immersed in phase a */
} or_params;

typedef struct or_sim or_sim;

or_sim *or_create(const or_params *p);
void    or_destroy(or_sim *s);
int     or_set_static_solid(or_sim *s, const unsigned char *mask);
int     or_init_fields(or_sim *s, const double *phi, const double *rho, const double *u);
int     or_set_pops(or_sim *s, const double *fa, const double *fb);
int     or_add_particle(or_sim *s, const double *x, const double *v, const double *w,
                        double R, double rho_p, double theta_deg, int kinematic);
int     or_step(or_sim *s, int n);
int     or_dem_only_step(or_sim *s, int n, double *traj /* [n][np][13] or NULL */);

void    or_get_pops(const or_sim *s, double *fa, double *fb);
void    or_get_fields(const or_sim *s, double *rho_a, double *rho_b, double *phi, double *u);
void    or_get_grad(const or_sim *s, double *grad /* [3][N] */);
void    or_get_owner(const or_sim *s, unsigned char *owner);
int     or_num_particles(const or_sim *s);
/* body force on phase a now and the phase-a velocity of the last controller update */
void    or_get_speed_control(const or_sim *s, double *out /* [6] */);
/* per particle 36 doubles: F_eta[3] T_eta[3] F_sig[3] T_sig[3] F_c[3] T_c[3]
   x[3] v[3] w[3] q[4] m, immersed volume fraction in phase a, buoyancy F_b[3]
   (the last two 0 while buoyancy_a is zero) */
void    or_get_particles(const or_sim *s, double *out);
/* per step: [0] bounce-back mass source, [1] refilled mass, [2] covered mass,
   [3] total fluid mass, [4..6] total fluid momentum (post-collision state) */
void    or_get_diag(const or_sim *s, double *out);

/* building blocks exposed for the pin tests */
void    or_lattice(int *c /* [19][3] */, double *w, int *opp);
void    or_mrt_matrices(double *M /* [19][19] */, double *Minv, double *S_pattern /* 1=omega,2=omega',0 */);
void    or_collide_node(const double *fa, const double *fb, const double *F_ext,
                        const double *nhat, double omega, double omega_p, double beta,
                        double *fa_out, double *fb_out, double *u_out);
double  or_omega_of_phi(const or_params *p, double phi, double rho);
void    or_wetting_rotate(double *g, const double *ns, double theta_rad);
int     or_capillary(const or_sim *s, int p, double *F, double *T);
double  or_immersed_fraction(const or_sim *s, int p);
int     or_eval_interface(or_sim *s);
void    or_get_phi(const or_sim *s, double *phi);

#ifdef __cplusplus
}
#endif
#endif
