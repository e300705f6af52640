/*
 * lbm.h - C ABI of the GB300 (sm_103a) hot path of the coupled colour-gradient
 * lattice Boltzmann / discrete element method for droplet-particle
 * interactions on solid surfaces (Naga, Zhang, Yang, Kusumaatmaja,
 * arXiv 2505.10171).
 *
 * One context holds one or more independent simulation instances (a batch of
 * uneven domains is stepped together).  Each instance is a periodic
 * nx x ny x nz D3Q19 lattice with two fluid components a (phi = +1) and b
 * (phi = -1), an optional solid substrate at the node plane z = 0, optional
 * static solid nodes, and up to LBM_MAX_PARTICLES rigid spheres.
 *
 * Conventions shared by every entry point:
 *  - Fields are z-major: node (x, y, z) sits at index (z*ny + y)*nx + x, and a
 *    vector field is three such blocks (x, y, z components).  Every value that
 *    crosses this boundary is IEEE double, whatever the storage precision.
 *  - Populations crossing the boundary are f^a_i then f^b_i, each [19][N], in
 *    the velocity order LBM_C below.
 *  - The caller owns every host buffer and every device buffer it passes; the
 *    library owns all device memory it allocates (released by lbm_destroy).
 *  - No C++ exception crosses this boundary.  Every call returns an
 *    lbm_status; lbm_last_error() gives a one-line description of the last
 *    failure on a context.  A device-side instability (non-finite or
 *    non-positive density) or an illegal particle displacement sets a sticky
 *    status reported by the next synchronising call.
 *  - lbm_step is asynchronous on the context's stream; the read functions
 *    synchronise that stream.
 *  - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19
#define LBM_MAX_PARTICLES 61

/* D3Q19 velocity order of every population array at this boundary
 * (Sec. IV: D3Q19 after Krueger et al.): rest, +-x, +-y, +-z, then the twelve
 * face diagonals in opposite pairs. */
#define LBM_C                                                                  \
    {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1},       \
     {0, 0, -1}, {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},    \
     {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1},  \
     {0, -1, 1}}

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument or physically invalid parameter */
    LBM_ERR_OOM = 2,         /* device allocation failed                        */
    LBM_ERR_CUDA = 3,        /* CUDA runtime error                              */
    LBM_ERR_STATE = 4,       /* call not valid in the current state             */
    LBM_ERR_UNSTABLE = 5,    /* non-finite/non-positive density seen on device  */
    LBM_ERR_TIMEOUT = 6,     /* a bounded device wait gave up (tensor-core GEMM) */
    LBM_ERR_UNSUPPORTED = 7  /* feature or precision not available              */
} lbm_status;

/* Population storage.  Every form stores the total populations as offsets
 * F_i = f_i/(w_i rho0) - 1: FP64, FP32, or half / bfloat16 with FP32
 * arithmetic.  The colour populations are not stored: after the recolouring
 * step of Sec. IV a node's colour offsets are
 * (f^a_i - f^b_i)/(w_i rho0) = phi (1 + F_i) + b (c_i . n)/|c_i|,
 * b = beta/2 (rho/rho0)(1 - phi^2), with the order parameter phi and the
 * interface normal n of that node's collision, so the state keeps phi, b and
 * n per node (FP64 in the FP64 form, FP32 otherwise) and every colour
 * population is rebuilt from them.  Particle sums, the DEM and mass sums are
 * FP64 in every form. */
typedef enum {
    LBM_FP64 = 0,
    LBM_FP32 = 1,
    LBM_FP16_OFFSET = 2,
    LBM_BF16_OFFSET = 3
} lbm_precision;

/* Physical parameters of one instance (lattice units, dt = dx = 1).
 * Table I of the paper gives the ranges used there. */
typedef struct {
    int nx, ny, nz;            /* lattice size, periodic in x, y and z (Sec. VI A);      */
                               /*    38 nx ny nz < 2^31 per instance                       */
    int wall_z0;               /* 1: node plane z = 0 is the substrate; its halfway wall  */
                               /*    sits at z = 0.5 (and z = nz - 0.5 through periodicity) */
    double wall_velocity[3];   /* substrate velocity (moving-wall bounce-back, Sec. V A)  */
    double theta_wall_deg;     /* substrate contact angle, measured in phase a (Sec. V E) */
    double rho0;               /* reference density                                       */
    double nu_a, nu_b;         /* kinematic viscosities; eta = rho0 nu, harmonic mean     */
                               /*    in phi (Sec. IV); must be > 0                         */
    double sigma;              /* interfacial tension (CSF force, Sec. IV)                */
    double beta;               /* recolouring segregation parameter in [0, 1] (Sec. IV)   */
    double cap_norm;           /* capillary prefactor C of Sec. V F; 0 selects 3 k beta,    */
                               /*    k = (1 + sqrt 2)/18 (the printed (9/2) k beta = 1.5x)   */
                               /*    with k = (1 + sqrt 2)/18                               */
    double body_force_a[3];    /* force density on phase a, weighted by (1 + phi)/2       */
    double body_force_b[3];    /* force density on phase b, weighted by (1 - phi)/2       */
    double kn, kt, kr;         /* DEM normal / sliding / rolling stiffness (Sec. III)     */
    double gn, gt, gr;         /* DEM damping constants                                   */
    double mu_s, mu_r;         /* sliding and rolling friction coefficients               */
    double delta_R;            /* mechanical minus hydrodynamic radius (Sec. V H)         */
    double g_particle[3];      /* external force on every particle (gravity, Sec. VI A)   */
    double grad_eps;           /* eps of the interface normal g/sqrt(|g|^2 + eps^2),       */
                               /*    g = grad phi; 0 selects 1e-4                          */
    double wet_phi_max;        /* wetting applied at nodes with |phi| < this; 0 -> 0.99   */
    int store_velocity;        /* 1: keep the collision velocity for lbm_read_fields(U)   */
    int diag_interval;         /* > 0: FP64 mass sums every that many steps               */
    double surrogate_u_ref;    /* surrogate inputs: velocity scale; 0 -> 1e-3             */
    double surrogate_r_ref;    /* surrogate inputs: radius scale; 0 -> 8                  */
    double surrogate_shell_gap;/* shell radius R_p + this; 0 -> 2                         */
    /* drop-speed control (driving of the drop by body_force_a): bit a of
     * drop_speed_control set -> every drop_speed_interval steps (0 -> 100) the
     * mass-weighted velocity of phase a over the fluid nodes,
     * U_a = sum (rho^a / rho) j / sum rho^a, j = sum_i c_i f_i, is compared with
     * drop_speed_target and body_force_a[a] = f0 + kp e + ki sum(e interval),
     * e = target - U_a, f0 = the body_force_a given here; kp = ki = 0 selects
     * kp = rho0/1000, ki = kp/5000 */
    int drop_speed_control;
    double drop_speed_target[3];
    double drop_speed_kp, drop_speed_ki;
    int drop_speed_interval;
    /* pressure boundaries (Sec. V D, anti-bounce-back): pressure_z = 1 makes the
     * node planes z = 0 and z = nz - 1 the outside of an inlet face at z = 0.5
     * with density rho_in and an outlet face at z = nz - 1.5 with rho_out
     * (pressure cs^2 rho); the fluid is then not periodic in z.  A link leaving
     * a boundary node x_b through a face takes
     * f_in = -f*_out(x_b) + 2 w_i rho_w [1 + (c_i.u_w)^2/(2 cs^4) - u_w^2/(2 cs^2)],
     * u_w and the colour split of rho_w from x_b's own post-collision state.
     * The faces carry no contact angle and no momentum-exchange force; keep
     * particles clear of them.  Needs nz >= 4 and wall_z0 = 0. */
    int pressure_z;
    double rho_in, rho_out;
    double surrogate_box;      /* surrogate inputs: box filter width (0: none), reading c30 */
    double buoyancy_a[3];      /* buoyancy, reading c28 (Sec. VI A): force per unit volume of a
                                  particle immersed in phase a, e.g. (0, 0, rho_a g); the
                                  particle receives (4/3) pi R^3 v buoyancy_a, v its immersed
                                  volume fraction in phase a (see LBM_PARTICLE_RECORD) */
} lbm_params;

/* One rigid sphere (Sec. III, V).  R_c = R_p + delta_R; m = rho_p 4/3 pi R_p^3;
 * I = 2/5 m R_p^2.  kinematic = 1 prescribes the motion (v, w kept constant). */
typedef struct {
    double x[3], v[3], w[3];
    double R_p, rho_p, theta_deg;
    int kinematic;
} lbm_particle;

/* lbm_read_fields mask bits; the output holds the selected fields one after
 * another in this bit order. */
enum {
    LBM_FIELD_RHO_A = 1,   /* sum_i f^a_i of the current state          [N]    */
    LBM_FIELD_RHO_B = 2,   /* sum_i f^b_i                                [N]    */
    LBM_FIELD_PHI = 4,     /* (rho^a - rho^b)/(rho^a + rho^b)            [N]    */
    LBM_FIELD_U = 8,       /* velocity of the last collision (Sec. IV)   [3][N] */
    LBM_FIELD_POPS = 16,   /* f^a then f^b, LBM_C order                  [38][N]*/
    LBM_FIELD_OWNER = 32   /* 0 fluid, 1 static solid, 2+p particle p    [N]    */
};

/* Number of doubles lbm_particle_forces writes per particle:
 * F_eta[3] T_eta[3] (momentum exchange, Sec. V B), F_sigma[3] T_sigma[3]
 * (capillary, Sec. V F), F_c[3] T_c[3] (contact, Sec. III), x[3] v[3] w[3],
 * orientation quaternion q[4] (w, x, y, z), m, then (reading c28) the
 * immersed volume fraction v in phase a and the buoyancy F_b[3].  v comes
 * from the phase-a share a of the capillary force's surface points,
 * s = (1 + phi)/2 clipped to [0, 1], area-weighted over the points with a
 * fluid corner: a flat interface at height (2a - 1) R above the centre leaves
 * v = (1 + t)^2 (2 - t)/4, t = 2a - 1, below it.  Both are those of the last
 * resolved-force step (0 before the first), and are computed only in contexts
 * where some instance has a nonzero buoyancy_a (0 otherwise). */
#define LBM_PARTICLE_RECORD 36

/* Create a context of n_instances instances; params points to n_instances
 * records (uneven sizes allowed).  stream is a cudaStream_t (NULL: the
 * library creates its own).  Validates every parameter (nu > 0, beta in
 * [0, 1], sizes > 0, finite values) -> LBM_ERR_ARG; allocates all lattice
 * memory -> LBM_ERR_OOM.  Populations start at rest with phi = -1 everywhere
 * until lbm_init_fields. */
lbm_status lbm_create(const lbm_params *params, int n_instances, lbm_precision prec,
                      void *stream, lbm_ctx **out);

/* Release all device memory of the context (NULL is ignored). */
void lbm_destroy(lbm_ctx *ctx);

/* One-line description of the last error on ctx (never NULL). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Mark static solid nodes of an instance (mask [N] host bytes, nonzero =
 * solid, e.g. a tube wall), in addition to the substrate plane.  Must come
 * before lbm_add_particles. */
lbm_status lbm_set_solid_mask(lbm_ctx *ctx, int inst, const uint8_t *mask);

/* Initialise the populations of an instance to the equilibrium (Sec. V C
 * form) of the given host fields: phi [N], rho [N] (NULL: rho0), u [3][N]
 * (NULL: at rest); rho^{a,b} = rho (1 +- phi)/2.  When pops is non-NULL it
 * holds f^a then f^b ([38][N], LBM_C order) and is stored instead (resume):
 * the total offsets as given, phi = (rho^a - rho^b)/rho, and b n from the
 * colour part beyond phi (1 + F_i) projected on (c_i . n)/|c_i|
 * (b n = 9/2 sum_i w_i c_i/|c_i| [G_i - phi (1 + F_i)]).  A state that
 * lbm_read_fields returned is restored exactly (to rounding); colour
 * populations of any other form keep only that projection.
 * Host buffers; synchronous. */
lbm_status lbm_init_fields(lbm_ctx *ctx, int inst, const double *phi, const double *rho,
                           const double *u, const double *pops);

/* As lbm_init_fields with device pointers (FP64), enqueued on the context's
 * stream; the buffers must stay valid until the stream reaches the call. */
lbm_status lbm_init_fields_device(lbm_ctx *ctx, int inst, const double *phi, const double *rho,
                                  const double *u);

/* Add n spheres to an instance (Sec. III, V).  Checks (-> LBM_ERR_ARG):
 * R_p > 0, rho_p > 0, 0 < theta < 180, hydrodynamic spheres clear of each
 * other and of the substrate, gamma_n < 2 sqrt(k_n m) and a collision time
 * t_c >= 10 (Sec. V H), at most LBM_MAX_PARTICLES per instance.  Only before
 * the first lbm_step (-> LBM_ERR_STATE). */
lbm_status lbm_add_particles(lbm_ctx *ctx, int inst, int n, const lbm_particle *parts);

/* Advance every instance by nsteps coupled time steps (Sec. IV-V, in the order
 * of the paper's flow chart of the coupled algorithm, Fig. 4): streaming with
 * bounce-back, momentum exchange, order parameter, gradient with wetting,
 * curvature and CSF force, MRT collision with Guo forcing, recolouring,
 * capillary force, DEM, geometry update and refill.  Asynchronous on the
 * context's stream; replays a captured CUDA graph (of two steps, or of one
 * step for a single-step call). */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* Set the velocity v and angular velocity w of particle p of an instance
 * (lattice units per step).  For a kinematic particle this is its prescribed
 * motion from the next step on; for a free one its current velocity.  Between
 * steps only, enqueued on the context stream (no synchronisation); the
 * captured step graph stays valid.  |v| or |w| R_p above 0.1 (the geometry
 * update assumes sub-lattice motion per step), a bad index or a null pointer ->
 * LBM_ERR_ARG. */
lbm_status lbm_set_particle_motion(lbm_ctx *ctx, int inst, int p, const double *v, const double *w);

/* Per-particle record (LBM_PARTICLE_RECORD doubles each) of an instance after
 * the last step; out holds n_particles records.  Synchronises. */
lbm_status lbm_particle_forces(lbm_ctx *ctx, int inst, double *out);

/* As lbm_particle_forces, enqueued on the context's stream without
 * synchronising.  If the device can address out (page-locked host memory,
 * which unified addressing maps, managed memory, or this device's memory),
 * one packing kernel writes the records there directly; otherwise (pageable host memory)
 * they are packed on the device and copied to out.  The values are valid once
 * the stream has passed that point, e.g. after the next synchronising call.
 * Lets a caller read every step's forces without stalling the device.  Bad
 * instance or null out -> LBM_ERR_ARG. */
lbm_status lbm_particle_forces_async(lbm_ctx *ctx, int inst, double *out);

/* Record ring: from the next step on, every step writes the records of all
 * particles of the context (instances in order, LBM_PARTICLE_RECORD doubles
 * each, the layout of lbm_particle_forces) into slot k mod slots of ring, k
 * counting the steps since this call (from 0).  The records are packed on the
 * device inside the step, right after the DEM (Sec. III) has updated the
 * particles, on the stream that runs the particle kernels: no launch and no
 * copy of the caller's.  ring must be page-locked host, managed or this
 * device's memory (the device writes it) of slots x n_particles_total x
 * LBM_PARTICLE_RECORD doubles, kept alive while set; a slot is valid once the
 * context's stream has passed its step (e.g. after the next synchronising
 * call).  ring NULL stops the recording; adding particles stops it too.
 * slots < 1, no particles, or memory the device cannot address ->
 * LBM_ERR_ARG.  Synchronises; invalidates the step graph. */
lbm_status lbm_set_record_ring(lbm_ctx *ctx, double *ring, int slots);

/* Measured FP32 multiply-add throughput of the current device in TFLOP/s
 * (2 FLOP per FMA): the non-tensor arithmetic ceiling of the 16-bit storage
 * modes, whose collision is held by instruction issue rather than by DRAM.
 * Eight CTAs of 256 threads per SM, eight independent chains per thread, the
 * best of five timed launches after a warm-up (about 2 ms each).  The paper
 * has no counterpart.  Null tflops -> LBM_ERR_ARG (no device call); a CUDA
 * failure -> LBM_ERR_CUDA.  Synchronises. */
lbm_status lbm_fp32_fma_peak(double *tflops);

/* Checkpoint of an instance's particles, for an exact resume with contacts
 * (the DEM of Sec. III carries state from step to step).  Per particle
 * LBM_PARTICLE_STATE doubles: x[3] v[3] w[3] q[4] (w, x, y, z), then the total
 * force and torque of the last DEM step F_prev[3] T_prev[3] (the next
 * velocity-Verlet step reads them); then the friction-spring histories of
 * Sec. III B-C: n_particles (n_particles + 1) slots of 6 doubles (sliding
 * xi[3], rolling xi_r[3]) in the library's order, to be handed back as read.
 * lbm_particle_state_size gives the total count (-1 for a bad instance). */
#define LBM_PARTICLE_STATE 19
long long lbm_particle_state_size(const lbm_ctx *ctx, int inst);

/* Read the checkpoint; n must equal lbm_particle_state_size (-> LBM_ERR_ARG).
 * Synchronises. */
lbm_status lbm_get_particle_state(lbm_ctx *ctx, int inst, double *out, size_t n);

/* Restore a checkpoint into a new context before its first step
 * (-> LBM_ERR_STATE after): the instance must hold the same particles, added
 * at exactly the checkpoint's positions (the solid map is built from them;
 * another position -> LBM_ERR_ARG), with the fields restored by
 * lbm_init_fields from the read populations.  Non-finite values or a speed
 * above 0.1 -> LBM_ERR_ARG.  Synchronises; invalidates the step graph. */
lbm_status lbm_set_particle_state(lbm_ctx *ctx, int inst, const double *in, size_t n);

/* Read the fields selected by mask (LBM_FIELD_*) of an instance into host
 * memory, FP64.  Solid nodes read 0 for the density, phi and population
 * fields.  LBM_FIELD_U requires store_velocity (-> LBM_ERR_STATE).
 * Synchronises. */
lbm_status lbm_read_fields(lbm_ctx *ctx, int inst, unsigned mask, double *out);

/* As lbm_read_fields into a device buffer; enqueued on the stream, no sync. */
lbm_status lbm_read_fields_device(lbm_ctx *ctx, int inst, unsigned mask, double *out);

/* Number of particles of an instance, or -1 for a bad instance index. */
int lbm_num_particles(const lbm_ctx *ctx, int inst);

/* Nodes (nx*ny*nz) of an instance, or -1. */
long long lbm_num_nodes(const lbm_ctx *ctx, int inst);

/* FP64 diagnostics of an instance, from the last time they were taken
 * (every diag_interval steps, or now when diag_interval is 0):
 * out[0] = sum rho^a, out[1] = sum rho^b over fluid nodes, out[2] = steps
 * taken so far, out[3] = sticky device status bits.  Synchronises. */
lbm_status lbm_diagnostics(lbm_ctx *ctx, int inst, double *out);

/* Launch shape of the fluid update.  form must be 2 (plain: order
 * parameter, solid phi, gradient + wetting + normal + curvature, collision,
 * with the nodes next to a solid in boundary passes beside the bulk kernels).
 * tile 0 (default): with 16-bit storage and an even nx in every instance the
 * bulk collision takes two nodes of a row per thread (pair loads and stores),
 * one node per thread otherwise; tile 1: one node per thread always.
 * zchunk: z-planes per work item of the gradient pass (0: 16).  Every shape
 * computes the same update; the node-pair collision agrees with the one-node
 * collision to the rounding of the storage type (the code generator may fuse
 * a different set of multiply-adds), the z-chunk gives the same bits.  Invalid
 * form, tile or zchunk -> LBM_ERR_ARG.  Invalidates the step graph. */
lbm_status lbm_set_fluid_kernel(lbm_ctx *ctx, int form, int tile, int zchunk);

/* Autotuner of the launch shape, on the context's own instances.  Instances
 * fall into size classes by nz (<= 64, <= 96, <= 128, larger); for each class
 * present, the z-planes per work item of the gradient pass are chosen from 8,
 * 16 and 32 (the other classes held at their current choice), then the
 * bulk-kernel variant (tile 0, 1).  Each candidate is re-planned, its step
 * graph captured and warmed up for 2 steps, then timed over `steps` (>= 2)
 * steps with CUDA events on the context stream; the fastest is kept.  The
 * simulation advances by all the trial steps (every shape computes the same
 * update).  *tile receives the variant; zchunks (may be NULL) one z-chunk per
 * instance; ms_best (may be NULL) the ms per step of the chosen shape.
 * lbm_set_fluid_kernel afterwards replaces the per-class choice by one
 * z-chunk for all.  Synchronises. */
lbm_status lbm_autotune(lbm_ctx *ctx, int steps, int *tile, int *zchunks, double *ms_best);

/* The fluid-update form the next step runs (2); -1 for a null context. */
int lbm_fluid_form_in_use(const lbm_ctx *ctx);

/* Count of kernel launches the last lbm_step call enqueued (graph nodes
 * included); for accounting in benchmarks. */
long long lbm_last_launch_count(const lbm_ctx *ctx);

/* Per-kernel timing.  With enable = 1, later lbm_step calls launch eagerly
 * (no graph replay) and bracket every kernel with CUDA events on the
 * context's stream; enabling again clears the record.  Synchronises. */
lbm_status lbm_profile(lbm_ctx *ctx, int enable);

/* Read the per-kernel record since lbm_profile(ctx, 1): for stage k
 * (order parameter, solid phi, gradient+wetting, collision [four-kernel
 * form], momentum exchange, capillary force, DEM, geometry owner, geometry
 * boundary, refill, fused fluid kernel, particle-region phi/gradient)
 * out[2k] = launches, out[2k+1] = total device milliseconds; at most
 * max_stages stages are written.  Synchronises. */
lbm_status lbm_profile_read(lbm_ctx *ctx, double *out, int max_stages);

/* Allocation-free FP64 component masses, for callers that cannot call
 * cudaMalloc (code running while a CUDA graph is captured, frameworks that own
 * all device memory through their own pool, loops where an allocation would
 * synchronise the device).  The paper has no counterpart; it is a variant of
 * the reduction behind lbm_diagnostics that needs no context.
 * pops: device pointer to FP64 populations, f^a then f^b, [38][n_nodes]
 * (the LBM_FIELD_POPS layout of lbm_read_fields_device; solid nodes 0);
 * masses: device pointer to 2 doubles, receives sum f^a, sum f^b.
 * stream: cudaStream_t the two kernels are enqueued on (NULL: legacy stream).
 * Allocates nothing: its scratch is a static device array of 4096 x 2 doubles
 * (64 KiB) that every GPU which loads the library keeps until the process
 * exits.  n_nodes must be in [1, 2^28] (-> LBM_ERR_ARG otherwise).  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  Every call shares
 * the one array, so calls that overlap on the GPU race.  Asynchronous; returns
 * LBM_ERR_CUDA if the lookup or a launch fails. */
lbm_status lbm_component_masses_noalloc(const double *pops, long long n_nodes, double *masses, void *stream);

/* Host-side fault injection, for testing the failure path of the bounded
 * device waits without a device fault.  fault = LBM_FAULT_GEMM_NO_COMMIT: every
 * tensor-core GEMM of the surrogate network on this context (predict,
 * gradient, train, the surrogate force model in a step) issues no MMA and
 * never signals its commit barrier, so its bounded wait on that barrier
 * (shortened to about a millisecond) finds nothing arriving, gives up, frees
 * its tensor memory and sets the sticky device status; the next synchronising
 * call returns LBM_ERR_TIMEOUT (outputs of the failed call are undefined).
 * LBM_FAULT_NONE switches it off.  The sticky status stays: create a new
 * context to continue.  Unknown fault -> LBM_ERR_ARG.  Synchronises. */
enum { LBM_FAULT_NONE = 0, LBM_FAULT_GEMM_NO_COMMIT = 1 };
lbm_status lbm_inject_fault(lbm_ctx *ctx, int fault);

/* Run state of a context, for an exact resume beside the populations
 * (lbm_read_fields / lbm_init_fields) and the particle checkpoint:
 * out[0] = steps taken (the drop-speed control and the diagnostics are
 * scheduled on it), then per instance 9 doubles: the body force on phase a
 * now [3], the drop-speed control's error integral [3] and the phase-a
 * velocity at its last update [3] (the PI law of lbm_params).
 * lbm_run_state_size gives 1 + 9 n_instances (-1 for a null context).
 * Get synchronises; set is valid before the first step only (-> LBM_ERR_STATE),
 * checks n and finiteness (-> LBM_ERR_ARG) and invalidates the step graph. */
long long lbm_run_state_size(const lbm_ctx *ctx);
lbm_status lbm_get_run_state(lbm_ctx *ctx, double *out, size_t n);
lbm_status lbm_set_run_state(lbm_ctx *ctx, const double *in, size_t n);

/* Drop-speed control state of an instance: out[0..2] the body force on phase
 * a now, out[3..5] U_a at the last update (zeros before the first).
 * Synchronises. */
lbm_status lbm_drop_speed_state(lbm_ctx *ctx, int inst, double *out);

/* ---------------------------------------------------------------------------
 * Learned force surrogate (an extension of the method; the paper has none).
 * On a coarse grid the momentum-exchange and capillary forces (Sec. V B, V F)
 * can be replaced by a network evaluated on samples of the flow around each
 * sphere:
 *   inputs (LBM_MLP_INPUTS = 387): at the 96 points of a Fibonacci sphere of
 *     radius R_p + surrogate_shell_gap around the centre (z_k = 1 - (2k+1)/96,
 *     azimuth k times the golden angle pi (3 - sqrt 5)), the order parameter
 *     and the velocity relative to the particle's rigid motion divided by
 *     surrogate_u_ref (phi, ux, uy, uz per point; trilinear over the fluid
 *     corners of the cell, zeros when none is fluid), then cos theta_p,
 *     sin theta_p, R_p / surrogate_r_ref;
 *   network: 400 (inputs zero-padded) -> 128 -> 128 -> 6, tanh hidden layers;
 *   outputs: F / (sigma R_p) (3) and T / (sigma R_p^2) (3), which replace
 *     F_eta + F_sigma and T_eta + T_sigma in the DEM.
 * Weights (LBM_MLP_PARAMS floats): W1 (128 x 400 row-major), b1 (128), W2
 * (128 x 128), b2 (128), W3 (6 x 128), b3 (6).  Products run on the tensor
 * cores with BF16 operands and FP32 accumulation; the master weights and Adam
 * state are FP32.  Training loss: mean over samples and the 6 outputs of the
 * squared error; Adam with beta1 = 0.9, beta2 = 0.999, eps = 1e-8; each epoch
 * visits the samples in the order of a Fisher-Yates shuffle driven by
 * SplitMix64 seeded once per call.
 * ------------------------------------------------------------------------- */
#define LBM_MLP_INPUTS 387
#define LBM_MLP_OUTPUTS 6
#define LBM_MLP_PARAMS 68614
#define LBM_MLP_MAX_BATCH 4096

typedef enum { LBM_FORCE_RESOLVED = 0, LBM_FORCE_SURROGATE = 1 } lbm_force_model;

/* Select how the fluid forces on the particles are computed from the next
 * step on.  LBM_FORCE_SURROGATE needs loaded weights and store_velocity in
 * every instance (-> LBM_ERR_STATE); it replaces the surface sums that the
 * buoyancy reads, so an instance with a nonzero buoyancy_a refuses it
 * (-> LBM_ERR_UNSUPPORTED).  Invalidates the step graph. */
lbm_status lbm_set_force_model(lbm_ctx *ctx, int model);

/* Copy n = LBM_MLP_PARAMS host floats in as the master weights (the BF16
 * copies follow) and reset the Adam state.  Wrong n -> LBM_ERR_ARG. */
lbm_status lbm_surrogate_load(lbm_ctx *ctx, const float *weights, size_t n);

/* Copy the FP32 master weights out (n = LBM_MLP_PARAMS).  Synchronises. */
lbm_status lbm_surrogate_save(lbm_ctx *ctx, float *weights, size_t n);

/* Network outputs Y [n][6] for host inputs X [n][387].  Synchronises. */
lbm_status lbm_surrogate_predict(lbm_ctx *ctx, const float *X, size_t n, float *Y);

/* Loss of one batch (X [n][387], targets Y [n][6], 1 <= n <=
 * LBM_MLP_MAX_BATCH) and its gradient with respect to the weights (grad
 * [LBM_MLP_PARAMS], same layout); no update.  Synchronises. */
lbm_status lbm_surrogate_gradient(lbm_ctx *ctx, const float *X, const float *Y, size_t n, float *grad,
                                  double *loss);

/* Mini-batch Adam over n samples for `epochs` epochs (batch in
 * [1, LBM_MLP_MAX_BATCH], lr > 0); *loss_out = mean batch loss of the last
 * epoch.  The Adam state carries over between calls until the next load.
 * Synchronises. */
lbm_status lbm_surrogate_train(lbm_ctx *ctx, const float *X, const float *Y, size_t n, int epochs, int batch,
                               double lr, uint64_t seed, double *loss_out);

/* Surrogate inputs of every particle of an instance for the current state,
 * out [n_particles][387].  Needs store_velocity (-> LBM_ERR_STATE).
 * Synchronises. */
lbm_status lbm_surrogate_features(lbm_ctx *ctx, int inst, float *out);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
