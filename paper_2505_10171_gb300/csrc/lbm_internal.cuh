// Internal device-side definitions of the sm_103a LBM-DEM library.
//
// Lattice: D3Q19 (Sec. IV of arXiv 2505.10171).  The device order is
// i = 0 rest, i = 1..9 the positive half-set h_k below, i = 10..18 their
// opposites, so that the opposite of i is i +- 9; the C ABI order (LBM_C in
// include/lbm.h) is mapped on the way in and out.
//
// Populations are stored as offsets (two-component encoding):
//   F_i = f_i/(w_i rho0) - 1,   G_i = (f^a_i - f^b_i)/(w_i rho0)
// structure of arrays: pop[q*N + n], q = 0..18 for F, 19..37 for G.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmg {

constexpr int Q = 19;
constexpr int NPOP = 38;

// positive half-set of D3Q19: +x, +y, +z, then the face diagonals
__host__ __device__ constexpr int hx(int k) { return (k == 0 || k == 3 || k == 4 || k == 5 || k == 6) ? 1 : 0; }
__host__ __device__ constexpr int hy(int k) { return (k == 1 || k == 3 || k == 7 || k == 8) ? 1 : (k == 4 ? -1 : 0); }
__host__ __device__ constexpr int hz(int k) { return (k == 2 || k == 5 || k == 7) ? 1 : ((k == 6 || k == 8) ? -1 : 0); }
__host__ __device__ constexpr int cx(int i) { return i == 0 ? 0 : (i <= 9 ? hx(i - 1) : -hx(i - 10)); }
__host__ __device__ constexpr int cy(int i) { return i == 0 ? 0 : (i <= 9 ? hy(i - 1) : -hy(i - 10)); }
__host__ __device__ constexpr int cz(int i) { return i == 0 ? 0 : (i <= 9 ? hz(i - 1) : -hz(i - 10)); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
template <class T>
__host__ __device__ constexpr T wgt(int i)
{
    return csq(i) == 0 ? T(1) / T(3) : (csq(i) == 1 ? T(1) / T(18) : T(1) / T(36));
}

// node flags: owner in the low 6 bits (0 fluid, 1 static solid, 2+p particle p
// of the instance), bit 6 = refilled this step, bit 7 = next to the other kind
constexpr uint8_t OWNER_MASK = 0x3f;
constexpr uint8_t FRESH_BIT = 0x40;
constexpr uint8_t BOUND_BIT = 0x80;
constexpr uint8_t OWN_FLUID = 0;
constexpr uint8_t OWN_WALL = 1;

// sticky status bits
constexpr unsigned ST_UNSTABLE = 1u;
constexpr unsigned ST_DISPLACEMENT = 2u;

constexpr int CAP_POINTS = 90 * 180;  // Sec. V E: 2 deg x 2 deg Lagrangian points
constexpr int CAP_THREADS = 256;
constexpr int CAP_BLOCKS = (CAP_POINTS + CAP_THREADS - 1) / CAP_THREADS;
constexpr int PART_THREADS = 256;
constexpr int GEOM_MARGIN = 3;  // lattice units a particle may move per step, < this

struct InstDev {
    int nx, ny, nz, np;
    long long N;         // nodes of the instance
    long long node_off;  // first node in the per-node arrays
    long long blk_start; // first fluid block of the instance
    int part_off;        // first particle of the instance
    int hist_off;        // first pair-history record of the instance
    int wall_z0, store_u;
    double rho0, sigma, beta, cap_norm, eta_a, eta_b;
    double body_a[3], body_b[3], wall_u[3];
    double cos_tw, sin_tw;
    double grad_eps, wet_max;
    double kn, kt, kr, gn, gt, gr, mu_s, mu_r, dR;
    double g_part[3];
};

struct PartDev {
    double x[3], v[3], w[3], q[4];
    double x_old[3];
    double R, Rc, m, I, cos_t, sin_t;
    double Fp[3], Tp[3];
    double Feta[3], Teta[3], Fsig[3], Tsig[3], Fc[3], Tc[3];
    int kin, inst, local, mem_side;
};

struct Lattice {
    const InstDev *inst;
    int n_inst;
    long long n_blocks;
    int bt;              // fluid block threads
    uint8_t *flags;
    void *pop[2];
    void *phi;           // [Ntot] real
    void *grad;          // [3][Ntot] real
    void *u;             // [3][Ntot] real (store_velocity)
    long long Ntot;
    PartDev *parts;
    int n_parts;
    int mem_blocks;      // blocks per particle of the momentum-exchange kernel
    int geom_blocks;     // blocks per particle of the geometry kernels
    int geom_side;       // side of the cube the geometry kernels cover
    double *mem_part;    // [n_parts][mem_blocks][6]
    double *cap_part;    // [n_parts][CAP_BLOCKS][6]
    double *hist;        // contact springs: per instance np*(np+1) records of 6
    unsigned *status;
};

template <class S>
struct Store;
template <>
struct Store<double> {
    using real = double;
    static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <>
struct Store<float> {
    using real = float;
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Store<__half> {
    using real = float;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
    using real = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ int find_inst(const InstDev *I, int n, long long blk)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (I[mid].blk_start <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ __forceinline__ double min_image(double d, int n)
{
    return d - n * floor(d / n + 0.5);
}

// periodic neighbourhood of one node
struct Nbr {
    int X[3], Y[3], Z[3];
    int nx;
    long long nxy;
    __device__ __forceinline__ void init(int x, int y, int z, int nx_, int ny_, int nz_)
    {
        nx = nx_;
        nxy = (long long)nx_ * ny_;
        X[0] = x == 0 ? nx_ - 1 : x - 1; X[1] = x; X[2] = x == nx_ - 1 ? 0 : x + 1;
        Y[0] = y == 0 ? ny_ - 1 : y - 1; Y[1] = y; Y[2] = y == ny_ - 1 ? 0 : y + 1;
        Z[0] = z == 0 ? nz_ - 1 : z - 1; Z[1] = z; Z[2] = z == nz_ - 1 ? 0 : z + 1;
    }
    __device__ __forceinline__ long long at(int dx, int dy, int dz) const
    {
        return (long long)Z[dz + 1] * nxy + (long long)Y[dy + 1] * nx + X[dx + 1];
    }
};

// velocity of the solid owning a node at the point xw (Sec. V A)
__device__ __forceinline__ void surface_velocity(const InstDev &I, const PartDev *parts, int owner,
                                                 double xw, double yw, double zw, double *u, double *lev)
{
    if (owner == OWN_WALL) {
        u[0] = I.wall_u[0]; u[1] = I.wall_u[1]; u[2] = I.wall_u[2];
        lev[0] = lev[1] = lev[2] = 0.0;
        return;
    }
    const PartDev &P = parts[I.part_off + owner - 2];
    double d0 = min_image(xw - P.x[0], I.nx);
    double d1 = min_image(yw - P.x[1], I.ny);
    double d2 = min_image(zw - P.x[2], I.nz);
    u[0] = P.v[0] + (P.w[1] * d2 - P.w[2] * d1);
    u[1] = P.v[1] + (P.w[2] * d0 - P.w[0] * d2);
    u[2] = P.v[2] + (P.w[0] * d1 - P.w[1] * d0);
    lev[0] = d0; lev[1] = d1; lev[2] = d2;
}

// Pull streaming of both components into node n (Sec. IV streaming), with the
// Sec. V A halfway bounce-back where the source node is solid:
//   f_i(x) = f*_ibar(x) + 6 w_i rho^{a,b}(x) c_i.u_w,  rho^{a,b}(x) taken from
// the node's own pre-streaming populations, u_w at the link midpoint.
template <class S>
__device__ __forceinline__ void gather(const InstDev &I, const PartDev *parts, const uint8_t *flags,
                                       const S *__restrict__ in, long long N, long long n, const Nbr &nb,
                                       uint8_t fl, typename Store<S>::real *F, typename Store<S>::real *G,
                                       int x, int y, int z)
{
    using R = typename Store<S>::real;
    const uint8_t *fli = flags + I.node_off;
    if (!(fl & BOUND_BIT)) {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            long long s = nb.at(-cx(i), -cy(i), -cz(i));
            F[i] = Store<S>::ld(in + (long long)i * N + s);
            G[i] = Store<S>::ld(in + (long long)(Q + i) * N + s);
        }
        return;
    }
    bool have_rho = false;
    double rr = 0.0, rd = 0.0;  // rho/rho0 and (rho^a - rho^b)/rho0 of this node
#pragma unroll
    for (int i = 0; i < Q; i++) {
        long long s = nb.at(-cx(i), -cy(i), -cz(i));
        int own = fli[s] & OWNER_MASK;
        if (own == OWN_FLUID) {
            F[i] = Store<S>::ld(in + (long long)i * N + s);
            G[i] = Store<S>::ld(in + (long long)(Q + i) * N + s);
            continue;
        }
        if (!have_rho) {
            double sF = 0.0, sG = 0.0;
#pragma unroll
            for (int j = 0; j < Q; j++) {
                sF += wgt<double>(j) * (double)Store<S>::ld(in + (long long)j * N + n);
                sG += wgt<double>(j) * (double)Store<S>::ld(in + (long long)(Q + j) * N + n);
            }
            rr = 1.0 + sF;
            rd = sG;
            have_rho = true;
        }
        double uw[3], lev[3];
        surface_velocity(I, parts, own, x - 0.5 * cx(i), y - 0.5 * cy(i), z - 0.5 * cz(i), uw, lev);
        double cu = cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2];
        const int ib = opp(i);
        F[i] = (R)((double)Store<S>::ld(in + (long long)ib * N + n) + 6.0 * rr * cu);
        G[i] = (R)((double)Store<S>::ld(in + (long long)(Q + ib) * N + n) + 6.0 * rd * cu);
    }
}

template <class R>
__device__ __forceinline__ R dsqrt(R v) { return sqrt(v); }

// Sec. V D geometric wetting: rotate g so that -g/|g| makes the angle theta
// with the outward solid normal ns, keeping |g|; of the two candidates the one
// closer to the original direction is kept.
template <class R>
__device__ __forceinline__ void wetting_rotate(R *g, const R *ns, R cth, R sth)
{
    R gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gm == R(0)) return;
    R st[3] = {-g[0] / gm, -g[1] / gm, -g[2] / gm};
    R ca = ns[0] * st[0] + ns[1] * st[1] + ns[2] * st[2];
    ca = ca > R(1) ? R(1) : (ca < R(-1) ? R(-1) : ca);
    R al = acos(ca);
    R sa = sin(al), cal = cos(al);
    if (sa < R(1e-4)) return;  // contact-line direction undefined (n* parallel to n_s)
    R ap1 = cth - sth * cal / sa, ap2 = sth / sa;
    R am1 = cth + sth * cal / sa, am2 = -sth / sa;
    R np_[3], nm_[3];
    for (int a = 0; a < 3; a++) {
        np_[a] = ap1 * ns[a] + ap2 * st[a];
        nm_[a] = am1 * ns[a] + am2 * st[a];
    }
    R dp = np_[0] * st[0] + np_[1] * st[1] + np_[2] * st[2];
    R dm = nm_[0] * st[0] + nm_[1] * st[1] + nm_[2] * st[2];
    const R *nc = dp >= dm ? np_ : nm_;
    for (int a = 0; a < 3; a++) g[a] = -gm * nc[a];
}

// kernel stages, in launch order within a step (for per-kernel timing)
enum Stage {
    STAGE_PHI = 0, STAGE_SOLIDPHI, STAGE_GRAD, STAGE_COLLIDE, STAGE_MEM, STAGE_CAPILLARY, STAGE_DEM,
    STAGE_GEOM_OWNER, STAGE_GEOM_BOUND, STAGE_REFILL, N_STAGES
};

// optional per-kernel marker: called right before and right after each launch
struct Marker {
    void (*fn)(void *self, int stage, int after) = nullptr;
    void *self = nullptr;
    void operator()(int stage, int after) const
    {
        if (fn) fn(self, stage, after);
    }
};

// host-side kernel launchers (defined in the .cu files)
template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_particle_forces(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_geometry(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk);
void launch_dem(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_init_fields(const Lattice &L, int cur, int inst, long long N, const double *phi, const double *rho,
                        const double *u, const double *pops, cudaStream_t st);
template <class S>
void launch_read_fields(const Lattice &L, int cur, int inst, long long N, unsigned mask, double *out,
                        cudaStream_t st);
template <class S>
void launch_mass_sums(const Lattice &L, int cur, int inst, long long N, double *partial, int nblk, double *out,
                      cudaStream_t st);
void launch_boundary_full(const Lattice &L, int inst, long long N, cudaStream_t st);
void launch_mark_particles(const Lattice &L, cudaStream_t st);

}  // namespace lbmg
