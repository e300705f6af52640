// Internal device-side definitions of the sm_103a LBM-DEM library.
//
// Lattice: D3Q19 (Sec. IV of arXiv 2505.10171).  The device order is
// i = 0 rest, i = 1..9 the positive half-set h_k below, i = 10..18 their
// opposites, so that the opposite of i is i +- 9; the C ABI order (LBM_C in
// include/lbm.h) is mapped on the way in and out.
//
// Populations are stored as total offsets F_i = f_i/(w_i rho0) - 1, structure
// of arrays pop[i*N + n].  The colour offsets G_i = (f^a_i - f^b_i)/(w_i rho0)
// are not stored: the recolouring step (Sec. IV) leaves every node with
//   G*_i = phi (1 + F*_i) + b (c_i . n)/|c_i|,   b = beta/2 (rho/rho0)(1 - phi^2),
// phi and n the order parameter and interface normal its collision used, so a
// state is F* plus one record (phi, a = b n) per node, and G is rebuilt where
// it is needed: G*_i = phi (1 + F*_i) + (c_i . a)/|c_i|.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
// outside of an inlet / outlet face of the Sec. V D pressure boundary (the
// node planes z = 0 and z = nz - 1); particles own 2 .. 62
constexpr uint8_t OWN_PRESS = 63;
__host__ __device__ __forceinline__ bool own_static(int o) { return o == OWN_WALL || o == OWN_PRESS; }

// sticky status bits
constexpr unsigned ST_UNSTABLE = 1u;
constexpr unsigned ST_DISPLACEMENT = 2u;
constexpr unsigned ST_TIMEOUT = 4u;  // a bounded wait for an asynchronous copy gave up

constexpr int CAP_POINTS = 90 * 180;  // Sec. V F: 2 deg x 2 deg Lagrangian points
constexpr int CAP_THREADS = 256;
constexpr int CAP_BLOCKS = (CAP_POINTS + CAP_THREADS - 1) / CAP_THREADS;
constexpr int CAP_PART = 8;  // per block: F_sig, T_sig, sum s dA, sum dA
constexpr int PART_THREADS = 256;
// doubles per block partial of the momentum exchange: force and torque of the
// small part, then the integer sums K and 2M of the rest part
constexpr int MEM_PART = 12;
constexpr int GEOM_MARGIN = 3;  // lattice units a particle may move per step, < this

// division by an integer fixed when the work items are planned (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// q = (mulhi(n, m) + n) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d)/d) + 1,
// exact for 0 <= n < 2^31 and 1 <= d < 2^31 (n + mulhi stays below 2^32); a
// handful of instructions instead of the runtime divide sequence
struct FastDiv {
    unsigned d, m;
    int l;
    void set(unsigned d_)
    {
        d = d_ ? d_ : 1;
        l = 0;
        while ((1ull << l) < d) l++;
        m = (unsigned)((((unsigned long long)1 << 32) * ((1ull << l) - d)) / d + 1);
    }
    __device__ __forceinline__ int div(int n) const { return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> l); }
};

struct InstDev {
    int nx, ny, nz, np;
    long long N;         // nodes of the instance
    long long node_off;  // first node in the per-node arrays
    long long pop_off;   // byte offset of the instance's population block
    int pstride;         // population stride (N)
    int part_off;        // first particle of the instance
    int hist_off;        // first pair-history record of the instance
    int crec_off;        // first DEM contact record of the instance
    int wall_z0, store_u;
    int press;                 // pressure faces at z = 0.5 and z = nz - 1.5 (Sec. V D)
    double rin, rout;          // their densities over rho0
    float f_rin, f_rout;
    double rho0, sigma, beta, cap_norm, eta_a, eta_b;
    double body_a[3], body_b[3], wall_u[3];
    double cos_tw, sin_tw;
    double grad_eps, wet_max;
    double kn, kt, kr, gn, gt, gr, mu_s, mu_r, dR;
    double g_part[3];
    double buoy[3];      // force per unit particle volume immersed in phase a (reading c28)
    // single-precision copies of the fluid parameters (no FP64 conversions in
    // the FP32 and 16-bit kernels)
    float f_rho0, f_sigma, f_beta, f_eta_a, f_eta_b, f_eps2, f_wet_max;
    float f_body_a[3], f_body_b[3];
    float f_ir0, f_h_ia, f_h_ib;
    // row-strip work items of the bulk kernels: st_rows whole x-rows of one z-plane per item
    // (st_nseg = 1, st_seg = nx), or one row cut into st_nseg segments of at
    // most st_seg nodes; st_ygroups items cover the y rows of a plane
    long long st_item_start;
    int st_rows, st_seg, st_nseg, st_ygroups;
    FastDiv fd_plane, fd_nseg, fd_nx;  // st_ygroups st_nseg, st_nseg, nx
    // surrogate inputs: shell gap, velocity and radius scales
    double sh_gap, sh_uref, sh_rref, sh_box;
    // gradient + curvature work items: gc_tiles_x * gc_tiles_y column tiles x
    // gc_nchunks z-chunks of gc_zc planes
    long long gc_item_start;
    int gc_tiles_x, gc_tiles_y, gc_nchunks, gc_zc;
    FastDiv fd_nchunks, fd_tiles_x;  // gc_nchunks, gc_tiles_x
    // drop-speed control (body force on phase a): component mask, interval,
    // target velocity, PI gains, base force
    int sp_mask, sp_interval;
    double sp_target[3], sp_kp, sp_ki, sp_f0[3];
};

// fluid parameters in the arithmetic precision R
template <class R>
struct FluidPar {
    R rho0, sigma, beta, eta_a, eta_b, eps2, wet_max, ba[3], bb[3];
    R ir0, h_ia, h_ib;  // 1/rho0, 1/(2 eta_a), 1/(2 eta_b)
};
__device__ __forceinline__ void load_par(const InstDev &I, FluidPar<double> &p)
{
    p.rho0 = I.rho0; p.sigma = I.sigma; p.beta = I.beta; p.eta_a = I.eta_a; p.eta_b = I.eta_b;
    p.eps2 = I.grad_eps * I.grad_eps; p.wet_max = I.wet_max;
    for (int a = 0; a < 3; a++) { p.ba[a] = I.body_a[a]; p.bb[a] = I.body_b[a]; }
    p.ir0 = 1.0 / I.rho0; p.h_ia = 0.5 / I.eta_a; p.h_ib = 0.5 / I.eta_b;
}
__device__ __forceinline__ void load_par(const InstDev &I, FluidPar<float> &p)
{
    p.rho0 = I.f_rho0; p.sigma = I.f_sigma; p.beta = I.f_beta; p.eta_a = I.f_eta_a; p.eta_b = I.f_eta_b;
    p.eps2 = I.f_eps2; p.wet_max = I.f_wet_max;
    for (int a = 0; a < 3; a++) { p.ba[a] = I.f_body_a[a]; p.bb[a] = I.f_body_b[a]; }
    p.ir0 = I.f_ir0; p.h_ia = I.f_h_ia; p.h_ib = I.f_h_ib;
}

struct PartDev {
    double x[3], v[3], w[3], q[4];
    double x_old[3];
    double R, Rc, m, I, cos_t, sin_t;
    double inv_m, inv_I;  // 1/m, 1/I
    double Fp[3], Tp[3];
    double Feta[3], Teta[3], Fsig[3], Tsig[3], Fc[3], Tc[3];
    double sub, Fb[3];    // immersed volume fraction in phase a, buoyancy
    float xf[3], xfo[3];  // single-precision copies of x and x_old
    float R2lo, R2hi;     // |x - x_p|^2 below / above these is inside / outside for sure
    int kin, inst, local, mem_side;
};

struct Lattice {
    const InstDev *inst;
    int n_inst;
    long long n_items;   // row-strip work items of all instances
    int buoyancy;        // some instance has a nonzero buoyancy_a: the immersed fractions are summed
    const long long *static_list;  // static solid nodes next to non-static ones (global node index)
    long long n_static;
    const long long *static_bfl;   // non-static nodes next to static solid ones
    long long n_static_bfl;
    uint8_t *flags;
    void *pop[2];
    void *phi;           // [Ntot] real: the order parameter of the step (outside a step: of the last one)
    void *col;           // [Ntot] ColRec<real>: colour record (phi, b n) of the stored state
    void *grad;          // [3][Ntot] real: regularised interface normal n
    void *gmag;          // [Ntot] real: sqrt(|grad phi|^2 + eps^2), so grad phi = n gmag
    void *kap;           // [Ntot] real: curvature div(n) of fluid nodes
    void *u;             // [3][Ntot] real (store_velocity)
    long long Ntot;
    PartDev *parts;
    int n_parts;
    int mem_blocks;      // blocks per particle of the momentum-exchange kernel
    int geom_blocks;     // blocks per particle of the geometry kernels
    int geom_side;       // side of the cube the geometry kernels cover
    int cap_side;        // side of the cube of phi around a particle for the capillary force
    long long *pbl;              // fluid nodes next to a solid inside the particle cubes (global index), this step
    unsigned long long *pbl_n;   // their number
    long long *psl;              // solid nodes next to fluid inside the particle cubes, this step
    unsigned long long *psl_n;   // their number
    int bound_ctas;              // CTAs of the grid-stride boundary passes
    int cap_blocks;      // blocks per particle covering that cube
    double *mem_part;    // [n_parts][mem_blocks][MEM_PART]
    double *cap_part;    // [n_parts][CAP_BLOCKS][CAP_PART]
    const double *cap_pts;  // [CAP_POINTS][4]: unit normal (3) and sin(alpha) of each surface point
    double *hist;        // contact springs: per instance np*(np+1) records of 6
    double *crec;        // DEM contact forces: per instance np + np(np-1)/2 records of 12
    unsigned *status;
};

// materialise a value here: the loads it depends on must be issued before
// any branch that follows, so the compiler cannot sink them into the one path
// that uses them (which would put the node's flag load and the population
// loads in series: two dependent DRAM round trips instead of one)
__device__ __forceinline__ void keep(float &v) { asm volatile("" : "+f"(v)); }
__device__ __forceinline__ void keep(double &v) { asm volatile("" : "+d"(v)); }

// programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream drains; it must
// wait here before touching anything the predecessor writes or reads.  A
// predecessor signals early that its dependent may be scheduled (all of its
// CTAs have started by then, so the dependent cannot take their places).
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// streamed populations are read through the read-only path (measured on this
// GPU: as fast as plain loads, faster than evict-first streaming loads)
template <class T>
__device__ __forceinline__ T pop_load(const T *p)
{
    return __ldg(p);
}

template <class S>
struct Store;
template <>
struct Store<double> {
    using real = double;
    static __device__ __forceinline__ double ld(const double *p) { return pop_load(p); }
    static __device__ __forceinline__ double lds(const double *p) { return *p; }  // shared memory
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <>
struct Store<float> {
    using real = float;
    static __device__ __forceinline__ float ld(const float *p) { return pop_load(p); }
    static __device__ __forceinline__ float lds(const float *p) { return *p; }  // shared memory
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Store<__half> {
    using real = float;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(pop_load(p)); }
    static __device__ __forceinline__ float lds(const __half *p) { return __half2float(*p); }  // shared memory
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
    using real = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(pop_load(p)); }
    static __device__ __forceinline__ float lds(const __nv_bfloat16 *p) { return __bfloat162float(*p); }  // shared memory
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// populations of one instance: F_i (i-major, stride pstride = N) at the
// instance block's byte offset; instance blocks follow one another in node order
template <class S>
struct Pop {
    using FT = S;
    using R = typename Store<S>::real;
    static constexpr size_t node_bytes = Q * sizeof(S);
    FT *f;
    int N;  // stride between directions (the instance's pstride)
    __host__ __device__ __forceinline__ Pop(const void *base, const InstDev &I)
        : f((FT *)((char *)base + I.pop_off)), N(I.pstride)
    {
    }
    __device__ __forceinline__ R F(int i, int m) const { return Store<FT>::ld(f + i * N + m); }
    __device__ __forceinline__ void setF(int i, int m, R v) const { Store<FT>::st(f + i * N + m, v); }
};

// two consecutive 16-bit values of a node pair (x even) as one 32-bit access,
// and the pair store of two reals
__device__ __forceinline__ void ld_pair(const __half *p, float &a, float &b)
{
    const __half2 v = __ldg(reinterpret_cast<const __half2 *>(p));
    a = __low2float(v);
    b = __high2float(v);
}
__device__ __forceinline__ void ld_pair(const __nv_bfloat16 *p, float &a, float &b)
{
    const __nv_bfloat162 v = __ldg(reinterpret_cast<const __nv_bfloat162 *>(p));
    a = __low2float(v);
    b = __high2float(v);
}
__device__ __forceinline__ void ld_pair(const float *p, float &a, float &b)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void st_pair(__half *p, float a, float b)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void st_pair(__nv_bfloat16 *p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void st_pair(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }

// minimum-image displacement on a periodic axis of n nodes (|d| < 3n/2): the
// same value as d - n floor(d/n + 1/2) without a double-precision division
__host__ __device__ __forceinline__ double min_image(double d, int n)
{
    const double h = 0.5 * n;
    return d >= h ? d - n : (d < -h ? d + n : d);
}

// the same in single precision (|d| < 3n/2)
__device__ __forceinline__ float min_image_f(float d, int n)
{
    const float h = 0.5f * n;
    return d >= h ? d - n : (d < -h ? d + n : d);
}

// periodic neighbourhood of one node: x coordinates and row/plane offsets of
// x-1..x+1, y-1..y+1, z-1..z+1 (instance-local 32-bit node indices; every
// instance has fewer than 2^31/38 nodes)
struct Nbr {
    int X[3], YO[3], ZO[3];
    __device__ __forceinline__ void init(int x, int y, int z, int nx_, int ny_, int nz_)
    {
        const int nxy = nx_ * ny_;
        X[0] = x == 0 ? nx_ - 1 : x - 1; X[1] = x; X[2] = x == nx_ - 1 ? 0 : x + 1;
        YO[0] = (y == 0 ? ny_ - 1 : y - 1) * nx_; YO[1] = y * nx_; YO[2] = (y == ny_ - 1 ? 0 : y + 1) * nx_;
        ZO[0] = (z == 0 ? nz_ - 1 : z - 1) * nxy; ZO[1] = z * nxy; ZO[2] = (z == nz_ - 1 ? 0 : z + 1) * nxy;
    }
    __device__ __forceinline__ int at(int dx, int dy, int dz) const { return ZO[dz + 1] + YO[dy + 1] + X[dx + 1]; }
    __device__ __forceinline__ int idx(int dx, int dy, int dz) const { return at(dx, dy, dz); }
};

// reciprocal and inverse square root: IEEE for double, the fast single-precision
// forms otherwise (the FP32 and 16-bit paths are held to 1e-4 / 2e-3)
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }

// velocity of the solid owning a node at the point xw (Sec. V A)
template <class R>
__device__ __forceinline__ void surface_velocity(const InstDev &I, const PartDev *parts, int owner, R xw, R yw, R zw,
                                                 R *u)
{
    // in R: double in the FP64 mode, float (with the float particle centres)
    // otherwise; the link midpoints are half-integers, exact in either
    if (owner == OWN_WALL) {
        u[0] = (R)I.wall_u[0]; u[1] = (R)I.wall_u[1]; u[2] = (R)I.wall_u[2];
        return;
    }
    const PartDev &P = parts[I.part_off + owner - 2];
    R d0, d1, d2;
    if (sizeof(R) == 8) {
        d0 = (R)min_image(xw - P.x[0], I.nx); d1 = (R)min_image(yw - P.x[1], I.ny); d2 = (R)min_image(zw - P.x[2], I.nz);
    } else {
        d0 = (R)min_image_f((float)xw - P.xf[0], I.nx); d1 = (R)min_image_f((float)yw - P.xf[1], I.ny);
        d2 = (R)min_image_f((float)zw - P.xf[2], I.nz);
    }
    const R w0 = (R)P.w[0], w1 = (R)P.w[1], w2 = (R)P.w[2];
    u[0] = (R)P.v[0] + (w1 * d2 - w2 * d1);
    u[1] = (R)P.v[1] + (w2 * d0 - w0 * d2);
    u[2] = (R)P.v[2] + (w0 * d1 - w1 * d0);
}

// cube of side `side` (clamped to the domain) centred on a particle's node
struct Region {
    int lo[3], sz[3];
    __device__ __forceinline__ void init(const double *xc, int side, int nx, int ny, int nz)
    {
        const int n[3] = {nx, ny, nz};
        for (int a = 0; a < 3; a++) {
            int s = side < n[a] ? side : n[a];
            sz[a] = s;
            int lo_ = (int)floor(xc[a]) - (s - 1) / 2;
            lo[a] = s == n[a] ? 0 : lo_;
        }
    }
    __device__ __forceinline__ long long count() const { return (long long)sz[0] * sz[1] * sz[2]; }
    // node t of the cube (t < count < 2^31); lo + i lies in (-n, 2n), so one
    // conditional wrap per axis suffices
    __device__ __forceinline__ void coord(long long t, int nx, int ny, int nz, int *x, int *y, int *z) const
    {
        const int tt = (int)t;
        const int ij = tt / sz[0];
        const int i = tt - ij * sz[0];
        const int k = ij / sz[1];
        const int j = ij - k * sz[1];
        int a = lo[0] + i, b = lo[1] + j, c = lo[2] + k;
        a += a < 0 ? nx : (a >= nx ? -nx : 0);
        b += b < 0 ? ny : (b >= ny ? -ny : 0);
        c += c < 0 ? nz : (c >= nz ? -nz : 0);
        *x = a;
        *y = b;
        *z = c;
    }
};

// neighbourhood of a node in global memory: node index and owner of the node
// at offset (dx, dy, dz), periodic
struct GlobalNbr {
    Nbr nb;
    const uint8_t *fli;  // flags of the instance
    __device__ __forceinline__ int idx(int dx, int dy, int dz) const { return nb.at(dx, dy, dz); }
    __device__ __forceinline__ int own(int dx, int dy, int dz) const { return fli[nb.at(dx, dy, dz)] & OWNER_MASK; }
};

// The colour record of a node of the stored state (see the top of this
// file): the order parameter phi of the collision that produced it and
// a = b n, one 16-byte (FP64: 32-byte) aligned record, so that a pulled source
// costs one vector load.
template <class R>
struct alignas(4 * sizeof(R)) ColRec {
    R p, a0, a1, a2;
};

// (c_i . a)/|c_i|: the colour offset G*_i of a record beyond phi (1 + F*_i)
template <class R>
__device__ __forceinline__ R col_rec(int i, const ColRec<R> &c)
{
    R t = 0;
    if (cx(i)) t += cx(i) * c.a0;
    if (cy(i)) t += cy(i) * c.a1;
    if (cz(i)) t += cz(i) * c.a2;
    return csq(i) == 1 ? t : t * R(0.70710678118654752440);
}

// one node's record slot (write side)
template <class R>
struct ColSlot {
    ColRec<R> *p;
    __device__ __forceinline__ void set(const ColRec<R> &c) const { *p = c; }
    // the slot n nodes further on
    __device__ __forceinline__ ColSlot shifted(long long n) const { return ColSlot{p + n}; }
    // phi of the record n nodes further on
    __device__ __forceinline__ R phi(long long n) const { return p[n].p; }
};

// the colour records of an instance (read side)
template <class R>
struct Colour {
    const ColRec<R> *c;
    __device__ __forceinline__ Colour(const Lattice &L, const InstDev &I)
        : c((const ColRec<R> *)L.col + I.node_off)
    {
    }
    __device__ __forceinline__ ColRec<R> at(int m) const { return c[m]; }
    // G*_i = phi (1 + F*_i) + (c_i . a)/|c_i| of the record at m
    __device__ __forceinline__ R G(int i, int m, R F) const
    {
        const ColRec<R> r = c[m];
        R g = r.p * (R(1) + F);
        if (i) g += col_rec(i, r);
        return g;
    }
};

template <class S>
using ColourOf = Colour<typename Store<S>::real>;
template <class S>
using ColSlotOf = ColSlot<typename Store<S>::real>;

// the record slot of global node g
template <class S>
__device__ __forceinline__ ColSlotOf<S> col_slot(const Lattice &L, long long g)
{
    return ColSlotOf<S>{(ColRec<typename Store<S>::real> *)L.col + g};
}

// Pull streaming (Sec. IV) into fluid node n, with the Sec. V A halfway
// bounce-back where the source node is solid:
//   f_i(x) = f*_ibar(x) + 6 w_i rho^{a,b}(x) c_i.u_w,
// rho^{a,b}(x) of the node's own pre-streaming state, u_w at the link midpoint.
// Every flag and population load is issued before any is used (one dependent
// round trip instead of one per link).  F receives the 19 total offsets.
// A source on a pressure face (Sec. V D) gives the anti-bounce-back value
//   f_i = -f*_ibar(x) + 2 w_i rho_w [1 + (c_i.u_w)^2/(2 cs^4) - u_w^2/(2 cs^2)],
// rho_w the face's density (inlet below, outlet above), u_w = j*/rho* of the
// node's own post-collision state; the colour split of rho_w follows that
// state's phi, so the colour offset is phi(x)(1 + F_i) + (c_i . a(x))/|c_i|.
// With C set, *sG receives sum_i w_i G_i of the streamed colour offsets:
// G_i(x) = G*_i(x - c_i) from a fluid source; from a solid one
// G*_ibar(x) + 6 (rho^a - rho^b)(x)/rho0 c_i.u_w, and since
// (rho^a - rho^b)(x) = phi(x) rho(x) that is phi(x)(1 + F_i(x)) - (c_i . a(x))/|c_i|.
template <class S, class A>
__device__ __forceinline__ void gather_all(const InstDev &I, const PartDev *parts, const A &nbr,
                                           const Pop<S> &in, const ColourOf<S> *C, int n,
                                           typename Store<S>::real *F, typename Store<S>::real *sG, int x, int y,
                                           int z)
{
    using R = typename Store<S>::real;
    int own[Q];
    R pF[Q], oF[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int s = nbr.idx(-cx(i), -cy(i), -cz(i));
        own[i] = nbr.own(-cx(i), -cy(i), -cz(i));
        pF[i] = in.F(i, s);
        oF[i] = in.F(i, n);
    }
    R sF = 0, jw[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < Q; j++) {
        sF += wgt<R>(j) * oF[j];
        if (cx(j)) jw[0] += wgt<R>(j) * cx(j) * oF[j];
        if (cy(j)) jw[1] += wgt<R>(j) * cy(j) * oF[j];
        if (cz(j)) jw[2] += wgt<R>(j) * cz(j) * oF[j];
    }
    const R rr = R(1) + sF;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (own[i] == OWN_FLUID) {
            F[i] = pF[i];
            continue;
        }
        if (own[i] == OWN_PRESS) {
            const R irr = R(1) / rr;
            const R u0 = jw[0] * irr, u1 = jw[1] * irr, u2 = jw[2] * irr;
            const R cu = cx(i) * u0 + cy(i) * u1 + cz(i) * u2;
            const R rw = sizeof(R) == 8 ? (R)(cz(i) > 0 ? I.rin : I.rout) : (R)(cz(i) > 0 ? I.f_rin : I.f_rout);
            F[i] = R(-2) - oF[opp(i)] + R(2) * rw * (R(1) + R(4.5) * cu * cu - R(1.5) * (u0 * u0 + u1 * u1 + u2 * u2));
            continue;
        }
        R uw[3];
        surface_velocity<R>(I, parts, own[i], x - R(0.5) * cx(i), y - R(0.5) * cy(i), z - R(0.5) * cz(i), uw);
        const R cu = cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2];
        F[i] = oF[opp(i)] + R(6) * rr * cu;
    }
    if (!C) return;
    const ColRec<R> cn = C->at(n);
    R g = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        R gi;
        if (own[i] == OWN_FLUID) {
            gi = C->G(i, nbr.idx(-cx(i), -cy(i), -cz(i)), F[i]);
        } else if (own[i] == OWN_PRESS) {
            gi = cn.p * (R(1) + F[i]) + col_rec(i, cn);
        } else {
            gi = cn.p * (R(1) + F[i]) - col_rec(i, cn);
        }
        g += wgt<R>(i) * gi;
    }
    *sG = g;
}

// order parameter after streaming of a fluid node none of whose neighbours is
// solid: phi = sum_i w_i G_i / (1 + sum_i w_i F_i) with G_i rebuilt from the
// source node's colour state
template <class S, class A>
__device__ __forceinline__ typename Store<S>::real phi_fluid(const A &nbr, const Pop<S> &in,
                                                             const ColourOf<S> &C)
{
    using R = typename Store<S>::real;
    R sF = 0, sG = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int s = nbr.idx(-cx(i), -cy(i), -cz(i));
        const R F = in.F(i, s);
        const ColRec<R> cs = C.at(s);
        sF += wgt<R>(i) * F;
        R g = cs.p * (R(1) + F);
        if (i) g += col_rec(i, cs);
        sG += wgt<R>(i) * g;
    }
    return sG / (R(1) + sF);
}

template <class R>
__device__ __forceinline__ R dsqrt(R v) { return sqrt(v); }

// Sec. V E geometric wetting: rotate g so that -g/|g| makes the angle theta
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
    // cos and sin of the angle alpha* between n* and n_s: the FP64 path takes
    // acos / sin / cos as the oracle does; single precision uses the dot and
    // the norm of the cross product (alpha* in [0, pi]), which need no
    // transcendental calls and keep sin alpha* to relative precision where
    // sqrt(1 - cos^2) would lose it (cos alpha* near +-1)
    R sa, cal;
    if (sizeof(R) == 8) {
        const R al = acos(ca);
        sa = sin(al);
        cal = cos(al);
    } else {
        cal = ca;
        const R x0 = ns[1] * st[2] - ns[2] * st[1], x1 = ns[2] * st[0] - ns[0] * st[2],
                x2 = ns[0] * st[1] - ns[1] * st[0];
        sa = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    }
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

// ---------------------------------------------------------------------------
// row-strip work items (all per-node kernels): a strip of one z-plane made of
// st_rows whole x-rows (at most ROW_NODES nodes), or one segment of a longer row
// ---------------------------------------------------------------------------
constexpr int ROW_NODES = 256;  // nodes per work item at most = threads per CTA

struct StItem {
    int k;       // instance
    int z, y0;   // plane and first row
    int nrows;   // rows (whole-row items)
    int x0, cnt; // first x and number of nodes
    bool whole;
};

__device__ __forceinline__ void st_item(const Lattice &L, long long item, StItem &it)
{
    int lo = 0, hi = L.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.inst[mid].st_item_start <= item) lo = mid;
        else hi = mid - 1;
    }
    const InstDev &I = L.inst[lo];
    const int loc = (int)(item - I.st_item_start);  // < 2^31: rows of one instance
    const int per_plane = I.st_ygroups * I.st_nseg;
    it.k = lo;
    it.z = I.fd_plane.div(loc);
    const int r = loc - it.z * per_plane;
    const int yg = I.fd_nseg.div(r), sg = r - yg * I.st_nseg;
    it.y0 = yg * I.st_rows;
    it.whole = I.st_nseg == 1;
    it.nrows = min(I.st_rows, I.ny - it.y0);
    it.x0 = sg * I.st_seg;
    it.cnt = it.whole ? it.nrows * I.nx : min(I.st_seg, I.nx - it.x0);
}

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// first node of the item in the per-node arrays and the 16-byte-aligned start
// of its flag copy
__device__ __forceinline__ long long item_node0(const InstDev &I, const StItem &it)
{
    return I.node_off + ((long long)it.z * I.ny + it.y0) * I.nx + it.x0;
}

// node j of a work item
__device__ __forceinline__ void item_node(const InstDev &I, const StItem &it, int j, int *x, int *y)
{
    int r = 0, xx = it.x0 + j;
    if (it.nrows > 1) {
        r = I.fd_nx.div(j);
        xx = j - r * I.nx;
    }
    *x = xx;
    *y = it.y0 + r;
}

// the nodes of work item `item` (CTAs launched in item order cover a
// contiguous band of rows, so the neighbour rows they share stay in L2):
// f(I, n, x, y, z) for the CTA's nodes
template <class F>
__device__ __forceinline__ void for_item_nodes(const Lattice &L, long long item, F &&f)
{
    StItem it;
    st_item(L, item, it);
    const int j = threadIdx.x;
    if (j >= it.cnt) return;
    const InstDev &I = L.inst[it.k];
    if (it.nrows == 1) {
        // one row or row segment per CTA: y and z are the same for every
        // thread, which lets the neighbour-row offsets be computed once per CTA
        const int x = it.x0 + j;
        f(I, (it.z * I.ny + it.y0) * I.nx + x, x, it.y0, it.z);
        return;
    }
    int x, y;
    item_node(I, it, j, &x, &y);
    f(I, (it.z * I.ny + y) * I.nx + x, x, y, it.z);
}

// kernel stages, in launch order within a step (for per-kernel timing)
enum Stage {
    STAGE_PHI = 0, STAGE_SOLIDPHI, STAGE_GRAD, STAGE_COLLIDE, STAGE_MEM, STAGE_CAPILLARY, STAGE_DEM,
    STAGE_GEOM_OWNER, STAGE_GEOM_BOUND, STAGE_REFILL, STAGE_FUSED, STAGE_REGION, STAGE_CURV, STAGE_SURROGATE,
    STAGE_PHI_BOUND, STAGE_COLLIDE_BOUND, N_STAGES
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

// host-side hook run by the fluid launcher once grad(phi), the normals and
// the curvature of the step are final
struct Hook {
    void (*fn)(void *self) = nullptr;
    void *self = nullptr;
    void operator()() const
    {
        if (fn) fn(self);
    }
};

// a second stream with two events: the plain form runs its boundary passes
// there, beside the bulk kernels (they write disjoint nodes)
struct SideLane {
    cudaStream_t side = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    Hook after_collide_bound;  // more side-stream work after the collision's boundary pass
};

// host-side kernel launchers (defined in the .cu files)
constexpr int FORM_PLAIN = 2;  // the launch form of the fluid update (the value the ABI names)
struct FluidLaunch {
    int tile;           // 0: node-pair bulk collision where possible; 1: one node per thread
    long long rows;     // row-strip work items (all instances): CTAs of each bulk kernel
    long long gc_items; // gradient + curvature work items (all instances)
    bool pair;          // every instance has an even nx: node-pair kernels for 16-bit storage
};
// plan the work items of the gradient + curvature kernel (z-planes per item:
// zc_inst[k] for instance k where set (> 0), else zc_request, else the default)
long long plan_gradcurv(std::vector<InstDev> &inst, int zc_request, const std::vector<int> &zc_inst);
// plan the row-strip work items of every instance; returns their number
long long plan_rows(std::vector<InstDev> &inst);
template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk,
                       const FluidLaunch &fz, const Hook &after_grad = Hook(), const SideLane &lane = SideLane());
template <class S>
void launch_particle_forces(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk);
// the two halves of it: momentum exchange (needs only the step's input
// populations) and capillary force (needs the step's phi and normals)
template <class S>
void launch_momentum_exchange(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_capillary(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_geometry(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk);
// its three parts: owners and fresh bits (first), then boundary bits and the
// refill of fresh nodes, which touch disjoint data and may run concurrently
void launch_geom_owner(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk);
void launch_geom_bound(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk);
template <class S>
void launch_refill(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk);
// sum_fluid: gather the momentum-exchange and capillary partial sums first
// (false when the surrogate has written the fluid forces)
template <class S>
void launch_dem(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk, bool sum_fluid);

// ---------------------------------------------------------------------------
// learned force surrogate (lbm_mlp.cu)
// ---------------------------------------------------------------------------
constexpr int MLP_NIN = 387, MLP_KIN = 400, MLP_HIDDEN = 128, MLP_NOUT = 6, MLP_SHELL = 96;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_HIDDEN * MLP_KIN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_HIDDEN;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_HIDDEN * MLP_HIDDEN;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_HIDDEN;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_NOUT * MLP_HIDDEN;
constexpr int MLP_NPARAM = MLP_OFF_B3 + MLP_NOUT;
constexpr int MLP_CAP = 4096;  // batch rows at most

struct Mlp {
    float *theta = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;  // [MLP_NPARAM]
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr;                   // BF16 operand copies
    __nv_bfloat16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dZ1 = nullptr, *dZ2 = nullptr, *dYb = nullptr;
    float *Y = nullptr, *dY = nullptr, *T = nullptr;  // [cap][16], [cap][16], [cap][6]
    double *loss_part = nullptr, *loss = nullptr;     // loss[0]: last batch, loss[1]: accumulator
    int cap = 0;
    long long t = 0;  // Adam steps taken
    bool fault_no_commit = false;  // host-set fault injection (lbm_inject_fault)
};
cudaError_t mlp_alloc(Mlp &m, int cap);
void mlp_free(Mlp &m);
void mlp_refresh(const Mlp &m, cudaStream_t st);
// rows idx[row0 + r] (or row0 + r) of fp32 features [*][387] (and targets [*][6]) into the batch buffers
void mlp_stage(const Mlp &m, const float *X, const float *Y, const long long *idx, long long row0, int n,
               cudaStream_t st);
cudaError_t mlp_forward(const Mlp &m, int n, unsigned *status, cudaStream_t st);
cudaError_t mlp_backward(const Mlp &m, int n, double *acc, unsigned *status, cudaStream_t st);
void mlp_adam(Mlp &m, double lr, cudaStream_t st);
template <class S>
void launch_shell_features(const Lattice &L, int p0, int np, float *feat, cudaStream_t st);
template <class S>
void launch_surrogate_forces(const Lattice &L, const Mlp &m, float *feat, cudaStream_t st, long long *launches,
                             const Marker &mk);
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
// count (list == null) or fill a static boundary list: mode 0 static solid
// nodes with a non-static neighbour, mode 1 non-static nodes with a static
// solid neighbour
void launch_static_bound(const Lattice &L, long long *list, unsigned long long *count, int mode, cudaStream_t st);
void launch_mark_particles(const Lattice &L, cudaStream_t st);

}  // namespace lbmg
