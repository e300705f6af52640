// Fluid update of one coupled time step (Sec. IV of arXiv 2505.10171).
//
// Per node: pull streaming with bounce-back -> order parameter phi -> phi on
// solid nodes next to fluid (w-weighted fluid mean) -> isotropic grad(phi)
// with the geometric wetting rotation (Sec. V D) -> regularised normal and its
// divergence (curvature) -> CSF + body force -> MRT with Guo forcing, evaluated
// in its two-relaxation-time form -> recolouring -> write.
//
// Two launch forms share the per-node device functions below and give
// bit-identical results:
//  * k_fused: one kernel per step.  A block owns a TX x TY column tile and a
//    chunk of z-planes and marches z: the order parameter of plane z+3 is
//    gathered into a shared-memory ring (with a 3-node halo, enough for the
//    solid-phi fill), solids of plane z+2 are filled, gradient/wetting/normal of
//    plane z+1 are formed, and plane z is collided.  Each population is read
//    from HBM about once and written once; halo re-reads hit L2.
//  * k_phi, k_solidphi, k_grad, k_collide: the four-kernel form over all nodes,
//    kept as the straightforward reference of the fused one.
// The particle-region kernels recompute phi and grad(phi) around each particle
// for the capillary force.
// Storage type S in {double, float, __half, __nv_bfloat16}; arithmetic in
// double for S = double and float otherwise.
#include "lbm_internal.cuh"

namespace lbmg {

// ---------------------------------------------------------------------------
// per-node device functions
// ---------------------------------------------------------------------------

// phi of a solid node: w-weighted mean over its fluid neighbours; phi_of(dx,
// dy, dz) returns the order parameter of the neighbour
template <class R, class A, class PhiF>
__device__ __forceinline__ R solid_fill(const A &nbr, const PhiF &phi_of)
{
    R sw = 0, sp = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (nbr.own(cx(i), cy(i), cz(i)) != OWN_FLUID) continue;
        sw += wgt<R>(i);
        sp += wgt<R>(i) * phi_of(cx(i), cy(i), cz(i));
    }
    return sw > R(0) ? sp / sw : R(0);
}

// outward solid normal and contact angle at a fluid node next to solid: the
// nearest particle surface if a neighbour belongs to a particle, otherwise the
// normalised -sum w_i c_i over substrate neighbours.
template <class R, class A>
__device__ __forceinline__ bool solid_normal(const InstDev &I, const PartDev *parts, const A &nbr, int x, int y,
                                             int z, R *ns, R *cth, R *sth)
{
    int best = -1;
    double bestd = 0.0;
    double ws[3] = {0.0, 0.0, 0.0};
    bool any = false;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int own = nbr.own(cx(i), cy(i), cz(i));
        if (own == OWN_FLUID) continue;
        any = true;
        if (own == OWN_WALL) {
            ws[0] -= wgt<double>(i) * cx(i);
            ws[1] -= wgt<double>(i) * cy(i);
            ws[2] -= wgt<double>(i) * cz(i);
        } else {
            const PartDev &P = parts[I.part_off + own - 2];
            double d0 = min_image(x - P.x[0], I.nx), d1 = min_image(y - P.x[1], I.ny),
                   d2 = min_image(z - P.x[2], I.nz);
            double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - P.R;
            int p = own - 2;
            if (best < 0 || dist < bestd || (dist == bestd && p < best)) {
                best = p;
                bestd = dist;
            }
        }
    }
    if (!any) return false;
    if (best >= 0) {
        const PartDev &P = parts[I.part_off + best];
        double d0 = min_image(x - P.x[0], I.nx), d1 = min_image(y - P.x[1], I.ny), d2 = min_image(z - P.x[2], I.nz);
        double dl = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        ns[0] = (R)(d0 / dl); ns[1] = (R)(d1 / dl); ns[2] = (R)(d2 / dl);
        *cth = (R)P.cos_t;
        *sth = (R)P.sin_t;
        return true;
    }
    double wl = sqrt(ws[0] * ws[0] + ws[1] * ws[1] + ws[2] * ws[2]);
    if (wl == 0.0) return false;
    ns[0] = (R)(ws[0] / wl); ns[1] = (R)(ws[1] / wl); ns[2] = (R)(ws[2] / wl);
    *cth = (R)I.cos_tw;
    *sth = (R)I.sin_tw;
    return true;
}

// grad(phi) = 3 sum_i w_i c_i phi(x + c_i) with the wetting rotation at
// boundary nodes inside the interface
template <class R, class A, class PhiF>
__device__ __forceinline__ void grad_node(const InstDev &I, const PartDev *parts, const A &nbr, const PhiF &phi_of,
                                          R phi_here, uint8_t fl, R wet_max, int x, int y, int z, R *gr)
{
    gr[0] = gr[1] = gr[2] = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        R p = phi_of(cx(i), cy(i), cz(i));
        R wc = R(3) * wgt<R>(i);
        gr[0] += wc * cx(i) * p;
        gr[1] += wc * cy(i) * p;
        gr[2] += wc * cz(i) * p;
    }
    if ((fl & BOUND_BIT) && fabs(phi_here) < wet_max) {
        R ns[3], cth, sth;
        if (solid_normal<R>(I, parts, nbr, x, y, z, ns, &cth, &sth)) wetting_rotate<R>(gr, ns, cth, sth);
    }
}

// force, velocity, MRT (two-relaxation-time form) with Guo forcing,
// recolouring and the write of node n.  F, G: streamed offsets; g: corrected
// grad(phi) of the node; nn: its regularised normal; kap: curvature.
template <class S>
__device__ __forceinline__ void collide_store(const FluidPar<typename Store<S>::real> &P, const typename Store<S>::real *F,
                                              const typename Store<S>::real *G, const typename Store<S>::real *g,
                                              const typename Store<S>::real *nn, typename Store<S>::real kap,
                                              S *__restrict__ out, int N, int n, typename Store<S>::real *U,
                                              long long Ustride, unsigned *status)
{
    using R = typename Store<S>::real;
    R sF = 0, sG = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const R w = wgt<R>(i);
        sF += w * F[i];
        sG += w * G[i];
        if (cx(i)) jx += w * cx(i) * F[i];
        if (cy(i)) jy += w * cy(i) * F[i];
        if (cz(i)) jz += w * cz(i) * F[i];
    }
    const R rr = R(1) + sF;  // rho / rho0
    const R phi = sG * frcp(rr);
    if (!(rr > R(0)) || !(phi == phi)) atomicOr(status, ST_UNSTABLE);
    // force density: CSF -1/2 sigma kappa grad(phi) plus phase-weighted body forces
    const R hs = R(-0.5) * P.sigma * kap;
    const R pa = R(0.5) * (R(1) + phi), pb = R(0.5) * (R(1) - phi);
    const R Fx = hs * g[0] + pa * P.ba[0] + pb * P.bb[0];
    const R Fy = hs * g[1] + pa * P.ba[1] + pb * P.bb[1];
    const R Fz = hs * g[2] + pa * P.ba[2] + pb * P.bb[2];
    // velocity: rho u = sum c f + F/2
    const R rho = P.rho0 * rr;
    const R irho = frcp(rho);
    const R ux = (P.rho0 * jx + R(0.5) * Fx) * irho;
    const R uy = (P.rho0 * jy + R(0.5) * Fy) * irho;
    const R uz = (P.rho0 * jz + R(0.5) * Fz) * irho;
    if (U) { U[n] = ux; U[Ustride + n] = uy; U[2 * Ustride + n] = uz; }
    // relaxation rates: harmonic-mean viscosity, tau = eta/(rho cs2) + 1/2
    const R inv_eta = (R(1) + phi) * P.h_ia + (R(1) - phi) * P.h_ib;
    const R tau = R(3) * frcp(inv_eta * rho) + R(0.5);
    const R om = frcp(tau);
    const R omp = R(8) * (R(2) - om) * frcp(R(8) - om);
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R cpe = R(1) - R(0.5) * om, cpo = R(1) - R(0.5) * omp;
    const R bq = R(0.5) * P.beta * rr * (R(1) - phi * phi);
    {
        const R feq0 = sF + rr * (R(-1.5) * uu);
        const R fb0 = R(-3) * uF * P.ir0;
        const R Fs = F[0] - om * (F[0] - feq0) + cpe * fb0;
        Store<S>::st(out + n, Fs);
        Store<S>::st(out + Q * N + n, phi * (R(1) + Fs));
    }
    // opposite pairs (i, i+9): the paper's S relaxes every even non-conserved
    // moment with omega and every odd one with omega', i.e. the MRT operator is
    // exactly the two-relaxation-time operator on the pair's even/odd parts
#pragma unroll
    for (int i = 1; i <= 9; i++) {
        const int ib = i + 9;
        const R cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const R cF = cx(i) * Fx + cy(i) * Fy + cz(i) * Fz;
        const R eqp = sF + rr * (R(4.5) * cu * cu - R(1.5) * uu);
        const R eqm = rr * R(3) * cu;
        const R fbp = (R(9) * cu * cF - R(3) * uF) * P.ir0;
        const R fbm = R(3) * cF * P.ir0;
        const R fp = R(0.5) * (F[i] + F[ib]);
        const R fm = R(0.5) * (F[i] - F[ib]);
        const R dp = -om * (fp - eqp) + cpe * fbp;
        const R dm = -omp * (fm - eqm) + cpo * fbm;
        const R Fi = F[i] + dp + dm;
        const R Fib = F[ib] + dp - dm;
        // recolouring: G* = phi (1 + F*) + beta/2 (rho/rho0)(1 - phi^2) c.n/|c|
        const R inv_len = csq(i) == 1 ? R(1) : R(0.70710678118654752440);
        const R cn = (cx(i) * nn[0] + cy(i) * nn[1] + cz(i) * nn[2]) * inv_len;
        const R rec = bq * cn;
        Store<S>::st(out + i * N + n, Fi);
        Store<S>::st(out + ib * N + n, Fib);
        Store<S>::st(out + (Q + i) * N + n, phi * (R(1) + Fi) + rec);
        Store<S>::st(out + (Q + ib) * N + n, phi * (R(1) + Fib) - rec);
    }
}

// curvature kappa = 3 sum_i w_i c_i . n(x + c_i), taken over opposite pairs as
// w_i c_i . (n(x + c_i) - n(x - c_i)) so that only the components along c_i
// are read; nf(dx, dy, dz, a) is component a of the neighbour's normal (the
// node's own normal for a solid neighbour)
template <class R, class NF>
__device__ __forceinline__ R curvature(const NF &nf)
{
    R k = 0;
#pragma unroll
    for (int i = 1; i <= 9; i++) {
        R t = 0;
        if (cx(i)) t += cx(i) * (nf(cx(i), cy(i), cz(i), 0) - nf(-cx(i), -cy(i), -cz(i), 0));
        if (cy(i)) t += cy(i) * (nf(cx(i), cy(i), cz(i), 1) - nf(-cx(i), -cy(i), -cz(i), 1));
        if (cz(i)) t += cz(i) * (nf(cx(i), cy(i), cz(i), 2) - nf(-cx(i), -cy(i), -cz(i), 2));
        k += wgt<R>(i) * t;
    }
    return R(3) * k;
}

// regularised interface normal n = g / sqrt(|g|^2 + eps^2); returns the norm
template <class R>
__device__ __forceinline__ R reg_normal(const R *g, R eps2, R *nn)
{
    const R m2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + eps2;
    const R im = frsqrt(m2);
    nn[0] = g[0] * im; nn[1] = g[1] * im; nn[2] = g[2] * im;
    return m2 * im;
}

// ---------------------------------------------------------------------------
// four-kernel form over all nodes (and the same bodies over particle regions)
// ---------------------------------------------------------------------------
#define LBM_NODE_PROLOGUE                                                                   \
    const long long blk = blockIdx.x;                                                        \
    const int k_inst = find_inst(L.inst, L.n_inst, blk);                                     \
    const InstDev &I = L.inst[k_inst];                                                       \
    const long long n_ = (blk - I.blk_start) * (long long)blockDim.x + threadIdx.x;          \
    if (n_ >= I.N) return;                                                                   \
    const int n = (int)n_;                                                                   \
    const int x = n % I.nx;                                                                  \
    const int y = (n / I.nx) % I.ny;                                                         \
    const int z = n / (I.nx * I.ny);

// region of particle blockIdx.y: nodes of a cube of side `side` around it
#define LBM_REGION_PROLOGUE                                                                  \
    const PartDev &P0 = L.parts[blockIdx.y];                                                 \
    const InstDev &I = L.inst[P0.inst];                                                      \
    Region reg;                                                                              \
    reg.init(P0.x, side, I.nx, I.ny, I.nz);                                                  \
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;                   \
    if (t >= reg.count()) return;                                                            \
    int x, y, z;                                                                             \
    reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);                                              \
    const int n = (z * I.ny + y) * I.nx + x;

template <class S>
__device__ __forceinline__ void phi_body(const Lattice &L, const InstDev &I, int cur, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    ((R *)L.phi)[g] = node_phi<S>(I, L.parts, nb, in, (int)I.N, n, fl, x, y, z);
}

template <class R>
__device__ __forceinline__ void solidphi_body(const Lattice &L, const InstDev &I, int n, int x, int y, int z)
{
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) == OWN_FLUID || !(fl & BOUND_BIT)) return;
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    const R *ph = (const R *)L.phi + I.node_off;
    auto phi_of = [&](int dx, int dy, int dz) { return ph[nb.idx(dx, dy, dz)]; };
    ((R *)L.phi)[g] = solid_fill<R>(nb, phi_of);
}

template <class R>
__device__ __forceinline__ void grad_body(const Lattice &L, const InstDev &I, int n, int x, int y, int z)
{
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    FluidPar<R> P;
    load_par(I, P);
    const R *ph = (const R *)L.phi + I.node_off;
    auto phi_of = [&](int dx, int dy, int dz) { return ph[nb.idx(dx, dy, dz)]; };
    R gr[3], nn[3];
    grad_node<R>(I, L.parts, nb, phi_of, ph[n], fl, P.wet_max, x, y, z, gr);
    const R m = reg_normal(gr, P.eps2, nn);
    R *Nn = (R *)L.grad;
    Nn[g] = nn[0];
    Nn[L.Ntot + g] = nn[1];
    Nn[2 * L.Ntot + g] = nn[2];
    ((R *)L.gmag)[g] = m;
}

template <class S>
__global__ void k_phi(Lattice L, int cur)
{
    LBM_NODE_PROLOGUE
    phi_body<S>(L, I, cur, n, x, y, z);
}

template <class R>
__global__ void k_solidphi(Lattice L)
{
    LBM_NODE_PROLOGUE
    solidphi_body<R>(L, I, n, x, y, z);
}

template <class R>
__global__ void k_grad(Lattice L)
{
    LBM_NODE_PROLOGUE
    grad_body<R>(L, I, n, x, y, z);
}

template <class S>
__global__ void __launch_bounds__(PART_THREADS) k_phi_region(Lattice L, int cur, int side)
{
    LBM_REGION_PROLOGUE
    phi_body<S>(L, I, cur, n, x, y, z);
}

template <class R>
__global__ void __launch_bounds__(PART_THREADS) k_solidphi_region(Lattice L, int side)
{
    LBM_REGION_PROLOGUE
    solidphi_body<R>(L, I, n, x, y, z);
}

template <class R>
__global__ void __launch_bounds__(PART_THREADS) k_grad_region(Lattice L, int side)
{
    LBM_REGION_PROLOGUE
    grad_body<R>(L, I, n, x, y, z);
}

template <class S>
__global__ void __launch_bounds__(256, sizeof(typename Store<S>::real) == 8 ? 1 : 2) k_collide(Lattice L, int cur)
{
    using R = typename Store<S>::real;
    LBM_NODE_PROLOGUE
    const int N = (int)I.N;
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
    if ((fl & OWNER_MASK) != OWN_FLUID) {
        if (U) { U[n] = 0; U[L.Ntot + n] = 0; U[2 * L.Ntot + n] = 0; }
        return;
    }
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    S *out = (S *)L.pop[cur ^ 1] + NPOP * I.node_off;
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    FluidPar<R> P;
    load_par(I, P);
    const R *Nn = (const R *)L.grad + I.node_off;
    const long long Nt = L.Ntot;
    const R nn[3] = {Nn[n], Nn[Nt + n], Nn[2 * Nt + n]};
    const R m = ((const R *)L.gmag)[g];
    const R gr[3] = {nn[0] * m, nn[1] * m, nn[2] * m};
    const bool bnd = fl & BOUND_BIT;
    auto nf = [&](int dx, int dy, int dz, int a) {
        if (bnd && nb.own(dx, dy, dz) != OWN_FLUID) return nn[a];
        return Nn[a * Nt + nb.idx(dx, dy, dz)];
    };
    const R kap = curvature<R>(nf);
    R F[Q], G[Q];
    gather<S>(I, L.parts, nb, in, N, n, fl, F, G, x, y, z);
    collide_store<S>(P, F, G, gr, nn, kap, out, N, n, U, L.Ntot, L.status);
}

// ---------------------------------------------------------------------------
// fused kernel
// ---------------------------------------------------------------------------
constexpr int FH = 3;     // halo of the phi ring (the solid fill needs 3 hops)
constexpr int NSLOT = 5;  // planes of phi and flags kept in the ring
template <int TX, int TY>
struct FusedGeom {
    static constexpr int NT = TX * TY;
    static constexpr int RW = TX + 2 * FH, RH = TY + 2 * FH, RN = RW * RH;
    static constexpr int W1 = TX + 2, H1 = TY + 2, R1N = W1 * H1;
};

template <class R, int TX, int TY>
constexpr size_t fused_smem_bytes()
{
    using Gm = FusedGeom<TX, TY>;
    return sizeof(R) * (NSLOT * Gm::RN + 9 * Gm::R1N + 2 * Gm::NT) + NSLOT * Gm::RN;
}

// neighbourhood of a fused-kernel node: node indices from its global
// coordinates, owners from the shared-memory flag ring
template <int TX, int TY>
struct RingNbr {
    Nbr nb;
    const uint8_t *flS;  // [NSLOT][RN]
    int r;               // region index of the node
    int slot[3];         // ring slots of the planes z-1, z, z+1
    __device__ __forceinline__ int idx(int dx, int dy, int dz) const { return nb.at(dx, dy, dz); }
    __device__ __forceinline__ int own(int dx, int dy, int dz) const
    {
        using Gm = FusedGeom<TX, TY>;
        return flS[slot[dz + 1] * Gm::RN + r + dy * Gm::RW + dx] & OWNER_MASK;
    }
};

__device__ __forceinline__ int wrapc(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ int find_item_inst(const InstDev *I, int n, long long item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (I[mid].item_start <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2) k_fused(Lattice L, int cur)
{
    using R = typename Store<S>::real;
    using Gm = FusedGeom<TX, TY>;
    constexpr int NT = Gm::NT, RW = Gm::RW, RN = Gm::RN, W1 = Gm::W1, R1N = Gm::R1N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *phiS = (R *)smem_raw;                  // [NSLOT][RN]
    R *nS = phiS + NSLOT * RN;                // [3 planes][3 comps][R1N]
    R *mS = nS + 9 * R1N;                     // [2 planes][NT]: |g| of the tile's nodes
    uint8_t *flS = (uint8_t *)(mS + 2 * NT);  // [NSLOT][RN]

    const long long item = blockIdx.x;
    const InstDev &I = L.inst[find_item_inst(L.inst, L.n_inst, item)];
    const long long local = item - I.item_start;
    const int chunk = (int)(local % I.nchunks);
    const long long t2 = local / I.nchunks;
    const int x0 = (int)(t2 % I.tiles_x) * TX;
    const int y0 = (int)(t2 / I.tiles_x) * TY;
    const int z0 = chunk * I.zc;
    const int z1 = min(z0 + I.zc, I.nz);
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const int N = (int)I.N;
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    S *out = (S *)L.pop[cur ^ 1] + NPOP * I.node_off;
    const uint8_t *fli = L.flags + I.node_off;
    R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
    FluidPar<R> P;
    load_par(I, P);

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool active = gx < nx && gy < ny;
    const int niter = (z1 - z0) + 6;

    for (int j = 0; j < niter; j++) {
        const int gp = z0 - 3 + j;  // plane gathered in this iteration
        // (1) flags and order parameter of plane gp over the whole region
        {
            const int s = j % NSLOT;
            const int Z = wrapc(gp, nz);
            for (int r = tid; r < RN; r += NT) {
                const int X = wrapc(x0 - FH + r % RW, nx);
                const int Y = wrapc(y0 - FH + r / RW, ny);
                const int n = (Z * ny + Y) * nx + X;
                const uint8_t fl = fli[n];
                flS[s * RN + r] = fl;
                R ph = 0;
                if ((fl & OWNER_MASK) == OWN_FLUID) {
                    GlobalNbr nb;
                    nb.nb.init(X, Y, Z, nx, ny, nz);
                    nb.fli = fli;
                    ph = node_phi<S>(I, L.parts, nb, in, N, n, fl, X, Y, Z);
                }
                phiS[s * RN + r] = ph;
            }
        }
        __syncthreads();
        // (2) phi on solid nodes of plane gp-1 (ring 1..RW-2 of the region)
        if (j >= 2) {
            const int sm = (j - 2) % NSLOT, s0 = (j - 1) % NSLOT, sp = j % NSLOT;
            for (int r = tid; r < RN; r += NT) {
                const int rx = r % RW, ry = r / RW;
                if (rx < 1 || rx >= RW - 1 || ry < 1 || ry >= Gm::RH - 1) continue;
                const uint8_t fl = flS[s0 * RN + r];
                if ((fl & OWNER_MASK) == OWN_FLUID || !(fl & BOUND_BIT)) continue;
                RingNbr<TX, TY> nb;
                nb.flS = flS;
                nb.r = r;
                nb.slot[0] = sm; nb.slot[1] = s0; nb.slot[2] = sp;
                auto phi_of = [&](int dx, int dy, int dz) { return phiS[nb.slot[dz + 1] * RN + r + dy * RW + dx]; };
                phiS[s0 * RN + r] = solid_fill<R>(nb, phi_of);
            }
        }
        __syncthreads();
        // (3) gradient, wetting and normal of plane gp-2 on the 1-halo tile
        if (j >= 4) {
            const int sm = (j - 3) % NSLOT, s0 = (j - 2) % NSLOT, sp = (j - 1) % NSLOT;
            const int ns = (j - 2) % 3, ms = (j - 2) % 2;
            const int Z = wrapc(gp - 2, nz);
            for (int r1 = tid; r1 < R1N; r1 += NT) {
                const int ax = r1 % W1, ay = r1 / W1;
                const int r = (ay + FH - 1) * RW + (ax + FH - 1);
                const uint8_t fl = flS[s0 * RN + r];
                R gr[3] = {0, 0, 0};
                if ((fl & OWNER_MASK) == OWN_FLUID) {
                    const int X = wrapc(x0 - 1 + ax, nx), Y = wrapc(y0 - 1 + ay, ny);
                    RingNbr<TX, TY> nb;
                    nb.flS = flS;
                    nb.r = r;
                    nb.slot[0] = sm; nb.slot[1] = s0; nb.slot[2] = sp;
                    auto phi_of = [&](int dx, int dy, int dz) { return phiS[nb.slot[dz + 1] * RN + r + dy * RW + dx]; };
                    grad_node<R>(I, L.parts, nb, phi_of, phiS[s0 * RN + r], fl, P.wet_max, X, Y, Z, gr);
                }
                R nn[3];
                const R m = reg_normal(gr, P.eps2, nn);
                nS[(ns * 3 + 0) * R1N + r1] = nn[0];
                nS[(ns * 3 + 1) * R1N + r1] = nn[1];
                nS[(ns * 3 + 2) * R1N + r1] = nn[2];
                if (ax >= 1 && ax <= TX && ay >= 1 && ay <= TY) mS[ms * NT + (ay - 1) * TX + (ax - 1)] = m;
            }
        }
        __syncthreads();
        // (4) collide plane gp-3 (the tile's own planes z0..z1-1)
        if (j >= 6 && active) {
            const int Z = wrapc(gp - 3, nz);
            const int n = (Z * ny + gy) * nx + gx;
            const int r = (ly + FH) * RW + (lx + FH);
            const int sm = (j - 4) % NSLOT, s0 = (j - 3) % NSLOT, sp = (j - 2) % NSLOT;
            const uint8_t fl = flS[s0 * RN + r];
            if ((fl & OWNER_MASK) != OWN_FLUID) {
                if (U) { U[n] = 0; U[L.Ntot + n] = 0; U[2 * L.Ntot + n] = 0; }
            } else {
                RingNbr<TX, TY> nb;
                nb.nb.init(gx, gy, Z, nx, ny, nz);
                nb.flS = flS;
                nb.r = r;
                nb.slot[0] = sm; nb.slot[1] = s0; nb.slot[2] = sp;
                const int nsl[3] = {(j - 4) % 3, (j - 3) % 3, (j - 2) % 3};
                const int r1 = (ly + 1) * W1 + (lx + 1);
                const R nn[3] = {nS[(nsl[1] * 3 + 0) * R1N + r1], nS[(nsl[1] * 3 + 1) * R1N + r1],
                                 nS[(nsl[1] * 3 + 2) * R1N + r1]};
                const R m = mS[((j - 3) % 2) * NT + tid];
                const R gr[3] = {nn[0] * m, nn[1] * m, nn[2] * m};
                const bool bnd = fl & BOUND_BIT;
                auto nf = [&](int dx, int dy, int dz, int a) {
                    if (bnd && nb.own(dx, dy, dz) != OWN_FLUID) return nn[a];
                    return nS[(nsl[dz + 1] * 3 + a) * R1N + r1 + dy * W1 + dx];
                };
                const R kap = curvature<R>(nf);
                R F[Q], G[Q];
                gather<S>(I, L.parts, nb, in, N, n, fl, F, G, gx, gy, Z);
                collide_store<S>(P, F, G, gr, nn, kap, out, N, n, U, L.Ntot, L.status);
            }
        }
        __syncthreads();
    }
}

// tile shapes of the fused kernel
int fused_tile_x(int tile) { return tile == 1 ? 64 : (tile == 2 ? 16 : 32); }
int fused_tile_y(int tile) { return tile == 1 ? 4 : (tile == 2 ? 16 : 8); }

template <class S, int TX, int TY>
static void launch_fused(const Lattice &L, int cur, long long items, cudaStream_t st)
{
    using R = typename Store<S>::real;
    constexpr size_t smem = fused_smem_bytes<R, TX, TY>();
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_fused<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    k_fused<S, TX, TY><<<(unsigned)items, TX * TY, smem, st>>>(L, cur);
}

template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk,
                       const FluidLaunch &fz)
{
    using R = typename Store<S>::real;
    if (fz.fused) {
        if (L.n_parts > 0) {
            // phi and grad(phi) around the particles, for the capillary force:
            // corners of the surface points lie within R_p + 2 of the centre,
            // their gradient reads phi within R_p + 3 (solid-filled), the fill
            // reads fluid phi within R_p + 4
            const int side = L.cap_side;
            mk(STAGE_REGION, 0);
            k_phi_region<S><<<dim3(L.cap_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, cur, side);
            k_solidphi_region<R><<<dim3(L.cap_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side - 2);
            k_grad_region<R><<<dim3(L.cap_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side - 4);
            mk(STAGE_REGION, 1);
            *launches += 3;
        }
        mk(STAGE_FUSED, 0);
        switch (fz.tile) {
        case 1: launch_fused<S, 64, 4>(L, cur, fz.items, st); break;
        case 2: launch_fused<S, 16, 16>(L, cur, fz.items, st); break;
        default: launch_fused<S, 32, 8>(L, cur, fz.items, st); break;
        }
        mk(STAGE_FUSED, 1);
        *launches += 1;
        return;
    }
    dim3 grid((unsigned)L.n_blocks), block(L.bt);
    mk(STAGE_PHI, 0);
    k_phi<S><<<grid, block, 0, st>>>(L, cur);
    mk(STAGE_PHI, 1);
    mk(STAGE_SOLIDPHI, 0);
    k_solidphi<R><<<grid, block, 0, st>>>(L);
    mk(STAGE_SOLIDPHI, 1);
    mk(STAGE_GRAD, 0);
    k_grad<R><<<grid, block, 0, st>>>(L);
    mk(STAGE_GRAD, 1);
    mk(STAGE_COLLIDE, 0);
    k_collide<S><<<grid, block, 0, st>>>(L, cur);
    mk(STAGE_COLLIDE, 1);
    *launches += 4;
}

#define INST(S)                                                                                                   \
    template void launch_fluid_step<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &,            \
                                       const FluidLaunch &);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
