// Fluid kernels of one coupled time step (Sec. IV of arXiv 2505.10171):
//   k_phi      pull streaming + bounce-back -> order parameter phi
//   k_solidphi phi on solid nodes next to fluid (w-weighted fluid mean)
//   k_grad     isotropic grad(phi) + geometric wetting rotation (Sec. V D)
//   k_collide  streaming again, curvature, CSF + body force, MRT with Guo
//              forcing (evaluated in its two-relaxation-time form), recolouring,
//              write of the post-collision offsets.
// Storage type S in {double, float, __half, __nv_bfloat16}; arithmetic in
// double for S = double and in float otherwise.
#include "lbm_internal.cuh"

namespace lbmg {

#define LBM_NODE_PROLOGUE                                                                   \
    const long long blk = blockIdx.x;                                                        \
    const int k_inst = find_inst(L.inst, L.n_inst, blk);                                     \
    const InstDev &I = L.inst[k_inst];                                                       \
    const long long n = (blk - I.blk_start) * (long long)blockDim.x + threadIdx.x;           \
    if (n >= I.N) return;                                                                    \
    const long long N = I.N;                                                                 \
    const long long g = I.node_off + n;                                                      \
    const int x = (int)(n % I.nx);                                                           \
    const int y = (int)((n / I.nx) % I.ny);                                                  \
    const int z = (int)(n / ((long long)I.nx * I.ny));

template <class S>
__global__ void k_phi(Lattice L, int cur)
{
    using R = typename Store<S>::real;
    LBM_NODE_PROLOGUE
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    R F[Q], G[Q];
    gather<S>(I, L.parts, L.flags, in, N, n, nb, fl, F, G, x, y, z);
    R sF = 0, sG = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        sF += wgt<R>(i) * F[i];
        sG += wgt<R>(i) * G[i];
    }
    ((R *)L.phi)[g] = sG / (R(1) + sF);
}

template <class R>
__global__ void k_solidphi(Lattice L)
{
    LBM_NODE_PROLOGUE
    (void)N;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) == OWN_FLUID || !(fl & BOUND_BIT)) return;
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    const uint8_t *fli = L.flags + I.node_off;
    const R *ph = (const R *)L.phi + I.node_off;
    R sw = 0, sp = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        long long m = nb.at(cx(i), cy(i), cz(i));
        if ((fli[m] & OWNER_MASK) != OWN_FLUID) continue;
        sw += wgt<R>(i);
        sp += wgt<R>(i) * ph[m];
    }
    ((R *)L.phi)[g] = sw > R(0) ? sp / sw : R(0);
}

// outward solid normal and contact angle at a fluid node next to solid: the
// nearest particle surface if a neighbour belongs to a particle, otherwise the
// normalised -sum w_i c_i over substrate neighbours.
template <class R>
__device__ __forceinline__ bool solid_normal(const Lattice &L, const InstDev &I, const Nbr &nb, int x, int y,
                                             int z, R *ns, R *cth, R *sth)
{
    const uint8_t *fli = L.flags + I.node_off;
    int best = -1;
    double bestd = 0.0;
    double ws[3] = {0.0, 0.0, 0.0};
    bool any = false;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int own = fli[nb.at(cx(i), cy(i), cz(i))] & OWNER_MASK;
        if (own == OWN_FLUID) continue;
        any = true;
        if (own == OWN_WALL) {
            ws[0] -= wgt<double>(i) * cx(i);
            ws[1] -= wgt<double>(i) * cy(i);
            ws[2] -= wgt<double>(i) * cz(i);
        } else {
            const PartDev &P = L.parts[I.part_off + own - 2];
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
        const PartDev &P = L.parts[I.part_off + best];
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

template <class R>
__global__ void k_grad(Lattice L)
{
    LBM_NODE_PROLOGUE
    (void)N;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    const R *ph = (const R *)L.phi + I.node_off;
    R gr[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; i++) {
        R p = ph[nb.at(cx(i), cy(i), cz(i))];
        R wc = R(3) * wgt<R>(i);
        gr[0] += wc * cx(i) * p;
        gr[1] += wc * cy(i) * p;
        gr[2] += wc * cz(i) * p;
    }
    if ((fl & BOUND_BIT) && fabs(ph[n]) < (R)I.wet_max) {
        R ns[3], cth, sth;
        if (solid_normal<R>(L, I, nb, x, y, z, ns, &cth, &sth)) wetting_rotate<R>(gr, ns, cth, sth);
    }
    R *G = (R *)L.grad;
    G[g] = gr[0];
    G[L.Ntot + g] = gr[1];
    G[2 * L.Ntot + g] = gr[2];
}

template <class S>
__global__ void k_collide(Lattice L, int cur)
{
    using R = typename Store<S>::real;
    LBM_NODE_PROLOGUE
    const uint8_t fl = L.flags[g];
    R *U = (R *)L.u;
    if ((fl & OWNER_MASK) != OWN_FLUID) {
        if (I.store_u) { U[g] = 0; U[L.Ntot + g] = 0; U[2 * L.Ntot + g] = 0; }
        return;
    }
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    S *out = (S *)L.pop[cur ^ 1] + NPOP * I.node_off;
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    R F[Q], G[Q];
    gather<S>(I, L.parts, L.flags, in, N, n, nb, fl, F, G, x, y, z);

    // moments of the streamed offsets
    R sF = 0, sG = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const R w = wgt<R>(i);
        sF += w * F[i];
        sG += w * G[i];
        jx += w * cx(i) * F[i];
        jy += w * cy(i) * F[i];
        jz += w * cz(i) * F[i];
    }
    const R rho0 = (R)I.rho0;
    const R rr = R(1) + sF;          // rho / rho0
    const R phi = sG / rr;
    if (!(rr > R(0)) || !(phi == phi)) atomicOr(L.status, ST_UNSTABLE);

    // interface normal n = g/sqrt(|g|^2 + eps^2) and curvature (div n; solid
    // neighbours contribute this node's own normal)
    const R *GR = (const R *)L.grad;
    const long long Nt = L.Ntot;
    const R eps2 = (R)(I.grad_eps * I.grad_eps);
    const R g0 = GR[g], g1 = GR[Nt + g], g2 = GR[2 * Nt + g];
    const R ig = R(1) / sqrt(g0 * g0 + g1 * g1 + g2 * g2 + eps2);
    const R n0 = g0 * ig, n1 = g1 * ig, n2 = g2 * ig;
    R kap = 0;
    const uint8_t *fli = L.flags + I.node_off;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        long long m = nb.at(cx(i), cy(i), cz(i));
        R a0 = n0, a1 = n1, a2 = n2;
        if (!(fl & BOUND_BIT) || (fli[m] & OWNER_MASK) == OWN_FLUID) {
            long long gmn = I.node_off + m;
            R h0 = GR[gmn], h1 = GR[Nt + gmn], h2 = GR[2 * Nt + gmn];
            R ih = R(1) / sqrt(h0 * h0 + h1 * h1 + h2 * h2 + eps2);
            a0 = h0 * ih; a1 = h1 * ih; a2 = h2 * ih;
        }
        kap += wgt<R>(i) * (cx(i) * a0 + cy(i) * a1 + cz(i) * a2);
    }
    kap *= R(3);

    // force density: CSF -1/2 sigma kappa grad(phi) plus phase-weighted body forces
    const R hs = R(-0.5) * (R)I.sigma * kap;
    const R pa = R(0.5) * (R(1) + phi), pb = R(0.5) * (R(1) - phi);
    const R Fx = hs * g0 + pa * (R)I.body_a[0] + pb * (R)I.body_b[0];
    const R Fy = hs * g1 + pa * (R)I.body_a[1] + pb * (R)I.body_b[1];
    const R Fz = hs * g2 + pa * (R)I.body_a[2] + pb * (R)I.body_b[2];

    // velocity: rho u = sum c f + F/2
    const R rho = rho0 * rr;
    const R ux = (rho0 * jx + R(0.5) * Fx) / rho;
    const R uy = (rho0 * jy + R(0.5) * Fy) / rho;
    const R uz = (rho0 * jz + R(0.5) * Fz) / rho;
    if (I.store_u) { U[g] = ux; U[Nt + g] = uy; U[2 * Nt + g] = uz; }

    // relaxation rates: harmonic-mean viscosity, tau = eta/(rho cs2) + 1/2
    const R inv_eta = (R(1) + phi) / (R(2) * (R)I.eta_a) + (R(1) - phi) / (R(2) * (R)I.eta_b);
    const R tau = R(3) / (inv_eta * rho) + R(0.5);
    const R om = R(1) / tau;
    const R omp = R(8) * (R(2) - om) / (R(8) - om);
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R ir0 = R(1) / rho0;
    const R cpe = R(1) - R(0.5) * om, cpo = R(1) - R(0.5) * omp;
    const R bq = R(0.5) * (R)I.beta * rr * (R(1) - phi * phi);

    // rest population
    {
        const R feq0 = sF + rr * (R(-1.5) * uu);
        const R fb0 = R(-3) * uF * ir0;
        const R Fs = F[0] - om * (F[0] - feq0) + cpe * fb0;
        Store<S>::st(out + n, Fs);
        Store<S>::st(out + (long long)Q * N + n, phi * (R(1) + Fs));
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
        const R fbp = (R(9) * cu * cF - R(3) * uF) * ir0;
        const R fbm = R(3) * cF * ir0;
        const R fp = R(0.5) * (F[i] + F[ib]);
        const R fm = R(0.5) * (F[i] - F[ib]);
        const R dp = -om * (fp - eqp) + cpe * fbp;
        const R dm = -omp * (fm - eqm) + cpo * fbm;
        const R Fi = F[i] + dp + dm;
        const R Fib = F[ib] + dp - dm;
        // recolouring: G* = phi (1 + F*) + beta/2 (rho/rho0)(1 - phi^2) c.n/|c|
        const R inv_len = csq(i) == 1 ? R(1) : R(0.70710678118654752440);
        const R cn = (cx(i) * n0 + cy(i) * n1 + cz(i) * n2) * inv_len;
        const R rec = bq * cn;
        Store<S>::st(out + (long long)i * N + n, Fi);
        Store<S>::st(out + (long long)ib * N + n, Fib);
        Store<S>::st(out + (long long)(Q + i) * N + n, phi * (R(1) + Fi) + rec);
        Store<S>::st(out + (long long)(Q + ib) * N + n, phi * (R(1) + Fib) - rec);
    }
}

template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk)
{
    using R = typename Store<S>::real;
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

template void launch_fluid_step<double>(const Lattice &, int, cudaStream_t, long long *, const Marker &);
template void launch_fluid_step<float>(const Lattice &, int, cudaStream_t, long long *, const Marker &);
template void launch_fluid_step<__half>(const Lattice &, int, cudaStream_t, long long *, const Marker &);
template void launch_fluid_step<__nv_bfloat16>(const Lattice &, int, cudaStream_t, long long *, const Marker &);

}  // namespace lbmg
