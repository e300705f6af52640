// Per-node device functions of the fluid update (Sec. IV, V E of arXiv
// 2505.10171), shared by every launch form so that all forms run the same
// arithmetic: solid-node phi, wetting normal, grad(phi), collision + recolouring
// + write, curvature and the regularised normal.
#pragma once

#include <type_traits>
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
    // arithmetic in R: FP64 in the FP64 mode, FP32 (with the float copies of
    // the particle centres) otherwise
    int best = -1;
    R bestd = 0;
    R ws[3] = {0, 0, 0};
    bool any = false;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int own = nbr.own(cx(i), cy(i), cz(i));
        if (own == OWN_FLUID || own == OWN_PRESS) continue;  // a pressure face carries no contact angle
        any = true;
        if (own == OWN_WALL) {
            ws[0] -= wgt<R>(i) * cx(i);
            ws[1] -= wgt<R>(i) * cy(i);
            ws[2] -= wgt<R>(i) * cz(i);
        } else {
            const PartDev &P = parts[I.part_off + own - 2];
            R d0, d1, d2;
            if (sizeof(R) == 8) {
                d0 = (R)min_image(x - P.x[0], I.nx); d1 = (R)min_image(y - P.x[1], I.ny);
                d2 = (R)min_image(z - P.x[2], I.nz);
            } else {
                d0 = (R)min_image_f((float)x - P.xf[0], I.nx); d1 = (R)min_image_f((float)y - P.xf[1], I.ny);
                d2 = (R)min_image_f((float)z - P.xf[2], I.nz);
            }
            const R dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - (R)P.R;
            const int p = own - 2;
            if (best < 0 || dist < bestd || (dist == bestd && p < best)) {
                best = p;
                bestd = dist;
            }
        }
    }
    if (!any) return false;
    if (best >= 0) {
        const PartDev &P = parts[I.part_off + best];
        R d0, d1, d2;
        if (sizeof(R) == 8) {
            d0 = (R)min_image(x - P.x[0], I.nx); d1 = (R)min_image(y - P.x[1], I.ny);
            d2 = (R)min_image(z - P.x[2], I.nz);
        } else {
            d0 = (R)min_image_f((float)x - P.xf[0], I.nx); d1 = (R)min_image_f((float)y - P.xf[1], I.ny);
            d2 = (R)min_image_f((float)z - P.xf[2], I.nz);
        }
        const R dl = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        ns[0] = d0 / dl; ns[1] = d1 / dl; ns[2] = d2 / dl;
        *cth = (R)P.cos_t;
        *sth = (R)P.sin_t;
        return true;
    }
    const R wl = sqrt(ws[0] * ws[0] + ws[1] * ws[1] + ws[2] * ws[2]);
    if (wl == R(0)) return false;
    ns[0] = ws[0] / wl; ns[1] = ws[1] / wl; ns[2] = ws[2] / wl;
    *cth = (R)I.cos_tw;
    *sth = (R)I.sin_tw;
    return true;
}

// grad(phi) = 3 sum_i w_i c_i phi(x + c_i)
template <class R, class PhiF>
__device__ __forceinline__ void grad_sum(const PhiF &phi_of, R *gr)
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
}

// the wetting rotation of grad(phi) at boundary nodes inside the interface
template <class R, class A>
__device__ __forceinline__ void grad_wet(const InstDev &I, const PartDev *parts, const A &nbr, R phi_here,
                                         uint8_t fl, R wet_max, int x, int y, int z, R *gr)
{
    if ((fl & BOUND_BIT) && fabs(phi_here) < wet_max) {
        R ns[3], cth, sth;
        if (solid_normal<R>(I, parts, nbr, x, y, z, ns, &cth, &sth)) wetting_rotate<R>(gr, ns, cth, sth);
    }
}

// both
template <class R, class A, class PhiF>
__device__ __forceinline__ void grad_node(const InstDev &I, const PartDev *parts, const A &nbr, const PhiF &phi_of,
                                          R phi_here, uint8_t fl, R wet_max, int x, int y, int z, R *gr)
{
    grad_sum<R>(phi_of, gr);
    grad_wet<R>(I, parts, nbr, phi_here, fl, wet_max, x, y, z, gr);
}

// the node's state before the per-direction updates of the collision
template <class R>
struct CollideState {
    R sF, rr, ux, uy, uz, Fx, Fy, Fz, om, omp, uu, uF, cpe, cpo, bq;
};

template <class R>
__device__ __forceinline__ CollideState<R> collide_state(const FluidPar<R> &P, const R *F, R phi, const R *g, R kap)
{
    CollideState<R> c;
    R sF = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const R w = wgt<R>(i);
        sF += w * F[i];
        if (cx(i)) jx += w * cx(i) * F[i];
        if (cy(i)) jy += w * cy(i) * F[i];
        if (cz(i)) jz += w * cz(i) * F[i];
    }
    c.sF = sF;
    c.rr = R(1) + sF;  // rho / rho0
    // force density: CSF -1/2 sigma kappa grad(phi) plus phase-weighted body forces
    const R hs = R(-0.5) * P.sigma * kap;
    const R pa = R(0.5) * (R(1) + phi), pb = R(0.5) * (R(1) - phi);
    c.Fx = hs * g[0] + pa * P.ba[0] + pb * P.bb[0];
    c.Fy = hs * g[1] + pa * P.ba[1] + pb * P.bb[1];
    c.Fz = hs * g[2] + pa * P.ba[2] + pb * P.bb[2];
    // velocity: rho u = sum c f + F/2
    const R rho = P.rho0 * c.rr;
    const R irho = frcp(rho);
    c.ux = (P.rho0 * jx + R(0.5) * c.Fx) * irho;
    c.uy = (P.rho0 * jy + R(0.5) * c.Fy) * irho;
    c.uz = (P.rho0 * jz + R(0.5) * c.Fz) * irho;
    // relaxation rates: harmonic-mean viscosity, tau = eta/(rho cs2) + 1/2
    const R inv_eta = (R(1) + phi) * P.h_ia + (R(1) - phi) * P.h_ib;
    const R tau = R(3) * frcp(inv_eta * rho) + R(0.5);
    c.om = frcp(tau);
    c.omp = R(8) * (R(2) - c.om) * frcp(R(8) - c.om);
    c.uu = c.ux * c.ux + c.uy * c.uy + c.uz * c.uz;
    c.uF = c.ux * c.Fx + c.uy * c.Fy + c.uz * c.Fz;
    c.cpe = R(1) - R(0.5) * c.om;
    c.cpo = R(1) - R(0.5) * c.omp;
    c.bq = R(0.5) * P.beta * c.rr * (R(1) - phi * phi);
    return c;
}

// post-collision rest population
template <class R>
__device__ __forceinline__ R collide_rest(const FluidPar<R> &P, const CollideState<R> &c, R F0)
{
    const R feq0 = c.sF + c.rr * (R(-1.5) * c.uu);
    const R fb0 = R(-3) * c.uF * P.ir0;
    return F0 - c.om * (F0 - feq0) + c.cpe * fb0;
}

// opposite pair (i, i+9): the paper's S relaxes every even non-conserved
// moment with omega and every odd one with omega', i.e. the MRT operator is
// exactly the two-relaxation-time operator on the pair's even/odd parts.
// Returns F*_i and F*_ib.
template <class R, int i>
__device__ __forceinline__ void collide_pair(const FluidPar<R> &P, const CollideState<R> &c, R Fi_in, R Fib_in,
                                             R &Fi, R &Fib)
{
    const R cu = cx(i) * c.ux + cy(i) * c.uy + cz(i) * c.uz;
    const R cF = cx(i) * c.Fx + cy(i) * c.Fy + cz(i) * c.Fz;
    const R eqp = c.sF + c.rr * (R(4.5) * cu * cu - R(1.5) * c.uu);
    const R eqm = c.rr * R(3) * cu;
    const R fbp = (R(9) * cu * cF - R(3) * c.uF) * P.ir0;
    const R fbm = R(3) * cF * P.ir0;
    const R fp = R(0.5) * (Fi_in + Fib_in);
    const R fm = R(0.5) * (Fi_in - Fib_in);
    const R dp = -c.om * (fp - eqp) + c.cpe * fbp;
    const R dm = -c.omp * (fm - eqm) + c.cpo * fbm;
    Fi = Fi_in + dp + dm;
    Fib = Fib_in + dp - dm;
}

template <class R, int i = 1>
struct PairLoop {
    template <class Fn>
    __device__ __forceinline__ static void run(Fn &&f)
    {
        f(std::integral_constant<int, i>());
        PairLoop<R, i + 1>::run(f);
    }
};
template <class R>
struct PairLoop<R, 10> {
    template <class Fn>
    __device__ __forceinline__ static void run(Fn &&) {}
};

// force, velocity, MRT (two-relaxation-time form) with Guo forcing (Sec. IV),
// recolouring and the write of node n.  F: streamed total offsets; phi: the
// order parameter after streaming (stored by the order-parameter pass); g:
// corrected grad(phi) of the node; nn: its regularised normal; kap: curvature.
// The recolouring of Sec. IV gives G*_i = phi (1 + F*_i) + b (c_i . n)/|c_i|
// with b = beta/2 (rho/rho0)(1 - phi^2): the state is complete with F* and
// the colour record (phi, b n), which are written (C).
template <class S>
__device__ __forceinline__ void collide_store_phi(const FluidPar<typename Store<S>::real> &P,
                                                  const typename Store<S>::real *F, typename Store<S>::real phi,
                                                  const typename Store<S>::real *g, const typename Store<S>::real *nn,
                                                  typename Store<S>::real kap, const Pop<S> &out, int n,
                                                  const ColSlotOf<S> &C, typename Store<S>::real *U,
                                                  long long Ustride, unsigned *status)
{
    using R = typename Store<S>::real;
    using FT = typename Pop<S>::FT;
    const int N = out.N;
    FT *const of = out.f + n;  // F_0 of this node; F_i at of + i N
    const CollideState<R> c = collide_state(P, F, phi, g, kap);
    if (status && (!(c.rr > R(0)) || !(phi == phi))) atomicOr(status, ST_UNSTABLE);
    if (U) { U[n] = c.ux; U[Ustride + n] = c.uy; U[2 * Ustride + n] = c.uz; }
    C.set(ColRec<R>{phi, c.bq * nn[0], c.bq * nn[1], c.bq * nn[2]});
    Store<FT>::st(of, collide_rest(P, c, F[0]));
    PairLoop<R>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value, ib = i + 9;
        R Fi, Fib;
        collide_pair<R, i>(P, c, F[i], F[ib], Fi, Fib);
        Store<FT>::st(of + i * N, Fi);
        Store<FT>::st(of + ib * N, Fib);
    });
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

}  // namespace lbmg
