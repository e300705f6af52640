// Particle kernels of one coupled time step (Sec. III and V of arXiv 2505.10171):
//   k_mem        momentum-exchange force and torque per particle (Sec. V B)
//   k_capillary  capillary force and torque from the Lagrangian surface points
//                (Sec. V F)
//   k_dem        fixed-order sums of the per-block partials of both, then
//                contacts (normal spring-dashpot, Luding sliding and rolling
//                friction) and velocity-Verlet update (Sec. III): one warp per
//                particle for the sums, one thread per contact, then one per
//                particle; positions and velocities FP64, contact arithmetic
//                FP64 in the FP64 mode and FP32 otherwise
//   k_geom_*     solid map update and refilling of uncovered nodes (Sec. V C)
// Per-link and per-point arithmetic runs in the storage precision's arithmetic
// type (double for FP64 storage, float otherwise); every sum over links,
// points or contacts is FP64 with a fixed order (warp shuffle, block tree,
// fixed block order), so results are reproducible run to run.  GB300 executes
// double precision at a small fraction of the single-precision rate, so the
// FP64 work is kept to the sums and the DEM.
#include "lbm_internal.cuh"

namespace lbmg {

// deterministic block sum of 6 doubles; thread 0 writes them to out
template <int K, class T>
__device__ __forceinline__ void block_sum(T *v, double *out)
{
    __shared__ T sm[PART_THREADS / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < K; a++)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    if (lane == 0)
        for (int a = 0; a < K; a++) sm[wid][a] = v[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < K; a++) {
            T s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sm[w][a];
            out[a] = (double)s;
        }
    }
    __syncthreads();  // sm is reused by a second call
}

template <class T>
__device__ __forceinline__ void block_sum6(T *v, double *out) { block_sum<6>(v, out); }

// particle centre in the arithmetic type R (single-precision copy for float)
__device__ __forceinline__ void centre(const PartDev &P, double *c) { c[0] = P.x[0]; c[1] = P.x[1]; c[2] = P.x[2]; }
__device__ __forceinline__ void centre(const PartDev &P, float *c) { c[0] = P.xf[0]; c[1] = P.xf[1]; c[2] = P.xf[2]; }

template <class R>
__device__ __forceinline__ R min_image_r(R d, int n)
{
    const R h = R(0.5) * n;
    return d >= h ? d - n : (d < -h ? d + n : d);
}

// Sec. V B momentum exchange (Wen 2014, Galilean invariant): per link from a
// fluid node x into particle p, force on p = (c_out - u_w) f_out - (c_in - u_w) f_in
// with f_out = f*_ibar(x) leaving towards the solid and f_in = f_i(x) bounced
// back; torque lever from the centre to the link midpoint.
//
// With f_out = w rho0 (1 + F), f_in = w rho0 (1 + F + 6 rr c.u_w) the link
// term is -2 w rho0 c (the rest part, order 0.1, cancelling over the closed
// surface) plus w rho0 (-c (2F + 6 rr c.u_w) + u_w 6 rr c.u_w) (order 1e-4).
// Rounding the sum in single precision would swamp the offsets, and FP64
// arithmetic per link is slow on this GPU, so the rest part is kept exactly in
// integers: with k = 36 w in {1, 2} and the lever d - delta, d the half-integer
// offset of the link midpoint from the integer point xr = floor(x_p), delta =
// x_p - xr, its force is -(rho0/18) K and its torque -(rho0/18) (M - delta x K)
// with K = sum k c and M = sum k d x c. The block partials hold the small
// part's force and torque, K and 2M; the DEM kernel assembles them in FP64.
template <class S>
__global__ void __launch_bounds__(PART_THREADS) k_mem(Lattice L, int cur)
{
    using R = typename Store<S>::real;
    const int p = blockIdx.y;
    const PartDev &P = L.parts[p];
    const InstDev &I = L.inst[P.inst];
    Region reg;
    reg.init(P.x, P.mem_side, I.nx, I.ny, I.nz);
    R acc[6] = {0, 0, 0, 0, 0, 0};
    int kin[6] = {0, 0, 0, 0, 0, 0};  // K, then 2M
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < reg.count()) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        const int n = (z * I.ny + y) * I.nx + x;
        const uint8_t *fli = L.flags + I.node_off;
        const uint8_t fl = fli[n];
        if ((fl & OWNER_MASK) == OWN_FLUID && (fl & BOUND_BIT)) {
            const Pop<S> in(L.pop[cur], I);
            Nbr nb;
            nb.init(x, y, z, I.nx, I.ny, I.nz);
            const int mine = 2 + P.local;
            // twice the node's offset from xr, minimum image (|.| < n)
            const int xr[3] = {(int)floor(P.x[0]), (int)floor(P.x[1]), (int)floor(P.x[2])};
            const int per[3] = {I.nx, I.ny, I.nz};
            const int pos[3] = {x, y, z};
            int D0[3];
            for (int a = 0; a < 3; a++) {
                int d = 2 * (pos[a] - xr[a]);
                d += d >= per[a] ? -2 * per[a] : (d < -per[a] ? 2 * per[a] : 0);
                D0[a] = d;
            }
            R rr = -1;
            R c[3], v[3], w[3];
            centre(P, c);
            for (int a = 0; a < 3; a++) { v[a] = (R)P.v[a]; w[a] = (R)P.w[a]; }
            const R r0 = (R)I.rho0;
            for (int i = 1; i < Q; i++) {
                if ((fli[nb.at(-cx(i), -cy(i), -cz(i))] & OWNER_MASK) != mine) continue;
                if (rr < R(0)) {
                    R sF = 0;
                    for (int j = 0; j < Q; j++) sF += wgt<R>(j) * in.F(j, n);
                    rr = R(1) + sF;
                }
                const int ci[3] = {cx(i), cy(i), cz(i)};
                const R lev[3] = {min_image_r<R>(x - R(0.5) * ci[0] - c[0], I.nx),
                                  min_image_r<R>(y - R(0.5) * ci[1] - c[1], I.ny),
                                  min_image_r<R>(z - R(0.5) * ci[2] - c[2], I.nz)};
                const R uw[3] = {v[0] + (w[1] * lev[2] - w[2] * lev[1]), v[1] + (w[2] * lev[0] - w[0] * lev[2]),
                                 v[2] + (w[0] * lev[1] - w[1] * lev[0])};
                const R wt = wgt<R>(i) * r0;
                const R Fo = in.F(opp(i), n);
                const R cu = ci[0] * uw[0] + ci[1] * uw[1] + ci[2] * uw[2];
                const R e = R(6) * rr * cu;
                const R q = R(2) * Fo + e;
                R dp[3];
                for (int a = 0; a < 3; a++) dp[a] = wt * (uw[a] * e - ci[a] * q);
                acc[0] += dp[0];
                acc[1] += dp[1];
                acc[2] += dp[2];
                acc[3] += lev[1] * dp[2] - lev[2] * dp[1];
                acc[4] += lev[2] * dp[0] - lev[0] * dp[2];
                acc[5] += lev[0] * dp[1] - lev[1] * dp[0];
                // rest part: k c and k (2d) x c, 2d = D0 - c
                const int k = csq(i) == 1 ? 2 : 1;
                const int D[3] = {D0[0] - ci[0], D0[1] - ci[1], D0[2] - ci[2]};
                kin[0] += k * ci[0];
                kin[1] += k * ci[1];
                kin[2] += k * ci[2];
                kin[3] += k * (D[1] * ci[2] - D[2] * ci[1]);
                kin[4] += k * (D[2] * ci[0] - D[0] * ci[2]);
                kin[5] += k * (D[0] * ci[1] - D[1] * ci[0]);
            }
        }
    }
    double *out = L.mem_part + ((long long)p * L.mem_blocks + blockIdx.x) * MEM_PART;
    double accd[6];
    for (int a = 0; a < 6; a++) accd[a] = (double)acc[a];
    block_sum6(accd, out);
    block_sum6(kin, out + 6);
}

// Sec. V F: dF = C sigma (1 - phi^2) dA (n x n_s) x n at the points
// alpha_j = (j + 1/2) 2 deg, varphi_k = k 2 deg on r = R_p, n the regularised
// normal of the trilinearly interpolated grad(phi) (fluid corners only);
// torque R_p n_s x dF.  With BUOY also the phase-a share of the surface for
// the buoyancy (reading c28): s = (1 + phi)/2 clipped to [0, 1] and dA, summed
// over the points with a fluid corner.
template <class R, bool BUOY>
__global__ void __launch_bounds__(CAP_THREADS) k_capillary(Lattice L)
{
    const int p = blockIdx.y;
    const PartDev &P = L.parts[p];
    const InstDev &I = L.inst[P.inst];
    double acc[CAP_PART] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt < CAP_POINTS) {
        const double *tp = L.cap_pts + 4 * pt;
        const R ns[3] = {(R)tp[0], (R)tp[1], (R)tp[2]};
        const R sa = (R)tp[3];
        const R da = R(2.0 * M_PI / 180.0);
        R c[3];
        centre(P, c);
        const R Rp = (R)P.R;
        const R xi[3] = {c[0] + Rp * ns[0], c[1] + Rp * ns[1], c[2] + Rp * ns[2]};
        const R dA = Rp * Rp * sa * da * da;
        int b[3];
        R fr[3];
        for (int a = 0; a < 3; a++) {
            const R fl = floor(xi[a]);
            b[a] = (int)fl;
            fr[a] = xi[a] - fl;
        }
        const int n3[3] = {I.nx, I.ny, I.nz};
        const uint8_t *fli = L.flags + I.node_off;
        const R *ph = (const R *)L.phi + I.node_off;
        const R *Gn = (const R *)L.grad + I.node_off;   // regularised normal
        const R *Gm = (const R *)L.gmag + I.node_off;   // its norm: grad phi = n gmag
        R ws = 0, phs = 0, gs[3] = {0, 0, 0};
        for (int cz_ = 0; cz_ < 2; cz_++)
            for (int cy_ = 0; cy_ < 2; cy_++)
                for (int cx_ = 0; cx_ < 2; cx_++) {
                    int X = b[0] + cx_, Y = b[1] + cy_, Z = b[2] + cz_;
                    X = X < 0 ? X + n3[0] : (X >= n3[0] ? X - n3[0] : X);
                    Y = Y < 0 ? Y + n3[1] : (Y >= n3[1] ? Y - n3[1] : Y);
                    Z = Z < 0 ? Z + n3[2] : (Z >= n3[2] ? Z - n3[2] : Z);
                    const long long m = ((long long)Z * I.ny + Y) * I.nx + X;
                    if ((fli[m] & OWNER_MASK) != OWN_FLUID) continue;
                    const R wgt_ = (cx_ ? fr[0] : R(1) - fr[0]) * (cy_ ? fr[1] : R(1) - fr[1]) *
                                   (cz_ ? fr[2] : R(1) - fr[2]);
                    const R mg = Gm[m];
                    ws += wgt_;
                    phs += wgt_ * ph[m];
                    gs[0] += wgt_ * (Gn[m] * mg);
                    gs[1] += wgt_ * (Gn[L.Ntot + m] * mg);
                    gs[2] += wgt_ * (Gn[2 * L.Ntot + m] * mg);
                }
        if (ws > R(0)) {
            const R phv = phs / ws;
            if (BUOY) {
                const R sa = fmin(fmax(R(0.5) * (R(1) + phv), R(0)), R(1));
                acc[6] = (double)(sa * dA);
                acc[7] = (double)dA;
            }
            const R g0 = gs[0] / ws, g1 = gs[1] / ws, g2 = gs[2] / ws;
            if (fabs(phv) < R(1)) {
                const R eps2 = (R)(I.grad_eps * I.grad_eps);
                const R gr = sqrt(g0 * g0 + g1 * g1 + g2 * g2 + eps2);
                const R nn[3] = {g0 / gr, g1 / gr, g2 / gr};
                const R c0 = nn[1] * ns[2] - nn[2] * ns[1], c1 = nn[2] * ns[0] - nn[0] * ns[2],
                        c2 = nn[0] * ns[1] - nn[1] * ns[0];
                const R mv[3] = {c1 * nn[2] - c2 * nn[1], c2 * nn[0] - c0 * nn[2], c0 * nn[1] - c1 * nn[0]};
                const R coef = (R)(I.cap_norm * I.sigma) * (R(1) - phv * phv) * dA;
                R dF[3];
                for (int a = 0; a < 3; a++) dF[a] = coef * mv[a];
                const R r[3] = {Rp * ns[0], Rp * ns[1], Rp * ns[2]};
                acc[0] = (double)dF[0];
                acc[1] = (double)dF[1];
                acc[2] = (double)dF[2];
                acc[3] = (double)(r[1] * dF[2] - r[2] * dF[1]);
                acc[4] = (double)(r[2] * dF[0] - r[0] * dF[2]);
                acc[5] = (double)(r[0] * dF[1] - r[1] * dF[0]);
            }
        }
    }
    block_sum<BUOY ? 8 : 6>(acc, L.cap_part + ((long long)p * CAP_BLOCKS + blockIdx.x) * CAP_PART);
}


// ---------------------------------------------------------------------------
// DEM (Sec. III).  Positions, velocities, spring histories and the Verlet
// sums are FP64; the contact arithmetic runs in T: double in the FP64 mode,
// float otherwise (FP64 issues at a small fraction of the FP32 rate here and
// the DEM is one serial chain of dependent operations).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T dot3(const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T>
__device__ __forceinline__ void cross3(const T *a, const T *b, T *r)
{
    T t0 = a[1] * b[2] - a[2] * b[1], t1 = a[2] * b[0] - a[0] * b[2], t2 = a[0] * b[1] - a[1] * b[0];
    r[0] = t0; r[1] = t1; r[2] = t2;
}

// Luding spring: project on the tangent plane, trial force, Coulomb cap,
// spring update (static: xi += v dt; sliding: xi = -(F + gamma v)/k).
template <class T>
__device__ void dem_spring(T *xi, const T *n, const T *v, T k, T gam, T FC, T *F)
{
    T xn = dot3(xi, n);
    for (int a = 0; a < 3; a++) xi[a] -= xn * n[a];
    T F0[3];
    for (int a = 0; a < 3; a++) F0[a] = -k * xi[a] - gam * v[a];
    T m = sqrt(dot3(F0, F0));
    if (m <= FC) {
        for (int a = 0; a < 3; a++) { F[a] = F0[a]; xi[a] += v[a]; }
    } else {
        for (int a = 0; a < 3; a++) F[a] = FC * F0[a] / m;
        for (int a = 0; a < 3; a++) xi[a] = k > T(0) ? -(F[a] + gam * v[a]) / k : T(0);
    }
}

// contact of particle i with partner j (j < 0: substrate); n from partner to
// i, delta > 0 the overlap.  Contact point X_i - (R_c,i - delta/2) n;
// F_n = [k_n delta - g_n v_rel.n] n; rolling velocity -a'(w_i - w_j) x n with
// torque -a' n x F_r on i (+a' n x F_r on j).  rec receives the force and
// torque on i, then on j.
template <class T>
__device__ void dem_contact(const InstDev &I, const PartDev *P, int i, int j, const T *vp, const T *wp, const T *n,
                            T delta, T *xi, T *xir, T *rec)
{
    const T Rci = (T)P[i].Rc;
    T bi[3], bj[3] = {0, 0, 0}, t[3], vi[3], vj[3];
    for (int a = 0; a < 3; a++) bi[a] = -(Rci - T(0.5) * delta) * n[a];
    cross3(wp + 3 * i, bi, t);
    for (int a = 0; a < 3; a++) vi[a] = vp[3 * i + a] + t[a];
    T ap;
    if (j >= 0) {
        const T Rcj = (T)P[j].Rc;
        for (int a = 0; a < 3; a++) bj[a] = (Rcj - T(0.5) * delta) * n[a];
        cross3(wp + 3 * j, bj, t);
        for (int a = 0; a < 3; a++) vj[a] = vp[3 * j + a] + t[a];
        ap = Rci * Rcj / (Rci + Rcj);
    } else {
        for (int a = 0; a < 3; a++) vj[a] = (T)I.wall_u[a];
        ap = Rci;
    }
    T vr[3];
    for (int a = 0; a < 3; a++) vr[a] = vi[a] - vj[a];
    const T vn = dot3(vr, n);
    const T Fnm = (T)I.kn * delta - (T)I.gn * vn;
    T vt[3];
    for (int a = 0; a < 3; a++) vt[a] = vr[a] - vn * n[a];
    T Ft[3];
    dem_spring(xi, n, vt, (T)I.kt, (T)I.gt, (T)I.mu_s * fabs(Fnm), Ft);
    T wrel[3], vrl[3];
    for (int a = 0; a < 3; a++) wrel[a] = wp[3 * i + a] - (j >= 0 ? wp[3 * j + a] : T(0));
    cross3(wrel, n, vrl);
    for (int a = 0; a < 3; a++) vrl[a] *= -ap;
    T Fr[3];
    dem_spring(xir, n, vrl, (T)I.kr, (T)I.gr, (T)I.mu_r * fabs(Fnm), Fr);
    T Tt[3], Tr[3];
    cross3(bi, Ft, Tt);
    cross3(n, Fr, Tr);
    T mFt[3] = {-Ft[0], -Ft[1], -Ft[2]}, Ttj[3];
    cross3(bj, mFt, Ttj);
    for (int a = 0; a < 3; a++) {
        rec[a] = Fnm * n[a] + Ft[a];
        rec[3 + a] = Tt[a] - ap * Tr[a];
        rec[6 + a] = -(Fnm * n[a] + Ft[a]);
        rec[9 + a] = Ttj[a] + ap * Tr[a];
    }
}

// orientation: exact rotation by |w| about w (unit quaternion, FP64 storage)
template <class T>
__device__ void quat_rotate(double *q, const T *w)
{
    T wm = sqrt(dot3(w, w));
    if (wm == T(0)) return;
    T h = T(0.5) * wm, s = sin(h) / wm;
    T d0 = cos(h), d1 = s * w[0], d2 = s * w[1], d3 = s * w[2];
    T q0 = (T)q[0], q1 = (T)q[1], q2 = (T)q[2], q3 = (T)q[3];
    T r0 = d0 * q0 - d1 * q1 - d2 * q2 - d3 * q3;
    T r1 = d0 * q1 + d1 * q0 + d2 * q3 - d3 * q2;
    T r2 = d0 * q2 - d1 * q3 + d2 * q0 + d3 * q1;
    T r3 = d0 * q3 + d1 * q2 - d2 * q1 + d3 * q0;
    T l = sqrt(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    q[0] = r0 / l; q[1] = r1 / l; q[2] = r2 / l; q[3] = r3 / l;
}

constexpr int DEM_MAXP = 61;
constexpr int DEM_THREADS = 256;  // a warp per particle for the fluid sums of up to 8 particles at once

// pair index c in [0, np(np-1)/2) -> (i, j), i < j, lexicographic
__device__ __forceinline__ void pair_of(int c, int np, int *i, int *j)
{
    int a = 0;
    while (c >= np - 1 - a) {
        c -= np - 1 - a;
        a++;
    }
    *i = a;
    *j = a + 1 + c;
}

__device__ __forceinline__ int pair_index(int i, int j, int np) { return i * np - i * (i + 1) / 2 + (j - i - 1); }

// one block per instance.  Velocity-Verlet predictor per particle; contact
// forces one thread per contact (substrate contacts, then pairs), kept per
// contact; corrector per particle, adding its contacts in a fixed order
// (substrate, then partners in increasing index).
template <class T, bool BUOY>
__global__ void __launch_bounds__(DEM_THREADS) k_dem(Lattice L, int sum_fluid)
{
    const InstDev &I = L.inst[blockIdx.x];
    const int np = I.np;
    if (np == 0) return;
    PartDev *P = L.parts + I.part_off;
    double *hist = L.hist + (long long)I.hist_off * 6;
    double *rec = L.crec + (long long)I.crec_off * 12;
    __shared__ double xn[3 * DEM_MAXP];
    __shared__ T vp[3 * DEM_MAXP], wp[3 * DEM_MAXP];
    const int tid = threadIdx.x;
    if (sum_fluid) {
        // fluid forces of this step: a warp per particle sums the block
        // partials of the momentum-exchange and capillary kernels, lanes over
        // a fixed block stride, then a fixed shuffle tree (deterministic)
        const int lane = tid & 31, wid = tid >> 5;
        for (int p = wid; p < np; p += DEM_THREADS / 32) {
            const long long pg = I.part_off + p;
            constexpr int NC = BUOY ? CAP_PART : 6;  // capillary partials used
            double s[12 + NC];
            for (int a = 0; a < 12 + NC; a++) s[a] = 0.0;
            for (int b = lane; b < L.mem_blocks; b += 32)
                for (int a = 0; a < MEM_PART; a++) s[a] += L.mem_part[(pg * L.mem_blocks + b) * MEM_PART + a];
            for (int b = lane; b < CAP_BLOCKS; b += 32)
                for (int a = 0; a < NC; a++) s[12 + a] += L.cap_part[(pg * CAP_BLOCKS + b) * CAP_PART + a];
            for (int o = 16; o > 0; o >>= 1)
                for (int a = 0; a < 12 + NC; a++) s[a] += __shfl_down_sync(0xffffffffu, s[a], o);
            if (lane == 0) {
                // momentum exchange: small part plus the exact rest part
                // -(rho0/18) K, -(rho0/18) (M - delta x K), M = (2M)/2
                const double g = -I.rho0 / 18.0;
                double dl[3], K[3], M[3];
                for (int a = 0; a < 3; a++) {
                    dl[a] = P[p].x[a] - floor(P[p].x[a]);
                    K[a] = s[6 + a];
                    M[a] = 0.5 * s[9 + a];
                }
                const double dK[3] = {dl[1] * K[2] - dl[2] * K[1], dl[2] * K[0] - dl[0] * K[2],
                                      dl[0] * K[1] - dl[1] * K[0]};
                for (int a = 0; a < 3; a++) {
                    P[p].Feta[a] = s[a] + g * K[a];
                    P[p].Teta[a] = s[3 + a] + g * (M[a] - dK[a]);
                    P[p].Fsig[a] = s[12 + a];
                    P[p].Tsig[a] = s[15 + a];
                }
                // buoyancy (reading c28): a flat interface at height h = (2a - 1) R
                // above the centre leaves the volume fraction (1 + t)^2 (2 - t)/4,
                // t = h/R, of the sphere below it (a spherical zone's area is
                // proportional to its height)
                if constexpr (BUOY) {
                    double sub = 0.0;
                    if (s[19] > 0.0) {
                        const double t = 2.0 * (s[18] / s[19]) - 1.0;
                        sub = (1.0 + t) * (1.0 + t) * (2.0 - t) / 4.0;
                    }
                    const double vol = 4.0 / 3.0 * M_PI * P[p].R * P[p].R * P[p].R;
                    P[p].sub = sub;
                    for (int a = 0; a < 3; a++) P[p].Fb[a] = vol * sub * I.buoy[a];
                }
            }
        }
        __syncthreads();
    }
    for (int p = tid; p < np; p += blockDim.x)
        for (int a = 0; a < 3; a++) {
            if (P[p].kin) {
                xn[3 * p + a] = P[p].x[a] + P[p].v[a];
                vp[3 * p + a] = (T)P[p].v[a];
                wp[3 * p + a] = (T)P[p].w[a];
            } else {
                const double acc = P[p].Fp[a] * P[p].inv_m, alp = P[p].Tp[a] * P[p].inv_I;
                xn[3 * p + a] = P[p].x[a] + P[p].v[a] + 0.5 * acc;
                vp[3 * p + a] = (T)(P[p].v[a] + acc);
                wp[3 * p + a] = (T)(P[p].w[a] + alp);
            }
        }
    __syncthreads();
    const int npair = np * (np - 1) / 2;
    for (int c = tid; c < np + npair; c += blockDim.x) {
        double *r = rec + 12 * c;
        T rt[12];
        for (int a = 0; a < 12; a++) rt[a] = T(0);
        double *hs;
        T xi[6];
        bool touch = false;
        if (c < np) {
            // particle-substrate contact, delta = R_c - (z_p - 0.5); history record c
            const int p = c;
            hs = hist + 6 * p;
            for (int a = 0; a < 6; a++) xi[a] = (T)hs[a];
            const double delta = P[p].Rc - (xn[3 * p + 2] - 0.5);
            if (I.wall_z0 && delta > 0.0) {
                const T n[3] = {T(0), T(0), T(1)};
                dem_contact<T>(I, P, p, -1, vp, wp, n, (T)delta, xi, xi + 3, rt);
                touch = true;
            }
        } else {
            // particle pair, delta_ij = R_c,i + R_c,j - |X_i - X_j|; history record np + i*np + j
            int i, j;
            pair_of(c - np, np, &i, &j);
            hs = hist + 6 * (np + i * np + j);
            for (int a = 0; a < 6; a++) xi[a] = (T)hs[a];
            const double d[3] = {min_image(xn[3 * i] - xn[3 * j], I.nx), min_image(xn[3 * i + 1] - xn[3 * j + 1], I.ny),
                                 min_image(xn[3 * i + 2] - xn[3 * j + 2], I.nz)};
            const double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double delta = P[i].Rc + P[j].Rc - dl;
            if (delta > 0.0 && dl > 0.0) {
                const T n[3] = {(T)(d[0] / dl), (T)(d[1] / dl), (T)(d[2] / dl)};
                dem_contact<T>(I, P, i, j, vp, wp, n, (T)delta, xi, xi + 3, rt);
                touch = true;
            }
        }
        for (int a = 0; a < 6; a++) hs[a] = touch ? (double)xi[a] : 0.0;
        for (int a = 0; a < 12; a++) r[a] = (double)rt[a];
    }
    __syncthreads();
    for (int p = tid; p < np; p += blockDim.x) {
        double Fc[3] = {0, 0, 0}, Tc[3] = {0, 0, 0};
        const double *r = rec + 12 * p;
        for (int a = 0; a < 3; a++) { Fc[a] += r[a]; Tc[a] += r[3 + a]; }
        for (int q = 0; q < np; q++) {
            if (q == p) continue;
            const double *rp = rec + 12 * (np + (q < p ? pair_index(q, p, np) : pair_index(p, q, np)));
            const int off = q < p ? 6 : 0;  // p is the second member of (q, p)
            for (int a = 0; a < 3; a++) { Fc[a] += rp[off + a]; Tc[a] += rp[off + 3 + a]; }
        }
        PartDev &Q_ = P[p];
        double F[3], Tq[3], wold[3];
        for (int a = 0; a < 3; a++) {
            Q_.Fc[a] = Fc[a];
            Q_.Tc[a] = Tc[a];
            F[a] = Fc[a] + I.g_part[a] + Q_.Feta[a] + Q_.Fsig[a] + Q_.Fb[a];
            Tq[a] = Tc[a] + Q_.Teta[a] + Q_.Tsig[a];
            wold[a] = Q_.w[a];
            Q_.x_old[a] = Q_.x[a];
            Q_.xfo[a] = Q_.xf[a];
        }
        if (!Q_.kin)
            for (int a = 0; a < 3; a++) {
                Q_.v[a] += 0.5 * (Q_.Fp[a] + F[a]) * Q_.inv_m;
                Q_.w[a] += 0.5 * (Q_.Tp[a] + Tq[a]) * Q_.inv_I;
            }
        const T wm[3] = {(T)(0.5 * (wold[0] + Q_.w[0])), (T)(0.5 * (wold[1] + Q_.w[1])),
                         (T)(0.5 * (wold[2] + Q_.w[2]))};
        quat_rotate<T>(Q_.q, wm);
        // the geometry kernels assume a move below the margin: a larger or
        // non-finite one sets the status and leaves the particle where it was
        // (the run is reported unstable), so that nothing indexes with it
        bool ok = true;
        for (int a = 0; a < 3; a++) ok = ok && fabs(xn[3 * p + a] - Q_.x[a]) < GEOM_MARGIN - 1;
        if (!ok) atomicOr(L.status, ST_DISPLACEMENT);
        const int per[3] = {I.nx, I.ny, I.nz};
        for (int a = 0; a < 3; a++) {
            // periodic domain: positions kept in [0, n)
            if (ok) Q_.x[a] = xn[3 * p + a] - per[a] * floor(xn[3 * p + a] / per[a]);
            Q_.xf[a] = (float)Q_.x[a];
            Q_.Fp[a] = F[a];
            Q_.Tp[a] = Tq[a];
        }
    }
}

// ---------------------------------------------------------------------------
// Geometry update and refilling (Sec. V C)
// ---------------------------------------------------------------------------
// owner of node (x,y,z) for the particle positions `which` (0: current, 1:
// previous): |x - x_p|^2 < R_p^2, decided in single precision when clear of
// the sphere surface by a margin and in double precision otherwise
__device__ __forceinline__ int particle_owner(const InstDev &I, const PartDev *parts, int x, int y, int z, int which)
{
    for (int p = 0; p < I.np; p++) {
        const PartDev &P = parts[I.part_off + p];
        const float *cf = which ? P.xfo : P.xf;
        const float e0 = min_image_r<float>((float)x - cf[0], I.nx);
        const float e1 = min_image_r<float>((float)y - cf[1], I.ny);
        const float e2 = min_image_r<float>((float)z - cf[2], I.nz);
        const float d2 = e0 * e0 + e1 * e1 + e2 * e2;
        if (d2 > P.R2hi) continue;
        if (d2 < P.R2lo) return 2 + p;
        const double *c = which ? P.x_old : P.x;
        const double d0 = min_image(x - c[0], I.nx), d1 = min_image(y - c[1], I.ny), dd = min_image(z - c[2], I.nz);
        if (d0 * d0 + d1 * d1 + dd * dd < P.R * P.R) return 2 + p;
    }
    return OWN_FLUID;
}

// new owner and fresh bit inside a particle's region (pure function of the
// particle positions, so overlapping regions write identical bytes)
__global__ void __launch_bounds__(PART_THREADS) k_geom_owner(Lattice L, int side)
{
    const PartDev &P = L.parts[blockIdx.y];
    const InstDev &I = L.inst[P.inst];
    Region reg;
    reg.init(P.x, side, I.nx, I.ny, I.nz);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < reg.count();
         t += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        const long long g = I.node_off + ((long long)z * I.ny + y) * I.nx + x;
        const uint8_t old = L.flags[g];
        if (own_static(old & OWNER_MASK)) continue;
        const int own = particle_owner(I, L.parts, x, y, z, 0);
        const int prev = particle_owner(I, L.parts, x, y, z, 1);
        uint8_t f = (uint8_t)own;
        if (own == OWN_FLUID && prev != OWN_FLUID) f |= FRESH_BIT;
        L.flags[g] = (uint8_t)(f | (old & BOUND_BIT));
    }
}

// boundary bit: fluid with a solid neighbour, or solid with a fluid neighbour
__device__ __forceinline__ void set_boundary(const Lattice &L, const InstDev &I, int x, int y, int z)
{
    const uint8_t *fli = L.flags + I.node_off;
    const int n = (z * I.ny + y) * I.nx + x;
    const uint8_t f = fli[n];
    const bool fluid = (f & OWNER_MASK) == OWN_FLUID;
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    bool b = false;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        bool nf = (fli[nb.at(cx(i), cy(i), cz(i))] & OWNER_MASK) == OWN_FLUID;
        b |= (nf != fluid);
    }
    L.flags[I.node_off + n] = (uint8_t)((f & ~BOUND_BIT) | (b ? BOUND_BIT : 0));
}

__global__ void __launch_bounds__(PART_THREADS) k_geom_bound(Lattice L, int side)
{
    const PartDev &P = L.parts[blockIdx.y];
    const InstDev &I = L.inst[P.inst];
    Region reg;
    reg.init(P.x, side, I.nx, I.ny, I.nz);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < reg.count();
         t += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        set_boundary(L, I, x, y, z);
    }
}

__global__ void k_boundary_full(Lattice L, int inst)
{
    const InstDev &I = L.inst[inst];
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < I.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x = (int)(n % I.nx), y = (int)((n / I.nx) % I.ny), z = (int)(n / ((long long)I.nx * I.ny));
        set_boundary(L, I, x, y, z);
    }
}

// Sec. V C refilling (Caiazzo 2008): a node uncovered this step gets
// f^{a,b} = feq(rho^{a,b}, u_p + w_p x (x - x_p)), rho^{a,b} the mean over the
// 18 moving-direction neighbours that are fluid and not fresh (two hops out if
// none; ambient (0, rho0) if still none).
//
// In the stored form (F* and the colour record (phi, b n) per node) the
// refilled state is F_i = (rho/rho0) e_i - 1 with the record
// (phi = (rho^a - rho^b)/rho, 0): its colour offsets (rho^a - rho^b)/rho0 e_i
// are phi (1 + F_i) exactly.  A neighbour's rho^a - rho^b is phi rho (its
// colour offsets sum to phi (1 + sum w F)).
//
// Few nodes are uncovered per step (about the swept surface area), so the
// kernel is a scan of the flags plus, per fresh node, one warp working on it:
// lane i-1 takes neighbour i and issues its 19 population loads at once, the
// sums meet in a shuffle reduction and lane i writes direction i.
template <class R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class S>
__device__ void refill_node(const InstDev &I, const PartDev *parts, const Pop<S> &pop,
                            typename Store<S>::real *ph, ColSlotOf<S> col, const uint8_t *fli,
                            int x, int y, int z, int lane)
{
    using R = typename Store<S>::real;
    R sF = 0, sG = 0;
    int nf = 0;
    for (int hop = 1; hop <= 2 && nf == 0; hop++) {
        R aF = 0, aG = 0;
        int ok = 0;
        if (lane < Q - 1) {
            const int i = lane + 1;
            const int X = ((x + hop * cx(i)) % I.nx + I.nx) % I.nx;
            const int Y = ((y + hop * cy(i)) % I.ny + I.ny) % I.ny;
            const int Z = ((z + hop * cz(i)) % I.nz + I.nz) % I.nz;
            const int m = (Z * I.ny + Y) * I.nx + X;
            const uint8_t fm = fli[m];
            if ((fm & OWNER_MASK) == OWN_FLUID && !(fm & FRESH_BIT)) {
                ok = 1;
#pragma unroll
                for (int j = 0; j < Q; j++) aF += wgt<R>(j) * (R(1) + pop.F(j, m));
                aG = col.phi(m) * aF;
            }
        }
        sF = warp_sum(aF);
        sG = warp_sum(aG);
        nf = __reduce_add_sync(0xffffffffu, ok);
    }
    // mean rho/rho0 and (rho^a - rho^b)/rho0 of the neighbours
    R rr, rd;
    if (nf > 0) { rr = sF / nf; rd = sG / nf; }
    else { rr = R(1); rd = R(-1); }
    if (lane >= Q) return;
    const int prev = particle_owner(I, parts, x, y, z, 1);
    const PartDev &P = parts[I.part_off + (prev >= 2 ? prev - 2 : 0)];
    R c[3];
    centre(P, c);
    const R d0 = min_image_r<R>(x - c[0], I.nx), d1 = min_image_r<R>(y - c[1], I.ny),
            d2 = min_image_r<R>(z - c[2], I.nz);
    const R w[3] = {(R)P.w[0], (R)P.w[1], (R)P.w[2]};
    const R u[3] = {(R)P.v[0] + w[1] * d2 - w[2] * d1, (R)P.v[1] + w[2] * d0 - w[0] * d2,
                    (R)P.v[2] + w[0] * d1 - w[1] * d0};
    const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const int i = lane;
    const int n = (z * I.ny + y) * I.nx + x;
    const R cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
    const R e = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
    pop.setF(i, n, rr * e - R(1));
    if (lane == 0) {
        ph[n] = rd / rr;
        col.shifted(n).set(ColRec<R>{rd / rr, R(0), R(0), R(0)});
    }
}

template <class S>
__global__ void __launch_bounds__(PART_THREADS) k_refill(Lattice L, int nxt, int side)
{
    using R = typename Store<S>::real;
    const PartDev &P0 = L.parts[blockIdx.y];
    const InstDev &I = L.inst[P0.inst];
    Region reg;
    reg.init(P0.x, side, I.nx, I.ny, I.nz);
    const Pop<S> pop(L.pop[nxt], I);
    const uint8_t *fli = L.flags + I.node_off;
    const int lane = threadIdx.x & 31;
    const long long count = reg.count();
    // warp-uniform trip count: every lane takes part in the ballots
    for (long long t0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < count;
         t0 += (long long)gridDim.x * blockDim.x) {
        const long long t = t0 + lane;
        int x = 0, y = 0, z = 0;
        bool fresh = false;
        if (t < count) {
            reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
            fresh = (fli[(z * I.ny + y) * I.nx + x] & FRESH_BIT) != 0;
        }
        unsigned todo = __ballot_sync(0xffffffffu, fresh);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int X = __shfl_sync(0xffffffffu, x, src), Y = __shfl_sync(0xffffffffu, y, src),
                      Z = __shfl_sync(0xffffffffu, z, src);
            refill_node<S>(I, L.parts, pop, (R *)L.phi + I.node_off, col_slot<S>(L, I.node_off), fli, X, Y, Z,
                           lane);
        }
    }
}

// initial particle marking: owner at the current positions, no fresh nodes
__global__ void __launch_bounds__(PART_THREADS) k_mark(Lattice L, int side)
{
    const PartDev &P = L.parts[blockIdx.y];
    const InstDev &I = L.inst[P.inst];
    Region reg;
    reg.init(P.x, side, I.nx, I.ny, I.nz);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < reg.count();
         t += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        const long long g = I.node_off + ((long long)z * I.ny + y) * I.nx + x;
        const uint8_t old = L.flags[g];
        if (own_static(old & OWNER_MASK)) continue;
        L.flags[g] = (uint8_t)(particle_owner(I, L.parts, x, y, z, 0) | (old & BOUND_BIT));
    }
}

// ---------------------------------------------------------------------------
template <class S>
void launch_momentum_exchange(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    mk(STAGE_MEM, 0);
    k_mem<S><<<dim3(L.mem_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, cur);
    mk(STAGE_MEM, 1);
    *launches += 1;
}

template <class S>
void launch_capillary(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk)
{
    using R = typename Store<S>::real;
    if (L.n_parts == 0) return;
    mk(STAGE_CAPILLARY, 0);
    if (L.buoyancy)
        k_capillary<R, true><<<dim3(CAP_BLOCKS, L.n_parts), CAP_THREADS, 0, st>>>(L);
    else
        k_capillary<R, false><<<dim3(CAP_BLOCKS, L.n_parts), CAP_THREADS, 0, st>>>(L);
    mk(STAGE_CAPILLARY, 1);
    *launches += 1;
}

template <class S>
void launch_particle_forces(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk)
{
    launch_momentum_exchange<S>(L, cur, st, launches, mk);
    launch_capillary<S>(L, st, launches, mk);
}

template <class S>
void launch_dem(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk, bool sum_fluid)
{
    using R = typename Store<S>::real;
    if (L.n_parts == 0) return;
    mk(STAGE_DEM, 0);
    if (L.buoyancy)
        k_dem<R, true><<<L.n_inst, DEM_THREADS, 0, st>>>(L, sum_fluid ? 1 : 0);
    else
        k_dem<R, false><<<L.n_inst, DEM_THREADS, 0, st>>>(L, sum_fluid ? 1 : 0);
    mk(STAGE_DEM, 1);
    *launches += 1;
}

void launch_geom_owner(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    // region sides: owner/refill cover the solid of the last two positions,
    // the boundary pass one more node around
    mk(STAGE_GEOM_OWNER, 0);
    k_geom_owner<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, L.geom_side);
    mk(STAGE_GEOM_OWNER, 1);
    *launches += 1;
}

void launch_geom_bound(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    mk(STAGE_GEOM_BOUND, 0);
    k_geom_bound<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, L.geom_side + 2);
    mk(STAGE_GEOM_BOUND, 1);
    *launches += 1;
}

template <class S>
void launch_refill(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    mk(STAGE_REFILL, 0);
    k_refill<S><<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, nxt, L.geom_side);
    mk(STAGE_REFILL, 1);
    *launches += 1;
}

template <class S>
void launch_geometry(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk)
{
    launch_geom_owner(L, st, launches, mk);
    launch_geom_bound(L, st, launches, mk);
    launch_refill<S>(L, nxt, st, launches, mk);
}

void launch_mark_particles(const Lattice &L, cudaStream_t st)
{
    if (L.n_parts == 0) return;
    const int side = L.geom_side;
    k_mark<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side);
    k_geom_bound<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side + 2);
}

void launch_boundary_full(const Lattice &L, int inst, long long N, cudaStream_t st)
{
    long long blocks = (N + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_boundary_full<<<(unsigned)blocks, 256, 0, st>>>(L, inst);
}

#define INST(S)                                                                                             \
    template void launch_particle_forces<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &); \
    template void launch_momentum_exchange<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &); \
    template void launch_capillary<S>(const Lattice &, cudaStream_t, long long *, const Marker &);           \
    template void launch_geometry<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &);     \
    template void launch_dem<S>(const Lattice &, cudaStream_t, long long *, const Marker &, bool);       \
    template void launch_refill<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
