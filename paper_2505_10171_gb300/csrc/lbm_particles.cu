// Particle kernels of one coupled time step (Sec. III and V of arXiv 2505.10171):
//   k_mem       momentum-exchange force and torque per particle (Sec. V B)
//   k_capillary capillary force and torque from the Lagrangian surface points
//               (Sec. V E)
//   k_dem       contacts (normal spring-dashpot, Luding sliding and rolling
//               friction) and velocity-Verlet update, FP64 (Sec. III)
//   k_geom_*    solid map update and refilling of uncovered nodes (Sec. V C)
// Per-particle sums are reduced in FP64 with a fixed order (warp shuffle,
// block tree, then a fixed-order sum over blocks inside k_dem), so results are
// reproducible run to run.
#include "lbm_internal.cuh"

namespace lbmg {

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
    __device__ __forceinline__ void coord(long long t, int nx, int ny, int nz, int *x, int *y, int *z) const
    {
        int i = (int)(t % sz[0]);
        int j = (int)((t / sz[0]) % sz[1]);
        int k = (int)(t / ((long long)sz[0] * sz[1]));
        *x = ((lo[0] + i) % nx + nx) % nx;
        *y = ((lo[1] + j) % ny + ny) % ny;
        *z = ((lo[2] + k) % nz + nz) % nz;
    }
};

// deterministic block sum of 6 doubles; thread 0 writes them to out
__device__ __forceinline__ void block_sum6(double *v, double *out)
{
    __shared__ double sm[PART_THREADS / 32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 6; a++)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    if (lane == 0)
        for (int a = 0; a < 6; a++) sm[wid][a] = v[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 6; a++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sm[w][a];
            out[a] = s;
        }
    }
}

// Sec. V B momentum exchange (Wen 2014, Galilean invariant): per link from a
// fluid node x into particle p, force on p = (c_out - u_w) f_out - (c_in - u_w) f_in
// with f_out = f*_ibar(x) leaving towards the solid and f_in = f_i(x) bounced
// back; torque lever from the centre to the link midpoint.
template <class S>
__global__ void __launch_bounds__(PART_THREADS) k_mem(Lattice L, int cur)
{
    const int p = blockIdx.y;
    const PartDev &P = L.parts[p];
    const InstDev &I = L.inst[P.inst];
    const long long N = I.N;
    Region reg;
    reg.init(P.x, P.mem_side, I.nx, I.ny, I.nz);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < reg.count()) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        const long long n = ((long long)z * I.ny + y) * I.nx + x;
        const uint8_t *fli = L.flags + I.node_off;
        const uint8_t fl = fli[n];
        if ((fl & OWNER_MASK) == OWN_FLUID && (fl & BOUND_BIT)) {
            const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
            Nbr nb;
            nb.init(x, y, z, I.nx, I.ny, I.nz);
            const int mine = 2 + P.local;
            double rr = -1.0;
            const double wr0 = I.rho0;
            for (int i = 1; i < Q; i++) {
                long long s = nb.at(-cx(i), -cy(i), -cz(i));
                if ((fli[s] & OWNER_MASK) != mine) continue;
                if (rr < 0.0) {
                    double sF = 0.0;
                    for (int j = 0; j < Q; j++) sF += wgt<double>(j) * (double)Store<S>::ld(in + (long long)j * N + n);
                    rr = 1.0 + sF;
                }
                double uw[3], lev[3];
                surface_velocity(I, L.parts, mine, x - 0.5 * cx(i), y - 0.5 * cy(i), z - 0.5 * cz(i), uw, lev);
                const int ib = opp(i);
                const double w = wgt<double>(i) * wr0;
                const double Fo = (double)Store<S>::ld(in + (long long)ib * N + n);
                const double cu = cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2];
                const double fout = w * (1.0 + Fo);
                const double fin = w * (1.0 + Fo + 6.0 * rr * cu);
                const double ci[3] = {(double)cx(i), (double)cy(i), (double)cz(i)};
                double dp[3];
                for (int a = 0; a < 3; a++) dp[a] = (-ci[a] - uw[a]) * fout - (ci[a] - uw[a]) * fin;
                acc[0] += dp[0];
                acc[1] += dp[1];
                acc[2] += dp[2];
                acc[3] += lev[1] * dp[2] - lev[2] * dp[1];
                acc[4] += lev[2] * dp[0] - lev[0] * dp[2];
                acc[5] += lev[0] * dp[1] - lev[1] * dp[0];
            }
        }
    }
    block_sum6(acc, L.mem_part + ((long long)p * L.mem_blocks + blockIdx.x) * 6);
}

// Sec. V E: dF = C sigma (1 - phi^2) dA [n_s - (n.n_s) n] at the points
// alpha_j = (j + 1/2) 2 deg, varphi_k = k 2 deg on r = R_p; phi and grad(phi)
// trilinearly interpolated over fluid corners only; torque R_p n_s x dF.
template <class R>
__global__ void __launch_bounds__(CAP_THREADS) k_capillary(Lattice L)
{
    const int p = blockIdx.y;
    const PartDev &P = L.parts[p];
    const InstDev &I = L.inst[P.inst];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt < CAP_POINTS) {
        const int j = pt / 180, k = pt % 180;
        const double da = 2.0 * M_PI / 180.0;
        const double al = (j + 0.5) * da, vp = k * da;
        const double sa = sin(al), ca = cos(al), sv = sin(vp), cv = cos(vp);
        const double ns[3] = {sa * cv, sa * sv, ca};
        const double xi[3] = {P.x[0] + P.R * ns[0], P.x[1] + P.R * ns[1], P.x[2] + P.R * ns[2]};
        const double dA = P.R * P.R * sa * da * da;
        int b[3];
        double fr[3];
        for (int a = 0; a < 3; a++) {
            double fl = floor(xi[a]);
            b[a] = (int)fl;
            fr[a] = xi[a] - fl;
        }
        const int n3[3] = {I.nx, I.ny, I.nz};
        const uint8_t *fli = L.flags + I.node_off;
        const R *ph = (const R *)L.phi + I.node_off;
        const R *G = (const R *)L.grad + I.node_off;
        double ws = 0.0, phs = 0.0, gs[3] = {0, 0, 0};
        for (int cz_ = 0; cz_ < 2; cz_++)
            for (int cy_ = 0; cy_ < 2; cy_++)
                for (int cx_ = 0; cx_ < 2; cx_++) {
                    int X = ((b[0] + cx_) % n3[0] + n3[0]) % n3[0];
                    int Y = ((b[1] + cy_) % n3[1] + n3[1]) % n3[1];
                    int Z = ((b[2] + cz_) % n3[2] + n3[2]) % n3[2];
                    long long m = ((long long)Z * I.ny + Y) * I.nx + X;
                    if ((fli[m] & OWNER_MASK) != OWN_FLUID) continue;
                    double wgt_ = (cx_ ? fr[0] : 1.0 - fr[0]) * (cy_ ? fr[1] : 1.0 - fr[1]) *
                                  (cz_ ? fr[2] : 1.0 - fr[2]);
                    ws += wgt_;
                    phs += wgt_ * (double)ph[m];
                    gs[0] += wgt_ * (double)G[m];
                    gs[1] += wgt_ * (double)G[L.Ntot + m];
                    gs[2] += wgt_ * (double)G[2 * L.Ntot + m];
                }
        if (ws > 0.0) {
            const double phv = phs / ws;
            const double g0 = gs[0] / ws, g1 = gs[1] / ws, g2 = gs[2] / ws;
            if (fabs(phv) < 1.0) {
                // regularised normal n = g/sqrt(|g|^2 + eps^2), m = (n x n_s) x n
                const double gr = sqrt(g0 * g0 + g1 * g1 + g2 * g2 + I.grad_eps * I.grad_eps);
                const double nn[3] = {g0 / gr, g1 / gr, g2 / gr};
                const double c0 = nn[1] * ns[2] - nn[2] * ns[1], c1 = nn[2] * ns[0] - nn[0] * ns[2],
                             c2 = nn[0] * ns[1] - nn[1] * ns[0];
                const double mv[3] = {c1 * nn[2] - c2 * nn[1], c2 * nn[0] - c0 * nn[2], c0 * nn[1] - c1 * nn[0]};
                const double coef = I.cap_norm * I.sigma * (1.0 - phv * phv) * dA;
                double dF[3];
                for (int a = 0; a < 3; a++) dF[a] = coef * mv[a];
                const double r[3] = {P.R * ns[0], P.R * ns[1], P.R * ns[2]};
                acc[0] = dF[0];
                acc[1] = dF[1];
                acc[2] = dF[2];
                acc[3] = r[1] * dF[2] - r[2] * dF[1];
                acc[4] = r[2] * dF[0] - r[0] * dF[2];
                acc[5] = r[0] * dF[1] - r[1] * dF[0];
            }
        }
    }
    block_sum6(acc, L.cap_part + ((long long)p * CAP_BLOCKS + blockIdx.x) * 6);
}

// ---------------------------------------------------------------------------
// DEM (Sec. III), one thread per instance, FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double *a, const double *b, double *r)
{
    double t0 = a[1] * b[2] - a[2] * b[1], t1 = a[2] * b[0] - a[0] * b[2], t2 = a[0] * b[1] - a[1] * b[0];
    r[0] = t0; r[1] = t1; r[2] = t2;
}

// Luding spring: project on the tangent plane, trial force, Coulomb cap,
// spring update (static: xi += v dt; sliding: xi = -(F + gamma v)/k).
__device__ void dem_spring(double *xi, const double *n, const double *v, double k, double gam, double FC, double *F)
{
    double xn = dot3(xi, n);
    for (int a = 0; a < 3; a++) xi[a] -= xn * n[a];
    double F0[3];
    for (int a = 0; a < 3; a++) F0[a] = -k * xi[a] - gam * v[a];
    double m = sqrt(dot3(F0, F0));
    if (m <= FC) {
        for (int a = 0; a < 3; a++) { F[a] = F0[a]; xi[a] += v[a]; }
    } else {
        for (int a = 0; a < 3; a++) F[a] = FC * F0[a] / m;
        for (int a = 0; a < 3; a++) xi[a] = k > 0.0 ? -(F[a] + gam * v[a]) / k : 0.0;
    }
}

// contact of particle i with partner j (j < 0: substrate); n from partner to
// i, delta > 0 the overlap.  Contact point X_i - (R_c,i - delta/2) n;
// F_n = [k_n delta - g_n v_rel.n] n; rolling velocity -a'(w_i - w_j) x n with
// torque -a' n x F_r on i (+a' n x F_r on j).
__device__ void dem_contact(const InstDev &I, PartDev *P, int i, int j, const double *vp, const double *wp,
                            const double *n, double delta, double *xi, double *xir)
{
    double bi[3], bj[3] = {0, 0, 0}, t[3], vi[3], vj[3];
    for (int a = 0; a < 3; a++) bi[a] = -(P[i].Rc - 0.5 * delta) * n[a];
    cross3(wp + 3 * i, bi, t);
    for (int a = 0; a < 3; a++) vi[a] = vp[3 * i + a] + t[a];
    double ap;
    if (j >= 0) {
        for (int a = 0; a < 3; a++) bj[a] = (P[j].Rc - 0.5 * delta) * n[a];
        cross3(wp + 3 * j, bj, t);
        for (int a = 0; a < 3; a++) vj[a] = vp[3 * j + a] + t[a];
        ap = P[i].Rc * P[j].Rc / (P[i].Rc + P[j].Rc);
    } else {
        for (int a = 0; a < 3; a++) vj[a] = I.wall_u[a];
        ap = P[i].Rc;
    }
    double vr[3];
    for (int a = 0; a < 3; a++) vr[a] = vi[a] - vj[a];
    const double vn = dot3(vr, n);
    const double Fnm = I.kn * delta - I.gn * vn;
    double vt[3];
    for (int a = 0; a < 3; a++) vt[a] = vr[a] - vn * n[a];
    double Ft[3];
    dem_spring(xi, n, vt, I.kt, I.gt, I.mu_s * fabs(Fnm), Ft);
    double wrel[3], vrl[3];
    for (int a = 0; a < 3; a++) wrel[a] = wp[3 * i + a] - (j >= 0 ? wp[3 * j + a] : 0.0);
    cross3(wrel, n, vrl);
    for (int a = 0; a < 3; a++) vrl[a] *= -ap;
    double Fr[3];
    dem_spring(xir, n, vrl, I.kr, I.gr, I.mu_r * fabs(Fnm), Fr);
    double Tt[3], Tr[3];
    cross3(bi, Ft, Tt);
    cross3(n, Fr, Tr);
    for (int a = 0; a < 3; a++) {
        P[i].Fc[a] += Fnm * n[a] + Ft[a];
        P[i].Tc[a] += Tt[a] - ap * Tr[a];
    }
    if (j >= 0) {
        double mFt[3] = {-Ft[0], -Ft[1], -Ft[2]}, Ttj[3];
        cross3(bj, mFt, Ttj);
        for (int a = 0; a < 3; a++) {
            P[j].Fc[a] -= Fnm * n[a] + Ft[a];
            P[j].Tc[a] += Ttj[a] + ap * Tr[a];
        }
    }
}

__device__ void quat_rotate(double *q, const double *w)
{
    double wm = sqrt(dot3(w, w));
    if (wm == 0.0) return;
    double h = 0.5 * wm, s = sin(h) / wm;
    double d0 = cos(h), d1 = s * w[0], d2 = s * w[1], d3 = s * w[2];
    double r0 = d0 * q[0] - d1 * q[1] - d2 * q[2] - d3 * q[3];
    double r1 = d0 * q[1] + d1 * q[0] + d2 * q[3] - d3 * q[2];
    double r2 = d0 * q[2] - d1 * q[3] + d2 * q[0] + d3 * q[1];
    double r3 = d0 * q[3] + d1 * q[2] - d2 * q[1] + d3 * q[0];
    double l = sqrt(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    q[0] = r0 / l; q[1] = r1 / l; q[2] = r2 / l; q[3] = r3 / l;
}

constexpr int DEM_MAXP = 61;

__global__ void k_dem(Lattice L, int mem_blocks)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.n_inst) return;
    const InstDev &I = L.inst[k];
    if (I.np == 0) return;
    PartDev *P = L.parts + I.part_off;
    const int np = I.np;
    double *hist = L.hist + (long long)I.hist_off * 6;
    // fluid forces of this step: fixed-order sums of the block partials
    for (int p = 0; p < np; p++) {
        const long long gp = I.part_off + p;
        double s[6] = {0, 0, 0, 0, 0, 0}, c[6] = {0, 0, 0, 0, 0, 0};
        for (int b = 0; b < mem_blocks; b++)
            for (int a = 0; a < 6; a++) s[a] += L.mem_part[(gp * mem_blocks + b) * 6 + a];
        for (int b = 0; b < CAP_BLOCKS; b++)
            for (int a = 0; a < 6; a++) c[a] += L.cap_part[(gp * CAP_BLOCKS + b) * 6 + a];
        for (int a = 0; a < 3; a++) {
            P[p].Feta[a] = s[a]; P[p].Teta[a] = s[3 + a];
            P[p].Fsig[a] = c[a]; P[p].Tsig[a] = c[3 + a];
        }
    }
    // velocity Verlet predictor (dt = 1)
    double vp[3 * DEM_MAXP], wp[3 * DEM_MAXP], xn[3 * DEM_MAXP];
    for (int p = 0; p < np; p++) {
        for (int a = 0; a < 3; a++) {
            P[p].x_old[a] = P[p].x[a];
            if (P[p].kin) {
                xn[3 * p + a] = P[p].x[a] + P[p].v[a];
                vp[3 * p + a] = P[p].v[a];
                wp[3 * p + a] = P[p].w[a];
            } else {
                double acc = P[p].Fp[a] / P[p].m, alp = P[p].Tp[a] / P[p].I;
                xn[3 * p + a] = P[p].x[a] + P[p].v[a] + 0.5 * acc;
                vp[3 * p + a] = P[p].v[a] + acc;
                wp[3 * p + a] = P[p].w[a] + alp;
            }
            P[p].Fc[a] = 0.0;
            P[p].Tc[a] = 0.0;
        }
    }
    // substrate contacts, delta = R_c - (z_p - 0.5); history record p
    for (int p = 0; p < np; p++) {
        double *xi = hist + 6 * p, *xir = xi + 3;
        double delta = P[p].Rc - (xn[3 * p + 2] - 0.5);
        if (I.wall_z0 && delta > 0.0) {
            const double n[3] = {0.0, 0.0, 1.0};
            dem_contact(I, P, p, -1, vp, wp, n, delta, xi, xir);
        } else {
            for (int a = 0; a < 6; a++) xi[a] = 0.0;
        }
    }
    // pair contacts, delta_ij = R_c,i + R_c,j - |X_i - X_j|; history record
    // np + i*np + j
    for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
            double *xi = hist + 6 * (np + i * np + j), *xir = xi + 3;
            double d[3] = {min_image(xn[3 * i] - xn[3 * j], I.nx), min_image(xn[3 * i + 1] - xn[3 * j + 1], I.ny),
                           min_image(xn[3 * i + 2] - xn[3 * j + 2], I.nz)};
            double dl = sqrt(dot3(d, d));
            double delta = P[i].Rc + P[j].Rc - dl;
            if (delta > 0.0 && dl > 0.0) {
                const double n[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
                dem_contact(I, P, i, j, vp, wp, n, delta, xi, xir);
            } else {
                for (int a = 0; a < 6; a++) xi[a] = 0.0;
            }
        }
    // corrector
    for (int p = 0; p < np; p++) {
        double F[3], T[3], wold[3];
        for (int a = 0; a < 3; a++) {
            F[a] = P[p].Fc[a] + I.g_part[a] + P[p].Feta[a] + P[p].Fsig[a];
            T[a] = P[p].Tc[a] + P[p].Teta[a] + P[p].Tsig[a];
            wold[a] = P[p].w[a];
        }
        if (!P[p].kin)
            for (int a = 0; a < 3; a++) {
                P[p].v[a] += 0.5 * (P[p].Fp[a] + F[a]) / P[p].m;
                P[p].w[a] += 0.5 * (P[p].Tp[a] + T[a]) / P[p].I;
            }
        double wm[3] = {0.5 * (wold[0] + P[p].w[0]), 0.5 * (wold[1] + P[p].w[1]), 0.5 * (wold[2] + P[p].w[2])};
        quat_rotate(P[p].q, wm);
        for (int a = 0; a < 3; a++) {
            if (fabs(xn[3 * p + a] - P[p].x[a]) >= GEOM_MARGIN - 1) atomicOr(L.status, ST_DISPLACEMENT);
            P[p].x[a] = xn[3 * p + a];
            P[p].Fp[a] = F[a];
            P[p].Tp[a] = T[a];
        }
    }
}

// ---------------------------------------------------------------------------
// Geometry update and refilling (Sec. V C)
// ---------------------------------------------------------------------------
// owner of node (x,y,z) for particle positions `which` (0: current, 1: previous)
__device__ __forceinline__ int particle_owner(const InstDev &I, const PartDev *parts, int x, int y, int z, int which)
{
    for (int p = 0; p < I.np; p++) {
        const PartDev &P = parts[I.part_off + p];
        const double *c = which ? P.x_old : P.x;
        double d0 = min_image(x - c[0], I.nx), d1 = min_image(y - c[1], I.ny), d2 = min_image(z - c[2], I.nz);
        if (d0 * d0 + d1 * d1 + d2 * d2 < P.R * P.R) return 2 + p;
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
        if ((old & OWNER_MASK) == OWN_WALL) continue;
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
    const long long n = ((long long)z * I.ny + y) * I.nx + x;
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
template <class S>
__global__ void __launch_bounds__(PART_THREADS) k_refill(Lattice L, int nxt, int side)
{
    const PartDev &P0 = L.parts[blockIdx.y];
    const InstDev &I = L.inst[P0.inst];
    Region reg;
    reg.init(P0.x, side, I.nx, I.ny, I.nz);
    const long long N = I.N;
    S *pop = (S *)L.pop[nxt] + NPOP * I.node_off;
    const uint8_t *fli = L.flags + I.node_off;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < reg.count();
         t += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        const long long n = ((long long)z * I.ny + y) * I.nx + x;
        if (!(fli[n] & FRESH_BIT)) continue;
        double sF = 0.0, sG = 0.0;
        int nf = 0;
        for (int hop = 1; hop <= 2 && nf == 0; hop++)
            for (int i = 1; i < Q; i++) {
                int X = ((x + hop * cx(i)) % I.nx + I.nx) % I.nx;
                int Y = ((y + hop * cy(i)) % I.ny + I.ny) % I.ny;
                int Z = ((z + hop * cz(i)) % I.nz + I.nz) % I.nz;
                long long m = ((long long)Z * I.ny + Y) * I.nx + X;
                uint8_t fm = fli[m];
                if ((fm & OWNER_MASK) != OWN_FLUID || (fm & FRESH_BIT)) continue;
                for (int j = 0; j < Q; j++) {
                    sF += wgt<double>(j) * (1.0 + (double)Store<S>::ld(pop + (long long)j * N + m));
                    sG += wgt<double>(j) * (double)Store<S>::ld(pop + (long long)(Q + j) * N + m);
                }
                nf++;
            }
        // mean rho/rho0 and (rho^a - rho^b)/rho0 of the neighbours
        double rr, rd;
        if (nf > 0) { rr = sF / nf; rd = sG / nf; }
        else { rr = 1.0; rd = -1.0; }
        const int prev = particle_owner(I, L.parts, x, y, z, 1);
        const PartDev &P = L.parts[I.part_off + (prev >= 2 ? prev - 2 : 0)];
        double d0 = min_image(x - P.x[0], I.nx), d1 = min_image(y - P.x[1], I.ny), d2 = min_image(z - P.x[2], I.nz);
        double u[3] = {P.v[0] + P.w[1] * d2 - P.w[2] * d1, P.v[1] + P.w[2] * d0 - P.w[0] * d2,
                       P.v[2] + P.w[0] * d1 - P.w[1] * d0};
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        for (int i = 0; i < Q; i++) {
            double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
            double e = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
            Store<S>::st(pop + (long long)i * N + n, (typename Store<S>::real)(rr * e - 1.0));
            Store<S>::st(pop + (long long)(Q + i) * N + n, (typename Store<S>::real)(rd * e));
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
        if ((old & OWNER_MASK) == OWN_WALL) continue;
        L.flags[g] = (uint8_t)(particle_owner(I, L.parts, x, y, z, 0) | (old & BOUND_BIT));
    }
}

// ---------------------------------------------------------------------------
template <class S>
void launch_particle_forces(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk)
{
    using R = typename Store<S>::real;
    if (L.n_parts == 0) return;
    mk(STAGE_MEM, 0);
    k_mem<S><<<dim3(L.mem_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, cur);
    mk(STAGE_MEM, 1);
    mk(STAGE_CAPILLARY, 0);
    k_capillary<R><<<dim3(CAP_BLOCKS, L.n_parts), CAP_THREADS, 0, st>>>(L);
    mk(STAGE_CAPILLARY, 1);
    *launches += 2;
}

void launch_dem(const Lattice &L, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    mk(STAGE_DEM, 0);
    k_dem<<<(L.n_inst + 31) / 32, 32, 0, st>>>(L, L.mem_blocks);
    mk(STAGE_DEM, 1);
    *launches += 1;
}

template <class S>
void launch_geometry(const Lattice &L, int nxt, cudaStream_t st, long long *launches, const Marker &mk)
{
    if (L.n_parts == 0) return;
    // region sides: owner/refill cover the solid of the last two positions,
    // the boundary pass one more node around
    const int side = L.geom_side;
    mk(STAGE_GEOM_OWNER, 0);
    k_geom_owner<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side);
    mk(STAGE_GEOM_OWNER, 1);
    mk(STAGE_GEOM_BOUND, 0);
    k_geom_bound<<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, side + 2);
    mk(STAGE_GEOM_BOUND, 1);
    mk(STAGE_REFILL, 0);
    k_refill<S><<<dim3(L.geom_blocks, L.n_parts), PART_THREADS, 0, st>>>(L, nxt, side);
    mk(STAGE_REFILL, 1);
    *launches += 3;
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
    template void launch_geometry<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
