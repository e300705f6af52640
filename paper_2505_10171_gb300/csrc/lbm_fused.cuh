// Fused z-marching form of the fluid update (one kernel per step).  Included
// once per storage type by lbm_fused_<type>.cu so that its instantiations
// compile in parallel.
#pragma once
#include "lbm_node.cuh"

namespace lbmg {

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
    const Pop<S> in(L.pop[cur], I);
    const Pop<S> out(L.pop[cur ^ 1], I);
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
                    ph = node_phi<S>(I, L.parts, nb, in, n, fl, X, Y, Z);
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
                R F[Q];
                gather_F<S>(I, L.parts, nb, in, n, fl, F, gx, gy, Z);
                collide_store_phi<S>(P, F, phiS[s0 * RN + r], gr, nn, kap, out, n, U, L.Ntot, L.status);
            }
        }
        __syncthreads();
    }
}

template <class S, int TX, int TY>
void launch_fused(const Lattice &L, int cur, long long items, cudaStream_t st)
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
void launch_fused_form(const Lattice &L, int cur, const FluidLaunch &fz, cudaStream_t st)
{
    if (fz.tile == 1) launch_fused<S, 32, 8>(L, cur, fz.items, st);
    else launch_fused<S, 16, 16>(L, cur, fz.items, st);
}

}  // namespace lbmg
