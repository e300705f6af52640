// Fluid update of one coupled time step (Sec. IV of arXiv 2505.10171).
//
// Per node: pull streaming with bounce-back -> order parameter phi -> phi on
// solid nodes next to fluid (w-weighted fluid mean) -> isotropic grad(phi)
// with the geometric wetting rotation (Sec. V D) -> regularised normal and its
// divergence (curvature) -> CSF + body force -> MRT with Guo forcing, evaluated
// in its two-relaxation-time form -> recolouring -> write.
//
// Three launch forms run the per-node device functions of lbm_node.cuh:
//  * plain (default): k_phi, k_solidphi, k_grad, k_curv, k_collide, one thread
//    per node with direct global loads.  The collision pulls only the 19 total
//    offsets F: the colour offsets enter it only through phi, which k_phi
//    stores.
//  * staged: the same kernels, with k_phi and k_collide replaced by persistent
//    kernels that bring their inputs into shared memory with asynchronous
//    copies (lbm_staged.cu).
//  * k_fused: one kernel per step.  A block owns a TX x TY column tile and a
//    chunk of z-planes and marches z: the order parameter of plane z+3 is
//    gathered into a shared-memory ring (with a 3-node halo, enough for the
//    solid-phi fill), solids of plane z+2 are filled, gradient/wetting/normal of
//    plane z+1 are formed, and plane z is collided.
// The staged and plain forms agree bit for bit; the fused form agrees bit for
// bit in FP32 and to rounding in FP64 (contraction into FMA may differ).
// The particle-region kernels recompute phi and grad(phi) around each particle
// for the capillary force.
// Storage type S in {double, float, __half, __nv_bfloat16}; arithmetic in
// double for S = double and float otherwise.
#include "lbm_node.cuh"

// CTAs of 256 threads per SM the single-precision order-parameter and
// collision kernels are compiled for (register budget 65536 / (256 x this))
#ifndef LBM_PHI_MINB
#define LBM_PHI_MINB 4
#endif
#ifndef LBM_COLLIDE_MINB
#define LBM_COLLIDE_MINB 4
#endif

namespace lbmg {

// ---------------------------------------------------------------------------
// four-kernel form over all nodes (and the same bodies over particle regions)
// ---------------------------------------------------------------------------
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
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    // the sums of a node without solid neighbours are formed before the flag
    // is tested (every neighbour address is valid), so that the 38 loads travel
    // with the flag load instead of after it
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    R v = phi_fluid<S>(nb, in, (int)I.N);
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    if (fl & BOUND_BIT) v = phi_node_cold<S>(&I, L.parts, L.flags + I.node_off, in, n, fl, x, y, z);
    ((R *)L.phi)[g] = v;
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
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    const R *ph = (const R *)L.phi + I.node_off;
    auto phi_of = [&](int dx, int dy, int dz) { return ph[nb.idx(dx, dy, dz)]; };
    R gr[3], nn[3];
    grad_sum<R>(phi_of, gr);  // loads issued before the flag is tested
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    FluidPar<R> P;
    load_par(I, P);
    grad_wet<R>(I, L.parts, nb, ph[n], fl, P.wet_max, x, y, z, gr);
    const R m = reg_normal(gr, P.eps2, nn);
    R *Nn = (R *)L.grad;
    Nn[g] = nn[0];
    Nn[L.Ntot + g] = nn[1];
    Nn[2 * L.Ntot + g] = nn[2];
    ((R *)L.gmag)[g] = m;
}

template <class S>
__global__ void __launch_bounds__(ROW_NODES, sizeof(S) == 8 ? 1 : LBM_PHI_MINB) k_phi(Lattice L, int cur)
{
    for_item_nodes(L, [&](const InstDev &I, int n, int x, int y, int z) { phi_body<S>(L, I, cur, n, x, y, z); });
}

template <class R>
__global__ void __launch_bounds__(ROW_NODES) k_solidphi(Lattice L)
{
    for_item_nodes(L, [&](const InstDev &I, int n, int x, int y, int z) { solidphi_body<R>(L, I, n, x, y, z); });
}

template <class R>
__global__ void __launch_bounds__(ROW_NODES) k_grad(Lattice L)
{
    for_item_nodes(L, [&](const InstDev &I, int n, int x, int y, int z) { grad_body<R>(L, I, n, x, y, z); });
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

// curvature of every fluid node from the stored normals (a solid neighbour
// contributes the node's own normal)
template <class R>
__device__ __forceinline__ void curv_body(const Lattice &L, const InstDev &I, int n, int x, int y, int z)
{
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    GlobalNbr nb;
    nb.nb.init(x, y, z, I.nx, I.ny, I.nz);
    nb.fli = L.flags + I.node_off;
    const R *Nn = (const R *)L.grad + I.node_off;
    const long long Nt = L.Ntot;
    // all-fluid neighbourhood first (loads issued with the flag load)
    R kap = curvature<R>([&](int dx, int dy, int dz, int a) { return Nn[a * Nt + nb.idx(dx, dy, dz)]; });
    if ((fl & OWNER_MASK) != OWN_FLUID) return;
    if (fl & BOUND_BIT)
        kap = curvature<R>([&](int dx, int dy, int dz, int a) {
            if (nb.own(dx, dy, dz) != OWN_FLUID) return Nn[a * Nt + n];
            return Nn[a * Nt + nb.idx(dx, dy, dz)];
        });
    ((R *)L.kap)[g] = kap;
}

template <class R>
__global__ void __launch_bounds__(ROW_NODES) k_curv(Lattice L)
{
    for_item_nodes(L, [&](const InstDev &I, int n, int x, int y, int z) { curv_body<R>(L, I, n, x, y, z); });
}

template <class S>
__device__ __forceinline__ void collide_body(const Lattice &L, const InstDev &I, int cur, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    const int N = (int)I.N;
    const long long g = I.node_off + n;
    const S *in = (const S *)L.pop[cur] + NPOP * I.node_off;
    S *out = (S *)L.pop[cur ^ 1] + NPOP * I.node_off;
    // every load of an interior fluid node is issued before the flag is tested
    const uint8_t fl = L.flags[g];
    const R *Nn = (const R *)L.grad + I.node_off;
    const long long Nt = L.Ntot;
    const R nn[3] = {Nn[n], Nn[Nt + n], Nn[2 * Nt + n]};
    const R m = ((const R *)L.gmag)[g];
    const R kap = ((const R *)L.kap)[g];
    const R phi = ((const R *)L.phi)[g];
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    R F[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) F[i] = Store<S>::ld(in + i * N + nb.at(-cx(i), -cy(i), -cz(i)));
    R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
    if ((fl & OWNER_MASK) != OWN_FLUID) {
        if (U) { U[n] = 0; U[L.Ntot + n] = 0; U[2 * L.Ntot + n] = 0; }
        return;
    }
    if (fl & BOUND_BIT) {
        collide_node_cold<S>(&I, L.parts, L.flags + I.node_off, in, out, n, fl, x, y, z, phi, nn[0], nn[1], nn[2], m,
                             kap, U, L.Ntot, L.status);
        return;
    }
    FluidPar<R> P;
    load_par(I, P);
    const R gr[3] = {nn[0] * m, nn[1] * m, nn[2] * m};
    collide_store_phi<S>(P, F, phi, gr, nn, kap, out, N, n, U, L.Ntot, L.status);
}

template <class S>
__global__ void __launch_bounds__(ROW_NODES, sizeof(S) == 8 ? 1 : LBM_COLLIDE_MINB) k_collide(Lattice L, int cur)
{
    for_item_nodes(L, [&](const InstDev &I, int n, int x, int y, int z) { collide_body<S>(L, I, cur, n, x, y, z); });
}

// tile shapes of the fused kernel: 0 -> 16 x 16, 1 -> 32 x 8
int fused_tile_x(int tile) { return tile == 1 ? 32 : 16; }
int fused_tile_y(int tile) { return tile == 1 ? 8 : 16; }

template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk,
                       const FluidLaunch &fz)
{
    using R = typename Store<S>::real;
    if (fz.form == FORM_FUSED) {
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
        launch_fused_form<S>(L, cur, fz, st);
        mk(STAGE_FUSED, 1);
        *launches += 1;
        return;
    }
    // staged form where every instance's rows are whole 16-byte units, plain otherwise
    const bool staged = fz.form == FORM_STAGED && fz.st_items > 0;
    const dim3 grid((unsigned)fz.rows);  // one CTA per row-strip work item
    mk(STAGE_PHI, 0);
    if (staged) launch_staged_phi<S>(L, cur, fz, st);
    else k_phi<S><<<grid, ROW_NODES, 0, st>>>(L, cur);
    mk(STAGE_PHI, 1);
    mk(STAGE_SOLIDPHI, 0);
    k_solidphi<R><<<grid, ROW_NODES, 0, st>>>(L);
    mk(STAGE_SOLIDPHI, 1);
    mk(STAGE_GRAD, 0);
    k_grad<R><<<grid, ROW_NODES, 0, st>>>(L);
    mk(STAGE_GRAD, 1);
    mk(STAGE_CURV, 0);
    k_curv<R><<<grid, ROW_NODES, 0, st>>>(L);
    mk(STAGE_CURV, 1);
    mk(STAGE_COLLIDE, 0);
    if (staged) launch_staged_collide<S>(L, cur, fz, st);
    else k_collide<S><<<grid, ROW_NODES, 0, st>>>(L, cur);
    mk(STAGE_COLLIDE, 1);
    *launches += 5;
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
