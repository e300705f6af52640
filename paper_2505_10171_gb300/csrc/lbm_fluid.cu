// Fluid update of one coupled time step (Sec. IV of arXiv 2505.10171).
//
// Per node: pull streaming with bounce-back -> order parameter phi -> phi on
// solid nodes next to fluid (w-weighted fluid mean) -> isotropic grad(phi)
// with the geometric wetting rotation (Sec. V E) -> regularised normal and its
// divergence (curvature) -> CSF + body force -> MRT with Guo forcing, evaluated
// in its two-relaxation-time form -> recolouring -> write.
//
// Kernels of a step: k_phi (one thread per node over row strips) stores phi;
// the solid-phi fill over the listed static solid nodes and the step's list
// of particle-surface solid nodes; k_gradcurv (z-marching tiles:
// gradient, wetting, normal, curvature); k_collide (or k_collide2).  Nodes next
// to a solid go to the boundary passes k_phi_bound and k_collide_bound, which
// run beside the bulk kernels on a second stream.
//
// The state between steps is the total offsets F* (pop[cur]) with one colour
// record per node: phi (the order parameter its collision used) and b n (the
// recolouring amplitude times the normal).  The order-parameter pass rebuilds
// each pulled colour offset G_i from its source node's record
// (lbm_internal.cuh); the collision needs the colour offsets only through phi.
// Storage type S in {double, float, __half, __nv_bfloat16}; arithmetic in
// double for S = double and float otherwise.
#include "lbm_node.cuh"

// CTAs of 256 threads per SM the single-precision order-parameter and
// collision kernels are compiled for (register budget 65536 / (256 x this)).
// The order-parameter pass holds 19 pulled offsets and 19 four-value colour
// records per node: with FP32 offsets 3 CTAs (85 registers) measured faster
// than 4 (106 against 115 us per 256x128x128 launch), with 16-bit offsets 4
// (91 against 125 us)
#ifndef LBM_PHI_MINB
#define LBM_PHI_MINB 4
#endif
#ifndef LBM_PHI_MINB_F32
#define LBM_PHI_MINB_F32 3
#endif
// CTAs per SM of the boundary passes, which run beside the bulk kernels
#ifndef LBM_BOUND_MINB
#define LBM_BOUND_MINB 2
#endif
// CTAs of 256 threads per SM of the one-node collision: 5 (48 registers, no
// spill) measured faster than 4 (64 registers) and 6 (40, spilling): 123
// against 127 and 148 us per FP32 256x128x128 launch
#ifndef LBM_COLLIDE_MINB
#define LBM_COLLIDE_MINB 5
#endif

namespace lbmg {

// ---------------------------------------------------------------------------
// bulk kernels over all nodes, list kernels over the nodes next to solids
// ---------------------------------------------------------------------------
// order parameter of a fluid node none of whose neighbours is solid; the
// boundary pass (k_phi_bound) does the others.  Keeping the bounce-back code
// out of the bulk kernel keeps its loads in flight (with it compiled in, the
// kernel ran 75% longer).
template <class S>
__device__ __forceinline__ void phi_body(const Lattice &L, const InstDev &I, int cur, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    const long long g = I.node_off + n;
    const uint8_t fl = L.flags[g];
    const Pop<S> in(L.pop[cur], I);
    const ColourOf<S> C(L, I);
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    R v = phi_fluid<S>(nb, in, C);
    keep(v);
    if ((fl & OWNER_MASK) != OWN_FLUID || (fl & BOUND_BIT)) return;
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

template <class S>
__global__ void __launch_bounds__(ROW_NODES, sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? LBM_PHI_MINB_F32 : LBM_PHI_MINB))
    k_phi(Lattice L, int cur)
{
    pdl_trigger();  // the gradient pass may be scheduled as this grid drains
    for_item_nodes(L, blockIdx.x, [&](const InstDev &I, int n, int x, int y, int z) { phi_body<S>(L, I, cur, n, x, y, z); });
}

// instance of global node g (binary search over the node offsets)
__device__ __forceinline__ int inst_of_node(const Lattice &L, long long g)
{
    int lo = 0, hi = L.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.inst[mid].node_off <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// static solid nodes with a neighbour that is not static solid: the only
// static nodes the solid-phi fill can reach.  count pass (list == null) or
// fill pass; the order of the list does not matter.
__global__ void k_static_bound(Lattice L, long long *list, unsigned long long *count, int mode)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L.Ntot || own_static(L.flags[g] & OWNER_MASK) != (mode == 0)) return;
    const InstDev &I = L.inst[inst_of_node(L, g)];
    const int n = (int)(g - I.node_off);
    const int x = n % I.nx, y = (n / I.nx) % I.ny, z = n / (I.nx * I.ny);
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    const uint8_t *fli = L.flags + I.node_off;
    bool hit = false;
#pragma unroll
    for (int i = 1; i < Q; i++) hit |= own_static(fli[nb.at(cx(i), cy(i), cz(i))] & OWNER_MASK) != (mode == 0);
    if (!hit) return;
    const unsigned long long k = atomicAdd(count, 1ull);
    if (list) list[k] = g;
}

// solid-phi fill of the listed static nodes
template <class R>
__global__ void k_solidphi_list(Lattice L)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n_static) return;
    const long long g = L.static_list[i];
    const InstDev &I = L.inst[inst_of_node(L, g)];
    const int n = (int)(g - I.node_off);
    const int x = n % I.nx, y = (n / I.nx) % I.ny, z = n / (I.nx * I.ny);
    solidphi_body<R>(L, I, n, x, y, z);
}

void launch_static_bound(const Lattice &L, long long *list, unsigned long long *count, int mode, cudaStream_t st)
{
    k_static_bound<<<(unsigned)((L.Ntot + 255) / 256), 256, 0, st>>>(L, list, count, mode);
}


// the fluid nodes next to a solid inside the particle cubes (cubes of side
// cap_side around each particle, cap_blocks CTAs each), appended to L.pbl
// with one atomic per warp: the particle part of the boundary passes' work
// list, rebuilt at the start of every step (the flags do not change within
// a step); likewise the solid nodes next to fluid, for the solid-phi fill,
// to L.psl.  Order within a list does not matter; a node in two cubes is
// listed twice and written twice with the same value.
__global__ void __launch_bounds__(PART_THREADS) k_bound_list(Lattice L)
{
    const long long b = blockIdx.x;
    const long long t = (b % L.cap_blocks) * blockDim.x + threadIdx.x;
    const PartDev &P0 = L.parts[b / L.cap_blocks];
    const InstDev &I = L.inst[P0.inst];
    Region reg;
    reg.init(P0.x, L.cap_side, I.nx, I.ny, I.nz);
    bool fluid = false, solid = false;
    long long g = 0;
    if (t < reg.count()) {
        int x, y, z;
        reg.coord(t, I.nx, I.ny, I.nz, &x, &y, &z);
        g = I.node_off + ((long long)z * I.ny + y) * I.nx + x;
        const uint8_t fl = L.flags[g];
        fluid = (fl & OWNER_MASK) == OWN_FLUID && (fl & BOUND_BIT);
        solid = (fl & OWNER_MASK) != OWN_FLUID && (fl & BOUND_BIT);
    }
    const int lane = threadIdx.x & 31;
    auto append = [&](bool take, long long *list, unsigned long long *count) {
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (!m) return;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (take) list[base + __popc(m & ((1u << lane) - 1u))] = g;
    };
    append(fluid, L.pbl, L.pbl_n);
    append(solid, L.psl, L.psl_n);
}

// work item t of the boundary passes: the listed particle nodes, then the
// static list of nodes next to static solids
__device__ __forceinline__ void bound_item(const Lattice &L, long long npb, long long t, const InstDev **Ip, int *n,
                                           int *x, int *y, int *z)
{
    const long long g = t < npb ? L.pbl[t] : L.static_bfl[t - npb];
    const InstDev &I = L.inst[inst_of_node(L, g)];
    *n = (int)(g - I.node_off);
    *x = *n % I.nx;
    *y = (*n / I.nx) % I.ny;
    *z = *n / (I.nx * I.ny);
    *Ip = &I;
}

// the boundary passes: fluid nodes next to a solid, with the bounce-back
// pull (Sec. V A), grid-stride over the work list; a node listed twice (two
// cubes, or a cube and the static list) is written twice with the same value
template <class S>
__device__ __forceinline__ void phi_bound_node(const Lattice &L, int cur, const InstDev *I, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    const long long g = I->node_off + n;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID || !(fl & BOUND_BIT)) return;
    const Pop<S> in(L.pop[cur], *I);
    const ColourOf<S> C(L, *I);
    GlobalNbr nb;
    nb.nb.init(x, y, z, I->nx, I->ny, I->nz);
    nb.fli = L.flags + I->node_off;
    R F[Q], sF = 0, sG = 0;
    gather_all<S>(*I, L.parts, nb, in, &C, n, F, &sG, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; i++) sF += wgt<R>(i) * F[i];
    ((R *)L.phi)[g] = sG / (R(1) + sF);
}

template <class S>
__global__ void __launch_bounds__(PART_THREADS, LBM_BOUND_MINB) k_phi_bound(Lattice L, int cur)
{
    const long long npb = L.pbl_n ? (long long)*L.pbl_n : 0;
    const long long total = npb + L.n_static_bfl;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const InstDev *I;
        int n, x, y, z;
        bound_item(L, npb, t, &I, &n, &x, &y, &z);
        phi_bound_node<S>(L, cur, I, n, x, y, z);
    }
}

template <class S>
__device__ __forceinline__ void collide_bound_node(const Lattice &L, int cur, const InstDev *I, int n, int x, int y,
                                                   int z)
{
    using R = typename Store<S>::real;
    const long long g = I->node_off + n;
    const uint8_t fl = L.flags[g];
    if ((fl & OWNER_MASK) != OWN_FLUID || !(fl & BOUND_BIT)) return;
    const Pop<S> in(L.pop[cur], *I);
    const Pop<S> out(L.pop[cur ^ 1], *I);
    const R *Nn = (const R *)L.grad + I->node_off;
    const long long Nt = L.Ntot;
    R *U = I->store_u ? (R *)L.u + I->node_off : nullptr;
    GlobalNbr nb;
    nb.nb.init(x, y, z, I->nx, I->ny, I->nz);
    nb.fli = L.flags + I->node_off;
    R F[Q];
    gather_all<S>(*I, L.parts, nb, in, (const ColourOf<S> *)nullptr, n, F, (R *)nullptr, x, y, z);
    FluidPar<R> P;
    load_par(*I, P);
    const R m = ((const R *)L.gmag)[g];
    const R gr[3] = {Nn[n] * m, Nn[Nt + n] * m, Nn[2 * Nt + n] * m};
    const R nn[3] = {Nn[n], Nn[Nt + n], Nn[2 * Nt + n]};
    collide_store_phi<S>(P, F, ((const R *)L.phi)[g], gr, nn, ((const R *)L.kap)[g], out, n,
                         col_slot<S>(L, g), U, L.Ntot, L.status);
}

template <class S>
__global__ void __launch_bounds__(PART_THREADS, LBM_BOUND_MINB) k_collide_bound(Lattice L, int cur)
{
    const long long npb = L.pbl_n ? (long long)*L.pbl_n : 0;
    const long long total = npb + L.n_static_bfl;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const InstDev *I;
        int n, x, y, z;
        bound_item(L, npb, t, &I, &n, &x, &y, &z);
        collide_bound_node<S>(L, cur, I, n, x, y, z);
    }
}

// solid-phi fill of the listed particle-surface solid nodes, grid-stride
template <class R>
__global__ void __launch_bounds__(PART_THREADS) k_solidphi_plist(Lattice L)
{
    const long long nps = (long long)*L.psl_n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nps;
         t += (long long)gridDim.x * blockDim.x) {
        const long long g = L.psl[t];
        const InstDev &I = L.inst[inst_of_node(L, g)];
        const int n = (int)(g - I.node_off);
        solidphi_body<R>(L, I, n, n % I.nx, (n / I.nx) % I.ny, n / (I.nx * I.ny));
    }
}

template <class S>
__device__ __forceinline__ void collide_body(const Lattice &L, const InstDev &I, int cur, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    const long long g = I.node_off + n;
    const Pop<S> in(L.pop[cur], I);
    const Pop<S> out(L.pop[cur ^ 1], I);
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
    for (int i = 0; i < Q; i++) F[i] = in.F(i, nb.at(-cx(i), -cy(i), -cz(i)));
#pragma unroll
    for (int i = 0; i < Q; i++) keep(F[i]);
    R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
    if ((fl & OWNER_MASK) != OWN_FLUID) {
        if (U) { U[n] = 0; U[L.Ntot + n] = 0; U[2 * L.Ntot + n] = 0; }
        return;
    }
    // nodes next to a solid belong to the boundary pass k_collide_bound
    if (fl & BOUND_BIT) return;
    FluidPar<R> P;
    load_par(I, P);
    const R gr[3] = {nn[0] * m, nn[1] * m, nn[2] * m};
    collide_store_phi<S>(P, F, phi, gr, nn, kap, out, n, col_slot<S>(L, g), U, L.Ntot, L.status);
}

// Node pairs (x even, x + 1) of one row per thread, for 16-bit storage: the
// pulls along directions with c_x = 0 are one 32-bit load of the pair, every
// output a pair store (half2, bfloat162 or float2), which halves the
// per-node load, store, conversion and address instructions.  Each node's
// arithmetic is that of collide_store_phi (the same expressions; the code
// generator may fuse a different set of multiply-adds, so the results agree
// to rounding); a node of the pair that the bulk kernel skips (solid, next to
// a solid) is computed but not written.
template <class S>
__device__ __forceinline__ void collide_body2(const Lattice &L, const InstDev &I, int cur, int n, int x, int y, int z)
{
    using R = typename Store<S>::real;
    using FT = typename Pop<S>::FT;
    static_assert(sizeof(FT) == 2 && sizeof(R) == 4, "pair kernel: 16-bit total offsets, FP32 arithmetic");
    const long long g = I.node_off + n;  // even
    const Pop<S> in(L.pop[cur], I);
    const Pop<S> out(L.pop[cur ^ 1], I);
    const int N = in.N;
    const uint8_t fl0 = L.flags[g], fl1 = L.flags[g + 1];
    const R *Nn = (const R *)L.grad + I.node_off;
    const long long Nt = L.Ntot;
    const float2 n0 = *reinterpret_cast<const float2 *>(Nn + n);
    const float2 n1 = *reinterpret_cast<const float2 *>(Nn + Nt + n);
    const float2 n2 = *reinterpret_cast<const float2 *>(Nn + 2 * Nt + n);
    const float2 mv = *reinterpret_cast<const float2 *>((const R *)L.gmag + g);
    const float2 kv = *reinterpret_cast<const float2 *>((const R *)L.kap + g);
    const float2 pv = *reinterpret_cast<const float2 *>((const R *)L.phi + g);
    Nbr nb;
    nb.init(x, y, z, I.nx, I.ny, I.nz);
    const int xp2 = x + 2 == I.nx ? 0 : x + 2;
    R F0[Q], F1[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const FT *row = in.f + i * N + nb.ZO[1 - cz(i)] + nb.YO[1 - cy(i)];
        if (cx(i) == 0) {
            ld_pair(row + x, F0[i], F1[i]);
        } else if (cx(i) == 1) {
            F0[i] = Store<FT>::ld(row + nb.X[0]);
            F1[i] = Store<FT>::ld(row + x);
        } else {
            F0[i] = Store<FT>::ld(row + x + 1);
            F1[i] = Store<FT>::ld(row + xp2);
        }
    }
#pragma unroll
    for (int i = 0; i < Q; i++) {
        keep(F0[i]);
        keep(F1[i]);
    }
    const bool fluid0 = (fl0 & OWNER_MASK) == OWN_FLUID, fluid1 = (fl1 & OWNER_MASK) == OWN_FLUID;
    const bool a0 = fluid0 && !(fl0 & BOUND_BIT), a1 = fluid1 && !(fl1 & BOUND_BIT);
    R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
    if (U) {
        if (!fluid0) { U[n] = 0; U[Nt + n] = 0; U[2 * Nt + n] = 0; }
        if (!fluid1) { U[n + 1] = 0; U[Nt + n + 1] = 0; U[2 * Nt + n + 1] = 0; }
    }
    if (!a0 && !a1) return;
    FluidPar<R> P;
    load_par(I, P);
    const R grA[3] = {n0.x * mv.x, n1.x * mv.x, n2.x * mv.x};
    const R grB[3] = {n0.y * mv.y, n1.y * mv.y, n2.y * mv.y};
    const R phA = pv.x, phB = pv.y;
    const CollideState<R> cA = collide_state(P, F0, phA, grA, kv.x);
    const CollideState<R> cB = collide_state(P, F1, phB, grB, kv.y);
    if ((a0 && (!(cA.rr > R(0)) || !(phA == phA))) || (a1 && (!(cB.rr > R(0)) || !(phB == phB))))
        atomicOr(L.status, ST_UNSTABLE);
    if (U) {
        if (a0) { U[n] = cA.ux; U[Nt + n] = cA.uy; U[2 * Nt + n] = cA.uz; }
        if (a1) { U[n + 1] = cB.ux; U[Nt + n + 1] = cB.uy; U[2 * Nt + n + 1] = cB.uz; }
    }
    FT *const of = out.f + n;
    const bool both = a0 && a1;
    auto put = [&](auto *p, R v0, R v1) {
        using T = std::remove_pointer_t<decltype(p)>;
        if (both) {
            st_pair(p, v0, v1);
        } else if (a0) {
            Store<T>::st(p, v0);
        } else {
            Store<T>::st(p + 1, v1);
        }
    };
    {
        if (a0) col_slot<S>(L, g).set(ColRec<R>{phA, cA.bq * n0.x, cA.bq * n1.x, cA.bq * n2.x});
        if (a1) col_slot<S>(L, g + 1).set(ColRec<R>{phB, cB.bq * n0.y, cB.bq * n1.y, cB.bq * n2.y});
    }
    put(of, collide_rest(P, cA, F0[0]), collide_rest(P, cB, F1[0]));
    PairLoop<R>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value, ib = i + 9;
        R FiA, FibA, FiB, FibB;
        collide_pair<R, i>(P, cA, F0[i], F0[ib], FiA, FibA);
        collide_pair<R, i>(P, cB, F1[i], F1[ib], FiB, FibB);
        put(of + i * N, FiA, FiB);
        put(of + ib * N, FibA, FibB);
    });
}

// CTAs of 128 threads per SM the node-pair collision is compiled for: 6 (80
// registers, 60 bytes spilled) measured faster than 4 (128 registers, no
// spill), 5, 7 and 8 (105, 102, 100 and 109 against 96 us per 256x128x128
// launch): the pulls of more node pairs in flight outweigh the spill traffic
#ifndef LBM_COLLIDE2_MINB
#define LBM_COLLIDE2_MINB 6
#endif
template <class S>
__global__ void __launch_bounds__(ROW_NODES / 2, LBM_COLLIDE2_MINB) k_collide2(Lattice L, int cur)
{
    StItem it;
    st_item(L, blockIdx.x, it);
    pdl_wait();  // the gradient pass's normals, |grad phi| and curvature
    const int j = 2 * (int)threadIdx.x;
    if (j >= it.cnt) return;
    const InstDev &I = L.inst[it.k];
    int x, y;
    item_node(I, it, j, &x, &y);
    collide_body2<S>(L, I, cur, (it.z * I.ny + y) * I.nx + x, x, y, it.z);
}

template <class S>
__global__ void __launch_bounds__(ROW_NODES, sizeof(S) == 8 ? 1 : LBM_COLLIDE_MINB) k_collide(Lattice L, int cur)
{
    for_item_nodes(L, blockIdx.x, [&](const InstDev &I, int n, int x, int y, int z) {
        pdl_wait();  // the gradient pass's normals, |grad phi| and curvature
        collide_body<S>(L, I, cur, n, x, y, z);
    });
}

// ---------------------------------------------------------------------------
// gradient, wetting, normal and curvature in one z-marching pass
// ---------------------------------------------------------------------------
// A CTA owns a GC_TX x GC_TY column tile and a chunk of z-planes.  Step j loads
// phi of plane z0-2+j (2-node halo) into a 3-plane ring, forms the normals of
// plane z0-3+j on the 1-halo tile into a second 3-plane ring (and writes
// those of its own planes), and the curvature of plane z0-4+j from the normal
// ring.  Each phi value is read from L2/HBM about 1.7 times, the normal once
// per CTA; the per-node arithmetic is that of grad_body and the curvature
// of the fused kernel.
constexpr int GC_TX = 32, GC_TY = 8, GC_ZC = 16;

// a mod n in [0, n): the in-range and one-period cases without a division
__device__ __forceinline__ int wrap_any(int a, int n)
{
    if (a >= 0 && a < n) return a;
    if (a < 0 && a >= -n) return a + n;
    if (a >= n && a < 2 * n) return a - n;
    a %= n;
    return a < 0 ? a + n : a;
}

// owners of the neighbours of a node from the shared-memory flag ring
template <int PW>
struct GcNbr {
    const uint8_t *fl[3];  // flag planes z-1, z, z+1
    int c;                 // index of the node in the plane region
    __device__ __forceinline__ int own(int dx, int dy, int dz) const
    {
        return fl[dz + 1][c + dy * PW + dx] & OWNER_MASK;
    }
};

template <class R>
#ifndef LBM_GC_MINB
#define LBM_GC_MINB 4
#endif
__global__ void __launch_bounds__(GC_TX *GC_TY, sizeof(R) == 8 ? 2 : LBM_GC_MINB) k_gradcurv(Lattice L)
{
    constexpr int NT = GC_TX * GC_TY;
    constexpr int PW = GC_TX + 4, PH = GC_TY + 4, PN = PW * PH;  // phi / flag region (2-node halo)
    constexpr int NW = GC_TX + 2, NH = GC_TY + 2, NN = NW * NH;  // normal region (1-node halo)
    constexpr int PER = (PN + NT - 1) / NT;                       // region values per thread
    __shared__ R phS[3][PN];
    __shared__ uint8_t flS[4][PN];
    __shared__ R nS[3][3][NN];

    const long long item = blockIdx.x;
    int k = 0;
    {
        int lo = 0, hi = L.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.inst[mid].gc_item_start <= item) lo = mid;
            else hi = mid - 1;
        }
        k = lo;
    }
    const InstDev &I = L.inst[k];
    const int loc = (int)(item - I.gc_item_start);
    const int t2 = I.fd_nchunks.div(loc);
    const int chunk = loc - t2 * I.gc_nchunks;
    const int ty = I.fd_tiles_x.div(t2);
    const int x0 = (t2 - ty * I.gc_tiles_x) * GC_TX, y0 = ty * GC_TY;
    const int z0 = chunk * I.gc_zc, z1 = min(z0 + I.gc_zc, I.nz);
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long off = I.node_off, Nt = L.Ntot;
    const uint8_t *fli = L.flags + off;
    const R *ph = (const R *)L.phi + off;
    R *Nn = (R *)L.grad + off;
    R *Gm = (R *)L.gmag + off;
    R *Kp = (R *)L.kap + off;
    FluidPar<R> P;
    load_par(I, P);
    const int tid = threadIdx.x, lx = tid % GC_TX, ly = tid / GC_TX;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool active = gx < nx && gy < ny;
    const int niter = (z1 - z0) + 4;

    // this thread's columns of the 1-halo normal region (fixed for all planes)
    constexpr int PER1 = (NN + NT - 1) / NT;
    int nX[PER1], nY[PER1];
    bool nOwn[PER1];
#pragma unroll
    for (int q = 0; q < PER1; q++) {
        const int r1 = tid + q * NT, ax = r1 % NW, ay = r1 / NW;
        nX[q] = wrap_any(x0 - 1 + ax, nx);
        nY[q] = wrap_any(y0 - 1 + ay, ny);
        nOwn[q] = r1 < NN && ax >= 1 && ax <= GC_TX && ay >= 1 && ay <= GC_TY && x0 - 1 + ax < nx && y0 - 1 + ay < ny;
    }
    // this thread's share of a plane region, prefetched one step ahead
    int roff[PER];
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int r = tid + q * NT;
        roff[q] = r < PN ? wrap_any(y0 - 2 + r / PW, ny) * nx + wrap_any(x0 - 2 + r % PW, nx) : -1;
    }
    pdl_trigger();  // the collision may be scheduled as this grid drains
    pdl_wait();     // phi of the order-parameter pass
    R pv[PER];
    uint8_t fv[PER];
    auto fetch = [&](int j) {
        const int zo = wrap_any(z0 - 2 + j, nz) * ny * nx;
#pragma unroll
        for (int q = 0; q < PER; q++)
            if (roff[q] >= 0) {
                pv[q] = ph[zo + roff[q]];
                fv[q] = fli[zo + roff[q]];
            }
    };
    fetch(0);

    for (int j = 0; j < niter; j++) {
        // (1) plane z0-2+j into the rings, then fetch the next one
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int r = tid + q * NT;
            if (r < PN) {
                phS[j % 3][r] = pv[q];
                flS[j % 4][r] = fv[q];
            }
        }
        if (j + 1 < niter) fetch(j + 1);
        __syncthreads();
        // (2) normals of plane zz = z0-3+j (phi planes of steps j-2..j) on the 1-halo tile
        if (j >= 2) {
            const int zz = z0 - 3 + j;
            const int Z = wrap_any(zz, nz);
            const R *pm = phS[(j - 2) % 3], *p0 = phS[(j - 1) % 3], *pp = phS[j % 3];
            const bool own_plane = zz >= z0 && zz < z1;
            GcNbr<PW> nb;
            nb.fl[0] = flS[(j - 2) % 4];
            nb.fl[1] = flS[(j - 1) % 4];
            nb.fl[2] = flS[j % 4];
#pragma unroll
            for (int q = 0; q < PER1; q++) {
                const int r1 = tid + q * NT;
                if (r1 >= NN) break;
                const int ax = r1 % NW, ay = r1 / NW;
                const int c = (ay + 1) * PW + (ax + 1);
                const uint8_t fl = nb.fl[1][c];
                R nn[3] = {0, 0, 0};
                if ((fl & OWNER_MASK) == OWN_FLUID) {
                    auto phi_of = [&](int dx, int dy, int dz) {
                        const R *pl = dz < 0 ? pm : (dz > 0 ? pp : p0);
                        return pl[c + dy * PW + dx];
                    };
                    R gr[3];
                    grad_sum<R>(phi_of, gr);
                    const int X = nX[q], Y = nY[q];
                    if (fl & BOUND_BIT) {
                        nb.c = c;
                        grad_wet<R>(I, L.parts, nb, p0[c], fl, P.wet_max, X, Y, Z, gr);
                    }
                    const R m = reg_normal(gr, P.eps2, nn);
                    if (own_plane && nOwn[q]) {
                        const int n = (Z * ny + Y) * nx + X;
                        Nn[n] = nn[0];
                        Nn[Nt + n] = nn[1];
                        Nn[2 * Nt + n] = nn[2];
                        Gm[n] = m;
                    }
                }
                nS[j % 3][0][r1] = nn[0];
                nS[j % 3][1][r1] = nn[1];
                nS[j % 3][2][r1] = nn[2];
            }
        }
        __syncthreads();
        // (3) curvature of plane z = z0-4+j (normals of steps j-2..j, flags of steps j-3..j-1)
        if (j >= 4 && active) {
            const int z = z0 - 4 + j;
            const int cp = (ly + 2) * PW + (lx + 2);
            const uint8_t fl = flS[(j - 2) % 4][cp];
            if ((fl & OWNER_MASK) == OWN_FLUID) {
                const int c = (ly + 1) * NW + (lx + 1);
                const int sl[3] = {(j - 2) % 3, (j - 1) % 3, j % 3};
                R kap = curvature<R>([&](int dx, int dy, int dz, int a) { return nS[sl[dz + 1]][a][c + dy * NW + dx]; });
                if (fl & BOUND_BIT) {
                    GcNbr<PW> fb;
                    fb.fl[0] = flS[(j - 3) % 4];
                    fb.fl[1] = flS[(j - 2) % 4];
                    fb.fl[2] = flS[(j - 1) % 4];
                    fb.c = cp;
                    kap = curvature<R>([&](int dx, int dy, int dz, int a) {
                        if (fb.own(dx, dy, dz) != OWN_FLUID) return nS[sl[1]][a][c];
                        return nS[sl[dz + 1]][a][c + dy * NW + dx];
                    });
                }
                Kp[(z * ny + gy) * nx + gx] = kap;
            }
        }
        __syncthreads();
    }
}

long long plan_gradcurv(std::vector<InstDev> &inst, int zc_request, const std::vector<int> &zc_inst)
{
    long long items = 0;
    for (size_t k = 0; k < inst.size(); k++) {
        InstDev &I = inst[k];
        const int req = k < zc_inst.size() && zc_inst[k] > 0 ? zc_inst[k] : zc_request;
        I.gc_tiles_x = (I.nx + GC_TX - 1) / GC_TX;
        I.gc_tiles_y = (I.ny + GC_TY - 1) / GC_TY;
        const int zc = std::min(req > 0 ? req : GC_ZC, I.nz);
        I.gc_nchunks = (I.nz + zc - 1) / zc;
        I.gc_zc = (I.nz + I.gc_nchunks - 1) / I.gc_nchunks;
        I.fd_nchunks.set(I.gc_nchunks);
        I.fd_tiles_x.set(I.gc_tiles_x);
        I.gc_item_start = items;
        items += (long long)I.gc_tiles_x * I.gc_tiles_y * I.gc_nchunks;
    }
    return items;
}

// row-strip work items of the bulk kernels: whole x-rows of one z-plane, at
// most ROW_NODES nodes per item, or one row cut into segments of at most
// ROW_NODES nodes
long long plan_rows(std::vector<InstDev> &inst)
{
    long long total = 0;
    for (auto &I : inst) {
        if (I.nx <= ROW_NODES) {
            I.st_rows = std::min(I.ny, ROW_NODES / I.nx);
            I.st_seg = I.nx;
            I.st_nseg = 1;
        } else {
            const int nseg = (I.nx + ROW_NODES - 1) / ROW_NODES;
            int seg = (I.nx + nseg - 1) / nseg;
            seg = (seg + 1) / 2 * 2;  // even: node pairs never straddle two items
            I.st_rows = 1;
            I.st_seg = seg;
            I.st_nseg = (I.nx + seg - 1) / seg;
        }
        I.st_ygroups = (I.ny + I.st_rows - 1) / I.st_rows;
        I.fd_plane.set(I.st_ygroups * I.st_nseg);
        I.fd_nseg.set(I.st_nseg);
        I.fd_nx.set(I.nx);
        I.st_item_start = total;
        total += (long long)I.nz * I.st_ygroups * I.st_nseg;
    }
    return total;
}

// launch with programmatic stream serialisation: the kernel may be scheduled
// while its predecessor in the stream drains (it calls pdl_wait first)
template <class... P, class... A>
static void launch_after(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class S>
void launch_fluid_step(const Lattice &L, int cur, cudaStream_t st, long long *launches, const Marker &mk,
                       const FluidLaunch &fz, const Hook &after_grad, const SideLane &lane)
{
    using R = typename Store<S>::real;
    const dim3 grid((unsigned)fz.rows);  // one CTA per row-strip work item
    const bool pair = sizeof(S) == 2 && fz.pair;
    // boundary passes: grid-stride over the listed particle nodes and the
    // static list of nodes next to walls
    const dim3 bgrid((unsigned)std::max(L.bound_ctas, 1));
    auto list_bound = [&](cudaStream_t s) {
        if (L.n_parts == 0) return;
        cudaMemsetAsync(L.pbl_n, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(L.psl_n, 0, sizeof(unsigned long long), s);
        k_bound_list<<<(unsigned)((long long)L.n_parts * L.cap_blocks), PART_THREADS, 0, s>>>(L);
        *launches += 1;
    };
    // phi of solid nodes next to fluid: the listed static nodes and the
    // particle-surface solid nodes the step's list scan found in the cubes.
    // It reads phi only at fluid nodes next to a solid, which the boundary
    // pass writes, so beside the bulk kernel it follows that pass on the side lane
    bool fill_done = false;
    auto fill_solid_phi = [&](cudaStream_t s) {
        if (L.n_static > 0) {
            k_solidphi_list<R><<<(unsigned)((L.n_static + 255) / 256), 256, 0, s>>>(L);
            *launches += 1;
        }
        if (L.n_parts > 0) {
            k_solidphi_plist<R><<<(unsigned)std::max(L.bound_ctas / 2, 1), PART_THREADS, 0, s>>>(L);
            *launches += 1;
        }
        fill_done = true;
    };
    // boundary pass beside (side lane) or after the bulk kernel; profiling
    // (no side lane) times the two separately
    auto bound_pass = [&](auto kernel, int bstage, int stage, auto &&bulk) {
        if (lane.side) {
            cudaEventRecord(lane.a, st);
            cudaStreamWaitEvent(lane.side, lane.a, 0);
            if (stage == STAGE_PHI) list_bound(lane.side);
            kernel<<<bgrid, PART_THREADS, 0, lane.side>>>(L, cur);
            if (stage == STAGE_PHI) fill_solid_phi(lane.side);
            cudaEventRecord(lane.b, lane.side);
            if (stage == STAGE_COLLIDE) lane.after_collide_bound();
            bulk();
            cudaStreamWaitEvent(st, lane.b, 0);
        } else {
            mk(stage, 0);
            bulk();
            mk(stage, 1);
            mk(bstage, 0);
            if (stage == STAGE_PHI) list_bound(st);
            kernel<<<bgrid, PART_THREADS, 0, st>>>(L, cur);
            mk(bstage, 1);
        }
        *launches += 1;
    };
    bound_pass(k_phi_bound<S>, STAGE_PHI_BOUND, STAGE_PHI, [&] { k_phi<S><<<grid, ROW_NODES, 0, st>>>(L, cur); });
    if (!fill_done) {
        mk(STAGE_SOLIDPHI, 0);
        fill_solid_phi(st);
        mk(STAGE_SOLIDPHI, 1);
    }
    mk(STAGE_GRAD, 0);
    launch_after(k_gradcurv<R>, dim3((unsigned)fz.gc_items), dim3(GC_TX * GC_TY), st, L);
    mk(STAGE_GRAD, 1);
    after_grad();
    bound_pass(k_collide_bound<S>, STAGE_COLLIDE_BOUND, STAGE_COLLIDE, [&] {
        if constexpr (sizeof(S) == 2) {
            if (pair) {
                launch_after(k_collide2<S>, grid, dim3(ROW_NODES / 2), st, L, cur);
                return;
            }
        }
        launch_after(k_collide<S>, grid, dim3(ROW_NODES), st, L, cur);
    });
    *launches += 3;
}


#define INST(S)                                                                                                   \
    template void launch_fluid_step<S>(const Lattice &, int, cudaStream_t, long long *, const Marker &,            \
                                       const FluidLaunch &, const Hook &, const SideLane &);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
