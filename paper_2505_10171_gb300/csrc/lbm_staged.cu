// Row-staged order-parameter and collision kernels (Sec. IV of arXiv
// 2505.10171): the same per-node arithmetic as the plain kernels, with the
// populations brought into shared memory by bulk asynchronous copies.
//
// A work item is a strip of one z-plane: st_rows whole x-rows (packed up to
// ST_SEGMAX nodes), or one segment of a longer row.  Pull streaming reads, for
// population q with velocity c, the strip shifted by -c; for a strip that is a
// run of whole rows that source is again a run of whole rows of plane z - c_z
// (two runs where it wraps in y), so each population of an item arrives with
// one or two cp.async.bulk copies and the x-shift (with its periodic wrap) is
// applied when reading shared memory.  A segment of a long row is copied with
// 16 bytes of halo on both sides; its two end nodes of the row, and every
// node next to a solid (bounce-back), take the plain global-memory gather.
//
// Each CTA is persistent: it walks items blockIdx.x, blockIdx.x + gridDim.x,
// ... through an NST-deep ring of shared-memory stages.  Warp 0 issues the
// copies of item k + NST while the CTA computes item k; each stage completes on
// an mbarrier that counts the bytes.  The HBM stream therefore stays busy
// independently of how many registers the collision needs.  Every wait is
// bounded: after about a second the kernel sets ST_TIMEOUT, waits (bounded)
// for its own copies in flight and returns.
#include "lbm_async.cuh"
#include "lbm_node.cuh"

namespace lbmg {

namespace {

// 16-byte asynchronous copy global -> shared (L2 only), and its group fences
__device__ __forceinline__ void cp16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// shared-memory stage: NROWS population strips of BUFW elements (all 38 for
// the order parameter, the 19 total offsets F for the collision), then (EXT)
// the normal n (3), |grad phi|_eps, curvature and order parameter of the
// strip's nodes, then its flags (from the 16-byte boundary below the first node)
// MINB CTAs share an SM; the ring is as deep as their share of the 228 KB of
// shared memory allows (2..8 stages)
template <class S, bool EXT, int MINB>
struct StLayout {
    using R = typename Store<S>::real;
    static constexpr int A = StagedCfg<S>::A;
    static constexpr int BUFW = ST_SEGMAX + 2 * A;
    static constexpr int NROWS = EXT ? Q : NPOP;
    static constexpr int NEXT = EXT ? 6 : 0;
    static constexpr size_t POP = (size_t)NROWS * BUFW * sizeof(S);
    static constexpr size_t EXTB = (size_t)NEXT * ST_SEGMAX * sizeof(R);
    static constexpr size_t FLB = ST_SEGMAX + 32;
    static constexpr size_t STAGE = (POP + EXTB + FLB + 127) / 128 * 128;
    static constexpr size_t HEAD = 128;  // the NST mbarriers
    static constexpr size_t BUDGET = (size_t)228 * 1024 / MINB - 1024 - HEAD;
    static constexpr int NST_FIT = (int)(BUDGET / STAGE);
    static constexpr int NST = NST_FIT > 8 ? 8 : NST_FIT;
    static_assert(NST >= 2, "two stages must fit");
    static constexpr size_t bytes() { return HEAD + NST * STAGE; }
};

// per-node arrays staged for the collision: n (3 components), |grad phi|_eps,
// curvature, order parameter
template <class R>
__device__ __forceinline__ const R *ext_array(const Lattice &L, int e)
{
    if (e < 3) return (const R *)L.grad + (long long)e * L.Ntot;
    return e == 3 ? (const R *)L.gmag : (e == 4 ? (const R *)L.kap : (const R *)L.phi);
}

// issue the copies of one item into a stage (all 32 lanes of warp 0)
template <class S, bool EXT, int MINB>
__device__ void st_issue(const Lattice &L, const void *pop_in, const StItem &it, unsigned char *stage, uint32_t bar,
                         int lane)
{
    using Ly = StLayout<S, EXT, MINB>;
    using R = typename Store<S>::real;
    constexpr int A = Ly::A;
    const InstDev &I = L.inst[it.k];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const S *in = (const S *)pop_in + NPOP * I.node_off;
    const int lo = it.whole ? 0 : max(it.x0 - A, 0);
    const int hi = it.whole ? nx : min(it.x0 + it.cnt + A, nx);
    const unsigned popb = (unsigned)(it.whole ? it.nrows * nx : hi - lo) * (unsigned)sizeof(S);
    const long long g0 = item_node0(I, it);
    const long long fst = g0 & ~15ll, fen = (g0 + it.cnt + 15) & ~15ll;
    const unsigned flb = (unsigned)(fen - fst);
    const unsigned extb = EXT ? (unsigned)it.cnt * (unsigned)sizeof(R) : 0u;
    if (lane == 0) mbar_arrive_expect_tx(bar, Ly::NROWS * popb + Ly::NEXT * extb + flb);
    __syncwarp();
    constexpr int NC = Ly::NROWS + Ly::NEXT + 1;
    for (int c = lane; c < NC; c += 32) {
        if (c < Ly::NROWS) {
            const int d = c < Q ? c : c - Q;
            const int zs = wrap1(it.z - cz(d), nz);
            const S *src = in + (long long)c * N + (long long)zs * ny * nx;
            unsigned char *dst = stage + (size_t)c * Ly::BUFW * sizeof(S);
            if (it.whole) {
                const int ys = wrap1(it.y0 - cy(d), ny);
                const int len1 = min(it.nrows, ny - ys);
                bulk_g2s(smem_addr(dst), src + (long long)ys * nx, (unsigned)(len1 * nx * sizeof(S)), bar);
                if (it.nrows > len1)
                    bulk_g2s(smem_addr(dst + (size_t)len1 * nx * sizeof(S)), src,
                             (unsigned)((it.nrows - len1) * nx * sizeof(S)), bar);
            } else {
                const int ys = wrap1(it.y0 - cy(d), ny);
                bulk_g2s(smem_addr(dst + (size_t)(lo - (it.x0 - A)) * sizeof(S)), src + (long long)ys * nx + lo,
                         popb, bar);
            }
        } else if (EXT && c < Ly::NROWS + Ly::NEXT) {
            const int e = c - Ly::NROWS;
            bulk_g2s(smem_addr(stage + Ly::POP + (size_t)e * ST_SEGMAX * sizeof(R)), ext_array<R>(L, e) + g0, extb,
                     bar);
        } else {
            bulk_g2s(smem_addr(stage + Ly::POP + Ly::EXTB), L.flags + fst, flb, bar);
        }
    }
}

// the same copies as st_issue, spread over all threads as 16-byte cp.async:
// warp w takes populations w, w + 8, ..., its lanes the 16-byte chunks of each
// source row; then the five per-node arrays and the flags
template <class S, bool EXT, int MINB>
__device__ __forceinline__ void st_issue_async(const Lattice &L, const void *pop_in, const StItem &it,
                                               unsigned char *stage)
{
    using Ly = StLayout<S, EXT, MINB>;
    using R = typename Store<S>::real;
    constexpr int A = Ly::A;
    constexpr int NW = ST_THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const InstDev &I = L.inst[it.k];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const S *in = (const S *)pop_in + NPOP * I.node_off;
    const int lo = it.whole ? 0 : max(it.x0 - A, 0);
    const int hi = it.whole ? nx : min(it.x0 + it.cnt + A, nx);
    const int nrows = it.whole ? it.nrows : 1;
    const int rowch = (hi - lo) * (int)sizeof(S) / 16;  // 16-byte chunks per copied row
    const int dst0 = it.whole ? 0 : (lo - (it.x0 - A)) * (int)sizeof(S);
    const int rowb = nx * (int)sizeof(S);
    for (int q = warp; q < Ly::NROWS; q += NW) {
        const int d = q < Q ? q : q - Q;
        const int zs = wrap1(it.z - cz(d), nz);
        const char *src = (const char *)(in + (long long)q * N + (long long)zs * ny * nx + lo);
        const uint32_t dst = smem_addr(stage + (size_t)q * Ly::BUFW * sizeof(S)) + dst0;
        for (int r = 0; r < nrows; r++) {
            const int ys = wrap1(it.y0 + r - cy(d), ny);
            const char *sr = src + (long long)ys * rowb;
            for (int ch = lane; ch < rowch; ch += 32) cp16(dst + r * rowb + 16 * ch, sr + 16 * ch);
        }
    }
    const long long g0 = item_node0(I, it);
    if (EXT && warp < Ly::NEXT) {
        const R *base = ext_array<R>(L, warp);
        const char *src = (const char *)(base + g0);
        const uint32_t dst = smem_addr(stage + Ly::POP + (size_t)warp * ST_SEGMAX * sizeof(R));
        const int nch = it.cnt * (int)sizeof(R) / 16;
        for (int ch = lane; ch < nch; ch += 32) cp16(dst + 16 * ch, src + 16 * ch);
    }
    if (warp == NW - 1) {
        const long long fst = g0 & ~15ll, fen = (g0 + it.cnt + 15) & ~15ll;
        const int nch = (int)(fen - fst) / 16;
        const uint32_t dst = smem_addr(stage + Ly::POP + Ly::EXTB);
        for (int ch = lane; ch < nch; ch += 32) cp16(dst + 16 * ch, L.flags + fst + 16 * ch);
    }
}

// shared-memory indices of the sources x-1, x, x+1 of node (x, row r) in a
// stage strip; `edge` marks the end nodes of a cut row, whose wrapped source
// is not in the strip
struct StSrc {
    int bm, b0, bp;
    bool edge;
};
template <int A>
__device__ __forceinline__ StSrc st_src(const StItem &it, int nx, int r, int x)
{
    StSrc s;
    if (it.whole) {
        const int rb = r * nx;
        s.bm = rb + (x == 0 ? nx - 1 : x - 1);
        s.b0 = rb + x;
        s.bp = rb + (x == nx - 1 ? 0 : x + 1);
        s.edge = false;
    } else {
        const int o = it.x0 - A;
        s.bm = x - 1 - o;
        s.b0 = x - o;
        s.bp = x + 1 - o;
        s.edge = x == 0 || x == nx - 1;
    }
    return s;
}

// the persistent pipeline shared by both kernels; body(it, stage) computes one
// item from a landed stage
template <class S, bool EXT, int MINB, class Body>
__device__ __forceinline__ void st_pipeline(const Lattice &L, const void *pop_in, long long n_items, Body &&body)
{
    using Ly = StLayout<S, EXT, MINB>;
    constexpr int NST = Ly::NST;
    extern __shared__ __align__(128) unsigned char st_smem[];
    const uint32_t bar0 = smem_addr(st_smem);
    auto bar = [&](int s) { return bar0 + 8u * (unsigned)s; };
    auto stage = [&](int s) { return st_smem + Ly::HEAD + (size_t)s * Ly::STAGE; };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; s++) mbar_init(bar(s), 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool producer = threadIdx.x < 32;
    if (producer)
        for (int s = 0; s < NST; s++) {
            const long long item = blockIdx.x + (long long)s * gridDim.x;
            if (item >= n_items) break;
            StItem it;
            st_item(L, item, it);
            st_issue<S, EXT, MINB>(L, pop_in, it, stage(s), bar(s), lane);
        }
    for (long long k = 0;; k++) {
        const long long item = blockIdx.x + k * gridDim.x;
        if (item >= n_items) break;
        const int s = (int)(k % NST);
        const bool ok = mbar_wait_bounded(bar(s), (unsigned)((k / NST) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(L.status, ST_TIMEOUT);
                // let this CTA's copies in flight land before it exits
                for (long long j = k; j < k + NST; j++) {
                    if (blockIdx.x + j * gridDim.x >= n_items) break;
                    mbar_wait_bounded(bar((int)(j % NST)), (unsigned)((j / NST) & 1));
                }
            }
            return;
        }
        StItem it;
        st_item(L, item, it);
        body(it, (const unsigned char *)stage(s));
        __syncthreads();  // every thread is done with stage s
        const long long nxt = item + (long long)NST * gridDim.x;
        if (producer && nxt < n_items) {
            StItem it2;
            st_item(L, nxt, it2);
            st_issue<S, EXT, MINB>(L, pop_in, it2, stage(s), bar(s), lane);
        }
    }
}

// the pipeline with cp.async staging: NST - 1 items in flight per thread; the
// barrier at the top of each iteration both publishes item k's copies and
// frees the stage of item k - 1 for item k + NST - 1 (no spin-waits)
template <class S, bool EXT, int MINB, class Body>
__device__ __forceinline__ void st_pipeline_async(const Lattice &L, const void *pop_in, long long n_items,
                                                  Body &&body)
{
    using Ly = StLayout<S, EXT, MINB>;
    constexpr int NST = Ly::NST;
    extern __shared__ __align__(128) unsigned char st_smem[];
    auto stage = [&](int s) { return st_smem + Ly::HEAD + (size_t)s * Ly::STAGE; };
    for (int s = 0; s < NST - 1; s++) {
        const long long item = blockIdx.x + (long long)s * gridDim.x;
        if (item < n_items) {
            StItem it;
            st_item(L, item, it);
            st_issue_async<S, EXT, MINB>(L, pop_in, it, stage(s));
        }
        cp_commit();
    }
    for (long long k = 0;; k++) {
        const long long item = blockIdx.x + k * gridDim.x;
        if (item >= n_items) break;
        cp_wait<NST - 2>();
        __syncthreads();
        const long long nxt = item + (long long)(NST - 1) * gridDim.x;
        if (nxt < n_items) {
            StItem it2;
            st_item(L, nxt, it2);
            st_issue_async<S, EXT, MINB>(L, pop_in, it2, stage((int)((k + NST - 1) % NST)));
        }
        cp_commit();
        StItem it;
        st_item(L, item, it);
        body(it, (const unsigned char *)stage((int)(k % NST)));
    }
    cp_wait<0>();
}

}  // namespace

// order parameter after streaming (same sums as node_phi)
template <class S, int MINB, bool ASYNC>
__global__ void __launch_bounds__(ST_THREADS, MINB) k_phi_staged(Lattice L, int cur, long long n_items)
{
    using R = typename Store<S>::real;
    using Ly = StLayout<S, false, MINB>;
    const void *pop_in = L.pop[cur];
    auto body = [&](const StItem &it, const unsigned char *stg) {
        const InstDev &I = L.inst[it.k];
        const int nx = I.nx, ny = I.ny, nz = I.nz;
        const Pop<S> in(pop_in, I);
        const S *sp = (const S *)stg;
        const long long g0 = item_node0(I, it);
        const uint8_t *sf = stg + Ly::POP + (g0 & 15);
        R *phi = (R *)L.phi;
        for (int j = threadIdx.x; j < it.cnt; j += ST_THREADS) {
            const uint8_t fl = sf[j];
            if ((fl & OWNER_MASK) != OWN_FLUID) continue;
            const int r = it.whole ? j / nx : 0;
            const int x = it.whole ? j - r * nx : it.x0 + j;
            const int y = it.y0 + r, z = it.z;
            const int n = (z * ny + y) * nx + x;
            const StSrc b = st_src<Ly::A>(it, nx, r, x);
            R v;
            if ((fl & BOUND_BIT) || b.edge) {
                v = phi_node_cold<S>(&I, L.parts, L.flags + I.node_off, in, n, fl, x, y, z);
            } else {
                R sF = 0, sG = 0;
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    const int o = cx(i) == 1 ? b.bm : (cx(i) == -1 ? b.bp : b.b0);
                    sF += wgt<R>(i) * Store<S>::lds(sp + i * Ly::BUFW + o);
                    sG += wgt<R>(i) * Store<S>::lds(sp + (Q + i) * Ly::BUFW + o);
                }
                v = sG / (R(1) + sF);
            }
            phi[I.node_off + n] = v;
        }
    };
    if constexpr (ASYNC) st_pipeline_async<S, false, MINB>(L, pop_in, n_items, body);
    else st_pipeline<S, false, MINB>(L, pop_in, n_items, body);
}

// force, collision, recolouring and write (same arithmetic as k_collide)
template <class S, int MINB, bool ASYNC>
__global__ void __launch_bounds__(ST_THREADS, MINB) k_collide_staged(Lattice L, int cur, long long n_items)
{
    using R = typename Store<S>::real;
    using Ly = StLayout<S, true, MINB>;
    const void *pop_in = L.pop[cur];
    auto body = [&](const StItem &it, const unsigned char *stg) {
        const InstDev &I = L.inst[it.k];
        const int nx = I.nx, ny = I.ny, nz = I.nz;
        const Pop<S> in(pop_in, I);
        const Pop<S> out(L.pop[cur ^ 1], I);
        const S *sp = (const S *)stg;
        const R *se = (const R *)(stg + Ly::POP);
        const long long g0 = item_node0(I, it);
        const uint8_t *sf = stg + Ly::POP + Ly::EXTB + (g0 & 15);
        R *U = I.store_u ? (R *)L.u + I.node_off : nullptr;
        FluidPar<R> P;
        load_par(I, P);
        for (int j = threadIdx.x; j < it.cnt; j += ST_THREADS) {
            const uint8_t fl = sf[j];
            const int r = it.whole ? j / nx : 0;
            const int x = it.whole ? j - r * nx : it.x0 + j;
            const int y = it.y0 + r, z = it.z;
            const int n = (z * ny + y) * nx + x;
            if ((fl & OWNER_MASK) != OWN_FLUID) {
                if (U) { U[n] = 0; U[L.Ntot + n] = 0; U[2 * L.Ntot + n] = 0; }
                continue;
            }
            const R nn[3] = {se[j], se[ST_SEGMAX + j], se[2 * ST_SEGMAX + j]};
            const R m = se[3 * ST_SEGMAX + j];
            const R kap = se[4 * ST_SEGMAX + j];
            const R phi = se[5 * ST_SEGMAX + j];
            const StSrc b = st_src<Ly::A>(it, nx, r, x);
            if ((fl & BOUND_BIT) || b.edge) {
                collide_node_cold<S>(&I, L.parts, L.flags + I.node_off, in, out, n, fl, x, y, z, phi, nn[0], nn[1],
                                     nn[2], m, kap, U, L.Ntot, L.status);
                continue;
            }
            const R gr[3] = {nn[0] * m, nn[1] * m, nn[2] * m};
            R F[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int o = cx(i) == 1 ? b.bm : (cx(i) == -1 ? b.bp : b.b0);
                F[i] = Store<S>::lds(sp + i * Ly::BUFW + o);
            }
            collide_store_phi<S>(P, F, phi, gr, nn, kap, out, n, U, L.Ntot, L.status);
        }
    };
    if constexpr (ASYNC) st_pipeline_async<S, true, MINB>(L, pop_in, n_items, body);
    else st_pipeline<S, true, MINB>(L, pop_in, n_items, body);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool plan_rows(std::vector<InstDev> &inst, size_t elem, long long *items)
{
    const int A = 16 / (int)elem;
    long long total = 0;
    bool ok = true;
    for (auto &I : inst) {
        if (I.nx % A) ok = false;
        if (I.nx <= ST_SEGMAX) {
            I.st_rows = std::min(I.ny, ST_SEGMAX / I.nx);
            I.st_seg = I.nx;
            I.st_nseg = 1;
        } else {
            const int nseg = (I.nx + ST_SEGMAX - 1) / ST_SEGMAX;
            int seg = (I.nx + nseg - 1) / nseg;
            seg = (seg + A - 1) / A * A;
            I.st_rows = 1;
            I.st_seg = seg;
            I.st_nseg = (I.nx + seg - 1) / seg;
        }
        I.st_ygroups = (I.ny + I.st_rows - 1) / I.st_rows;
        I.st_item_start = total;
        total += (long long)I.nz * I.st_ygroups * I.st_nseg;
    }
    *items = total;
    return ok;
}


// staged variants: 0 cp.async copies, two CTAs per SM; 1 bulk copies, two
// CTAs per SM; 2 cp.async copies, one CTA per SM with a deeper ring.  FP64
// keeps one CTA per SM throughout (its collision needs the full register file).
template <class S>
constexpr int minb_of(int variant)
{
    return sizeof(S) == 8 ? 1 : (variant == 2 ? 1 : 2);
}

template <class S, int V>
struct StVariant {
    static constexpr int MINB = minb_of<S>(V);
    static constexpr bool ASYNC = V != 1;
};

template <class S, int V>
static void grids_v(int *grid_phi, int *grid_collide, int cap)
{
    using Vt = StVariant<S, V>;
    grid_phi[V] =
        persistent_grid(k_phi_staged<S, Vt::MINB, Vt::ASYNC>, StLayout<S, false, Vt::MINB>::bytes(), cap);
    grid_collide[V] =
        persistent_grid(k_collide_staged<S, Vt::MINB, Vt::ASYNC>, StLayout<S, true, Vt::MINB>::bytes(), cap);
}

template <class S>
void staged_grids(int *grid_phi, int *grid_collide, int cap)
{
    grids_v<S, 0>(grid_phi, grid_collide, cap);
    grids_v<S, 1>(grid_phi, grid_collide, cap);
    grids_v<S, 2>(grid_phi, grid_collide, cap);
}

template <class S, int V>
static void staged_phi_v(const Lattice &L, int cur, const FluidLaunch &fz, cudaStream_t st)
{
    using Vt = StVariant<S, V>;
    const int grid = (int)std::min<long long>(fz.st_grid_phi[V], fz.st_items);
    k_phi_staged<S, Vt::MINB, Vt::ASYNC>
        <<<grid, ST_THREADS, StLayout<S, false, Vt::MINB>::bytes(), st>>>(L, cur, fz.st_items);
}

template <class S, int V>
static void staged_collide_v(const Lattice &L, int cur, const FluidLaunch &fz, cudaStream_t st)
{
    using Vt = StVariant<S, V>;
    const int grid = (int)std::min<long long>(fz.st_grid_collide[V], fz.st_items);
    k_collide_staged<S, Vt::MINB, Vt::ASYNC>
        <<<grid, ST_THREADS, StLayout<S, true, Vt::MINB>::bytes(), st>>>(L, cur, fz.st_items);
}

// variant fz.tile (0, 1 or 2)
template <class S>
void launch_staged_phi(const Lattice &L, int cur, const FluidLaunch &fz, cudaStream_t st)
{
    if (fz.tile == 1) staged_phi_v<S, 1>(L, cur, fz, st);
    else if (fz.tile == 2) staged_phi_v<S, 2>(L, cur, fz, st);
    else staged_phi_v<S, 0>(L, cur, fz, st);
}

template <class S>
void launch_staged_collide(const Lattice &L, int cur, const FluidLaunch &fz, cudaStream_t st)
{
    if (fz.tile == 1) staged_collide_v<S, 1>(L, cur, fz, st);
    else if (fz.tile == 2) staged_collide_v<S, 2>(L, cur, fz, st);
    else staged_collide_v<S, 0>(L, cur, fz, st);
}

#define INST(S)                                                                                   \
    template void staged_grids<S>(int *, int *, int);                                             \
    template void launch_staged_phi<S>(const Lattice &, int, const FluidLaunch &, cudaStream_t); \
    template void launch_staged_collide<S>(const Lattice &, int, const FluidLaunch &, cudaStream_t);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
