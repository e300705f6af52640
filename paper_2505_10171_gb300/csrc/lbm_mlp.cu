// Learned particle-force surrogate (an extension of the method, not in the
// paper): samples of the flow on a shell around each sphere feed a
// 400-128-128-6 tanh network whose output replaces the momentum-exchange and
// capillary forces.  The network runs and trains with BF16 operands on the
// fifth-generation tensor cores: tcgen05.mma with the accumulator in tensor
// memory, operands staged in shared memory, FP32 master weights, Adam.
//
// GEMM: C[m][n] = sum_k A(m,k) B(n,k), A(m,k) = A[m sam + k sak],
// B(n,k) = B[n sbn + k sbk] (bf16; zero outside the valid extents), one CTA of
// 128 threads per 128-row by BN-column tile.  Per 64-wide chunk of k the CTA
// writes A (128 x 64) and B (BN x 64) into shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices: along k
// LBO apart, along rows 128 bytes apart), with 16-byte loads where the operand
// is contiguous along k or along its rows; thread 0 issues four
// tcgen05.mma.kind::f16 (K = 16 each) and commits them to the stage's
// mbarrier.  Two stages: the chunk after is staged while the tensor core
// works on the one before, and a stage is refilled only once the commit of the
// chunk that read it has arrived (bounded waits).  The epilogue reads the FP32
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows)
// and applies bias, tanh or the tanh derivative.
#include <cmath>
#include <mutex>
#include <vector>

#include "lbm_async.cuh"
#include "lbm_internal.cuh"

namespace lbmg {

using bf16 = __nv_bfloat16;

namespace {

// ---------------------------------------------------------------------------
// tcgen05 wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// shared-memory matrix descriptor: start address, leading (k) and stride
// (row-group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D,
// M = 128, N = BN
template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

constexpr int GM = 128;  // tile rows (TMEM lanes)
constexpr int GK = 64;   // k per staged chunk
#ifndef LBM_GEMM_BN
#define LBM_GEMM_BN 64
#endif
constexpr int BNH = LBM_GEMM_BN;  // column tile of the GEMMs with 128 or more columns

// shared memory: two barriers and the TMEM slot, then two stages of A and B.
// A stage holds exactly its tile: the four MMAs of a chunk read core matrices
// 2j LBO + {0, LBO} + 16 row groups x 128 bytes, j < 4, i.e. 8 LBO bytes.
template <int BN>
struct GemmSmem {
    static constexpr int HEAD = 128;
    static constexpr int A_LBO = GM / 8 * 128;  // bytes between core matrices along k
    static constexpr int B_LBO = BN / 8 * 128;
    static constexpr int A_STAGE = GM * GK * 2;
    static constexpr int B_STAGE = BN * GK * 2;
    static constexpr int BYTES = HEAD + 2 * (A_STAGE + B_STAGE);
};
static_assert(GemmSmem<128>::BYTES <= 227 * 1024, "two stages fit in shared memory");

struct GemmArgs {
    int Mv, Nv, Kv;  // valid extents
    const bf16 *A;
    long long sam, sak;
    const bf16 *B;
    long long sbn, sbk;
    const float *bias;  // [n] or null
    int act;            // 0: none, 1: tanh, 2: times (1 - g(m,n)^2)
    const bf16 *g;
    long long sgm, sgn;
    float *C32;
    long long scm, scn;
    bf16 *C16;
    long long s16m, s16n;
    unsigned *status;
    int no_mma;            // fault injection: issue no MMA and no commit (the wait finds nothing arriving)
    long long wait_limit;  // clock cycles a wait on the commit barrier may take
};

// one chunk of rows r0.. (ROWS of them) and k0..k0+GK into the canonical
// layout.  vec: 1 = the operand is contiguous along k (sk = 1), 2 = along its
// rows (sr = 1), both with 16-byte aligned runs of 8 (checked by the caller):
// runs of 8 elements wholly inside the valid extents move as one 16-byte load;
// the rest element by element, zero outside the extents.
template <int ROWS>
__device__ __forceinline__ void stage_tile(const bf16 *P, long long sr, long long sk, int r0, int rv, int k0, int kv,
                                           int vec, unsigned char *dst)
{
    auto at = [&](int r, int k) {
        return (bf16 *)(dst + ((k >> 3) * (ROWS / 8) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
    };
    auto scalar8 = [&](int r, int k, int dr, int dk) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int gr = r0 + r + e * dr, gk = k0 + k + e * dk;
            bf16 v = __float2bfloat16_rn(0.0f);
            if (gr < rv && gk < kv) v = P[(long long)gr * sr + (long long)gk * sk];
            *at(r + e * dr, k + e * dk) = v;
        }
    };
    if (vec == 1) {
        // one core-matrix row (8 k values, 16 bytes) per vector
        for (int i = threadIdx.x; i < ROWS * (GK / 8); i += GM) {
            const int r = i / (GK / 8), k = (i % (GK / 8)) * 8;
            const int gr = r0 + r, gk = k0 + k;
            if (gr < rv && gk + 8 <= kv)
                *(uint4 *)at(r, k) = *(const uint4 *)(P + (long long)gr * sr + gk);
            else
                scalar8(r, k, 0, 1);
        }
    } else if (vec == 2) {
        // 8 rows at one k: a core-matrix column (consecutive threads take
        // consecutive k, whose 2-byte stores share 32-bit words)
        for (int i = threadIdx.x; i < (ROWS / 8) * GK; i += GM) {
            const int r = (i / GK) * 8, k = i % GK;
            const int gr = r0 + r, gk = k0 + k;
            if (gr + 8 <= rv && gk < kv) {
                const uint4 w = *(const uint4 *)(P + gr + (long long)gk * sk);
                const bf16 *h = (const bf16 *)&w;
#pragma unroll
                for (int e = 0; e < 8; e++) *at(r + e, k) = h[e];
            } else {
                scalar8(r, k, 1, 0);
            }
        }
    } else {
        for (int i = threadIdx.x; i < ROWS * GK; i += GM) {
            const int r = i / GK, k = i % GK;
            const int gr = r0 + r, gk = k0 + k;
            bf16 v = __float2bfloat16_rn(0.0f);
            if (gr < rv && gk < kv) v = P[(long long)gr * sr + (long long)gk * sk];
            *at(r, k) = v;
        }
    }
}

// which staging path an operand takes (the same for every thread of the grid)
__device__ __forceinline__ int vec_mode(const bf16 *P, long long sr, long long sk)
{
    if (((uintptr_t)P & 15) != 0) return 0;
    if (sk == 1 && sr % 8 == 0) return 1;
    if (sr == 1 && sk % 8 == 0) return 2;
    return 0;
}

template <int BN>
__global__ void __launch_bounds__(GM) k_gemm_tc(GemmArgs g)
{
    using Sm = GemmSmem<BN>;
    extern __shared__ __align__(1024) unsigned char gsm[];
    // stage st: A at As0 + st A_STAGE, B at Bs0 + st B_STAGE, barrier bar0 + 8 st
    unsigned char *const As0 = gsm + Sm::HEAD;
    unsigned char *const Bs0 = gsm + Sm::HEAD + 2 * Sm::A_STAGE;
    const uint32_t bar0 = smem_addr(gsm);
    const uint32_t slot = smem_addr(gsm + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * BN;
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;

    if (warp == 0) {
        tmem_alloc(slot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *(volatile uint32_t *)(gsm + 16);
    const int va = vec_mode(g.A, g.sam, g.sak), vb = vec_mode(g.B, g.sbn, g.sbk);

    // chunk c uses stage c & 1 and commits to that stage's barrier, whose
    // phases complete in chunk order, the one of chunk c having parity
    // (c >> 1) & 1, and at most one of its phases is ever pending
    const int nchunks = (g.Kv + GK - 1) / GK;
    bool ok = true;
    int last = -1;  // last chunk whose MMAs were committed
    for (int c = 0; c < nchunks; c++) {
        const int st = c & 1;
        if (c >= 2) {
            // the MMAs of chunk c - 2 read this stage
            ok = mbar_wait_bounded(bar0 + 8 * st, (unsigned)(((c - 2) >> 1) & 1), g.wait_limit);
            if (__syncthreads_or(!ok)) break;
            tc_fence_after();
        }
        unsigned char *const As = As0 + st * Sm::A_STAGE;
        unsigned char *const Bs = Bs0 + st * Sm::B_STAGE;
        stage_tile<GM>(g.A, g.sam, g.sak, m0, g.Mv, c * GK, g.Kv, va, As);
        stage_tile<BN>(g.B, g.sbn, g.sbk, n0, g.Nv, c * GK, g.Kv, vb, Bs);
        fence_async_smem();
        __syncthreads();
        if (tid == 0 && !g.no_mma) {
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < GK / 16; j++) {
                const uint64_t ad = smem_desc(smem_addr(As) + j * 2 * Sm::A_LBO, Sm::A_LBO, 128);
                const uint64_t bd = smem_desc(smem_addr(Bs) + j * 2 * Sm::B_LBO, Sm::B_LBO, 128);
                tc_mma_bf16(tmem, ad, bd, idesc_bf16<BN>(), (c > 0 || j > 0) ? 1u : 0u);
            }
            tc_commit(bar0 + 8 * st);
        }
        last = c;
    }
    // a commit covers every MMA this thread issued before it: the last one's
    // arrival means the accumulator is complete
    if (ok && last >= 0) {
        ok = mbar_wait_bounded(bar0 + 8 * (last & 1), (unsigned)((last >> 1) & 1), g.wait_limit);
        ok = !__syncthreads_or(!ok);
        tc_fence_after();
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(g.status, ST_TIMEOUT);
            // MMAs still in flight (none are issued under the fault injection)
            // must finish before the tensor memory is freed
            if (!g.no_mma && last >= 0) mbar_wait_bounded(bar0 + 8 * (last & 1), (unsigned)((last >> 1) & 1));
        }
    } else if (nchunks > 0) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (m < g.Mv) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int n = n0 + c0 + i;
                    if (n >= g.Nv) break;
                    float x = v[i];
                    if (g.bias) x += g.bias[n];
                    if (g.act == 1) {
                        x = tanhf(x);
                    } else if (g.act == 2) {
                        const float h = __bfloat162float(g.g[(long long)m * g.sgm + (long long)n * g.sgn]);
                        x *= 1.0f - h * h;
                    }
                    if (g.C32) g.C32[(long long)m * g.scm + (long long)n * g.scn] = x;
                    if (g.C16) g.C16[(long long)m * g.s16m + (long long)n * g.s16n] = __float2bfloat16_rn(x);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// k_gemm_tc<BN> needs more than 48 KiB of dynamic shared memory, a function
// attribute of each device: set once per device (under a lock, since
// contexts on several threads may reach here first together), with its result
// checked, before the first launch there
template <int BN>
static cudaError_t gemm_setup()
{
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static bool done[MAXDEV] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, GemmSmem<BN>::BYTES);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// returns the set-up's or this launch's own error
template <int BN>
cudaError_t gemm(const GemmArgs &a, int M, int N, cudaStream_t st)
{
    const cudaError_t e = gemm_setup<BN>();
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + BN - 1) / BN));
    void *args[] = {(void *)&a};
    return cudaLaunchKernel((const void *)k_gemm_tc<BN>, grid, dim3(GM), args, GemmSmem<BN>::BYTES, st);
}

GemmArgs gargs(int Mv, int Nv, int Kv, const bf16 *A, long long sam, long long sak, const bf16 *B, long long sbn,
               long long sbk, unsigned *status)
{
    GemmArgs a;
    memset(&a, 0, sizeof a);
    a.Mv = Mv; a.Nv = Nv; a.Kv = Kv;
    a.A = A; a.sam = sam; a.sak = sak;
    a.B = B; a.sbn = sbn; a.sbk = sbk;
    a.status = status;
    a.wait_limit = WAIT_CYCLES;
    return a;
}

// the GEMM arguments under the network's fault-injection setting: with it on,
// no MMA is issued and the commit barrier is never signalled, so the bounded
// wait (shortened to about a millisecond) runs out and reports a timeout
static GemmArgs mode(GemmArgs a, const Mlp &m)
{
    a.no_mma = m.fault_no_commit ? 1 : 0;
    if (a.no_mma) a.wait_limit = 1ll << 21;
    return a;
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------
constexpr int EW = 256;

// master weights -> bf16 copies used as GEMM operands
__global__ void k_refresh(const float *theta, bf16 *W1b, bf16 *W2b, bf16 *W3b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_HIDDEN * MLP_KIN) W1b[i] = __float2bfloat16_rn(theta[MLP_OFF_W1 + i]);
    if (i < MLP_HIDDEN * MLP_HIDDEN) W2b[i] = __float2bfloat16_rn(theta[MLP_OFF_W2 + i]);
    if (i < MLP_NOUT * MLP_HIDDEN) W3b[i] = __float2bfloat16_rn(theta[MLP_OFF_W3 + i]);
}

// rows idx[r] (or r) of fp32 features [*][387] -> bf16 inputs [n][400]
__global__ void k_stage_inputs(const float *X, const long long *idx, long long row0, int n, bf16 *Xb)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * MLP_KIN) return;
    const int r = (int)(t / MLP_KIN), c = (int)(t % MLP_KIN);
    const long long src = idx ? idx[row0 + r] : row0 + r;
    Xb[t] = __float2bfloat16_rn(c < MLP_NIN ? X[src * MLP_NIN + c] : 0.0f);
}

// targets of the batch rows -> T [n][6]
__global__ void k_stage_targets(const float *Y, const long long *idx, long long row0, int n, float *T)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * MLP_NOUT) return;
    const int r = t / MLP_NOUT, c = t % MLP_NOUT;
    const long long src = idx ? idx[row0 + r] : row0 + r;
    T[t] = Y[src * MLP_NOUT + c];
}

// dY = 2 (Y - T) / (6 n) (fp32 and bf16, ld 16 with zero columns 6..15),
// per-block partial sums of the squared error in FP64
__global__ void k_loss(const float *Y, const float *T, int n, float *dY, bf16 *dYb, double *part)
{
    __shared__ double sh[EW];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (t < n * 16) {
        const int r = t / 16, c = t % 16;
        float d = 0.0f;
        if (c < MLP_NOUT) {
            const float diff = Y[r * 16 + c] - T[r * MLP_NOUT + c];
            e2 = (double)diff * diff;
            d = 2.0f * diff / (float)(MLP_NOUT * n);
        }
        dY[t] = d;
        dYb[t] = __float2bfloat16_rn(d);
    }
    sh[threadIdx.x] = e2;
    __syncthreads();
    for (int s = EW / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// loss of the batch: fixed-order sum of the block partials; optionally added
// to an accumulator
__global__ void k_loss_final(const double *part, int nblk, int n, double *loss, double *acc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nblk; i++) s += part[i];
    const double l = s / ((double)n * MLP_NOUT);
    *loss = l;
    if (acc) *acc += l;
}

// column sums (bias gradients): out[c] = sum_r src[r ld + c], one block per column
template <class T>
__global__ void k_colsum(const T *src, int rows, int ld, float *out)
{
    __shared__ float sh[EW];
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int r = threadIdx.x; r < rows; r += EW) s += (float)src[(long long)r * ld + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = EW / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// Adam (Kingma and Ba 2015) on the FP32 master weights
__global__ void k_adam(float *theta, const float *grad, float *m, float *v, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
cudaError_t mlp_alloc(Mlp &m, int cap)
{
    m.cap = cap;
    auto A = [&](void **p, size_t b) { return cudaMalloc(p, b); };
    cudaError_t e;
    if ((e = A((void **)&m.theta, sizeof(float) * MLP_NPARAM)) || (e = A((void **)&m.grad, sizeof(float) * MLP_NPARAM)) ||
        (e = A((void **)&m.adam_m, sizeof(float) * MLP_NPARAM)) ||
        (e = A((void **)&m.adam_v, sizeof(float) * MLP_NPARAM)) ||
        (e = A((void **)&m.W1b, sizeof(bf16) * MLP_HIDDEN * MLP_KIN)) ||
        (e = A((void **)&m.W2b, sizeof(bf16) * MLP_HIDDEN * MLP_HIDDEN)) ||
        (e = A((void **)&m.W3b, sizeof(bf16) * MLP_NOUT * MLP_HIDDEN)) ||
        (e = A((void **)&m.X, sizeof(bf16) * (size_t)cap * MLP_KIN)) ||
        (e = A((void **)&m.H1, sizeof(bf16) * (size_t)cap * MLP_HIDDEN)) ||
        (e = A((void **)&m.H2, sizeof(bf16) * (size_t)cap * MLP_HIDDEN)) ||
        (e = A((void **)&m.dZ1, sizeof(bf16) * (size_t)cap * MLP_HIDDEN)) ||
        (e = A((void **)&m.dZ2, sizeof(bf16) * (size_t)cap * MLP_HIDDEN)) ||
        (e = A((void **)&m.dYb, sizeof(bf16) * (size_t)cap * 16)) || (e = A((void **)&m.Y, sizeof(float) * (size_t)cap * 16)) ||
        (e = A((void **)&m.dY, sizeof(float) * (size_t)cap * 16)) ||
        (e = A((void **)&m.T, sizeof(float) * (size_t)cap * MLP_NOUT)) ||
        (e = A((void **)&m.loss_part, sizeof(double) * ((size_t)cap * 16 / EW + 1))) ||
        (e = A((void **)&m.loss, sizeof(double) * 2)))
        return e;
    cudaMemset(m.adam_m, 0, sizeof(float) * MLP_NPARAM);
    cudaMemset(m.adam_v, 0, sizeof(float) * MLP_NPARAM);
    cudaMemset(m.loss, 0, sizeof(double) * 2);
    return cudaSuccess;
}

void mlp_free(Mlp &m)
{
    void *ps[] = {m.theta, m.grad, m.adam_m, m.adam_v, m.W1b, m.W2b, m.W3b, m.X, m.H1, m.H2,
                  m.dZ1, m.dZ2, m.dYb, m.Y, m.dY, m.T, m.loss_part, m.loss};
    for (void *p : ps) cudaFree(p);
    m = Mlp();
}

void mlp_refresh(const Mlp &m, cudaStream_t st)
{
    k_refresh<<<(MLP_HIDDEN * MLP_KIN + EW - 1) / EW, EW, 0, st>>>(m.theta, m.W1b, m.W2b, m.W3b);
}

void mlp_stage(const Mlp &m, const float *X, const float *Y, const long long *idx, long long row0, int n,
               cudaStream_t st)
{
    const long long t = (long long)n * MLP_KIN;
    k_stage_inputs<<<(unsigned)((t + EW - 1) / EW), EW, 0, st>>>(X, idx, row0, n, m.X);
    if (Y) k_stage_targets<<<(n * MLP_NOUT + EW - 1) / EW, EW, 0, st>>>(Y, idx, row0, n, m.T);
}

cudaError_t mlp_forward(const Mlp &m, int n, unsigned *status, cudaStream_t st)
{
    cudaError_t e;
    const float *b1 = m.theta + MLP_OFF_B1, *b2 = m.theta + MLP_OFF_B2, *b3 = m.theta + MLP_OFF_B3;
    // h1 = tanh(X W1^T + b1)
    GemmArgs a = gargs(n, MLP_HIDDEN, MLP_KIN, m.X, MLP_KIN, 1, m.W1b, MLP_KIN, 1, status);
    a.bias = b1; a.act = 1; a.C16 = m.H1; a.s16m = MLP_HIDDEN; a.s16n = 1;
    if ((e = gemm<BNH>(mode(a, m), n, MLP_HIDDEN, st)) != cudaSuccess) return e;
    // h2 = tanh(h1 W2^T + b2)
    a = gargs(n, MLP_HIDDEN, MLP_HIDDEN, m.H1, MLP_HIDDEN, 1, m.W2b, MLP_HIDDEN, 1, status);
    a.bias = b2; a.act = 1; a.C16 = m.H2; a.s16m = MLP_HIDDEN; a.s16n = 1;
    if ((e = gemm<BNH>(mode(a, m), n, MLP_HIDDEN, st)) != cudaSuccess) return e;
    // y = h2 W3^T + b3  ([n][16], columns 6..15 unused)
    a = gargs(n, MLP_NOUT, MLP_HIDDEN, m.H2, MLP_HIDDEN, 1, m.W3b, MLP_HIDDEN, 1, status);
    a.bias = b3; a.C32 = m.Y; a.scm = 16; a.scn = 1;
    if ((e = gemm<16>(mode(a, m), n, 16, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t mlp_backward(const Mlp &m, int n, double *acc, unsigned *status, cudaStream_t st)
{
    cudaError_t e;
    float *g = m.grad;
    const int nl = (n * 16 + EW - 1) / EW;
    k_loss<<<nl, EW, 0, st>>>(m.Y, m.T, n, m.dY, m.dYb, m.loss_part);
    k_loss_final<<<1, 32, 0, st>>>(m.loss_part, nl, n, m.loss, acc);
    // dW3[j][i] = sum_b dY[b][j] h2[b][i]   (M = hidden i, N = output j, K = batch)
    GemmArgs a = gargs(MLP_HIDDEN, MLP_NOUT, n, m.H2, 1, MLP_HIDDEN, m.dYb, 1, 16, status);
    a.C32 = g + MLP_OFF_W3; a.scm = 1; a.scn = MLP_HIDDEN;
    if ((e = gemm<16>(mode(a, m), MLP_HIDDEN, 16, st)) != cudaSuccess) return e;
    k_colsum<float><<<MLP_NOUT, EW, 0, st>>>(m.dY, n, 16, g + MLP_OFF_B3);
    // dz2 = (dY W3) * (1 - h2^2)
    a = gargs(n, MLP_HIDDEN, MLP_NOUT, m.dYb, 16, 1, m.W3b, 1, MLP_HIDDEN, status);
    a.act = 2; a.g = m.H2; a.sgm = MLP_HIDDEN; a.sgn = 1; a.C16 = m.dZ2; a.s16m = MLP_HIDDEN; a.s16n = 1;
    if ((e = gemm<BNH>(mode(a, m), n, MLP_HIDDEN, st)) != cudaSuccess) return e;
    // dW2[o][i] = sum_b dz2[b][o] h1[b][i]
    a = gargs(MLP_HIDDEN, MLP_HIDDEN, n, m.dZ2, 1, MLP_HIDDEN, m.H1, 1, MLP_HIDDEN, status);
    a.C32 = g + MLP_OFF_W2; a.scm = MLP_HIDDEN; a.scn = 1;
    if ((e = gemm<BNH>(mode(a, m), MLP_HIDDEN, MLP_HIDDEN, st)) != cudaSuccess) return e;
    k_colsum<bf16><<<MLP_HIDDEN, EW, 0, st>>>(m.dZ2, n, MLP_HIDDEN, g + MLP_OFF_B2);
    // dz1 = (dz2 W2) * (1 - h1^2)
    a = gargs(n, MLP_HIDDEN, MLP_HIDDEN, m.dZ2, MLP_HIDDEN, 1, m.W2b, 1, MLP_HIDDEN, status);
    a.act = 2; a.g = m.H1; a.sgm = MLP_HIDDEN; a.sgn = 1; a.C16 = m.dZ1; a.s16m = MLP_HIDDEN; a.s16n = 1;
    if ((e = gemm<BNH>(mode(a, m), n, MLP_HIDDEN, st)) != cudaSuccess) return e;
    // dW1[o][i] = sum_b dz1[b][o] x[b][i]
    a = gargs(MLP_HIDDEN, MLP_KIN, n, m.dZ1, 1, MLP_HIDDEN, m.X, 1, MLP_KIN, status);
    a.C32 = g + MLP_OFF_W1; a.scm = MLP_KIN; a.scn = 1;
    if ((e = gemm<BNH>(mode(a, m), MLP_HIDDEN, MLP_KIN, st)) != cudaSuccess) return e;
    k_colsum<bf16><<<MLP_HIDDEN, EW, 0, st>>>(m.dZ1, n, MLP_HIDDEN, g + MLP_OFF_B1);
    return cudaSuccess;
}

void mlp_adam(Mlp &m, double lr, cudaStream_t st)
{
    m.t += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m.t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)m.t));
    k_adam<<<(MLP_NPARAM + EW - 1) / EW, EW, 0, st>>>(m.theta, m.grad, m.adam_m, m.adam_v, (float)lr, c1, c2);
    mlp_refresh(m, st);
}

// ---------------------------------------------------------------------------
// shell sampling and the surrogate forces in the step
// ---------------------------------------------------------------------------
namespace {

// fields at point X (lattice units, wrapped) as the trilinear mean over the
// fluid corners of its cell; false when no corner is fluid
template <class R>
__device__ bool interp_fluid(const Lattice &L, const InstDev &I, const double *X, double *phi, double *u)
{
    const int b[3] = {(int)floor(X[0]), (int)floor(X[1]), (int)floor(X[2])};
    const double f[3] = {X[0] - b[0], X[1] - b[1], X[2] - b[2]};
    const R *ph = (const R *)L.phi + I.node_off;
    const R *U = (const R *)L.u + I.node_off;
    double ap = 0.0, au[3] = {0.0, 0.0, 0.0}, ws = 0.0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                const int x = (b[0] + dx) % I.nx, y = (b[1] + dy) % I.ny, z = (b[2] + dz) % I.nz;
                const int n = (z * I.ny + y) * I.nx + x;
                if ((L.flags[I.node_off + n] & OWNER_MASK) != OWN_FLUID) continue;
                ap = ap + w * (double)ph[n];
                for (int a = 0; a < 3; a++) au[a] = au[a] + w * (double)U[a * L.Ntot + n];
                ws += w;
            }
    if (ws <= 0.0) return false;
    *phi = ap / ws;
    for (int a = 0; a < 3; a++) u[a] = au[a] / ws;
    return true;
}

// features of particles p0..p0+gridDim.x-1: 96 shell points (one thread
// each), then cos(theta), sin(theta), R/R_ref
template <class R>
__global__ void __launch_bounds__(128) k_shell(Lattice L, int p0, float *feat)
{
    const int p = p0 + blockIdx.x;
    const PartDev &P = L.parts[p];
    const InstDev &I = L.inst[P.inst];
    float *f = feat + (long long)blockIdx.x * MLP_NIN;
    const int k = threadIdx.x;
    if (k < MLP_SHELL) {
        const double ez = 1.0 - (2.0 * k + 1.0) / MLP_SHELL;
        const double er = sqrt(1.0 - ez * ez);
        const double az = k * (3.14159265358979323846 * (3.0 - sqrt(5.0)));
        const double e[3] = {er * cos(az), er * sin(az), ez};
        const double rs = P.R + I.sh_gap;
        const int n3[3] = {I.nx, I.ny, I.nz};
        double lev[3];
        for (int a = 0; a < 3; a++) lev[a] = rs * e[a];
        // with a box filter (width sh_box) the mean over the 3 x 3 x 3 points
        // of the box, offsets -w/3, 0, +w/3 per axis, of those whose cell has
        // a fluid corner (the midpoint rule of the box average); with a wall
        // at z = 0 a point outside [0, nz) in z lies in or beyond the wall and
        // is left out (no wrap across the wall)
        const int nsub = I.sh_box > 0.0 ? 27 : 1;
        double ph = 0.0, u[3] = {0.0, 0.0, 0.0};
        int used = 0;
        for (int s = 0; s < nsub; s++) {
            const double d[3] = {nsub == 1 ? 0.0 : (s % 3 - 1) * I.sh_box / 3.0,
                                 nsub == 1 ? 0.0 : ((s / 3) % 3 - 1) * I.sh_box / 3.0,
                                 nsub == 1 ? 0.0 : (s / 9 - 1) * I.sh_box / 3.0};
            double X[3];
            bool in_wall = false;
            for (int a = 0; a < 3; a++) {
                const double v = P.x[a] + lev[a] + d[a];
                if (a == 2 && I.wall_z0 && !(v >= 0.0 && v < n3[2])) in_wall = true;
                X[a] = v - n3[a] * floor(v / n3[a]);
            }
            if (in_wall) continue;
            double p1 = 0.0, u1[3] = {0.0, 0.0, 0.0};
            if (!interp_fluid<R>(L, I, X, &p1, u1)) continue;
            ph += p1;
            for (int a = 0; a < 3; a++) u[a] += u1[a];
            used++;
        }
        float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (used > 0) {
            ph /= used;
            for (int a = 0; a < 3; a++) u[a] /= used;
            const double us[3] = {P.v[0] + (P.w[1] * lev[2] - P.w[2] * lev[1]),
                                  P.v[1] + (P.w[2] * lev[0] - P.w[0] * lev[2]),
                                  P.v[2] + (P.w[0] * lev[1] - P.w[1] * lev[0])};
            o[0] = (float)ph;
            for (int a = 0; a < 3; a++) o[1 + a] = (float)((u[a] - us[a]) / I.sh_uref);
        }
        for (int a = 0; a < 4; a++) f[4 * k + a] = o[a];
    } else if (k == MLP_SHELL) {
        f[4 * MLP_SHELL] = (float)P.cos_t;
        f[4 * MLP_SHELL + 1] = (float)P.sin_t;
        f[4 * MLP_SHELL + 2] = (float)(P.R / I.sh_rref);
    }
}

// surrogate output -> fluid forces of the particles: F = sigma R_p y[0..2],
// T = sigma R_p^2 y[3..5]; the capillary share is folded into these
__global__ void k_surrogate_apply(Lattice L, const float *Y, int p0, int np)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= np) return;
    PartDev &P = L.parts[p0 + r];
    const double s = L.inst[P.inst].sigma * P.R;
    for (int a = 0; a < 3; a++) {
        P.Feta[a] = s * (double)Y[r * 16 + a];
        P.Teta[a] = s * P.R * (double)Y[r * 16 + 3 + a];
        P.Fsig[a] = 0.0;
        P.Tsig[a] = 0.0;
    }
}

}  // namespace

template <class S>
void launch_shell_features(const Lattice &L, int p0, int np, float *feat, cudaStream_t st)
{
    using R = typename Store<S>::real;
    k_shell<R><<<np, 128, 0, st>>>(L, p0, feat);
}

template <class S>
void launch_surrogate_forces(const Lattice &L, const Mlp &m, float *feat, cudaStream_t st, long long *launches,
                             const Marker &mk)
{
    if (L.n_parts == 0) return;
    mk(STAGE_SURROGATE, 0);
    for (int p0 = 0; p0 < L.n_parts; p0 += m.cap) {
        const int np = std::min(m.cap, L.n_parts - p0);
        launch_shell_features<S>(L, p0, np, feat, st);
        mlp_stage(m, feat, nullptr, nullptr, 0, np, st);
        // a failed set-up or launch stays in the runtime's last error, which
        // lbm_step checks after enqueueing the step
        if (mlp_forward(m, np, L.status, st) != cudaSuccess) return;
        k_surrogate_apply<<<(np + 127) / 128, 128, 0, st>>>(L, m.Y, p0, np);
        *launches += 6;
    }
    mk(STAGE_SURROGATE, 1);
}

#define INST(S)                                                                                        \
    template void launch_shell_features<S>(const Lattice &, int, int, float *, cudaStream_t);          \
    template void launch_surrogate_forces<S>(const Lattice &, const Mlp &, float *, cudaStream_t, long long *, \
                                             const Marker &);
INST(double)
INST(float)
INST(__half)
INST(__nv_bfloat16)
#undef INST

}  // namespace lbmg
