// Allocation-free variant of the FP64 component-mass reduction.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, host frameworks that hand out all device memory from their
// own pool and forbid other allocations, or latency-critical loops where an
// allocation would synchronise the device.  lbm_component_masses_noalloc lets
// them take the FP64 mass sums of a population array they already hold,
// without the library allocating anything: its scratch (one pair of partial
// sums per block) is a file-scope __device__ array of fixed size, which every
// GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_NODES_PER_BLOCK = 65536;  // 256 threads x 256 nodes
constexpr int NA_MAX_BLOCKS = 4096;              // scratch slots -> at most 2^28 nodes

// shared by every call: one (sum f^a, sum f^b) pair per block
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS][2];

constexpr int NA_MAX_DEVICES = 64;
double *g_partials_addr[NA_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

__global__ void k_noalloc_partial(const double *__restrict__ pops, long long n, double (*part)[2])
{
    const long long begin = (long long)blockIdx.x * NA_NODES_PER_BLOCK;
    const long long end = begin + NA_NODES_PER_BLOCK < n ? begin + NA_NODES_PER_BLOCK : n;
    double sa = 0.0, sb = 0.0;
    for (long long k = begin + threadIdx.x; k < end; k += NA_THREADS)
        for (int q = 0; q < LBM_Q; q++) {
            sa += pops[(long long)q * n + k];
            sb += pops[(long long)(LBM_Q + q) * n + k];
        }
    __shared__ double sh[2][NA_THREADS];
    sh[0][threadIdx.x] = sa;
    sh[1][threadIdx.x] = sb;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    // every slot this call reads is written here first, so nothing needs clearing
    if (threadIdx.x == 0) {
        part[blockIdx.x][0] = sh[0][0];
        part[blockIdx.x][1] = sh[1][0];
    }
}

__global__ void k_noalloc_final(const double (*part)[2], int nblk, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < nblk; i++) {
            a += part[i][0];
            b += part[i][1];
        }
        out[0] = a;
        out[1] = b;
    }
}

}  // namespace

extern "C" lbm_status lbm_component_masses_noalloc(const double *pops, long long n_nodes, double *masses,
                                                   void *stream)
{
    if (!pops || !masses || n_nodes < 1) return LBM_ERR_ARG;
    if (n_nodes > NA_NODES_PER_BLOCK * NA_MAX_BLOCKS) return LBM_ERR_ARG;  // more than 2^28 nodes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return LBM_ERR_UNSUPPORTED;
    double *part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            // the array's name is a host-side stand-in; kernels need its device
            // address, looked up once per device with that device current
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return LBM_ERR_CUDA;
            }
            g_partials_addr[dev] = (double *)p;
        }
        part = g_partials_addr[dev];
    }
    int nblk = (int)((n_nodes + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
    cudaStream_t st = (cudaStream_t)stream;
    // launched through cudaLaunchKernel, whose return code is that launch's
    // own: an earlier, unrelated error left in the runtime is neither reported
    // as this call's failure nor cleared
    double(*pp)[2] = (double(*)[2])part;
    void *a1[] = {(void *)&pops, (void *)&n_nodes, (void *)&pp};
    if (cudaLaunchKernel((const void *)k_noalloc_partial, dim3(nblk), dim3(NA_THREADS), a1, 0, st) != cudaSuccess) {
        cudaGetLastError();  // this launch's error, reported by the return value
        return LBM_ERR_CUDA;
    }
    const double(*cp)[2] = pp;
    void *a2[] = {(void *)&cp, (void *)&nblk, (void *)&masses};
    if (cudaLaunchKernel((const void *)k_noalloc_final, dim3(1), dim3(32), a2, 0, st) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
