// Residual and squared norm of a caller-held CSR matrix, with no device
// allocation at all: the per-block partial sums of the norm live in a
// file-scope device array instead of memory the library would allocate.
//
// Who needs this: code that cannot call cudaMalloc when it wants a residual.
// A framework or serving process often hands all device memory to its own
// pool allocator at start-up and accounts for every byte, so a raw cudaMalloc
// from a library either fails (the pool already holds the memory) or breaks
// its budget; and a latency-bound loop cannot afford cudaMalloc/cudaFree
// inside it (both can take milliseconds, and cudaFree waits for the device).
// Such a caller keeps the matrix and vectors in memory it already owns and
// gets the residual without a setup handle.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/amgdd.h"

namespace {

// Rows handled by one block of the residual kernel (four per thread), and the
// largest number of blocks whose partial sums the static scratch holds: n is
// limited to kRowsPerBlock * kMaxBlocks = 16,777,216 rows.
constexpr int kThreads = 1024;
constexpr int kRowsPerBlock = 4096;
constexpr int kMaxBlocks = 4096;

// 32 KiB scratch, held by every GPU that loads the library until the process
// exits. Shared by all calls: it keeps the last call's partial sums, which
// the next call overwrites completely before reading them (nothing in it has
// to start at zero). Calls whose kernels overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_partial[kMaxBlocks];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double *g_partial_ptr[kMaxDevices] = {};


// r_i = b_i - (sum_k a_ik x_k as an ascending fma chain); block partial of r^2.
__global__ void __launch_bounds__(kThreads) k_residual_csr(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const double *__restrict__ val, const double *__restrict__ b,
                               const double *__restrict__ x, double *__restrict__ r, double *__restrict__ partial)
{
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int64_t r1 = r0 + kRowsPerBlock < n ? r0 + kRowsPerBlock : n;
    double acc = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], x[col[k]], s);
        const double ri = b[i] - s;
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

// out[0] = sum of partial[0..nb) in a fixed order.
__global__ void k_sum_partials(const double *__restrict__ partial, int nb, double *__restrict__ out)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[0] = v;
    }
}

}  // namespace

namespace amgdd {
void set_last_error(const std::string &msg);  // capi.cpp: text for amgdd_last_error(NULL)
}

namespace {
amgdd_status fail(amgdd_status s, const std::string &m)
{
    amgdd::set_last_error(m);
    return s;
}
}  // namespace

extern "C" amgdd_status amgdd_residual_csr_noalloc(int32_t n, const int32_t *rowptr, const int32_t *col,
                                                   const double *val, const double *b, const double *x, double *r,
                                                   double *nrm2, void *stream)
{
    if (n < 0) return fail(AMGDD_ERR_INVALID_ARG, "n must be >= 0");
    if ((int64_t)n > (int64_t)kRowsPerBlock * kMaxBlocks)
        return fail(AMGDD_ERR_INVALID_ARG, "n = " + std::to_string(n) +
                                               " exceeds the 16,777,216-row limit of the static scratch");
    if (!rowptr || !col || !val || !b || !x || !r || !nrm2) return fail(AMGDD_ERR_INVALID_ARG, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(AMGDD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(AMGDD_ERR_INVALID_ARG, "device ordinal out of range");
    double *partial;
    {
        // Once per device, with that device current: the device address of the
        // static scratch (its host-side name is only a stand-in). The address
        // is kept for the life of the process, so a device reset
        // (cudaDeviceReset) between calls is not supported.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_partial_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partial);
            if (e != cudaSuccess || !p)
                return fail(AMGDD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_partial_ptr[dev] = static_cast<double *>(p);
        }
        partial = g_partial_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = n == 0 ? 1 : (int)(((int64_t)n + kRowsPerBlock - 1) / kRowsPerBlock);
    k_residual_csr<<<nb, kThreads, 0, st>>>(n, rowptr, col, val, b, x, r, partial);
    k_sum_partials<<<1, 1024, 0, st>>>(partial, nb, nrm2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AMGDD_ERR_CUDA, std::string("residual kernels: ") + cudaGetErrorString(e));
    return AMGDD_OK;
}
