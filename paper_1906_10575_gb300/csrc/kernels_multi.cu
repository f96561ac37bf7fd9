// Several right-hand sides at once (R = 2 or 4) on the global levels:
// residual, column norms and SpMV over vectors stored row by row with their R
// values side by side (v[i * R + j]); one load of an operator entry feeds R
// independent fma chains, each the single-column chain. The composite-grid
// kernel and its variants are in fac_multi.cuh.
#include <cstdint>

#include "fac_multi.cuh"
#include "kernels.cuh"

namespace amgdd {
namespace dev {

// ---- global levels (FP64) -------------------------------------------------

template <int R>
__global__ void k_residual_r(SellView A, const double *__restrict__ b, const double *__restrict__ x,
                             double *__restrict__ r, double *__restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nslices = (A.rows + 31) / 32;
    double acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = 0.0;
    for (int64_t q = warp; q < nslices; q += nwarps) {
        const int64_t row = q * 32 + lane;
        if (row < A.rows) {
            const int32_t i = A.rowid ? __ldg(A.rowid + row) : (int32_t)row;
            const VecR<double, R> s = sell_dot_r<int32_t, double, R, 1>(A.soff, A.rlen, A.col, A.val, q, lane, row, x);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double ri = b[(int64_t)i * R + j] - s.v[j];
                r[(int64_t)i * R + j] = ri;
                acc[j] = fma(ri, ri, acc[j]);
            }
        }
    }
    __shared__ double red[R][32];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            double v = threadIdx.x < (blockDim.x >> 5) ? red[j][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = v;
        }
    }
}

template <int R>
__global__ void k_sumsq_r(const double *__restrict__ v, int64_t n, double *__restrict__ partial)
{
    double acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] = fma(v[i * R + j], v[i * R + j], acc[j]);
    __shared__ double red[R][32];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        double x = acc[j];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[j][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            double x = threadIdx.x < (blockDim.x >> 5) ? red[j][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = x;
        }
    }
}

// out[j] = sum over blocks of partial[j * n + b], fixed order.
template <int R>
__global__ void k_finish_r(const double *__restrict__ partial, int n, double *__restrict__ out)
{
    __shared__ double red[32];
    for (int j = 0; j < R; ++j) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[(int64_t)j * n + i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) out[j] = v;
        }
        __syncthreads();
    }
}

template <int R>
__global__ void k_spmv_r(SellView M, const double *__restrict__ x, double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nslices = (M.rows + 31) / 32;
    for (int64_t q = warp; q < nslices; q += nwarps) {
        const int64_t row = q * 32 + lane;
        if (row >= M.rows) continue;
        const int32_t i = M.rowid ? __ldg(M.rowid + row) : (int32_t)row;
        const VecR<double, R> s = sell_dot_r<int32_t, double, R, 1>(M.soff, M.rlen, M.col, M.val, q, lane, row, x);
#pragma unroll
        for (int j = 0; j < R; ++j) y[(int64_t)i * R + j] = s.v[j];
    }
}

}  // namespace dev

// ---------------------------------------------------------------------------

cudaError_t launch_fac_multi(const FacParams &P, int nsub, int nrhs, int variant, cudaStream_t st)
{
    if (P.nbins < 1 || !P.ctr || !P.bin_off || !P.bin_grid || !P.desc || !P.u) return cudaErrorInvalidValue;
    switch (nrhs) {
    case 1: return launch_fac_multi_1(P, nsub, variant, st);
    case 2: return launch_fac_multi_2(P, nsub, variant, st);
    case 4: return launch_fac_multi_4(P, nsub, variant, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t residual_r(const SellView &A, const double *b, const double *x, double *r, double *partial,
                              int nblocks, double *out, cudaStream_t st)
{
    dev::k_residual_r<R><<<nblocks, 256, 0, st>>>(A, b, x, r, partial);
    dev::k_finish_r<R><<<1, 1024, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_residual_multi(const SellView &A, const double *b, const double *x, double *r, double *partial,
                                  int nblocks, double *out, int nrhs, cudaStream_t st)
{
    switch (nrhs) {
    case 2: return residual_r<2>(A, b, x, r, partial, nblocks, out, st);
    case 4: return residual_r<4>(A, b, x, r, partial, nblocks, out, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t sumsq_r(const double *v, int64_t n, double *partial, int nblocks, double *out, cudaStream_t st)
{
    dev::k_sumsq_r<R><<<nblocks, 256, 0, st>>>(v, n, partial);
    dev::k_finish_r<R><<<1, 1024, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_sumsq_multi(const double *v, int64_t n, double *partial, int nblocks, double *out, int nrhs,
                               cudaStream_t st)
{
    switch (nrhs) {
    case 2: return sumsq_r<2>(v, n, partial, nblocks, out, st);
    case 4: return sumsq_r<4>(v, n, partial, nblocks, out, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spmv_multi(const SellView &M, const double *x, double *y, int nrhs, cudaStream_t st)
{
    const int64_t warps = (M.rows + 31) / 32;
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    switch (nrhs) {
    case 2: dev::k_spmv_r<2><<<(int)blocks, 256, 0, st>>>(M, x, y); break;
    case 4: dev::k_spmv_r<4><<<(int)blocks, 256, 0, st>>>(M, x, y); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace amgdd
