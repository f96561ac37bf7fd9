// Several right-hand sides at once (R = 2 or 4): every vector is stored row by
// row with its R values side by side (v[i * R + j]), and one load of an
// operator entry feeds R independent fma chains. Column j's chain is exactly
// the single-right-hand-side chain (same entries, same ascending order), so
// each column reproduces the one-at-a-time result bit for bit.
#include <cstdint>

#include "fac_device.cuh"
#include "kernels.cuh"

namespace amgdd {
namespace dev {

template <class T, int R>
struct VecR {
    T v[R];
};

// R consecutive values of the gathered vector (16- or 32-byte aligned groups
// are loaded as vectors).
template <class T, int R>
__device__ __forceinline__ VecR<T, R> load_r(const T *__restrict__ p)
{
    VecR<T, R> o;
    if constexpr (sizeof(T) == 4 && R == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        o.v[0] = q.x; o.v[1] = q.y; o.v[2] = q.z; o.v[3] = q.w;
    } else if constexpr (sizeof(T) == 8 && R == 2) {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        o.v[0] = q.x; o.v[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && R == 4) {
        const double2 q0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 q1 = reinterpret_cast<const double2 *>(p)[1];
        o.v[0] = q0.x; o.v[1] = q0.y; o.v[2] = q1.x; o.v[3] = q1.y;
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) o.v[j] = p[j];
    }
    return o;
}

// s_j = sum_k a_k x[c_k * R + j] for the lane's row, one fma chain per column.
template <class CI, class T, int R, class SV>
__device__ __forceinline__ VecR<T, R> sell_dot_r(const int64_t *soff, const uint16_t *rlen, const CI *col,
                                                 const SV *val, int64_t slice, int lane, int64_t row,
                                                 const T *__restrict__ x)
{
    const int64_t base = __ldg(soff + slice) + lane;
    const int len = __ldg(rlen + row);
    VecR<T, R> s;
#pragma unroll
    for (int j = 0; j < R; ++j) s.v[j] = T(0);
#pragma unroll 1
    for (int k = 0; k < len; ++k) {
        const int c = ld_op<true>(col + base + 32 * k);
        const T a = (T)ld_op<true>(val + base + 32 * k);
        const VecR<T, R> xv = load_r<T, R>(x + (int64_t)c * R);
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = fma(a, xv.v[j], s.v[j]);
    }
    return s;
}

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
            const VecR<double, R> s = sell_dot_r<int32_t, double, R>(A.soff, A.rlen, A.col, A.val, q, lane, row, x);
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
        const VecR<double, R> s = sell_dot_r<int32_t, double, R>(M.soff, M.rlen, M.col, M.val, q, lane, row, x);
#pragma unroll
        for (int j = 0; j < R; ++j) y[(int64_t)i * R + j] = s.v[j];
    }
}

// ---- composite grids ------------------------------------------------------

template <class CI, class T, int R>
__device__ __forceinline__ VecR<T, R> view_dot_r(const FacViewDev &V, int64_t slice0, int64_t row0, int first,
                                                 int r, const T *__restrict__ x)
{
    const int v = r - first;
    return sell_dot_r<CI, T, R>(V.soff, V.rlen, static_cast<const CI *>(V.col), static_cast<const T *>(V.val),
                                slice0 + (v >> 5), v & 31, row0 + r, x);
}

template <class CI, class T, int R>
__device__ __forceinline__ void relax_pass_r(const FacParams &P, const Block &B, const FacLevelDesc &d,
                                             const FacViewDev &V, int64_t s0, int first, int r0, int r1)
{
    T *__restrict__ u = static_cast<T *>(P.u) + d.row0 * R;
    T *__restrict__ t = static_cast<T *>(P.t) + d.row0 * R;
    T *__restrict__ dd = static_cast<T *>(P.d) + d.row0 * R;
    const T *__restrict__ f = static_cast<const T *>(P.f) + d.row0 * R;
    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
    for_rows(B, first, r0, r1, [&](int r) {
        const VecR<T, R> s = view_dot_r<CI, T, R>(V, s0, d.row0, first, r, u);
#pragma unroll
        for (int j = 0; j < R; ++j) dd[r * R + j] = (f[r * R + j] - s.v[j]) * l1[r];
    });
    __syncthreads();
    for_rows(B, first, r0, r1, [&](int r) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const T v = dd[r * R + j];
            u[r * R + j] = u[r * R + j] + v;
            t[r * R + j] = t[r * R + j] + v;
        }
    });
    __syncthreads();
}

template <class CI, class T, int R>
__global__ void __launch_bounds__(512, 2) k_fac_all_grids_r(FacParams P)
{
    Block B;
    B.tid = threadIdx.x;
    B.nt = blockDim.x;
    B.lane = threadIdx.x & 31;
    B.warp = threadIdx.x >> 5;
    B.nw = blockDim.x >> 5;
    T *__restrict__ Pu = static_cast<T *>(P.u);
    T *__restrict__ Pf = static_cast<T *>(P.f);
    T *__restrict__ Pt = static_cast<T *>(P.t);
    T *__restrict__ Ps = static_cast<T *>(P.s);
    T *__restrict__ Pw = static_cast<T *>(P.w);
    const T *__restrict__ Pl1 = static_cast<const T *>(P.l1inv);
    __shared__ int claimed;
    for (;;) {
        __syncthreads();
        if (B.tid == 0) {
            unsigned sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            int g = -1;
            for (int probe = 0; probe < P.nbins && g < 0; ++probe) {
                const int b = (int)((sm + (unsigned)probe) % (unsigned)P.nbins);
                const int k = atomicAdd(P.ctr + b, 1);
                if (k < P.bin_off[b + 1] - P.bin_off[b]) g = P.bin_grid[P.bin_off[b] + k];
            }
            claimed = g;
        }
        __syncthreads();
        const int p = claimed;
        if (p < 0) break;
        const FacLevelDesc *D = P.desc + (int64_t)p * P.nlev;
        const int L = P.nlev - 1;

        for (int l = 0; l <= L; ++l) {
            const FacLevelDesc d = D[l];
            const double *__restrict__ rl = P.r_all + P.level_off[l] * R;
            for (int r = B.tid; r < d.nBar; r += B.nt) {
                const int64_t i = d.row0 + r;
                const int64_t g = P.gmap[i];
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    Pu[i * R + j] = T(0);
                    Pt[i * R + j] = T(0);
                    Ps[i * R + j] = T(0);
                    if (r < d.nReal) Pf[i * R + j] = (T)rl[g * R + j];
                }
            }
        }
        __syncthreads();

        for (int c = 1; c <= P.nfac; ++c) {
            for (int l = 0; l < L; ++l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                if (l > 0) {
                    T *__restrict__ u = Pu + d.row0 * R;
                    T *__restrict__ t = Pt + d.row0 * R;
                    const T *__restrict__ f = Pf + d.row0 * R;
                    const T *__restrict__ l1 = Pl1 + d.row0;
                    for (int r = B.tid; r < d.nBar; r += B.nt) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (r < d.nC) {
                                const T v = f[r * R + j] * l1[r];
                                u[r * R + j] = T(0) + v;
                                t[r * R + j] = t[r * R + j] + v;
                            } else {
                                u[r * R + j] = T(0);
                            }
                        }
                    }
                    __syncthreads();
                    relax_pass_r<CI, T, R>(P, B, d, P.AFc, d.sAFc, d.nC, d.nC, d.nReal);
                } else {
                    relax_pass_r<CI, T, R>(P, B, d, P.A, d.sA, 0, 0, d.nC);
                    relax_pass_r<CI, T, R>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                }
                {
                    const T *__restrict__ t = Pt + d.row0 * R;
                    const T *__restrict__ s = Ps + d.row0 * R;
                    T *__restrict__ w = Pw + d.row0 * R;
                    for_rows(B, 0, 0, d.nBar, [&](int r) {
                        const VecR<T, R> at = view_dot_r<CI, T, R>(P.At, d.sAt, d.row0, 0, r, t);
#pragma unroll
                        for (int j = 0; j < R; ++j) w[r * R + j] = s[r * R + j] + at.v[j];
                    });
                }
                __syncthreads();
                {
                    const T *__restrict__ w = Pw + d.row0 * R;
                    T *__restrict__ s1 = Ps + dn.row0 * R;
                    T *__restrict__ f1 = Pf + dn.row0 * R;
                    const T *__restrict__ u1 = Pu + dn.row0 * R;
                    for_rows(B, 0, 0, dn.nBar, [&](int r) {
                        const VecR<T, R> sv = view_dot_r<CI, T, R>(P.R, dn.sR, dn.row0, 0, r, w);
#pragma unroll
                        for (int j = 0; j < R; ++j) s1[r * R + j] = sv.v[j];
                        if (r < dn.nReal) {
                            if (c > 1) {
                                const VecR<T, R> au = view_dot_r<CI, T, R>(P.A, dn.sA, dn.row0, 0, r, u1);
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = (f1[r * R + j] - au.v[j]) - sv.v[j];
                            } else {
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = f1[r * R + j] - sv.v[j];
                            }
                        }
                    });
                    T *__restrict__ t = Pt + d.row0 * R;
                    T *__restrict__ s = Ps + d.row0 * R;
                    for (int r = B.tid; r < d.nBar * R; r += B.nt) {
                        t[r] = T(0);
                        s[r] = T(0);
                    }
                }
                __syncthreads();
            }
            {
                const FacLevelDesc d = D[L];
                const T *__restrict__ f = Pf + d.row0 * R;
                T *__restrict__ u = Pu + d.row0 * R;
                for (int e = B.tid; e < P.nL * R; e += B.nt) {
                    const int I = e / R, j = e % R;
                    double s = 0.0;
                    const double *__restrict__ a = P.ainv + (int64_t)I * P.nL;
                    for (int J = 0; J < P.nL; ++J) s = fma(__ldg(a + J), (double)f[J * R + j], s);
                    u[I * R + j] = (T)s;
                }
            }
            __syncthreads();
            for (int l = L - 1; l >= 0; --l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                T *__restrict__ u = Pu + d.row0 * R;
                const T *__restrict__ u1 = Pu + dn.row0 * R;
                for_rows(B, 0, 0, d.nBar, [&](int r) {
                    const VecR<T, R> pu = view_dot_r<CI, T, R>(P.P, d.sP, d.row0, 0, r, u1);
#pragma unroll
                    for (int j = 0; j < R; ++j) u[r * R + j] = u[r * R + j] + pu.v[j];
                });
                __syncthreads();
                relax_pass_r<CI, T, R>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                relax_pass_r<CI, T, R>(P, B, d, P.A, d.sA, 0, 0, d.nC);
            }
        }

        const FacLevelDesc d0 = D[0];
        const int64_t o0 = P.owned0[p], o1 = P.owned0[p + 1];
        for (int64_t k = o0 + B.tid; k < o1; k += B.nt) {
            const int64_t i = d0.row0 + P.owned[k];
            const int64_t g = P.gmap[i];
#pragma unroll
            for (int j = 0; j < R; ++j) P.x[g * R + j] = P.x[g * R + j] + (double)Pu[i * R + j];
        }
    }
}

}  // namespace dev

// ---------------------------------------------------------------------------

template <int R>
static cudaError_t launch_fac_r_ci(const FacParams &P, int nsub, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e;
    if (P.fp32) {
        auto kern = P.col16 ? dev::k_fac_all_grids_r<uint16_t, float, R> : dev::k_fac_all_grids_r<int32_t, float, R>;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, 0);
        if (e != cudaSuccess) return e;
        int ctas = (per_sm < 1 ? 1 : per_sm) * P.nbins;
        if (ctas > nsub) ctas = nsub;
        if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t) * (size_t)P.nbins, st)) != cudaSuccess) return e;
        kern<<<ctas, 512, 0, st>>>(P);
    } else {
        auto kern = P.col16 ? dev::k_fac_all_grids_r<uint16_t, double, R> : dev::k_fac_all_grids_r<int32_t, double, R>;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, 0);
        if (e != cudaSuccess) return e;
        int ctas = (per_sm < 1 ? 1 : per_sm) * P.nbins;
        if (ctas > nsub) ctas = nsub;
        if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t) * (size_t)P.nbins, st)) != cudaSuccess) return e;
        kern<<<ctas, 512, 0, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_fac_multi(const FacParams &P, int nsub, int nrhs, cudaStream_t st)
{
    if (P.nbins < 1 || !P.ctr || !P.bin_off || !P.bin_grid || !P.desc || !P.u) return cudaErrorInvalidValue;
    switch (nrhs) {
    case 2: return launch_fac_r_ci<2>(P, nsub, st);
    case 4: return launch_fac_r_ci<4>(P, nsub, st);
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
