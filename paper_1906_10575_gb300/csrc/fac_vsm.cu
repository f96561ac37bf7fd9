// Composite-grid FAC kernel for small grids: each grid's six work vectors
// live in the block's shared memory while the block cycles it (autotuner
// candidates 26 and 27). On small grids every AlgFAC phase (Algorithm 4) is
// bound by the latency of reading the values the previous phase wrote; held
// on chip, that read costs a shared-memory access instead of a round trip
// through L2. Operations and their order are those of k_fac_all_grids_r
// (fac_multi.cuh), so the results are the same bit for bit.
#include "fac_multi.cuh"

namespace amgdd {
namespace dev {

// The six work vectors of the grid a block is working on, R values per row.
// Row i of the composite layout (row0 + local row) is entry i - rb: rb = 0
// where they are the global arrays, rb = the grid's first row where they sit
// in the block's shared memory.
template <class T>
struct WorkVecs {
    T *u, *f, *t, *s, *w, *d;
    int64_t rb;
};

// Elements of one work vector of a grid with `rows` rows held in shared
// memory: R values per row, rounded up to 16 bytes.
template <class T, int R>
__host__ __device__ __forceinline__ int64_t vsm_stride(int64_t rows)
{
    constexpr int64_t q = 16 / (int64_t)sizeof(T);
    return (rows * R + q - 1) / q * q;
}

// Row r (local, of a view whose slices start at local row `first`) of V
// times x, one fma chain per column in ascending entry order: the chain of
// sell_dot_r without prefetch, its UNR operator entries per step loaded
// through the read-only path so that they stay cacheable in L1.
template <class CI, class T, int R, int UNR>
__device__ __forceinline__ VecR<T, R> view_dot_v(const FacViewDev &V, int64_t s0, int64_t row0, int first, int r,
                                                 const T *__restrict__ x)
{
    const int v = r - first;
    const CI *__restrict__ col = static_cast<const CI *>(V.col);
    const T *__restrict__ val = static_cast<const T *>(V.val);
    const int64_t base = __ldg(V.soff + s0 + (v >> 5)) + (v & 31);
    const int len = __ldg(V.rlen + row0 + r);
    VecR<T, R> s;
#pragma unroll
    for (int j = 0; j < R; ++j) s.v[j] = T(0);
    int k = 0;
#pragma unroll 1
    for (; k + UNR <= len; k += UNR) {
        int c[UNR];
        T a[UNR];
        VecR<T, R> xv[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) c[u] = __ldg(col + base + 32 * (k + u));
#pragma unroll
        for (int u = 0; u < UNR; ++u) a[u] = __ldg(val + base + 32 * (k + u));
#pragma unroll
        for (int u = 0; u < UNR; ++u) xv[u] = load_r<T, R>(x + (int64_t)c[u] * R);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
            for (int j = 0; j < R; ++j) s.v[j] = fma(a[u], xv[u].v[j], s.v[j]);
    }
#pragma unroll 1
    for (; k < len; ++k) {
        const int c = __ldg(col + base + 32 * k);
        const T a = __ldg(val + base + 32 * k);
        const VecR<T, R> xv = load_r<T, R>(x + (int64_t)c * R);
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = fma(a, xv.v[j], s.v[j]);
    }
    return s;
}

// V . x for rows [r0, r1) of a view, one row per lane (the tile schedule).
template <class CI, class T, int R, int UNR, class Fn>
__device__ __forceinline__ void rows_dot_v(const Block &B, const FacViewDev &V, int64_t s0, int64_t row0, int first,
                                           int r0, int r1, const T *x, Fn &&fn)
{
    for_rows(B, first, r0, r1, [&](int r) { fn(r, view_dot_v<CI, T, R, UNR>(V, s0, row0, first, r, x)); });
}

// relax_pass_r on the work vectors W.
template <class CI, class T, int R, int UNR>
__device__ __forceinline__ void relax_pass_v(const FacParams &P, const WorkVecs<T> &W, const Block &B,
                                             const FacLevelDesc &d, const FacViewDev &V, int64_t s0, int first,
                                             int r0, int r1, bool in_place = false)
{
    const int64_t o = (d.row0 - W.rb) * R;
    T *__restrict__ u = W.u + o;
    T *__restrict__ t = W.t + o;
    T *__restrict__ dd = W.d + o;
    const T *__restrict__ f = W.f + o;
    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
    if (in_place) {
        rows_dot_v<CI, T, R, UNR>(B, V, s0, d.row0, first, r0, r1, u, [&](int r, const VecR<T, R> &s) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const T v = (f[r * R + j] - s.v[j]) * l1[r];
                u[r * R + j] = u[r * R + j] + v;
                t[r * R + j] = t[r * R + j] + v;
            }
        });
        __syncthreads();
        return;
    }
    rows_dot_v<CI, T, R, UNR>(B, V, s0, d.row0, first, r0, r1, u, [&](int r, const VecR<T, R> &s) {
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

// The cycles of k_fac_all_grids_r (tile schedule, no prefetch), for small
// grids: a grid whose six work vectors fit the block's P.vsm_bytes of dynamic
// shared memory keeps them there from its prologue to its epilogue, so every
// phase reads what the previous one wrote without a round trip through L2;
// operators are loaded cacheable in L1, where a small grid's operators stay
// from phase to phase. Its final u and f are copied to the global arrays
// (what amgdd_get_fac_state reads). A grid that does not fit uses the global
// arrays. Every operation and its order are those of k_fac_all_grids_r.
template <class CI, class T, int R, int UNR, int MINB>
__global__ void __launch_bounds__(512, MINB) k_fac_grids_vsm(FacParams P)
{
    extern __shared__ __align__(16) unsigned char fac_vecs[];
    Block B;
    B.tid = threadIdx.x;
    B.nt = blockDim.x;
    B.lane = threadIdx.x & 31;
    B.warp = threadIdx.x >> 5;
    B.nw = blockDim.x >> 5;
    T *__restrict__ Pu = static_cast<T *>(P.u);
    T *__restrict__ Pf = static_cast<T *>(P.f);
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

        // the grid's rows are [D[0].row0, D[L].row0 + D[L].nBar): levels back to back
        const int64_t grow0 = D[0].row0;
        const int64_t grows = D[L].row0 + D[L].nBar - grow0;
        const int64_t st = vsm_stride<T, R>(grows);
        const bool on_chip = 6 * st * (int64_t)sizeof(T) <= P.vsm_bytes;
        T *sm = reinterpret_cast<T *>(fac_vecs);
        const WorkVecs<T> W = on_chip ? WorkVecs<T>{sm, sm + st, sm + 2 * st, sm + 3 * st, sm + 4 * st, sm + 5 * st,
                                                    grow0}
                                      : WorkVecs<T>{Pu, Pf, static_cast<T *>(P.t), static_cast<T *>(P.s),
                                                    static_cast<T *>(P.w), static_cast<T *>(P.d), 0};

        for (int l = 0; l <= L; ++l) {
            const FacLevelDesc d = D[l];
            const double *__restrict__ rl = P.r_all + P.level_off[l] * R;
            for (int r = B.tid; r < d.nBar; r += B.nt) {
                const int64_t i = d.row0 + r;
                const int64_t ii = i - W.rb;
                const int64_t g = P.gmap[i];
                // as in k_fac_all_grids_r: t, u_0, s_0 from zero, f on real
                // rows; every other entry is written before it is read
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    W.t[ii * R + j] = T(0);
                    if (l == 0) {
                        W.u[ii * R + j] = T(0);
                        W.s[ii * R + j] = T(0);
                    }
                    if (r < d.nReal) W.f[ii * R + j] = (T)rl[g * R + j];
                }
            }
        }
        __syncthreads();

        for (int c = 1; c <= P.nfac; ++c) {
            for (int l = 0; l < L; ++l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                if (l > 0) {
                    T *__restrict__ u = W.u + (d.row0 - W.rb) * R;
                    T *__restrict__ t = W.t + (d.row0 - W.rb) * R;
                    const T *__restrict__ f = W.f + (d.row0 - W.rb) * R;
                    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
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
                    relax_pass_v<CI, T, R, UNR>(P, W, B, d, P.AFc, d.sAFc, d.nC, d.nC, d.nReal, true);
                } else {
                    relax_pass_v<CI, T, R, UNR>(P, W, B, d, P.A, d.sA, 0, 0, d.nC);
                    relax_pass_v<CI, T, R, UNR>(P, W, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                }
                {
                    const T *__restrict__ s = W.s + (d.row0 - W.rb) * R;
                    T *__restrict__ w = W.w + (d.row0 - W.rb) * R;
                    const T *t = W.t + (d.row0 - W.rb) * R;
                    rows_dot_v<CI, T, R, UNR>(B, P.At, d.sAt, d.row0, 0, 0, d.nBar, t, [&](int r, const VecR<T, R> &at) {
#pragma unroll
                        for (int j = 0; j < R; ++j) w[r * R + j] = s[r * R + j] + at.v[j];
                    });
                }
                __syncthreads();
                {
                    const T *w = W.w + (d.row0 - W.rb) * R;
                    T *__restrict__ s1 = W.s + (dn.row0 - W.rb) * R;
                    T *__restrict__ f1 = W.f + (dn.row0 - W.rb) * R;
                    const T *__restrict__ u1 = W.u + (dn.row0 - W.rb) * R;
                    // s_{l+1} = R_l w_l on every row of level l+1; then, on its
                    // real rows, f_{l+1} -= A_{l+1} u_{l+1} (cycles after the
                    // first) and f_{l+1} -= s_{l+1}
                    for_rows(B, 0, 0, dn.nBar, [&](int r) {
                        const VecR<T, R> sv = view_dot_v<CI, T, R, UNR>(P.R, dn.sR, dn.row0, 0, r, w);
#pragma unroll
                        for (int j = 0; j < R; ++j) s1[r * R + j] = sv.v[j];
                        if (r < dn.nReal) {
                            if (c > 1) {
                                const VecR<T, R> au = view_dot_v<CI, T, R, UNR>(P.A, dn.sA, dn.row0, 0, r, u1);
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = (f1[r * R + j] - au.v[j]) - sv.v[j];
                            } else {
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = f1[r * R + j] - sv.v[j];
                            }
                        }
                    });
                    T *__restrict__ t = W.t + (d.row0 - W.rb) * R;
                    for (int r = B.tid; r < d.nBar * R; r += B.nt) t[r] = T(0);
                }
                __syncthreads();
            }
            {
                const FacLevelDesc d = D[L];
                const T *__restrict__ f = W.f + (d.row0 - W.rb) * R;
                T *__restrict__ u = W.u + (d.row0 - W.rb) * R;
                // u_L = A_L^{-1} f_L in FP64 over the nonzeros of the inverse
                for (int e = B.tid; e < P.nL * R; e += B.nt) {
                    const int I = e / R, j = e % R;
                    double s = 0.0;
                    const int32_t k1 = __ldg(P.ainv_ptr + I + 1);
                    for (int32_t k = __ldg(P.ainv_ptr + I); k < k1; ++k)
                        s = fma(__ldg(P.ainv_val + k), (double)f[__ldg(P.ainv_col + k) * R + j], s);
                    u[I * R + j] = (T)s;
                }
            }
            __syncthreads();
            for (int l = L - 1; l >= 0; --l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                T *__restrict__ u = W.u + (d.row0 - W.rb) * R;
                const T *u1 = W.u + (dn.row0 - W.rb) * R;
                rows_dot_v<CI, T, R, UNR>(B, P.P, d.sP, d.row0, 0, 0, d.nBar, u1, [&](int r, const VecR<T, R> &pu) {
#pragma unroll
                    for (int j = 0; j < R; ++j) u[r * R + j] = u[r * R + j] + pu.v[j];
                });
                __syncthreads();
                relax_pass_v<CI, T, R, UNR>(P, W, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                relax_pass_v<CI, T, R, UNR>(P, W, B, d, P.A, d.sA, 0, 0, d.nC);
            }
        }

        const FacLevelDesc d0 = D[0];
        const int64_t o0 = P.owned0[p], o1 = P.owned0[p + 1];
        for (int64_t k = o0 + B.tid; k < o1; k += B.nt) {
            const int64_t i = d0.row0 + P.owned[k];
            const int64_t g = P.gmap[i];
#pragma unroll
            for (int j = 0; j < R; ++j) P.x[g * R + j] = P.x[g * R + j] + (double)W.u[(i - W.rb) * R + j];
        }
        if (on_chip) {
            // the final u and f of the grid where the global-memory path leaves them
            for (int64_t e = B.tid; e < grows * R; e += B.nt) {
                Pu[grow0 * R + e] = W.u[e];
                Pf[grow0 * R + e] = W.f[e];
            }
        }
    }
}

}  // namespace dev

namespace {

// One launch of k_fac_grids_vsm: the dynamic shared memory holds the six work
// vectors of the largest grid (P.max_grid_rows rows) when that fits the
// opt-in limit next to the kernel's static shared memory; otherwise none is
// requested and every grid keeps its vectors in global memory.
template <class CI, class T, int R, int UNR, int MINB>
cudaError_t launch_vsm_kernel(const FacParams &P0, int nsub, cudaStream_t st)
{
    auto kern = dev::k_fac_grids_vsm<CI, T, R, UNR, MINB>;
    FacParams P = P0;
    int dev = 0, nsm = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int64_t need = 6 * dev::vsm_stride<T, R>(P.max_grid_rows) * (int64_t)sizeof(T);
    const int64_t room = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
    P.vsm_bytes = need <= room ? need : 0;
    const size_t smem = (size_t)P.vsm_bytes;
    if (smem > 48 * 1024 && (int64_t)fa.maxDynamicSharedSizeBytes < (int64_t)smem) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem)) != cudaSuccess) return e;
    int ctas = (per_sm < 1 ? 1 : per_sm) * (nsm < 1 ? 1 : nsm);
    if (ctas > nsub) ctas = nsub;
    if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t) * (size_t)P.nbins, st)) != cudaSuccess) return e;
    kern<<<ctas, 512, smem, st>>>(P);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_vsm_typed(const FacParams &P, int nsub, int nrhs, int variant, cudaStream_t st)
{
    const bool unr4 = variant == 2;
    switch (nrhs) {
    case 1: return unr4 ? launch_vsm_kernel<uint16_t, T, 1, 4, 1>(P, nsub, st)
                        : launch_vsm_kernel<uint16_t, T, 1, 2, 2>(P, nsub, st);
    case 2: return unr4 ? launch_vsm_kernel<uint16_t, T, 2, 4, 1>(P, nsub, st)
                        : launch_vsm_kernel<uint16_t, T, 2, 2, 2>(P, nsub, st);
    case 4: return unr4 ? launch_vsm_kernel<uint16_t, T, 4, 4, 1>(P, nsub, st)
                        : launch_vsm_kernel<uint16_t, T, 4, 2, 2>(P, nsub, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fac_vsm(const FacParams &P, int nsub, int nrhs, int variant, cudaStream_t st)
{
    if (!P.col16) return cudaErrorInvalidValue;
    return P.fp32 ? launch_vsm_typed<float>(P, nsub, nrhs, variant, st)
                  : launch_vsm_typed<double>(P, nsub, nrhs, variant, st);
}

}  // namespace amgdd
