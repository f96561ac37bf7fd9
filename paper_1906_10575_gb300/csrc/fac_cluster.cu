// Composite-grid FAC kernel for few, large grids: each grid is cycled by a
// thread-block cluster of K blocks (autotuner candidates 28-30: K = 2, 4, 8)
// instead of one block. With one block per grid, a launch over fewer grids
// than SMs leaves most of the GPU idle while each block walks its grid's
// levels slice by slice; a cluster spreads every AlgFAC phase (Algorithm 4)
// of one grid over K SMs and separates the phases by cluster barriers.
//
// Operations and their order are those of k_fac_all_grids_r (fac_multi.cuh):
// every row product is the same ascending fma chain, so the results are the
// same bit for bit. The work vectors stay in global memory; the blocks of a
// cluster run on different SMs, so every read of a work vector goes to L2
// (ld.global.cg), and the cluster barrier (release / acquire at cluster
// scope) makes one phase's writes visible to the next phase's reads.
//
// No wait here can outlast the work: the blocks of a cluster execute the
// same sequence of cluster barriers (all control flow depends only on the
// claimed grid and its descriptors, which are the same for every block), the
// grid index is claimed once per cluster by block 0 and read by all blocks
// from its shared memory before a further barrier, and clusters never wait
// for one another.
#include <cstdint>

#include "fac_multi.cuh"

namespace amgdd {
namespace dev {
namespace {

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_blocks()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// The int at shared-memory address p of block 0 of this cluster.
__device__ __forceinline__ int ld_rank0(const int *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned ra;
    int v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(ra) : "r"(a));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

// Work-vector reads from L2 (coherent across the cluster's SMs).
template <class T>
__device__ __forceinline__ T ldv(const T *p)
{
    return __ldcg(p);
}

template <class T, int R>
__device__ __forceinline__ VecR<T, R> ldv_r(const T *p)
{
    VecR<T, R> o;
    if constexpr (sizeof(T) == 4 && R == 4) {
        const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
        o.v[0] = q.x; o.v[1] = q.y; o.v[2] = q.z; o.v[3] = q.w;
    } else if constexpr (sizeof(T) == 8 && R == 2) {
        const double2 q = __ldcg(reinterpret_cast<const double2 *>(p));
        o.v[0] = q.x; o.v[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && R == 4) {
        const double2 q0 = __ldcg(reinterpret_cast<const double2 *>(p));
        const double2 q1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
        o.v[0] = q0.x; o.v[1] = q0.y; o.v[2] = q1.x; o.v[3] = q1.y;
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) o.v[j] = __ldcg(p + j);
    }
    return o;
}

// Row r (local, of a view whose slices start at local row `first`) of V
// times x: the ascending fma chain of sell_dot_r (no prefetch), UNR operator
// entries per step, the gathered values read from L2.
template <class CI, class T, int R, int UNR>
__device__ __forceinline__ VecR<T, R> view_dot_c(const FacViewDev &V, int64_t s0, int64_t row0, int first, int r,
                                                 const T *x)
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
        for (int u = 0; u < UNR; ++u) c[u] = __ldcs(col + base + 32 * (k + u));
#pragma unroll
        for (int u = 0; u < UNR; ++u) a[u] = __ldcs(val + base + 32 * (k + u));
#pragma unroll
        for (int u = 0; u < UNR; ++u) xv[u] = ldv_r<T, R>(x + (int64_t)c[u] * R);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
            for (int j = 0; j < R; ++j) s.v[j] = fma(a[u], xv[u].v[j], s.v[j]);
    }
#pragma unroll 1
    for (; k < len; ++k) {
        const int c = __ldcs(col + base + 32 * k);
        const T a = __ldcs(val + base + 32 * k);
        const VecR<T, R> xv = ldv_r<T, R>(x + (int64_t)c * R);
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = fma(a, xv.v[j], s.v[j]);
    }
    return s;
}

template <class CI, class T, int R, int UNR, class Fn>
__device__ __forceinline__ void rows_dot_c(const Block &B, const FacViewDev &V, int64_t s0, int64_t row0, int first,
                                           int r0, int r1, const T *x, Fn &&fn)
{
    for_rows(B, first, r0, r1, [&](int r) { fn(r, view_dot_c<CI, T, R, UNR>(V, s0, row0, first, r, x)); });
}

// One Jacobi half-sweep over rows [r0, r1) of level d (see relax_pass_r),
// phases separated by cluster barriers.
template <class CI, class T, int R, int UNR>
__device__ __forceinline__ void relax_pass_c(const FacParams &P, const Block &B, const FacLevelDesc &d,
                                             const FacViewDev &V, int64_t s0, int first, int r0, int r1,
                                             bool in_place = false)
{
    T *u = static_cast<T *>(P.u) + d.row0 * R;
    T *t = static_cast<T *>(P.t) + d.row0 * R;
    T *dd = static_cast<T *>(P.d) + d.row0 * R;
    const T *f = static_cast<const T *>(P.f) + d.row0 * R;
    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
    if (in_place) {
        rows_dot_c<CI, T, R, UNR>(B, V, s0, d.row0, first, r0, r1, u, [&](int r, const VecR<T, R> &s) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const T v = (ldv(f + r * R + j) - s.v[j]) * __ldg(l1 + r);
                u[r * R + j] = ldv(u + r * R + j) + v;
                t[r * R + j] = ldv(t + r * R + j) + v;
            }
        });
        cluster_barrier();
        return;
    }
    rows_dot_c<CI, T, R, UNR>(B, V, s0, d.row0, first, r0, r1, u, [&](int r, const VecR<T, R> &s) {
#pragma unroll
        for (int j = 0; j < R; ++j) dd[r * R + j] = (ldv(f + r * R + j) - s.v[j]) * __ldg(l1 + r);
    });
    cluster_barrier();
    for_rows(B, first, r0, r1, [&](int r) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const T v = ldv(dd + r * R + j);
            u[r * R + j] = ldv(u + r * R + j) + v;
            t[r * R + j] = ldv(t + r * R + j) + v;
        }
    });
    cluster_barrier();
}

template <class CI, class T, int R, int UNR>
__global__ void __launch_bounds__(512, 1) k_fac_cluster(FacParams P)
{
    const unsigned rank = cluster_rank(), K = cluster_blocks();
    Block B;
    B.tid = (int)(rank * blockDim.x + threadIdx.x);
    B.nt = (int)(K * blockDim.x);
    B.lane = threadIdx.x & 31;
    B.warp = B.tid >> 5;
    B.nw = B.nt >> 5;
    T *Pu = static_cast<T *>(P.u);
    T *Pf = static_cast<T *>(P.f);
    T *Pt = static_cast<T *>(P.t);
    T *Ps = static_cast<T *>(P.s);
    T *Pw = static_cast<T *>(P.w);
    const T *__restrict__ Pl1 = static_cast<const T *>(P.l1inv);
    __shared__ int claimed;
    for (;;) {
        // every block is done with the previous grid; block 0 claims the next
        cluster_barrier();
        if (rank == 0 && threadIdx.x == 0) {
            const int k = atomicAdd(P.ctr, 1);
            claimed = k < P.bin_off[1] - P.bin_off[0] ? P.bin_grid[P.bin_off[0] + k] : -1;
        }
        cluster_barrier();
        const int p = ld_rank0(&claimed);
        // every block has read the claim before block 0 may overwrite it or exit
        cluster_barrier();
        if (p < 0) break;
        const FacLevelDesc *D = P.desc + (int64_t)p * P.nlev;
        const int L = P.nlev - 1;

        for (int l = 0; l <= L; ++l) {
            const FacLevelDesc d = D[l];
            const double *__restrict__ rl = P.r_all + P.level_off[l] * R;
            for (int r = B.tid; r < d.nBar; r += B.nt) {
                const int64_t i = d.row0 + r;
                const int64_t g = P.gmap[i];
                // as in k_fac_all_grids_r: t, u_0, s_0 from zero, f on real
                // rows; every other entry is written before it is read
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    Pt[i * R + j] = T(0);
                    if (l == 0) {
                        Pu[i * R + j] = T(0);
                        Ps[i * R + j] = T(0);
                    }
                    if (r < d.nReal) Pf[i * R + j] = (T)rl[g * R + j];
                }
            }
        }
        cluster_barrier();

        for (int c = 1; c <= P.nfac; ++c) {
            for (int l = 0; l < L; ++l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                if (l > 0) {
                    T *u = Pu + d.row0 * R;
                    T *t = Pt + d.row0 * R;
                    const T *f = Pf + d.row0 * R;
                    const T *__restrict__ l1 = Pl1 + d.row0;
                    for (int r = B.tid; r < d.nBar; r += B.nt) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (r < d.nC) {
                                const T v = ldv(f + r * R + j) * __ldg(l1 + r);
                                u[r * R + j] = T(0) + v;
                                t[r * R + j] = ldv(t + r * R + j) + v;
                            } else {
                                u[r * R + j] = T(0);
                            }
                        }
                    }
                    cluster_barrier();
                    relax_pass_c<CI, T, R, UNR>(P, B, d, P.AFc, d.sAFc, d.nC, d.nC, d.nReal, true);
                } else {
                    relax_pass_c<CI, T, R, UNR>(P, B, d, P.A, d.sA, 0, 0, d.nC);
                    relax_pass_c<CI, T, R, UNR>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                }
                {
                    const T *s = Ps + d.row0 * R;
                    T *w = Pw + d.row0 * R;
                    const T *t = Pt + d.row0 * R;
                    rows_dot_c<CI, T, R, UNR>(B, P.At, d.sAt, d.row0, 0, 0, d.nBar, t, [&](int r, const VecR<T, R> &at) {
#pragma unroll
                        for (int j = 0; j < R; ++j) w[r * R + j] = ldv(s + r * R + j) + at.v[j];
                    });
                }
                cluster_barrier();
                {
                    const T *w = Pw + d.row0 * R;
                    T *s1 = Ps + dn.row0 * R;
                    T *f1 = Pf + dn.row0 * R;
                    const T *u1 = Pu + dn.row0 * R;
                    // s_{l+1} = R_l w_l on every row of level l+1; then, on its
                    // real rows, f_{l+1} -= A_{l+1} u_{l+1} (cycles after the
                    // first) and f_{l+1} -= s_{l+1}
                    for_rows(B, 0, 0, dn.nBar, [&](int r) {
                        const VecR<T, R> sv = view_dot_c<CI, T, R, UNR>(P.R, dn.sR, dn.row0, 0, r, w);
#pragma unroll
                        for (int j = 0; j < R; ++j) s1[r * R + j] = sv.v[j];
                        if (r < dn.nReal) {
                            if (c > 1) {
                                const VecR<T, R> au = view_dot_c<CI, T, R, UNR>(P.A, dn.sA, dn.row0, 0, r, u1);
#pragma unroll
                                for (int j = 0; j < R; ++j)
                                    f1[r * R + j] = (ldv(f1 + r * R + j) - au.v[j]) - sv.v[j];
                            } else {
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = ldv(f1 + r * R + j) - sv.v[j];
                            }
                        }
                    });
                    T *t = Pt + d.row0 * R;
                    for (int r = B.tid; r < d.nBar * R; r += B.nt) t[r] = T(0);
                }
                cluster_barrier();
            }
            {
                const FacLevelDesc d = D[L];
                const T *f = Pf + d.row0 * R;
                T *u = Pu + d.row0 * R;
                // u_L = A_L^{-1} f_L in FP64 over the nonzeros of the inverse
                for (int e = B.tid; e < P.nL * R; e += B.nt) {
                    const int I = e / R, j = e % R;
                    double s = 0.0;
                    const int32_t k1 = __ldg(P.ainv_ptr + I + 1);
                    for (int32_t k = __ldg(P.ainv_ptr + I); k < k1; ++k)
                        s = fma(__ldg(P.ainv_val + k), (double)ldv(f + __ldg(P.ainv_col + k) * R + j), s);
                    u[I * R + j] = (T)s;
                }
            }
            cluster_barrier();
            for (int l = L - 1; l >= 0; --l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                T *u = Pu + d.row0 * R;
                const T *u1 = Pu + dn.row0 * R;
                rows_dot_c<CI, T, R, UNR>(B, P.P, d.sP, d.row0, 0, 0, d.nBar, u1, [&](int r, const VecR<T, R> &pu) {
#pragma unroll
                    for (int j = 0; j < R; ++j) u[r * R + j] = ldv(u + r * R + j) + pu.v[j];
                });
                cluster_barrier();
                relax_pass_c<CI, T, R, UNR>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal);
                relax_pass_c<CI, T, R, UNR>(P, B, d, P.A, d.sA, 0, 0, d.nC);
            }
        }

        const FacLevelDesc d0 = D[0];
        const int64_t o0 = P.owned0[p], o1 = P.owned0[p + 1];
        for (int64_t k = o0 + B.tid; k < o1; k += B.nt) {
            const int64_t i = d0.row0 + P.owned[k];
            const int64_t g = P.gmap[i];
#pragma unroll
            for (int j = 0; j < R; ++j) P.x[g * R + j] = P.x[g * R + j] + (double)ldv(Pu + i * R + j);
        }
    }
}

}  // namespace
}  // namespace dev

namespace {

// One launch of k_fac_cluster with clusters of K blocks of 512 threads,
// claiming grids from one queue (P.nbins must be 1): as many clusters as can
// be resident at once, never more than there are grids.
template <class CI, class T, int R, int UNR>
cudaError_t launch_cluster_kernel(const FacParams &P, int nsub, int K, cudaStream_t st)
{
    if (P.nbins != 1 || K < 1 || K > 8) return cudaErrorInvalidValue;
    auto kern = dev::k_fac_cluster<CI, T, R, UNR>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(512, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cfg.gridDim = dim3((unsigned)K, 1, 1);
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    if (nclusters > nsub) nclusters = nsub;
    cfg.gridDim = dim3((unsigned)(nclusters * K), 1, 1);
    if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaLaunchKernelEx(&cfg, kern, P)) != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_cluster_typed(const FacParams &P, int nsub, int nrhs, int K, cudaStream_t st)
{
    switch (nrhs) {
    case 1: return launch_cluster_kernel<uint16_t, T, 1, 2>(P, nsub, K, st);
    case 2: return launch_cluster_kernel<uint16_t, T, 2, 2>(P, nsub, K, st);
    case 4: return launch_cluster_kernel<uint16_t, T, 4, 2>(P, nsub, K, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fac_cluster(const FacParams &P, int nsub, int nrhs, int K, cudaStream_t st)
{
    if (!P.col16) return cudaErrorInvalidValue;
    return P.fp32 ? launch_cluster_typed<float>(P, nsub, nrhs, K, st)
                  : launch_cluster_typed<double>(P, nsub, nrhs, K, st);
}

}  // namespace amgdd
