// sm_103a kernels of the AMG-DD solve phase.
//
// Every sparse row product is computed by one thread as the chain
// s = 0; s = fma(a_k, x[col_k], s) over the row's entries in ascending column
// order of the level's global numbering (SELL-32 storage: entry k of row
// 32*q + lane sits at soff[q] + 32*k + lane, so a warp's loads of entry k are
// one coalesced 256-byte line of values and a 128-byte line of indices).
// Built with -fmad=false: only the explicit fma() calls fuse.
#include <cstdint>

#include "fac_device.cuh"
#include "kernels.cuh"

namespace amgdd {
namespace dev {

__device__ __forceinline__ double sell_dot(const int64_t *__restrict__ soff, const uint16_t *__restrict__ rlen,
                                           const int32_t *__restrict__ col, const double *__restrict__ val,
                                           int64_t slice, int lane, int64_t row, const double *__restrict__ x)
{
    const int64_t base = __ldg(soff + slice) + lane;
    const int len = __ldg(rlen + row);
    double s = 0.0;
    const int32_t *c = col + base;
    const double *v = val + base;
    int k = 0;
#pragma unroll 1
    for (; k + 4 <= len; k += 4) {
        const int32_t c0 = __ldg(c + 32 * (k + 0)), c1 = __ldg(c + 32 * (k + 1));
        const int32_t c2 = __ldg(c + 32 * (k + 2)), c3 = __ldg(c + 32 * (k + 3));
        const double v0 = __ldg(v + 32 * (k + 0)), v1 = __ldg(v + 32 * (k + 1));
        const double v2 = __ldg(v + 32 * (k + 2)), v3 = __ldg(v + 32 * (k + 3));
        const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
        s = fma(v0, x0, s);
        s = fma(v1, x1, s);
        s = fma(v2, x2, s);
        s = fma(v3, x3, s);
    }
    for (; k < len; ++k) s = fma(__ldg(v + 32 * k), x[__ldg(c + 32 * k)], s);
    return s;
}

// ---------------------------------------------------------------------------
// Global-level kernels (one thread per row, one warp per SELL slice).

// r = b - A x over all rows; per-block partial sums of r^2.
__global__ void k_residual(SellView A, const double *__restrict__ b, const double *__restrict__ x,
                           double *__restrict__ r, double *__restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nslices = (A.rows + 31) / 32;
    double acc = 0.0;
    for (int64_t q = warp; q < nslices; q += nwarps) {
        const int64_t row = q * 32 + lane;
        if (row < A.rows) {
            const int32_t i = A.rowid ? __ldg(A.rowid + row) : (int32_t)row;
            const double s = sell_dot(A.soff, A.rlen, A.col, A.val, q, lane, row, x);
            const double ri = b[i] - s;
            r[i] = ri;
            acc = fma(ri, ri, acc);
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

// sum of squares of v (partial per block)
__global__ void k_sumsq(const double *__restrict__ v, int64_t n, double *__restrict__ partial)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(v[i], v[i], acc);
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = x;
    }
}

// out[0] = sum of partial[0..n) in a fixed order (deterministic).
__global__ void k_finish_sum(const double *__restrict__ partial, int n, double *__restrict__ out)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[0] = v;
    }
}

// sell_dot with the gathered vector read through L2 (ld.global.cg): the
// single-block chain reads vectors that it wrote itself one step earlier.
// The single block is latency bound, so up to eight entries of the row are
// loaded (indices, then values and gathered x) before their fmas, which stay
// in ascending entry order.
__device__ __forceinline__ double sell_dot_cg(const int64_t *__restrict__ soff, const uint16_t *__restrict__ rlen,
                                              const int32_t *__restrict__ col, const double *__restrict__ val,
                                              int64_t slice, int lane, int64_t row, const double *x)
{
    const int64_t base = __ldg(soff + slice) + lane;
    const int len = __ldg(rlen + row);
    double s = 0.0;
    const int32_t *c = col + base;
    const double *v = val + base;
#pragma unroll 1
    for (int k = 0; k < len; k += 8) {
        int32_t ci[8];
        double a[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) ci[u] = k + u < len ? __ldg(c + 32 * (k + u)) : 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = k + u < len ? __ldg(v + 32 * (k + u)) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = k + u < len ? __ldcg(x + ci[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k + u < len) s = fma(a[u], xv[u], s);
    }
    return s;
}

// One convergence check of a solve graph's while node (one thread): rel =
// sqrt(nr2) / ref (first: k = 0, ref = sqrt(*ref2), or the residual norm
// itself when that is zero), hist[k] = rel, the node's condition set to
// "rel > tol (or NaN) and k < max_iter", k advancing by the iteration
// about to run.
__device__ __forceinline__ void converge_step(cudaGraphConditionalHandle hc, double nr2, const double *ref2,
                                              ConvState *cs, double *hist, double tol, int32_t max_iter, int first)
{
    const double nr = sqrt(nr2);
    int32_t k = first ? 0 : cs->k;
    double ref = first ? sqrt(ref2[0]) : cs->ref;
    if (first && ref == 0.0) ref = nr;
    const double rel = ref > 0.0 ? nr / ref : 0.0;
    hist[k] = rel;
    const bool more = !(rel <= tol) && k < max_iter;
    cs->k = more ? k + 1 : k;
    cs->ref = ref;
    cudaGraphSetConditional(hc, more ? 1u : 0u);
}

// Barrier between the steps of the chain: the whole cluster (release and
// acquire at cluster scope, so every block sees what the others wrote in
// global memory) or, launched without a cluster, the block.
template <bool CL>
__device__ __forceinline__ void chain_sync()
{
    if constexpr (CL)
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else __syncthreads();
}

// The work of ChainParams on one cluster of blocks (CL) or one block, one SELL
// slice per warp at a time, the cluster's warps numbered block by block.
template <bool CL>
__global__ void __launch_bounds__(512, 2) k_chain(ChainParams C)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int warp = (int)blockIdx.x * nwb + wib, nw = (int)gridDim.x * nwb;
    if (C.residual) {
        const SellView &A = C.A;
        const int64_t nslices = (A.rows + 31) / 32;
        double acc = 0.0;
        for (int64_t q = warp; q < nslices; q += nw) {
            const int64_t row = q * 32 + lane;
            if (row < A.rows) {
                const int32_t i = A.rowid ? __ldg(A.rowid + row) : (int32_t)row;
                const double s = sell_dot_cg(A.soff, A.rlen, A.col, A.val, q, lane, row, C.x);
                const double ri = C.b[i] - s;
                C.r[i] = ri;
                acc = fma(ri, ri, acc);
            }
        }
        __shared__ double red[32];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) red[wib] = acc;
        __syncthreads();
        if (wib == 0) {
            double v = lane < nwb ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) C.partial[blockIdx.x] = v;
        }
        chain_sync<CL>();
        // the blocks' partial sums in block order
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double t = 0.0;
            for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(C.partial + k);
            C.nrm2[0] = t;
            const ChainCheck &K = C.check;
            if (K.on) converge_step(K.hc, t, K.ref2, K.cs, K.hist, K.tol, K.max_iter, K.first);
        }
    }
    for (int k = 0; k < C.nsteps; ++k) {
        const ChainStep &S = C.step[k];
        const int64_t nslices = (S.M.rows + 31) / 32;
        for (int64_t q = warp; q < nslices; q += nw) {
            const int64_t row = q * 32 + lane;
            if (row < S.M.rows) {
                const int32_t i = S.M.rowid ? __ldg(S.M.rowid + row) : (int32_t)row;
                S.y[i] = sell_dot_cg(S.M.soff, S.M.rlen, S.M.col, S.M.val, q, lane, row, S.x);
            }
        }
        if (k + 1 < C.nsteps) chain_sync<CL>();
    }
}

__global__ void k_converge(cudaGraphConditionalHandle hc, const double *nrm2, const double *ref2, ConvState *cs,
                           double *hist, double tol, int32_t max_iter, int first)
{
    if (threadIdx.x != 0) return;
    converge_step(hc, nrm2[0], ref2, cs, hist, tol, max_iter, first);
}

// y[i] = M_i . x (mode 0) or y[i] = y[i] + M_i . x (mode 1) over rows [r0, r1).
__global__ void k_spmv(SellView M, int64_t r0, int64_t r1, const double *__restrict__ x, double *__restrict__ y,
                       int mode)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t q0 = r0 / 32, q1 = (r1 + 31) / 32;
    for (int64_t q = q0 + warp; q < q1; q += nwarps) {
        const int64_t row = q * 32 + lane;
        if (row < r0 || row >= r1) continue;
        const int32_t i = M.rowid ? __ldg(M.rowid + row) : (int32_t)row;
        const double s = sell_dot(M.soff, M.rlen, M.col, M.val, q, lane, row, x);
        y[i] = mode ? y[i] + s : s;
    }
}

// CF l1-Jacobi, first half: d_i = (f_i - A_i u) * l1inv_i over device rows
// [r0, r1); mode 1 computes the residual res_i = f_i - A_i u instead.
__global__ void k_relax_compute(SellView A, int64_t r0, int64_t r1, const double *__restrict__ f,
                                const double *__restrict__ u, const double *__restrict__ l1inv,
                                double *__restrict__ d, int mode)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t q0 = r0 / 32, q1 = (r1 + 31) / 32;
    for (int64_t q = q0 + warp; q < q1; q += nwarps) {
        const int64_t row = q * 32 + lane;
        if (row < r0 || row >= r1) continue;
        const int32_t i = A.rowid ? __ldg(A.rowid + row) : (int32_t)row;
        const double s = sell_dot(A.soff, A.rlen, A.col, A.val, q, lane, row, u);
        const double res = f[i] - s;
        d[i] = mode ? res : res * l1inv[i];
    }
}

// second half: u_i = u_i + d_i over the same device rows
__global__ void k_relax_apply(const int32_t *__restrict__ rowid, int64_t r0, int64_t r1, const double *__restrict__ d,
                              double *__restrict__ u)
{
    for (int64_t row = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < r1;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = rowid[row];
        u[i] = u[i] + d[i];
    }
}

// u = Ainv f (dense, row-major), one thread per row.
__global__ void k_coarse_solve(const double *__restrict__ ainv, int n, const double *__restrict__ f,
                               double *__restrict__ u)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < n; I += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int J = 0; J < n; ++J) s = fma(ainv[(int64_t)I * n + J], f[J], s);
        u[I] = s;
    }
}

// ---------------------------------------------------------------------------
// All composite grids, one CTA each: gather f_l = r_l on D_l, n_fac AlgFAC
// V(1,1)-cycles (Algorithm 4), add u_0 on the owned points into x.

// Row product of local row `r` of a composite-grid view whose slices start at
// local row `first`: slice q = (r - first) / 32, lane = (r - first) % 32. T is
// the arithmetic type of the composite grid (double, or float in the mixed-
// precision mode): s = 0; s = fma(a_k, x_k, s) in T over ascending entries.
template <class CI, int UNR, bool STREAM = false, class T = double>
__device__ __forceinline__ T view_dot(const FacViewDev &V, int64_t slice0, int64_t row0, int first, int r,
                                      const T *__restrict__ x)
{
    const int v = r - first;
    const int64_t base = __ldg(V.soff + slice0 + (v >> 5)) + (v & 31);
    const int len = __ldg(V.rlen + row0 + r);
    const CI *__restrict__ c = static_cast<const CI *>(V.col) + base;
    const T *__restrict__ a = static_cast<const T *>(V.val) + base;
    T s = T(0);
    int k = 0;
    if constexpr (UNR == 2) {
#pragma unroll 1
        for (; k + 2 <= len; k += 2) {
            const int c0 = ld_op<STREAM>(c + 32 * k), c1 = ld_op<STREAM>(c + 32 * (k + 1));
            const T a0 = ld_op<STREAM>(a + 32 * k), a1 = ld_op<STREAM>(a + 32 * (k + 1));
            const T x0 = x[c0], x1 = x[c1];
            s = fma(a0, x0, s);
            s = fma(a1, x1, s);
        }
        if (k < len) s = fma(ld_op<STREAM>(a + 32 * k), x[ld_op<STREAM>(c + 32 * k)], s);
        return s;
    } else {
#pragma unroll 1
        for (; k + UNR <= len; k += UNR) {
            int ci[UNR];
            T av[UNR], xv[UNR];
#pragma unroll
            for (int j = 0; j < UNR; ++j) ci[j] = ld_op<STREAM>(c + 32 * (k + j));
#pragma unroll
            for (int j = 0; j < UNR; ++j) av[j] = ld_op<STREAM>(a + 32 * (k + j));
#pragma unroll
            for (int j = 0; j < UNR; ++j) xv[j] = x[ci[j]];
#pragma unroll
            for (int j = 0; j < UNR; ++j) s = fma(av[j], xv[j], s);
        }
        for (; k < len; ++k) s = fma(ld_op<STREAM>(a + 32 * k), x[ld_op<STREAM>(c + 32 * k)], s);
        return s;
    }
}

// --- asynchronous staging of SELL slices (cp.async into shared memory) ----
// Each warp owns a ring of S stages; a stage holds K consecutive k-steps of the
// slice being multiplied: K x 32 values, then K x 32 column indices. The
// copies hold no registers while in flight, so a lane can keep S*K entries
// outstanding within the 32-register budget. (FP64 composite grids only.)
template <class CI, int K, int S>
struct Ring {
    static constexpr int kVal = K * 32 * 8;
    static constexpr int kCol = K * 32 * (int)sizeof(CI);
    static constexpr int kStage = kVal + kCol;
    static constexpr int kWarp = S * kStage;
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copies chunk `ch` (k-steps [ch*K, ch*K+K) clipped to the slice width W) into
// its stage; always commits a group, empty past the end of the slice.
template <class CI, int K, int S>
__device__ __forceinline__ void issue_chunk(unsigned char *ring, const double *gval, const CI *gcol, int W, int ch,
                                            int lane)
{
    using R = Ring<CI, K, S>;
    const int k0 = ch * K;
    if (k0 < W) {
        const int kc = K < W - k0 ? K : W - k0;
        unsigned char *st = ring + (ch % S) * R::kStage;
        const unsigned char *sv = reinterpret_cast<const unsigned char *>(gval + (int64_t)k0 * 32);
        const int nv = kc * 16;
        for (int v = lane; v < nv; v += 32) cp_async16(st + 16 * v, sv + 16 * v);
        const unsigned char *sc = reinterpret_cast<const unsigned char *>(gcol + (int64_t)k0 * 32);
        const int nc = kc * 2 * (int)sizeof(CI);
        for (int v = lane; v < nc; v += 32) cp_async16(st + R::kVal + 16 * v, sc + 16 * v);
    }
    cp_async_commit();
}

// Row product of slice `slice` for this lane's row (len entries; 0 for lanes
// without a row). All 32 lanes of the warp must call it together.
template <class CI, int K, int S>
__device__ __forceinline__ double view_dot_async(const FacViewDev &V, int64_t slice, int len, int lane,
                                                 const double *__restrict__ x, unsigned char *ring)
{
    using R = Ring<CI, K, S>;
    const int64_t a = __ldg(V.soff + slice), b = __ldg(V.soff + slice + 1);
    const int W = (int)((b - a) >> 5);
    const double *gval = static_cast<const double *>(V.val) + a;
    const CI *gcol = static_cast<const CI *>(V.col) + a;
#pragma unroll
    for (int c = 0; c < S - 1; ++c) issue_chunk<CI, K, S>(ring, gval, gcol, W, c, lane);
    double s = 0.0;
    const int nch = (W + K - 1) / K;
    for (int ch = 0; ch < nch; ++ch) {
        issue_chunk<CI, K, S>(ring, gval, gcol, W, ch + S - 1, lane);
        cp_async_wait<S - 1>();
        __syncwarp();
        const unsigned char *st = ring + (ch % S) * R::kStage;
        const double *sv = reinterpret_cast<const double *>(st);
        const CI *sc = reinterpret_cast<const CI *>(st + R::kVal);
        double xv[K], av[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const bool on = ch * K + kk < len;
            av[kk] = on ? sv[kk * 32 + lane] : 0.0;
            xv[kk] = on ? x[sc[kk * 32 + lane]] : 0.0;
        }
#pragma unroll
        for (int kk = 0; kk < K; ++kk)
            if (ch * K + kk < len) s = fma(av[kk], xv[kk], s);
        __syncwarp();
    }
    return s;
}

// Row product of local row r of a view: direct loads (K == 0) or staged
// through the warp's cp.async ring (K > 0, FP64 only). `active` rows only
// accumulate.
template <class CI, int UNR, int K, int S, bool STREAM, class T>
__device__ __forceinline__ T row_dot(const FacViewDev &V, int64_t slice0, int64_t row0, int first, int q, int r,
                                     bool active, const T *__restrict__ x, unsigned char *ring, int lane)
{
    if constexpr (K == 0) {
        return active ? view_dot<CI, UNR, STREAM, T>(V, slice0, row0, first, r, x) : T(0);
    } else {
        static_assert(sizeof(T) == 8, "cp.async staging is built for FP64 composite grids");
        const int len = active ? (int)__ldg(V.rlen + row0 + r) : 0;
        return view_dot_async<CI, K, S>(V, slice0 + q, len, lane, x, ring);
    }
}

// One Jacobi half-sweep over local rows [r0, r1) with view V (slices from
// `first`): d = (f - V u) * (1/l1) for every row, then u += d, t += d.
template <class CI, int UNR, int K, int S, bool STREAM, class T>
__device__ __forceinline__ void relax_pass(const FacParams &P, const Block &B, const FacLevelDesc &d,
                                           const FacViewDev &V, int64_t s0, int first, int r0, int r1,
                                           unsigned char *ring)
{
    T *__restrict__ u = static_cast<T *>(P.u) + d.row0;
    T *__restrict__ t = static_cast<T *>(P.t) + d.row0;
    T *__restrict__ dd = static_cast<T *>(P.d) + d.row0;
    const T *__restrict__ f = static_cast<const T *>(P.f) + d.row0;
    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
    for_slices(B, first, r0, r1, [&](int q, int r, bool on) {
        const T s = row_dot<CI, UNR, K, S, STREAM, T>(V, s0, d.row0, first, q, r, on, u, ring, B.lane);
        if (on) dd[r] = (f[r] - s) * l1[r];
    });
    __syncthreads();
    for_rows(B, first, r0, r1, [&](int r) {
        const T v = dd[r];
        u[r] = u[r] + v;
        t[r] = t[r] + v;
    });
    __syncthreads();
}

template <class CI, int MINB, int UNR, int K, int S, int NT = 512, bool STREAM = false, class T = double>
__global__ void __launch_bounds__(NT, MINB) k_fac_all_grids(FacParams P)
{
    extern __shared__ __align__(16) unsigned char fac_smem[];
    Block B;
    B.tid = threadIdx.x;
    B.nt = blockDim.x;
    B.lane = threadIdx.x & 31;
    B.warp = threadIdx.x >> 5;
    B.nw = blockDim.x >> 5;
    unsigned char *ring = K > 0 ? fac_smem + (size_t)B.warp * Ring<CI, (K > 0 ? K : 1), (S > 0 ? S : 1)>::kWarp : nullptr;
    T *__restrict__ Pu = static_cast<T *>(P.u);
    T *__restrict__ Pf = static_cast<T *>(P.f);
    T *__restrict__ Pt = static_cast<T *>(P.t);
    T *__restrict__ Ps = static_cast<T *>(P.s);
    T *__restrict__ Pw = static_cast<T *>(P.w);
    const T *__restrict__ Pl1 = static_cast<const T *>(P.l1inv);
    __shared__ int claimed;
    for (;;) {
    // claim the next grid: own SM's bin first, then the others (each probe
    // is one atomic; at most nbins probes, no waiting)
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
        const double *__restrict__ rl = P.r_all + P.level_off[l];
        for (int r = B.tid; r < d.nBar; r += B.nt) {
            const int64_t i = d.row0 + r;
            Pu[i] = T(0);
            Pt[i] = T(0);
            Ps[i] = T(0);
            if (r < d.nReal) Pf[i] = (T)rl[P.gmap[i]];
        }
    }
    __syncthreads();

    for (int c = 1; c <= P.nfac; ++c) {
        for (int l = 0; l < L; ++l) {
            const FacLevelDesc d = D[l];
            const FacLevelDesc dn = D[l + 1];
            if (l > 0) {
                // u_l <- 0, then the C half-sweep, which with u = 0 is
                // delta = (f - 0) * (1/l1); the F half-sweep then only sees the
                // C values of u (view AFc)
                T *__restrict__ u = Pu + d.row0;
                T *__restrict__ t = Pt + d.row0;
                const T *__restrict__ f = Pf + d.row0;
                const T *__restrict__ l1 = Pl1 + d.row0;
                for (int r = B.tid; r < d.nBar; r += B.nt) {
                    if (r < d.nC) {
                        const T v = f[r] * l1[r];
                        u[r] = T(0) + v;
                        t[r] = t[r] + v;
                    } else {
                        u[r] = T(0);
                    }
                }
                __syncthreads();
                relax_pass<CI, UNR, K, S, STREAM, T>(P, B, d, P.AFc, d.sAFc, d.nC, d.nC, d.nReal, ring);
            } else {
                relax_pass<CI, UNR, K, S, STREAM, T>(P, B, d, P.A, d.sA, 0, 0, d.nC, ring);
                relax_pass<CI, UNR, K, S, STREAM, T>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal, ring);
            }
            // w_l = s_l + A_l t_l on Dbar_l (t_l is zero off the real points)
            {
                const T *__restrict__ t = Pt + d.row0;
                const T *__restrict__ s = Ps + d.row0;
                T *__restrict__ w = Pw + d.row0;
                for_slices(B, 0, 0, d.nBar, [&](int q, int r, bool on) {
                    const T at = row_dot<CI, UNR, K, S, STREAM, T>(P.At, d.sAt, d.row0, 0, q, r, on, t, ring, B.lane);
                    if (on) w[r] = s[r] + at;
                });
            }
            __syncthreads();
            // s_{l+1} = R_l w_l on Dbar_{l+1}; f_{l+1} -= A_{l+1} u_{l+1} (c > 1);
            // f_{l+1} -= s_{l+1}; then t_l = s_l = 0
            {
                const T *__restrict__ w = Pw + d.row0;
                T *__restrict__ s1 = Ps + dn.row0;
                T *__restrict__ f1 = Pf + dn.row0;
                const T *__restrict__ u1 = Pu + dn.row0;
                for_slices(B, 0, 0, dn.nBar, [&](int q, int r, bool on) {
                    const T sv = row_dot<CI, UNR, K, S, STREAM, T>(P.R, dn.sR, dn.row0, 0, q, r, on, w, ring, B.lane);
                    if (on) s1[r] = sv;
                    const bool real = on && r < dn.nReal;
                    if (c > 1) {
                        // A_{l+1}'s slices cover the real rows only: lanes of slices
                        // past them have no row
                        const bool qa = (q << 5) < dn.nReal;
                        if (qa) {
                            const T au =
                                row_dot<CI, UNR, K, S, STREAM, T>(P.A, dn.sA, dn.row0, 0, q, r, real, u1, ring, B.lane);
                            if (real) f1[r] = (f1[r] - au) - sv;
                        }
                    } else if (real) {
                        f1[r] = f1[r] - sv;
                    }
                });
                T *__restrict__ t = Pt + d.row0;
                T *__restrict__ s = Ps + d.row0;
                for (int r = B.tid; r < d.nBar; r += B.nt) {
                    t[r] = T(0);
                    s[r] = T(0);
                }
            }
            __syncthreads();
        }
        // coarsest level: u_L = A_L^{-1} f_L in FP64 (local order = global order)
        {
            const FacLevelDesc d = D[L];
            const T *__restrict__ f = Pf + d.row0;
            T *__restrict__ u = Pu + d.row0;
            for (int I = B.tid; I < P.nL; I += B.nt) {
                double s = 0.0;
                const double *__restrict__ a = P.ainv + (int64_t)I * P.nL;
                for (int J = 0; J < P.nL; ++J) s = fma(__ldg(a + J), (double)f[J], s);
                u[I] = (T)s;
            }
        }
        __syncthreads();
        for (int l = L - 1; l >= 0; --l) {
            const FacLevelDesc d = D[l];
            const FacLevelDesc dn = D[l + 1];
            T *__restrict__ u = Pu + d.row0;
            const T *__restrict__ u1 = Pu + dn.row0;
            for_slices(B, 0, 0, d.nBar, [&](int q, int r, bool on) {
                const T pu = row_dot<CI, UNR, K, S, STREAM, T>(P.P, d.sP, d.row0, 0, q, r, on, u1, ring, B.lane);
                if (on) u[r] = u[r] + pu;
            });
            __syncthreads();
            relax_pass<CI, UNR, K, S, STREAM, T>(P, B, d, P.A, d.sA, 0, d.nC, d.nReal, ring);
            relax_pass<CI, UNR, K, S, STREAM, T>(P, B, d, P.A, d.sA, 0, 0, d.nC, ring);
        }
    }

    const FacLevelDesc d0 = D[0];
    const int64_t o0 = P.owned0[p], o1 = P.owned0[p + 1];
    for (int64_t k = o0 + B.tid; k < o1; k += B.nt) {
        const int64_t i = d0.row0 + P.owned[k];
        const int32_t g = P.gmap[i];
        P.x[g] = P.x[g] + (double)Pu[i];
    }
    }
}

}  // namespace dev

// ---------------------------------------------------------------------------
// Launchers (host).

static int blocks_for(int64_t rows, int threads, int cap)
{
    const int64_t warps = (rows + 31) / 32;
    int64_t b = (warps * 32 + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_residual(const SellView &A, const double *b, const double *x, double *r, double *partial,
                            int nblocks, double *out, cudaStream_t st)
{
    dev::k_residual<<<nblocks, 256, 0, st>>>(A, b, x, r, partial);
    dev::k_finish_sum<<<1, 1024, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_chain(const ChainParams &C, cudaStream_t st)
{
    if (!C.residual && C.nsteps <= 0) return cudaSuccess;
    // a cluster of kChainBlocks blocks when the device can hold one, else
    // one block (cached per device)
    static int cluster_ok[64];   // 0 unknown, 1 cluster, 2 single block
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int &ok = cluster_ok[dev & 63];
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)kChainBlocks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)kChainBlocks, 1, 1);
    cfg.blockDim = dim3(512, 1, 1);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ok == 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, dev::k_chain<true>, &cfg);
        if (e != cudaSuccess) return e;
        ok = n >= 1 ? 1 : 2;
    }
    if (ok == 1) {
        if ((e = cudaLaunchKernelEx(&cfg, dev::k_chain<true>, C)) != cudaSuccess) return e;
    } else {
        dev::k_chain<false><<<1, 512, 0, st>>>(C);
    }
    return cudaGetLastError();
}

cudaError_t launch_converge(cudaGraphConditionalHandle hc, const double *nrm2, const double *ref2, ConvState *cs,
                            double *hist, double tol, int32_t max_iter, int first, cudaStream_t st)
{
    dev::k_converge<<<1, 32, 0, st>>>(hc, nrm2, ref2, cs, hist, tol, max_iter, first);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double *v, int64_t n, double *partial, int nblocks, double *out, cudaStream_t st)
{
    dev::k_sumsq<<<nblocks, 256, 0, st>>>(v, n, partial);
    dev::k_finish_sum<<<1, 1024, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_spmv(const SellView &M, int64_t r0, int64_t r1, const double *x, double *y, int mode,
                        cudaStream_t st)
{
    if (r1 <= r0) return cudaSuccess;
    dev::k_spmv<<<blocks_for(r1 - r0 + 32, 256, 152 * 16), 256, 0, st>>>(M, r0, r1, x, y, mode);
    return cudaGetLastError();
}

cudaError_t launch_relax_compute(const SellView &A, int64_t r0, int64_t r1, const double *f, const double *u,
                                 const double *l1inv, double *d, int mode, cudaStream_t st)
{
    if (r1 <= r0) return cudaSuccess;
    dev::k_relax_compute<<<blocks_for(r1 - r0 + 32, 256, 152 * 16), 256, 0, st>>>(A, r0, r1, f, u, l1inv, d, mode);
    return cudaGetLastError();
}

cudaError_t launch_relax_apply(const int32_t *rowid, int64_t r0, int64_t r1, const double *d, double *u,
                               cudaStream_t st)
{
    if (r1 <= r0) return cudaSuccess;
    dev::k_relax_apply<<<blocks_for(r1 - r0, 256, 152 * 16), 256, 0, st>>>(rowid, r0, r1, d, u);
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const double *ainv, int n, const double *f, double *u, cudaStream_t st)
{
    dev::k_coarse_solve<<<(n + 255) / 256, 256, 0, st>>>(ainv, n, f, u);
    return cudaGetLastError();
}

template <class CI, int MINB, int UNR, int K, int S, int NT = 512, bool STREAM = false, class T = double>
static cudaError_t launch_variant(const FacParams &P, int nsub, int threads, cudaStream_t st, int *blocks_per_sm)
{
    if (threads > NT) threads = NT;
    if (NT > 512) threads = NT;
    size_t smem = 0;
    if constexpr (K > 0) smem = (size_t)(threads / 32) * dev::Ring<CI, K, S>::kWarp;
    auto kern = dev::k_fac_all_grids<CI, MINB, UNR, K, S, NT, STREAM, T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm) {
        *blocks_per_sm = per_sm;
        return cudaSuccess;
    }
    // persistent: every resident slot gets a CTA (never more CTAs than grids)
    int ctas = per_sm * P.nbins;
    if (ctas > nsub) ctas = nsub;
    e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t) * (size_t)P.nbins, st);
    if (e != cudaSuccess) return e;
    kern<<<ctas, threads, smem, st>>>(P);
    return cudaGetLastError();
}

template <class CI>
static cudaError_t launch_fac_ci(const FacParams &P, int nsub, int threads, cudaStream_t st, int *bps)
{
    if (P.fp32) {  // FP32 composite grids: direct-load schedules only
        if (P.schedule == 1) return launch_variant<CI, 4, 2, 0, 0, 512, false, float>(P, nsub, threads, st, bps);
        return launch_variant<CI, 4, 2, 0, 0, 512, true, float>(P, nsub, threads, st, bps);
    }
    switch (P.schedule) {
    case 2: return launch_variant<CI, 3, 4, 0, 0>(P, nsub, threads, st, bps);  // 3 CTAs/SM, 4 entries per step
    case 3: return launch_variant<CI, 4, 2, 4, 2>(P, nsub, threads, st, bps);  // 4 CTAs/SM, cp.async ring 2 x 4
    case 4: return launch_variant<CI, 3, 2, 4, 3>(P, nsub, threads, st, bps);  // 3 CTAs/SM, cp.async ring 3 x 4
    case 5: return launch_variant<CI, 4, 2, 2, 4>(P, nsub, threads, st, bps);  // 4 CTAs/SM, cp.async ring 4 x 2
    case 6: return launch_variant<CI, 2, 2, 0, 0, 1024>(P, nsub, threads, st, bps);  // 2 CTAs of 1024/SM
    case 7: return launch_variant<CI, 2, 2, 4, 2, 1024>(P, nsub, threads, st, bps);  // same, cp.async ring 2 x 4
    case 8: return launch_variant<CI, 4, 2, 0, 0, 512, true>(P, nsub, threads, st, bps);  // 1 + evict-first operator loads
    case 9: return launch_variant<CI, 2, 2, 0, 0, 1024, true>(P, nsub, threads, st, bps); // 6 + evict-first operator loads
    case 1: return launch_variant<CI, 4, 2, 0, 0>(P, nsub, threads, st, bps);  // 4 CTAs/SM, 2 entries per step
    default: return launch_variant<CI, 4, 2, 0, 0, 512, true>(P, nsub, threads, st, bps);  // schedule 8
    }
}

cudaError_t launch_fac_all_grids(const FacParams &P, int nsub, int threads, cudaStream_t st)
{
    if (P.nbins < 1 || !P.ctr || !P.bin_off || !P.bin_grid || !P.desc || !P.u) return cudaErrorInvalidValue;
    return P.col16 ? launch_fac_ci<uint16_t>(P, nsub, threads, st, nullptr)
                   : launch_fac_ci<int32_t>(P, nsub, threads, st, nullptr);
}

cudaError_t fac_blocks_per_sm(const FacParams &P, int threads, int *blocks)
{
    return P.col16 ? launch_fac_ci<uint16_t>(P, 0, threads, nullptr, blocks)
                   : launch_fac_ci<int32_t>(P, 0, threads, nullptr, blocks);
}

}  // namespace amgdd
