// Composite-grid FAC kernel for small grids: each grid's work vectors
// live in the block's shared memory while the block cycles it (autotuner
// candidates 26 and 27). On small grids every AlgFAC phase (Algorithm 4) is
// bound by the latency of reading the values the previous phase wrote; held
// on chip, that read costs a shared-memory access instead of a round trip
// through L2. Operations and their order are those of k_fac_all_grids_r
// (fac_multi.cuh), so the results are the same bit for bit.
#include "fac_multi.cuh"

namespace amgdd {
namespace dev {

// Elements of one work vector of a grid with `rows` rows held in shared
// memory: R values per row, rounded up to 16 bytes.
template <class T, int R>
__host__ __device__ __forceinline__ int64_t vsm_stride(int64_t rows)
{
    constexpr int64_t q = 16 / (int64_t)sizeof(T);
    return (rows * R + q - 1) / q * q;
}

// Work vectors a grid keeps on chip: u in its two buffers, f, t and s.
constexpr int kVsmVectors = 5;

// The cycles of k_fac_all_grids_r (tile schedule, no prefetch), for small
// grids: a grid whose five work vectors fit the block's P.vsm_bytes of
// dynamic shared memory keeps them there from its prologue to its epilogue,
// so every phase reads what the previous one wrote without a round trip
// through L2; operators are loaded through the read-only path, cacheable in
// L1, where a small grid's operators stay from phase to phase. Its final u
// and f are copied to the global arrays (what amgdd_get_fac_state reads). A
// grid that does not fit uses the global arrays. The per-grid cycle is
// fac_grid_r itself, so every operation and its order are those of
// k_fac_all_grids_r.
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
        const bool on_chip = kVsmVectors * st * (int64_t)sizeof(T) <= P.vsm_bytes;
        T *sm = reinterpret_cast<T *>(fac_vecs);
        const WorkVecs<T> W = on_chip ? WorkVecs<T>{sm, sm + st, sm + 2 * st, sm + 3 * st, sm + 4 * st, grow0}
                                      : global_vecs<T>(P);
        fac_grid_r<CI, T, R, UNR, 0, false, 0, false>(P, B, p, W, nullptr);
        if (on_chip) {
            // the final u and f of the grid where the global-memory path
            // leaves them (the last half-sweep ended at a barrier)
            for (int64_t e = B.tid; e < grows * R; e += B.nt) {
                Pu[grow0 * R + e] = W.u[e];
                Pf[grow0 * R + e] = W.f[e];
            }
        }
    }
}

}  // namespace dev

namespace {

// One launch of k_fac_grids_vsm: the dynamic shared memory holds the five work
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
    const int64_t need = dev::kVsmVectors * dev::vsm_stride<T, R>(P.max_grid_rows) * (int64_t)sizeof(T);
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
