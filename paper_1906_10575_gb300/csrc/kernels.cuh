// Plain-data views and launchers shared by the host library and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace amgdd {

// Device view of a SELL-32 matrix (see amgdd_internal.hpp for the layout).
struct SellView {
    int64_t rows;
    const int64_t *soff;
    const uint16_t *rlen;
    const int32_t *col;
    const double *val;
    const int32_t *rowid;   // device row -> output index (nullptr: identity)
};

// Per-grid, per-level descriptor of the composite-grid layout. Local rows
// are ordered [real C | real F | ghost]; every view is a SELL-32 block whose
// slices start at the view's first row.
struct FacLevelDesc {
    int32_t nC;        // real C rows: local [0, nC)
    int32_t nReal;     // real rows: local [0, nReal)
    int32_t nBar;      // all rows: local [0, nBar)
    int32_t pad;
    int64_t row0;      // offset into the per-row arrays (nBar entries per level)
    int64_t sA;        // slices of A_l real rows (full rows), rows [0, nReal)
    int64_t sAt;       // slices of A_l all rows, real columns only, rows [0, nBar)
    int64_t sAFc;      // slices of A_l real F rows, real C columns only, rows [nC, nReal)
    int64_t sP;        // slices of P_l, rows [0, nBar), columns on level l+1
    int64_t sR;        // slices of R_{l-1} on this level's rows, columns on level l-1
};

// One SELL family (all grids and levels back to back). rlen is indexed by
// row0 + local row; col holds uint16_t or int32_t local indices.
struct FacViewDev {
    const int64_t *soff;
    const uint16_t *rlen;
    const void *col;
    const void *val;            // double or float (the composite grid's type)
};

constexpr int kMaxLevels = 40;

// Teams of the team-partitioned FAC kernel (variant 16): block b of the
// launch holds teams [block_off[b], block_off[b + 1]); team k is warps
// [w0[k], w0[k] + nw[k]) of its block and cycles grids
// grid[grid_off[k] .. grid_off[k + 1]) in order.
struct FacTeams {
    int nblocks;
    const int32_t *block_off, *w0, *nw, *grid_off, *grid;
};

struct FacParams {
    int nlev, nsub, nfac, nL;
    int col16;                  // 1: local columns are uint16_t
    int schedule;               // kernel variant (see launch_fac_all_grids)
    // Work distribution: grids are packed into one bin per SM (by estimated
    // work); a CTA claims grids from the bin of the SM it runs on, then from
    // the other bins. ctr holds one claim counter per bin (zeroed per launch).
    int nbins;
    const int32_t *bin_off;     // nbins + 1
    const int32_t *bin_grid;    // nsub
    int32_t *ctr;               // nbins
    const FacLevelDesc *desc;   // [p * nlev + l]
    const int32_t *order;       // launch order of the grids
    const int32_t *gmap;        // per row: level index
    const void *l1inv;          // per row, composite grid's type
    FacViewDev A, At, AFc, P, R;
    const int32_t *owned;       // level-0 local indices of owned points
    const int64_t *owned0;      // per grid offset (nsub + 1)
    const double *ainv;         // n_L x n_L
    // the nonzeros of ainv row by row, ascending columns (nL + 1 offsets);
    // a block-diagonal coarsest level (independent systems) leaves most of
    // the dense inverse exactly zero
    const int32_t *ainv_ptr, *ainv_col;
    const double *ainv_val;
    const double *r_all;        // restricted residuals, levels back to back
    int64_t level_off[kMaxLevels + 1];
    double *x;
    void *u, *f, *t, *s, *w, *d;    // per-row workspace, composite grid's type
    int fp32;                   // 1: composite grids in FP32 (mixed precision)
    // lanes per row on each level in the group-per-row kernel variant
    // (powers of two up to 32; 1 = one row per lane)
    int8_t grp[kMaxLevels + 1];
    // rows of the largest composite grid (all its levels), and the dynamic
    // shared memory per block that holds a grid's work vectors in the
    // variants that keep them on chip (0: none; set by their launcher)
    int64_t max_grid_rows;
    int64_t vsm_bytes;
    FacTeams teams;
};

cudaError_t launch_residual(const SellView &A, const double *b, const double *x, double *r, double *partial,
                            int nblocks, double *out, cudaStream_t st);

// Small sparse products run back to back by one cluster of kChainBlocks
// blocks of 512 threads (one block where the device cannot hold the
// cluster), with a cluster barrier between them (no launch and no grid-wide
// wait per step): optionally r = b - A x with sum r_i^2 in *nrm2 (the
// blocks' partial sums in partial[0 .. kChainBlocks), added in block order),
// then y = M x for each step in order (step k may read what step k - 1
// wrote). Each row keeps the ascending fma chain of the multi-block kernels.
constexpr int kChainBlocks = 8;
struct ChainStep {
    SellView M;
    const double *x;
    double *y;
};
struct ConvState;
// The convergence check of a solve graph's while node (see launch_converge),
// done by the chain itself right after the norm when `on` is set.
struct ChainCheck {
    int on, first;
    int32_t max_iter;
    double tol;
    cudaGraphConditionalHandle hc;
    const double *ref2;
    ConvState *cs;
    double *hist;
};
struct ChainParams {
    int residual;               // 1: the residual comes first
    SellView A;
    const double *b, *x;
    double *r, *nrm2, *partial;
    int nsteps;
    ChainStep step[kMaxLevels];
    ChainCheck check;           // only with the residual
};
cudaError_t launch_chain(const ChainParams &C, cudaStream_t st);

// Convergence state of a solve that runs its iterations in a graph's while
// node: k = iterations done, ref = the norm relative residuals divide by.
struct ConvState {
    int32_t k;
    int32_t pad;
    double ref;
};
// One thread: rel = sqrt(*nrm2) / ref (first: k = 0, ref = sqrt(*ref2), or
// the residual norm itself when that is zero), hist[k] = rel, and the while
// node's condition set to "rel > tol (or NaN) and k < max_iter", k advancing
// by the iteration about to run.
cudaError_t launch_converge(cudaGraphConditionalHandle hc, const double *nrm2, const double *ref2, ConvState *cs,
                            double *hist, double tol, int32_t max_iter, int first, cudaStream_t st);
cudaError_t launch_sumsq(const double *v, int64_t n, double *partial, int nblocks, double *out, cudaStream_t st);
cudaError_t launch_spmv(const SellView &M, int64_t r0, int64_t r1, const double *x, double *y, int mode,
                        cudaStream_t st);
cudaError_t launch_relax_compute(const SellView &A, int64_t r0, int64_t r1, const double *f, const double *u,
                                 const double *l1inv, double *d, int mode, cudaStream_t st);
cudaError_t launch_relax_apply(const int32_t *rowid, int64_t r0, int64_t r1, const double *d, double *u,
                               cudaStream_t st);
cudaError_t launch_coarse_solve(const double *ainv, int n, const double *f, double *u, cudaStream_t st);
cudaError_t launch_fac_all_grids(const FacParams &P, int nsub, int threads, cudaStream_t st);
// several right-hand sides (nrhs = 2 or 4), vectors stored row by row
// Composite-grid kernel for nrhs = 1, 2 or 4 columns, variant 1..15 (see
// fac_multi.cuh; every variant but the group-per-row variant 10 keeps each
// row's ascending fma chain, and 10 reorders row sums the same way for every
// column); the per-column launchers live in fac_multi_r*.cu.
cudaError_t launch_fac_multi(const FacParams &P, int nsub, int nrhs, int variant, cudaStream_t st);
cudaError_t launch_fac_multi_1(const FacParams &P, int nsub, int variant, cudaStream_t st);
cudaError_t launch_fac_multi_2(const FacParams &P, int nsub, int variant, cudaStream_t st);
cudaError_t launch_fac_multi_4(const FacParams &P, int nsub, int variant, cudaStream_t st);
// Composite-grid kernel with each grid's work vectors in shared memory
// (fac_vsm.cu) for nrhs = 1, 2 or 4 columns: variant 1 = two operator entries
// in flight, two blocks per SM; 2 = four entries, one block. Needs 16-bit
// local columns.
cudaError_t launch_fac_vsm(const FacParams &P, int nsub, int nrhs, int variant, cudaStream_t st);
// Composite-grid kernel cycling each grid with a cluster of K = 1..8 blocks
// (fac_cluster.cu), grids claimed from one queue (P.nbins == 1), for nrhs =
// 1, 2 or 4 columns. Needs 16-bit local columns.
cudaError_t launch_fac_cluster(const FacParams &P, int nsub, int nrhs, int K, cudaStream_t st);
cudaError_t launch_residual_multi(const SellView &A, const double *b, const double *x, double *r, double *partial,
                                  int nblocks, double *out, int nrhs, cudaStream_t st);
cudaError_t launch_sumsq_multi(const double *v, int64_t n, double *partial, int nblocks, double *out, int nrhs,
                               cudaStream_t st);
cudaError_t launch_spmv_multi(const SellView &M, const double *x, double *y, int nrhs, cudaStream_t st);
// resident CTAs per SM of the selected FAC kernel variant
cudaError_t fac_blocks_per_sm(const FacParams &P, int threads, int *blocks);

}  // namespace amgdd
