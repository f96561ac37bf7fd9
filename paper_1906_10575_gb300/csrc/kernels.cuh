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

// Per-grid, per-level descriptor of the composite-grid layout.
struct FacLevelDesc {
    int32_t nC;        // real C rows: local [0, nC)
    int32_t nReal;     // real rows: local [0, nReal)
    int32_t nBar;      // all rows: local [0, nBar)
    int32_t pad;
    int64_t row0;      // offset into the per-row arrays
    int64_t slice0;    // offset into the slice-offset arrays
};

constexpr int kMaxLevels = 40;

struct FacParams {
    int nlev, nsub, nfac, nL;
    const FacLevelDesc *desc;   // [p * nlev + l]
    const int32_t *order;       // launch order of the grids
    const int32_t *gmap;        // per row: level index
    const double *l1inv;        // per row
    const uint16_t *rlenA, *rlenP, *rlenR;
    const int64_t *soffA, *soffP, *soffR;
    const int32_t *colA, *colP, *colR;
    const double *valA, *valP, *valR;
    const int32_t *owned;       // level-0 local indices of owned points
    const int64_t *owned0;      // per grid offset (nsub + 1)
    const double *ainv;         // n_L x n_L
    const double *r_all;        // restricted residuals, levels back to back
    int64_t level_off[kMaxLevels + 1];
    double *x;
    double *u, *f, *t, *s, *w, *d;  // per-row workspace
};

cudaError_t launch_residual(const SellView &A, const double *b, const double *x, double *r, double *partial,
                            int nblocks, double *out, cudaStream_t st);
cudaError_t launch_sumsq(const double *v, int64_t n, double *partial, int nblocks, double *out, cudaStream_t st);
cudaError_t launch_spmv(const SellView &M, int64_t r0, int64_t r1, const double *x, double *y, int mode,
                        cudaStream_t st);
cudaError_t launch_relax_compute(const SellView &A, int64_t r0, int64_t r1, const double *f, const double *u,
                                 const double *l1inv, double *d, int mode, cudaStream_t st);
cudaError_t launch_relax_apply(const int32_t *rowid, int64_t r0, int64_t r1, const double *d, double *u,
                               cudaStream_t st);
cudaError_t launch_coarse_solve(const double *ainv, int n, const double *f, double *u, cudaStream_t st);
cudaError_t launch_fac_all_grids(const FacParams &P, int nsub, int threads, cudaStream_t st);

}  // namespace amgdd
