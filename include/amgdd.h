/*
 * amgdd.h - C ABI of the GB300 AMG-DD solve-phase library.
 *
 * Method: algebraic multigrid domain decomposition (AMG-DD) of Mitchell,
 * Strzodka and Falgout, "Parallel Performance of Algebraic Multigrid Domain
 * Decomposition" (arXiv 1906.10575). On one GPU the paper's processors become
 * virtual subdomains: every composite grid is solved by the same kernel launch.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an amgdd_status and never aborts, traps or exits.
 *     On failure amgdd_last_error(h) describes the cause (thread-local text
 *     when no handle exists yet).
 *   - Host pointers are caller-owned and only read during the call, unless
 *     stated otherwise. Device pointers are caller-owned CUDA global-memory
 *     buffers (for example torch tensor storage) on the current device.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream. Device work is ordered on that stream; calls that
 *     return host data synchronise it.
 *   - Values are IEEE FP64, indices int32. Matrices are CSR with ascending,
 *     unique column indices in each row.
 *   - Every row product in the solve phase is computed as the chain
 *     s = 0; s = fma(a_ik, x_k, s) over ascending column index k, so results
 *     do not depend on the kernel's launch shape.
 *   - One handle may be used by one host thread / stream at a time.
 */
#ifndef AMGDD_H
#define AMGDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amgdd_handle_s *amgdd_handle;

typedef enum {
    AMGDD_OK = 0,
    AMGDD_ERR_INVALID_ARG = 1,         /* bad size, pointer, range or CSR structure */
    AMGDD_ERR_NOT_SYMMETRIC = 2,       /* A is not structurally/numerically symmetric */
    AMGDD_ERR_HIERARCHY_ASSUMPTION = 3,/* connectivity assumption of Sections 4.2/4.5 fails */
    AMGDD_ERR_OOM = 4,                 /* host or device allocation failed */
    AMGDD_ERR_CUDA = 5,                /* a CUDA runtime call failed */
    AMGDD_ERR_NO_CONVERGENCE = 6,      /* max_iter reached before tol */
    AMGDD_ERR_DEVICE_TIMEOUT = 7,      /* never returned by this version: no kernel of the
                                          library waits on another block (grids are claimed
                                          with atomicAdd, teams wait only on their own named
                                          barrier, clusters on the hardware cluster barrier);
                                          kept so that the code stays stable */
    AMGDD_ERR_SINGULAR = 8,            /* coarsest matrix is singular */
    AMGDD_ERR_NOT_ON_DEVICE = 9        /* handle was set up with host_only = 1 */
} amgdd_status;

/* Input matrix A_0 (HOST pointers, copied by amgdd_setup). */
typedef struct {
    int32_t n;              /* rows = columns */
    int64_t nnz;            /* = rowptr[n] */
    const int32_t *rowptr;  /* n+1 entries, rowptr[0] = 0, non-decreasing */
    const int32_t *col;     /* nnz entries in [0,n), ascending within a row */
    const double *val;      /* nnz entries; positive diagonal required */
} amgdd_csr;

/* Setup and solve options. amgdd_options_default fills the defaults. */
typedef struct {
    double theta;           /* strength threshold (Section 2), default 0.25 */
    int32_t max_coarse;     /* stop coarsening at n_l <= max_coarse, default 16 */
    int32_t max_levels;     /* maximum number of levels, default 25 */
    int32_t n_fac;          /* AlgFAC V(1,1)-cycles per AMG-DD iteration, default 2 */
    int32_t strict_assumption; /* 1: fail setup when the assumption is violated */
    int32_t host_only;      /* 1: build hierarchy and maps on the host only, no
                               device upload (inspection / CPU testing);
                               2: also build and range-check the device layouts,
                               still without touching the device, holding the
                               composite-grid layout whole on the host;
                               3: as 2, but the composite-grid layout is packed,
                               checked and dropped chunk by chunk, the way a
                               device setup streams it to the device */
    int32_t threads;        /* FAC kernel threads per block (0 = default 512) */
    int32_t schedule;       /* single-column FAC kernel schedule, all giving
                               identical results: 0 = none (the default
                               kernel is candidate 15 of amgdd_autotune at
                               every width); 1 = four resident blocks of 512
                               threads per SM; 2 = three blocks, deeper
                               unrolling; 3-5 = operators staged through
                               cp.async rings of different depths; 6, 7 = two
                               blocks of 1024 threads (7 with a cp.async ring);
                               8, 9 = 1 and 6 with evict-first operator loads */
    int32_t precision;      /* 0 = FP64 throughout (default); 1 = mixed: AlgFAC
                               cycles on the composite grids in FP32 (operators
                               rounded to FP32, fp32 fma chains), inside FP64
                               iterative refinement: residual, restriction,
                               coarsest solve and x += u_0 stay FP64 */
    int32_t hybrid_level;   /* 0 = none; Lt >= 1 also builds the composite grids of
                               the hierarchy from level Lt down for hybrid AMG-DD
                               (Algorithm 3, amg_hybrid_cycle / amg_hybrid_solve);
                               subdomains on level Lt are inherited from the
                               partition through the C points (FP64) */
    int32_t interp;         /* interpolation (Section 2; the paper uses hypre
                               defaults it does not restate): 0 = direct over
                               strong C neighbours (default); 1 = extended+i
                               (distance two: strong C neighbours plus those
                               of strong F neighbours, with the "+i" term and
                               weak connections lumped into the diagonal) */
    int32_t p_max;          /* extended+i only: keep the p_max largest |weights|
                               per row, rescaled to the row's sum (0 = keep
                               all; default 4) */
    int32_t coarsen;        /* C/F splitting (Section 2; the paper uses the HMIS
                               of the hypre defaults without restating it):
                               0 = Ruge-Stueben first pass (default); 1 = HMIS
                               with the subdomains as the processors: the first
                               pass on each subdomain's own strong connections,
                               its C points at subdomain-interior points seeding
                               PMIS on the whole strength graph, whose random
                               tie-break is SplitMix64 of (level << 40) + point
                               index (reproducible) */
    int32_t reserved[2];
} amgdd_options;

/* Statistics of a completed setup. */
#define AMGDD_MAX_LEVELS 40
typedef struct {
    int32_t num_levels;
    int32_t nsub;
    int32_t n[AMGDD_MAX_LEVELS];        /* n_l */
    int64_t nnz[AMGDD_MAX_LEVELS];      /* nnz(A_l) */
    int64_t nnz_P[AMGDD_MAX_LEVELS];    /* nnz(P_l), l < L */
    int64_t comp_real[AMGDD_MAX_LEVELS];   /* sum_p |D_l^p| */
    int64_t comp_ghost[AMGDD_MAX_LEVELS];  /* sum_p |Dbar_l^p \ D_l^p| */
    int64_t comp_nnz_real[AMGDD_MAX_LEVELS]; /* sum_p nnz of A_l rows of D_l^p */
    int64_t comp_nnz_A[AMGDD_MAX_LEVELS];  /* stored local A_l entries (real + ghost rows) */
    int64_t comp_nnz_P[AMGDD_MAX_LEVELS];  /* stored local P_l entries */
    int64_t comp_nnz_R[AMGDD_MAX_LEVELS];  /* stored local R_l entries */
    double operator_complexity;         /* sum_l nnz(A_l) / nnz(A_0) */
    double grid_complexity;             /* sum_l n_l / n_0 */
    double composite_overhead;          /* Section 6.1 definition */
    int64_t assumption_violations;      /* grid-level pairs that break the assumption */
    int64_t device_bytes;               /* device memory held by the handle */
    int64_t fac_fma;                    /* FP64 fused multiply-adds one all-grids
                                           FAC launch executes (n_fac cycles) */
    int64_t fac_entry_bytes;            /* bytes per stored local operator entry */
    double setup_seconds;
} amgdd_setup_stats;

/* Per-solve report. history: caller-provided HOST buffer of max_iter+1
 * doubles (or NULL); history[k] = ||b - A x_k|| / ||b|| (||r_0|| if b = 0). */
typedef struct {
    int32_t iterations;
    int32_t converged;
    double final_relres;
    double *history;
    double seconds;         /* host wall time of the solve call */
    int64_t kernel_launches;/* kernels launched by the call */
} amgdd_solve_info;

amgdd_status amgdd_options_default(amgdd_options *opts);

/* Box partition helper (the paper partitions with METIS, Section 6; boxes
 * stand in): unknown (i,j,k) of an nx*ny*nz lexicographic grid (i fastest) goes
 * to box (i/bx, j/by, k/bz), boxes numbered lexicographically. part: HOST,
 * nx*ny*nz entries. *nsub receives the number of boxes. nz = bz = 1 for 2D. */
amgdd_status amgdd_box_partition(int32_t nx, int32_t ny, int32_t nz, int32_t bx, int32_t by,
                                 int32_t bz, int32_t *part, int32_t *nsub);

/* Setup (Sections 2 and 3): classical AMG hierarchy of A (strength, Ruge-
 * Stueben first-pass C/F splitting, direct interpolation P_l, R_l = P_l^T,
 * Galerkin A_{l+1} = R_l A_l P_l), then the composite grid of every subdomain
 * p: D_0 = points within distance padding[0] of {i : part[i] = p} in graph(A_0),
 * D_{l+1} = points within padding[l+1] of the C points of D_l in graph(A_{l+1}),
 * the coarsest level whole, plus one ghost layer Dbar_l (eq. (1)).
 *   A       : HOST CSR, copied; must be symmetric with a positive diagonal.
 *   part    : HOST, A->n entries in [0, nsub); every subdomain non-empty.
 *   padding : HOST, npadding entries eta_0..; the last value repeats for
 *             deeper levels (npadding >= 1).
 *   stream  : stream for the upload (ignored when opts->host_only).
 *   out     : receives the handle (NULL on failure).
 * Errors: INVALID_ARG, NOT_SYMMETRIC, SINGULAR, HIERARCHY_ASSUMPTION (only with
 * opts->strict_assumption), OOM, CUDA. A failed setup frees everything it had
 * allocated. Testing of those paths: with AMGDD_FAULT_ALLOC=k (k >= 1) in the
 * environment, the k-th device or pinned host allocation of this call fails
 * as if memory were exhausted (OOM), without allocating. */
amgdd_status amgdd_setup(const amgdd_csr *A, const int32_t *part, int32_t nsub,
                         const int32_t *padding, int32_t npadding, const amgdd_options *opts,
                         void *stream, amgdd_handle *out);

/* Frees host and device memory of the handle (after synchronising its last
 * stream). NULL is accepted. */
void amgdd_destroy(amgdd_handle h);

const char *amgdd_last_error(amgdd_handle h);

amgdd_status amgdd_get_stats(amgdd_handle h, amgdd_setup_stats *stats);

/* Composite-grid index map of subdomain `sub` on `level` (Section 3), local
 * order: owned points of D_l ascending, other real points ascending, ghost
 * points ascending. global_idx / kind: HOST buffers of at least *count entries;
 * with global_idx == NULL only *count = |Dbar_l| is returned.
 * kind: 0 owned, 1 real (not owned), 2 ghost. */
amgdd_status amgdd_get_maps(amgdd_handle h, int32_t sub, int32_t level, int32_t *global_idx,
                            uint8_t *kind, int32_t *count);

/* Host copy of a hierarchy operator. which: 0 = A_l, 1 = P_l, 2 = R_l.
 * With rowptr == NULL only rows/cols/nnz are returned. Buffers: HOST,
 * rowptr rows+1 (int64), col nnz, val nnz. */
amgdd_status amgdd_get_operator(amgdd_handle h, int32_t level, int32_t which, int32_t *rows,
                                int32_t *cols, int64_t *nnz, int64_t *rowptr, int32_t *col,
                                double *val);

/* C/F flags (1 = C) of level l < L and 1/l1 row norms of level l (HOST, n_l). */
amgdd_status amgdd_get_cf(amgdd_handle h, int32_t level, int32_t *cf, double *l1inv);

/* Row-major explicit inverse of the coarsest matrix (HOST, n_L*n_L). */
amgdd_status amgdd_get_coarse_inverse(amgdd_handle h, double *ainv);

/* The team plan of FAC candidate 31 (no counterpart in the paper; the host
 * planner setup uses, exposed for inspection, no handle, no GPU): nsub
 * composite grids with work[g] (FMA counts, HOST) over nblocks blocks of 32
 * warps, at most 15 teams per block. Up to two grids per block on average,
 * every grid gets a team of its own whose warps follow its work; with more
 * grids, every block has two teams of 16 warps with lists of grids (largest
 * first, each to the least-loaded team). Outputs (HOST, caller-allocated):
 * block_off[nblocks + 1] (teams of block b: [block_off[b], block_off[b+1])),
 * w0 and nw (first warp and warps of each team; room for 15 * nblocks),
 * grid_off (room for 15 * nblocks + 1) and grid[nsub] (the grids of team k:
 * grid[grid_off[k] .. grid_off[k+1])), *nteams. INVALID_ARG for nsub < 1,
 * nblocks < 1, null pointers or negative work. */
amgdd_status amgdd_plan_teams(const int64_t *work, int32_t nsub, int32_t nblocks, int32_t *block_off,
                              int32_t *w0, int32_t *nw, int32_t *grid_off, int32_t *grid, int32_t *nteams);

/* ---- solve phase (device pointers, stream-ordered) ---------------------- */

/* Algorithm 2, step 1: r = b - A_0 x on all n rows; *nrm2 (HOST, may be NULL)
 * receives ||r||_2^2 (order of the reduction is fixed, not sequential).
 * b, x, r: DEVICE, n doubles each. */
amgdd_status amgdd_residual(amgdd_handle h, const double *b, const double *x, double *r,
                            double *nrm2, void *stream);

/* Algorithm 2, step 2: r_{l+1} = R_l r_l for all l. r_all: DEVICE buffer of
 * sum_l n_l doubles, levels back to back; level 0 is the input. */
amgdd_status amgdd_restrict(amgdd_handle h, double *r_all, void *stream);

/* Algorithm 2, steps 3-5 in one launch: every composite grid gathers its
 * right-hand sides f_l = r_l on D_l, runs n_fac AlgFAC V(1,1)-cycles
 * (Algorithm 4) and adds u_0 on its owned points into x.
 * r_all: DEVICE (as amgdd_restrict); x: DEVICE, n doubles, updated in place. */
amgdd_status amgdd_fac(amgdd_handle h, const double *r_all, double *x, void *stream);

/* After amgdd_fac: u_l on Dbar_l and f_l on D_l (zero at ghost points) of one
 * composite grid, in the amgdd_get_maps order. u, f: HOST, |Dbar_l| each. */
amgdd_status amgdd_get_fac_state(amgdd_handle h, int32_t sub, int32_t level, double *u, double *f);

/* One AMG-DD iteration (Algorithm 2): residual, restriction, AlgFAC on every
 * composite grid, owned corrections added into x. b, x: DEVICE, n doubles. */
amgdd_status amgdd_iterate(amgdd_handle h, const double *b, double *x, void *stream);

/* AMG-DD solver: iterate until ||b - A x|| / ||b|| <= tol or max_iter
 * iterations. x holds x_0 on entry and the last iterate on exit (also on
 * NO_CONVERGENCE). b, x: DEVICE. info may be NULL.
 * The whole solve runs as one CUDA graph on `stream`: |b|^2, the first
 * residual and its restriction, then the iterations in a conditional while
 * node whose condition a one-thread kernel sets from the relative residual
 * (so no host round trip per iteration). The graph is captured on the
 * handle's own streams the first time a (b, x, tol, max_iter) combination is
 * used and kept until one of them changes or the FAC kernel choice changes.
 * The call then waits for the stream and reads the iteration count and the
 * history; it cannot itself be recorded into a caller's stream capture.
 * max_iter >= 0 (0 computes the initial relative residual only). */
amgdd_status amgdd_solve(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter,
                         void *stream, amgdd_solve_info *info);

/* One AMG V(1,1)-cycle (Algorithm 1) with CF l1-Jacobi on the same hierarchy,
 * applied in place to x with right-hand side b. b, x: DEVICE. */
amgdd_status amg_vcycle(amgdd_handle h, const double *b, double *x, void *stream);

/* V-cycle solver on the same hierarchy, same stopping rule and the same
 * one-graph execution as amgdd_solve. */
amgdd_status amg_vcycle_solve(amgdd_handle h, const double *b, double *x, double tol,
                              int32_t max_iter, void *stream, amgdd_solve_info *info);

/* Hybrid AMG-DD V(1,1)-cycle (Section 3.1, Algorithm 3) in place on x with
 * right-hand side b: CF l1-Jacobi V-cycle relaxation and restriction on levels
 * 0 .. Lt-1, then one AMG-DD cycle (Algorithm 2 with AlgFAC, from the current
 * level-Lt correction) in place of the coarse solve on level Lt, then the
 * V-cycle's interpolation and relaxation. Lt = opts->hybrid_level (>= 1);
 * b, x: DEVICE, n doubles. */
amgdd_status amg_hybrid_cycle(amgdd_handle h, const double *b, double *x, void *stream);

/* Hybrid AMG-DD solver, same stopping rule as amgdd_solve. */
amgdd_status amg_hybrid_solve(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter,
                              void *stream, amgdd_solve_info *info);

/* ---- several right-hand sides at once --------------------------------------
 * Right-hand sides of the same matrix solved together (nrhs = 2 or 4): B and X
 * are DEVICE arrays of n x nrhs doubles stored row by row (X[i * nrhs + j] is
 * unknown i of column j, i.e. a contiguous torch tensor of shape (n, nrhs)).
 * Every operator entry is loaded once per use and feeds nrhs independent fma
 * chains; column j follows exactly the single-column arithmetic of
 * amgdd_iterate / amgdd_solve, so its iterates are the ones that a solve of
 * column j alone would produce after the same number of iterations. The first
 * call with a given nrhs allocates that width's device work space. */

/* One AMG-DD iteration (Algorithm 2) for all columns. */
amgdd_status amgdd_iterate_multi(amgdd_handle h, const double *B, double *X, int32_t nrhs, void *stream);

/* Algorithm 2, steps 3-5 for all columns in one launch (amgdd_fac for nrhs
 * columns). R_all: DEVICE, the restricted residuals of every level, level l
 * at row offset sum_{k<l} n_k, each level stored row by row with its nrhs
 * values side by side (R_all[(off_l + i) * nrhs + j]); X: DEVICE, n x nrhs
 * row by row, updated in place. */
amgdd_status amgdd_fac_multi(amgdd_handle h, const double *R_all, double *X, int32_t nrhs, void *stream);

/* AMG-DD solver for all columns: iterates until every column satisfies
 * ||b_j - A x_j|| / ||b_j|| <= tol (or max_iter). info->history (HOST, may be
 * NULL) receives nrhs * (max_iter + 1) doubles, column j's history at
 * history[j * (max_iter + 1) + k]; info->final_relres is the largest final
 * relative residual over the columns. */
amgdd_status amgdd_solve_multi(amgdd_handle h, const double *B, double *X, int32_t nrhs, double tol,
                               int32_t max_iter, void *stream, amgdd_solve_info *info);

/* ---- FAC kernel choice -------------------------------------------------------
 * The paper leaves the mapping of the composite-grid cycles onto hardware
 * open; these calls choose among kernels that all compute the same values
 * (every row product is the same ascending fma chain, so iterates do not
 * depend on the choice). Candidates, numbered k = 0 .. AMGDD_FAC_CANDIDATES-1:
 *   k = 0..8  : the single-column kernel with schedule k + 1 (amgdd_options
 *               .schedule; one column only; FP32 composite grids: k = 0, 7);
 *   k = 9..17 : the several-column kernel (one column is a width of 1),
 *               variant k - 8: operator entries in flight per row (1, 2 or 4)
 *               and resident blocks of 512 threads per SM (2, 3 or 4):
 *               9: 1/2, 10: 2/2, 11: 2/3, 12: 4/2, 13: 1/4, 14: 2/4; and with
 *               the operator entries 2 or 4 steps ahead prefetched into L2:
 *               15: 2/4 (2 ahead), 16: 2/3 (2 ahead), 17: 2/4 (4 ahead).
 *   k = 18, 19: candidate 16 with g lanes per row ("warp-per-row" for
 *               g = 32) instead of one: lane j of a group sums entries j,
 *               j+g, ... and the group adds its partial sums by an xor
 *               butterfly, so a small level's rows spread over all warps.
 *               18: g per level from the level's size (g doubles, up to 32,
 *               while mean slices of 32 rows per grid times g stay below 16
 *               and 2g stays within the mean row length; 1 on large levels);
 *               19: g = 32 on every level. These two REORDER each row sum:
 *               results then differ from the other candidates by rounding
 *               (they need 16-bit local columns).
 *   k = 20, 21: as 15 with the operator entries 2 (20) or 4 (21) steps ahead
 *               prefetched into L1 instead of L2 (16-bit local columns).
 *   k = 22..24: as 15, and every pass whose gathered level vector fits 16,
 *               32 or 44 KB copies it to shared memory first (16-bit local
 *               columns).
 *   k = 25:     as 15, but blocks claim grids from one queue, largest first,
 *               instead of from per-SM bins of estimated work.
 *   k = 26, 27: one queue as 25, no prefetch, and each grid's six work
 *               vectors held in the block's shared memory from its prologue
 *               to its epilogue, operators loaded cacheable in L1 (for small
 *               grids, whose phases are bound by the latency of reading what
 *               the previous phase wrote): 26: 2 entries in flight, 2 blocks
 *               per SM; 27: 4 entries, 1 block. The shared memory is sized
 *               for the largest grid; when that exceeds the per-block limit,
 *               the vectors stay in global memory (16-bit local columns).
 *   k = 28..30: one queue as 25, each grid cycled by a thread-block cluster
 *               of 2, 4 or 8 blocks of 512 threads instead of one block, the
 *               phases separated by cluster barriers (for launches over fewer
 *               grids than SMs; 16-bit local columns).
 *   k = 31:     as 15 (2 entries in flight, L2 prefetch 2 ahead) in blocks
 *               of 1024 threads, two per SM, each split into teams of whole
 *               warps on their own named barriers; setup sizes every team
 *               by its grids' work so that all teams finish together (one
 *               grid per team while there are at most two grids per block,
 *               else two teams of 16 warps per block with lists of grids;
 *               16-bit local columns).
 * Default before any amgdd_set_fac_kernel or amgdd_autotune: k = 15 for
 * every width (k = schedule - 1 for one column when amgdd_options.schedule
 * is 1..9). */
#define AMGDD_FAC_CANDIDATES 32
/* amgdd_autotune flags: also time candidates 18 and 19 (reordered row sums) */
#define AMGDD_TUNE_ALLOW_REORDERED 1

/* Uses candidate k for the FAC step of nrhs (1, 2 or 4) columns from now on.
 * Returns AMGDD_ERR_INVALID_ARG when k does not apply (see above). Drops the
 * handle's captured solver graphs (they are captured again when next used). */
amgdd_status amgdd_set_fac_kernel(amgdd_handle h, int32_t nrhs, int32_t candidate);

/* Autotuner: times one warm-up and `reps` FAC launches of every candidate
 * that applies to nrhs (1, 2 or 4) columns on this handle's composite grids
 * (zero restricted residuals, a scratch solution allocated and freed here),
 * with CUDA events on `stream`, and keeps the fastest as amgdd_set_fac_kernel
 * would (candidates within 1 % of the fastest count as ties, which go to the
 * lowest-numbered one). Candidates that reorder row sums take part only with flags &
 * AMGDD_TUNE_ALLOW_REORDERED. ms (HOST, may be NULL): AMGDD_FAC_CANDIDATES
 * doubles, the mean milliseconds per launch, -1 where a candidate does not
 * apply or was not timed. best (may be NULL): the chosen candidate.
 * Overwrites the FAC work space (what amgdd_get_fac_state reads) and the
 * handle's residual buffers. */
amgdd_status amgdd_autotune(amgdd_handle h, int32_t nrhs, int32_t reps, int32_t flags, double *ms, int32_t *best,
                            void *stream);

/* ---- adjoint: gradient with respect to diffusion coefficients -------------
 * The paper has no adjoint; this supports differentiating solves of the 3D
 * 7-point diffusion operator -div(kappa grad u) with node-wise kappa, face
 * coefficients 2 k_i k_j / (k_i + k_j) and Dirichlet faces using k_i
 * (lexicographic numbering, i fastest). For vectors x, lam it computes
 *   grad[m] = d(-lam^T A(kappa) x)/d kappa_m
 *           = -( sum over neighbours j of m of 2 k_j^2/(k_m + k_j)^2 (lam_m - lam_j)(x_m - x_j)
 *                + (boundary faces of m) lam_m x_m ),
 * which is dL/dkappa when x solves A x = b and lam solves A lam = dL/dx.
 * kappa, x, lam, grad: DEVICE, nx*ny*nz doubles each; stream-ordered. */
amgdd_status amgdd_kappa_grad_3d(int32_t nx, int32_t ny, int32_t nz, const double *kappa, const double *x,
                                 const double *lam, double *grad, void *stream);

/* ---- residual without any device allocation ------------------------------
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot call cudaMalloc at the moment they need a residual, for example a
 * process whose device memory was handed to its own pool allocator at start-up
 * (a raw allocation then fails or breaks its memory budget), or a latency-bound
 * loop that cannot pay for cudaMalloc/cudaFree (which can take milliseconds;
 * cudaFree waits for the device). It needs no setup handle and allocates nothing: the matrix and
 * vectors are the caller's, and the per-block partial sums of the norm live in
 * a 32 KiB file-scope device array that every GPU loading the library holds
 * until the process exits.
 *
 * Computes r = b - A x (each row as the ascending fma chain, like
 * amgdd_residual) and nrm2[0] = ||r||_2^2 (fixed-order reduction).
 *   n        : rows, 0 <= n <= 16,777,216 (the scratch holds one partial sum per
 *              4096 rows); a larger n returns AMGDD_ERR_INVALID_ARG.
 *   rowptr, col, val : DEVICE CSR of A (n+1, nnz, nnz entries); the caller
 *              guarantees a valid structure (columns in [0, n)): device data is
 *              not inspected.
 *   b, x, r  : DEVICE, n doubles; nrm2: DEVICE, 1 double.
 *   stream   : cudaStream_t (NULL = legacy default stream); stream-ordered,
 *              nothing is synchronised.
 * The first call on a device looks up the scratch's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not reset the device
 * (cudaDeviceReset) between calls: the kept address would be stale. Every call
 * shares the one scratch array, so calls whose kernels overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised.
 * Errors: INVALID_ARG (size, null pointer), CUDA; text via amgdd_last_error(NULL). */
amgdd_status amgdd_residual_csr_noalloc(int32_t n, const int32_t *rowptr, const int32_t *col,
                                        const double *val, const double *b, const double *x, double *r,
                                        double *nrm2, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* AMGDD_H */
