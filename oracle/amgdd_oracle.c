/*
 * AMG-DD oracle: a plain, slow CPU FP64 implementation of the AMG-DD solve
 * phase and of the setup it needs (Mitchell, Strzodka, Falgout, "Parallel
 * Performance of Algebraic Multigrid Domain Decomposition", arXiv 1906.10575).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header, table or helper with the CUDA
 * library: both are written independently from the same definitions.
 *
 * What it computes, and where the paper defines it:
 *   - classical AMG setup: strength of connection, Ruge-Stueben first-pass
 *     C/F splitting, direct interpolation P_l, R_l = P_l^T, Galerkin
 *     A_{l+1} = R_l A_l P_l (Section 2);
 *   - composite grids D_l, ghost layers Dbar_l (Section 3, Fig. 1; eq. (1) of
 *     Section 4.1);
 *   - the AlgFAC V-cycle (Algorithm 4, Sections 4.2-4.5);
 *   - the global cycle with relaxation suppressed outside D_l, which the
 *     AlgFAC cycle must reproduce exactly (Section 4, opening paragraphs);
 *   - the AMG-DD iteration (Algorithm 2) and the AMG V(1,1)-cycle
 *     (Algorithm 1).
 *
 * Readings where the paper is silent (it uses hypre defaults it does not
 * print):
 *   - strength: j strongly influences i iff -a_ij >= theta * max_{k!=i}(-a_ik),
 *     and a row whose largest -a_ik is <= 0 has no strong connections;
 *   - coarsening: Ruge-Stueben first pass, measure
 *     lambda_i = |S_i^T n U| + 2 |S_i^T n F|, largest measure first, ties to
 *     the smallest index; points with no strong connection in either
 *     direction become F points with an empty interpolation row; or
 *     (coarsen = 1) HMIS with the subdomains as processors and a SplitMix64
 *     draw in place of PMIS's random numbers (hmis_coarsen below);
 *   - interpolation: direct interpolation over strong C neighbours with
 *     positive off-diagonals lumped into the diagonal; or (interp = 1) the
 *     extended+i interpolation of the hypre defaults the paper names, with
 *     truncation to pmax entries per row (exti_interp below);
 *   - smoother: CF l1-Jacobi, l1_i = sum_j |a_ij| over the whole row,
 *     delta_i = (f_i - (A u)_i) * (1 / l1_i); pre-smoothing C then F points,
 *     post-smoothing F then C points;
 *   - coarsest solve: product with the explicit inverse of A_L formed by
 *     Gauss-Jordan elimination with partial pivoting.
 *
 * Floating-point convention (so that an independent implementation that
 * follows the same definitions reproduces every bit): this file is compiled
 * with -ffp-contract=off; every sparse row product is the chain
 * s = 0; s = fma(a_ik, x_col(k), s) over the row's entries in ascending column
 * order; setup products (Galerkin, Gauss-Jordan) use separate multiply and
 * add/subtract. Only the residual 2-norm is order-dependent.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXLEV 40
#define ORC_MAX_COARSE_DENSE 8192

typedef struct {
    int n, m;       /* rows, columns */
    int64_t *rp;    /* n+1 */
    int *ci;        /* nnz, ascending within a row */
    double *v;      /* nnz */
} Mat;

typedef struct {
    int nlev;                 /* levels 0 .. nlev-1; coarsest L = nlev-1 */
    Mat A[ORC_MAXLEV];
    Mat P[ORC_MAXLEV];        /* n_l x n_{l+1}, l < L */
    Mat R[ORC_MAXLEV];        /* n_{l+1} x n_l, R_l = P_l^T */
    int *cf[ORC_MAXLEV];      /* l < L: 1 = C point, 0 = F point */
    int *cmap[ORC_MAXLEV];    /* l < L: coarse index of a C point, -1 for F */
    double *l1inv[ORC_MAXLEV];/* 1 / sum_j |a_ij| */
    double *ainv;             /* n_L x n_L row-major inverse of A_L */
    int status;               /* 0 ok, 1 singular coarsest matrix, 2 coarsest too large */
} Hier;

static void *xmalloc(size_t n) { void *p = malloc(n ? n : 1); if (!p) abort(); return p; }
static void *xcalloc(size_t n, size_t s) { void *p = calloc(n ? n : 1, s ? s : 1); if (!p) abort(); return p; }

static void mat_free(Mat *M) { free(M->rp); free(M->ci); free(M->v); memset(M, 0, sizeof *M); }

/* Sparse row product s = sum_k a_ik x_{c(k)} as an ascending fma chain. */
static inline double rowdot(const Mat *A, int i, const double *x)
{
    double s = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
        s = fma(A->v[k], x[A->ci[k]], s);
    return s;
}

/* ------------------------------------------------------------------ */
/* Setup (Section 2)                                                   */
/* ------------------------------------------------------------------ */

/* Strength of connection: S_i = { j != i : -a_ij >= theta * max_{k!=i}(-a_ik) }.
 * Returned as a pattern CSR (ascending j). */
static void strength(const Mat *A, double theta, int64_t **srp_out, int **sci_out)
{
    int n = A->n;
    int64_t *srp = xcalloc((size_t)n + 1, sizeof(int64_t));
    int64_t cnt = 0;
    int *sci = xmalloc(sizeof(int) * (size_t)(A->rp[n] > 0 ? A->rp[n] : 1));
    for (int i = 0; i < n; ++i) {
        double mx = 0.0;
        int any = 0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            if (A->ci[k] == i) continue;
            double nv = -A->v[k];
            if (!any || nv > mx) { mx = nv; any = 1; }
        }
        if (any && mx > 0.0) {
            double thr = theta * mx;
            for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
                if (A->ci[k] == i) continue;
                if (-A->v[k] >= thr) sci[cnt++] = A->ci[k];
            }
        }
        srp[i + 1] = cnt;
    }
    *srp_out = srp;
    *sci_out = sci;
}

/* Transpose of a pattern: row j of the result lists the i with j in row i,
 * ascending. */
static void pattern_transpose(int n, const int64_t *rp, const int *ci, int64_t **trp_out, int **tci_out)
{
    int64_t *trp = xcalloc((size_t)n + 1, sizeof(int64_t));
    int64_t nnz = rp[n];
    int *tci = xmalloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t k = 0; k < nnz; ++k) trp[ci[k] + 1]++;
    for (int i = 0; i < n; ++i) trp[i + 1] += trp[i];
    int64_t *pos = xmalloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) pos[i] = trp[i];
    for (int i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) tci[pos[ci[k]]++] = i;
    free(pos);
    *trp_out = trp;
    *tci_out = tci;
}

/* Max-heap of (lambda, index); larger lambda first, equal lambda -> smaller
 * index first. Entries may be stale; the caller checks them when popped. */
typedef struct { int64_t lam; int idx; } HItem;
typedef struct { HItem *a; int64_t n, cap; } Heap;

static int hbefore(HItem x, HItem y) { return x.lam > y.lam || (x.lam == y.lam && x.idx < y.idx); }

static void hpush(Heap *h, int64_t lam, int idx)
{
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = realloc(h->a, sizeof(HItem) * (size_t)h->cap);
        if (!h->a) abort();
    }
    int64_t c = h->n++;
    h->a[c].lam = lam;
    h->a[c].idx = idx;
    while (c > 0) {
        int64_t p = (c - 1) / 2;
        if (!hbefore(h->a[c], h->a[p])) break;
        HItem t = h->a[c]; h->a[c] = h->a[p]; h->a[p] = t;
        c = p;
    }
}

static HItem hpop(Heap *h)
{
    HItem top = h->a[0];
    h->a[0] = h->a[--h->n];
    int64_t c = 0;
    for (;;) {
        int64_t l = 2 * c + 1, r = l + 1, b = c;
        if (l < h->n && hbefore(h->a[l], h->a[b])) b = l;
        if (r < h->n && hbefore(h->a[r], h->a[b])) b = r;
        if (b == c) break;
        HItem t = h->a[c]; h->a[c] = h->a[b]; h->a[b] = t;
        c = b;
    }
    return top;
}

/* Ruge-Stueben first pass (Section 2: a maximal set of C points that do not
 * strongly influence each other but strongly influence the F points).
 * state: 1 = C, 2 = F. */
static int *rs_coarsen(int n, const int64_t *srp, const int *sci)
{
    int64_t *trp;
    int *tci;
    pattern_transpose(n, srp, sci, &trp, &tci);   /* S^T: row i = points depending on i */
    int *state = xcalloc((size_t)n, sizeof(int)); /* 0 = undecided */
    int64_t *lam = xcalloc((size_t)n, sizeof(int64_t));
    Heap h = {0};
    for (int i = 0; i < n; ++i) {
        lam[i] = trp[i + 1] - trp[i];
        if (srp[i + 1] == srp[i] && trp[i + 1] == trp[i]) state[i] = 2;
    }
    for (int i = 0; i < n; ++i)
        if (state[i] == 0) hpush(&h, lam[i], i);
    while (h.n > 0) {
        HItem it = hpop(&h);
        int i = it.idx;
        if (state[i] != 0 || it.lam != lam[i]) continue;
        state[i] = 1;
        for (int64_t k = trp[i]; k < trp[i + 1]; ++k) {
            int j = tci[k];
            if (state[j] != 0) continue;
            state[j] = 2;
            for (int64_t q = srp[j]; q < srp[j + 1]; ++q) {
                int m = sci[q];
                if (state[m] == 0) { lam[m] += 1; hpush(&h, lam[m], m); }
            }
        }
        for (int64_t k = srp[i]; k < srp[i + 1]; ++k) {
            int j = sci[k];
            if (state[j] == 0) { lam[j] -= 1; hpush(&h, lam[j], j); }
        }
    }
    free(h.a);
    free(lam);
    free(trp);
    free(tci);
    return state;
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the output for counter x. It stands in for the
 * random part of the PMIS measure below, so that the coarsening is
 * reproducible: point i of level l draws splitmix64((l << 40) + i). */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* PMIS order of two points: i before j when |S_i^T| is larger, then when
 * its SplitMix64 draw is larger, then when its index is smaller. */
static int pmis_before(int i, int j, const int64_t *trp, const uint64_t *draw)
{
    int64_t ci = trp[i + 1] - trp[i], cj = trp[j + 1] - trp[j];
    if (ci != cj) return ci > cj;
    if (draw[i] != draw[j]) return draw[i] > draw[j];
    return i < j;
}

/* HMIS coarsening (the coarsening of the hypre defaults that Section 6 names;
 * the paper does not restate it, this follows the published definition of De
 * Sterck, Yang and Heys, SIAM J. Matrix Anal. Appl. 27 (2006)), with the
 * subdomains in the role of the processors (sub[i] = subdomain of point i):
 *  1. the Ruge-Stueben first pass (rs_coarsen) on each subdomain alone, i.e.
 *     on the strong connections between points of the same subdomain;
 *  2. its C points that are interior (no strong connection, in either
 *     direction, to a point of another subdomain) are the first independent
 *     set of PMIS on the whole strength graph: they are C, everything else
 *     undecided;
 *  3. PMIS: undecided points on which no point depends strongly (|S_i^T| = 0)
 *     become F; then repeat: every undecided point that strongly depends on a
 *     C point becomes F; stop when none is undecided; else every undecided
 *     point that comes before all its undecided strong neighbours (S_i and
 *     S_i^T, in the order of pmis_before) becomes C.
 * With one subdomain every point is interior and the result is the first
 * pass itself. Returns 1 (C) / 2 (F) per point, like rs_coarsen. */
static int *hmis_coarsen(int n, const int64_t *srp, const int *sci, const int *sub, int level)
{
    /* 1. first pass on the same-subdomain connections */
    int64_t *lrp = xmalloc(sizeof(int64_t) * ((size_t)n + 1));
    int *lci = xmalloc(sizeof(int) * (size_t)(srp[n] > 0 ? srp[n] : 1));
    lrp[0] = 0;
    for (int i = 0; i < n; ++i) {
        int64_t o = lrp[i];
        for (int64_t k = srp[i]; k < srp[i + 1]; ++k)
            if (sub[sci[k]] == sub[i]) lci[o++] = sci[k];
        lrp[i + 1] = o;
    }
    int *first = rs_coarsen(n, lrp, lci);
    free(lrp);
    free(lci);
    /* 2. interior C points of the first pass */
    int64_t *trp;
    int *tci;
    pattern_transpose(n, srp, sci, &trp, &tci);
    int *state = xcalloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int interior = 1;
        for (int64_t k = srp[i]; k < srp[i + 1] && interior; ++k) interior = sub[sci[k]] == sub[i];
        for (int64_t k = trp[i]; k < trp[i + 1] && interior; ++k) interior = sub[tci[k]] == sub[i];
        if (interior && first[i] == 1) state[i] = 1;
    }
    free(first);
    /* 3. PMIS */
    uint64_t *draw = xmalloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) draw[i] = splitmix64(((uint64_t)level << 40) + (uint64_t)i);
    for (int i = 0; i < n; ++i)
        if (state[i] == 0 && trp[i + 1] == trp[i]) state[i] = 2;
    int *pick = xcalloc((size_t)n, sizeof(int));
    for (;;) {
        for (int i = 0; i < n; ++i) {
            if (state[i] != 0) continue;
            for (int64_t k = srp[i]; k < srp[i + 1]; ++k)
                if (state[sci[k]] == 1) { state[i] = 2; break; }
        }
        int left = 0;
        for (int i = 0; i < n; ++i) left += state[i] == 0;
        if (left == 0) break;
        for (int i = 0; i < n; ++i) {
            pick[i] = 0;
            if (state[i] != 0) continue;
            int first_among = 1;
            for (int64_t k = srp[i]; k < srp[i + 1] && first_among; ++k) {
                int j = sci[k];
                if (j != i && state[j] == 0 && pmis_before(j, i, trp, draw)) first_among = 0;
            }
            for (int64_t k = trp[i]; k < trp[i + 1] && first_among; ++k) {
                int j = tci[k];
                if (j != i && state[j] == 0 && pmis_before(j, i, trp, draw)) first_among = 0;
            }
            pick[i] = first_among;
        }
        for (int i = 0; i < n; ++i)
            if (pick[i]) state[i] = 1;
    }
    free(pick);
    free(draw);
    free(trp);
    free(tci);
    return state;
}

/* Direct interpolation (Section 2: P_l built from the connections in A_l):
 * C point: injection. F point i with strong C neighbours C_i:
 *   alpha = (sum_{j!=i, a_ij<0} a_ij) / (sum_{k in C_i} a_ik),
 *   d     = a_ii + sum_{j!=i, a_ij>0} a_ij,
 *   w_ik  = (-alpha * a_ik) / d.
 * All sums run over ascending column index. */
static void direct_interp(const Mat *A, const int64_t *srp, const int *sci, const int *state,
                          const int *cmap, int nc, Mat *P)
{
    int n = A->n;
    P->n = n;
    P->m = nc;
    P->rp = xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int i = 0; i < n; ++i) {
        int64_t c = 0;
        if (state[i] == 1) c = 1;
        else
            for (int64_t q = srp[i]; q < srp[i + 1]; ++q) c += (state[sci[q]] == 1);
        P->rp[i + 1] = P->rp[i] + c;
    }
    P->ci = xmalloc(sizeof(int) * (size_t)(P->rp[n] > 0 ? P->rp[n] : 1));
    P->v = xmalloc(sizeof(double) * (size_t)(P->rp[n] > 0 ? P->rp[n] : 1));
    for (int i = 0; i < n; ++i) {
        int64_t o = P->rp[i];
        if (state[i] == 1) {
            P->ci[o] = cmap[i];
            P->v[o] = 1.0;
            continue;
        }
        if (P->rp[i + 1] == o) continue;
        double num = 0.0, d = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
            if (A->ci[k] == i) d = A->v[k];
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            if (A->ci[k] == i) continue;
            if (A->v[k] < 0.0) num = num + A->v[k];
            else if (A->v[k] > 0.0) d = d + A->v[k];
        }
        /* entries a_ij for the strong C neighbours, ascending j (S_i is
         * ascending and so is row i of A) */
        double den = 0.0;
        int64_t k = A->rp[i];
        for (int64_t q = srp[i]; q < srp[i + 1]; ++q) {
            int j = sci[q];
            if (state[j] != 1) continue;
            while (A->ci[k] != j) ++k;
            den = den + A->v[k];
        }
        double alpha = num / den;
        k = A->rp[i];
        for (int64_t q = srp[i]; q < srp[i + 1]; ++q) {
            int j = sci[q];
            if (state[j] != 1) continue;
            while (A->ci[k] != j) ++k;
            P->ci[o] = cmap[j];
            P->v[o] = (-alpha * A->v[k]) / d;
            ++o;
        }
    }
}

/* Extended+i interpolation (the distance-two interpolation of the hypre
 * defaults that Section 6 names; the paper does not restate it, this follows
 * its published definition). For an F point i with strong influencers S_i:
 *   C_i = S_i n C, F_i = S_i n F (ascending),
 *   Chat_i = C_i u (union over k in F_i of S_k n C), ascending;
 *   abar_kl = a_kl if a_kl * a_kk < 0, else 0;
 *   D_k = sum over l in Chat_i u {i} of abar_kl (row k ascending), k in F_i;
 *   d   = a_ii + sum over the other entries n of row i (ascending) of
 *           (a_in * abar_ni) / D_n   if n in F_i and D_n != 0,
 *           a_in                     if n in F_i and D_n == 0,
 *           a_in                     if n not in Chat_i u F_i,
 *         nothing                    if n in Chat_i;
 *   num_j = a_ij (0 if absent) + sum over k in F_i with D_k != 0 (ascending)
 *           of (a_ik * abar_kj) / D_k,   j in Chat_i;
 *   w_ij  = (-num_j) / d.
 * Truncation (pmax > 0, rows with more than pmax entries): keep the pmax
 * entries of largest |w| (ties to the smaller column), multiply them by
 * (sum of all w, ascending) / (sum of the kept w, ascending) when the latter
 * is nonzero, keep ascending columns. C points: injection; an F point with
 * empty Chat_i: empty row. */
static void exti_interp(const Mat *A, const int64_t *srp, const int *sci, const int *state,
                        const int *cmap, int nc, int pmax, Mat *P)
{
    int n = A->n;
    int *inC = xmalloc(sizeof(int) * (size_t)(n > 0 ? n : 1));   /* Chat membership: owner row */
    int *inF = xmalloc(sizeof(int) * (size_t)(n > 0 ? n : 1));   /* F_i membership: owner row */
    double *Dk = xmalloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) inC[i] = inF[i] = -1;
    int64_t cap = 1024, used = 0;
    int *rc = xmalloc(sizeof(int) * (size_t)cap);
    double *rv = xmalloc(sizeof(double) * (size_t)cap);
    int64_t *rp = xcalloc((size_t)n + 1, sizeof(int64_t));
    int *ch = xmalloc(sizeof(int) * 64), chcap = 64;
    double *wv = xmalloc(sizeof(double) * 64);
    int *ord = xmalloc(sizeof(int) * 64);
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        if (state[i] == 1) {
            ch[0] = cmap[i];
            wv[0] = 1.0;
            cnt = 1;
        } else {
            /* Chat_i and F_i */
            for (int64_t q = srp[i]; q < srp[i + 1]; ++q) {
                int j = sci[q];
                if (state[j] == 1) {
                    if (inC[j] != i) {
                        inC[j] = i;
                        if (cnt == chcap) {
                            chcap *= 2;
                            ch = realloc(ch, sizeof(int) * (size_t)chcap);
                            wv = realloc(wv, sizeof(double) * (size_t)chcap);
                            ord = realloc(ord, sizeof(int) * (size_t)chcap);
                        }
                        ch[cnt++] = j;
                    }
                } else {
                    inF[j] = i;
                    for (int64_t q2 = srp[j]; q2 < srp[j + 1]; ++q2) {
                        int m = sci[q2];
                        if (state[m] == 1 && inC[m] != i) {
                            inC[m] = i;
                            if (cnt == chcap) {
                                chcap *= 2;
                                ch = realloc(ch, sizeof(int) * (size_t)chcap);
                                wv = realloc(wv, sizeof(double) * (size_t)chcap);
                                ord = realloc(ord, sizeof(int) * (size_t)chcap);
                            }
                            ch[cnt++] = m;
                        }
                    }
                }
            }
            /* ascending Chat_i (insertion sort: the sets are small) */
            for (int a = 1; a < cnt; ++a) {
                int v = ch[a], b = a - 1;
                while (b >= 0 && ch[b] > v) { ch[b + 1] = ch[b]; --b; }
                ch[b + 1] = v;
            }
            if (cnt > 0) {
                /* D_k for k in F_i */
                for (int64_t q = srp[i]; q < srp[i + 1]; ++q) {
                    int k = sci[q];
                    if (inF[k] != i) continue;
                    double akk = 0.0, D = 0.0;
                    for (int64_t e = A->rp[k]; e < A->rp[k + 1]; ++e)
                        if (A->ci[e] == k) akk = A->v[e];
                    for (int64_t e = A->rp[k]; e < A->rp[k + 1]; ++e) {
                        int l = A->ci[e];
                        if (l != i && inC[l] != i) continue;
                        double a = A->v[e];
                        if (a * akk < 0.0) D = D + a;
                    }
                    Dk[k] = D;
                }
                /* d */
                double d = 0.0;
                for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
                    if (A->ci[e] == i) d = A->v[e];
                for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e) {
                    int nn = A->ci[e];
                    if (nn == i) continue;
                    double a = A->v[e];
                    if (inF[nn] == i) {
                        if (Dk[nn] != 0.0) {
                            double akk = 0.0, aki = 0.0;
                            for (int64_t f = A->rp[nn]; f < A->rp[nn + 1]; ++f) {
                                if (A->ci[f] == nn) akk = A->v[f];
                                if (A->ci[f] == i) aki = A->v[f];
                            }
                            double abar = aki * akk < 0.0 ? aki : 0.0;
                            d = d + (a * abar) / Dk[nn];
                        } else {
                            d = d + a;
                        }
                    } else if (inC[nn] != i) {
                        d = d + a;
                    }
                }
                /* num_j, w_ij */
                for (int t = 0; t < cnt; ++t) {
                    int j = ch[t];
                    double num = 0.0;
                    for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
                        if (A->ci[e] == j) num = A->v[e];
                    for (int64_t q = srp[i]; q < srp[i + 1]; ++q) {
                        int k = sci[q];
                        if (inF[k] != i || Dk[k] == 0.0) continue;
                        double aik = 0.0, akk = 0.0, akj = 0.0;
                        for (int64_t e = A->rp[i]; e < A->rp[i + 1]; ++e)
                            if (A->ci[e] == k) aik = A->v[e];
                        for (int64_t f = A->rp[k]; f < A->rp[k + 1]; ++f) {
                            if (A->ci[f] == k) akk = A->v[f];
                            if (A->ci[f] == j) akj = A->v[f];
                        }
                        double abar = akj * akk < 0.0 ? akj : 0.0;
                        num = num + (aik * abar) / Dk[k];
                    }
                    wv[t] = (-num) / d;
                }
                /* truncation */
                if (pmax > 0 && cnt > pmax) {
                    for (int t = 0; t < cnt; ++t) ord[t] = t;
                    for (int a = 1; a < cnt; ++a) {   /* by |w| descending, then column */
                        int v = ord[a], b = a - 1;
                        while (b >= 0 && (fabs(wv[ord[b]]) < fabs(wv[v]) ||
                                          (fabs(wv[ord[b]]) == fabs(wv[v]) && ch[ord[b]] > ch[v]))) {
                            ord[b + 1] = ord[b];
                            --b;
                        }
                        ord[b + 1] = v;
                    }
                    char keep[4096];
                    char *kp = cnt <= 4096 ? keep : xmalloc((size_t)cnt);
                    for (int t = 0; t < cnt; ++t) kp[t] = 0;
                    for (int t = 0; t < pmax; ++t) kp[ord[t]] = 1;
                    double all = 0.0, kept = 0.0;
                    for (int t = 0; t < cnt; ++t) all = all + wv[t];
                    for (int t = 0; t < cnt; ++t)
                        if (kp[t]) kept = kept + wv[t];
                    int o = 0;
                    for (int t = 0; t < cnt; ++t) {
                        if (!kp[t]) continue;
                        ch[o] = ch[t];
                        wv[o] = kept != 0.0 ? wv[t] * (all / kept) : wv[t];
                        ++o;
                    }
                    if (kp != keep) free(kp);
                    cnt = o;
                }
                for (int t = 0; t < cnt; ++t) ch[t] = cmap[ch[t]];
            }
        }
        if (used + cnt > cap) {
            while (used + cnt > cap) cap *= 2;
            rc = realloc(rc, sizeof(int) * (size_t)cap);
            rv = realloc(rv, sizeof(double) * (size_t)cap);
        }
        for (int t = 0; t < cnt; ++t) {
            rc[used + t] = ch[t];
            rv[used + t] = wv[t];
        }
        used += cnt;
        rp[i + 1] = used;
    }
    P->n = n;
    P->m = nc;
    P->rp = rp;
    P->ci = rc;
    P->v = rv;
    free(inC); free(inF); free(Dk); free(ch); free(wv); free(ord);
}

/* R = P^T with ascending fine index in each row. */
static void transpose(const Mat *P, Mat *R)
{
    int n = P->n, m = P->m;
    R->n = m;
    R->m = n;
    R->rp = xcalloc((size_t)m + 1, sizeof(int64_t));
    int64_t nnz = P->rp[n];
    R->ci = xmalloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    R->v = xmalloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t k = 0; k < nnz; ++k) R->rp[P->ci[k] + 1]++;
    for (int I = 0; I < m; ++I) R->rp[I + 1] += R->rp[I];
    int64_t *pos = xmalloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int I = 0; I < m; ++I) pos[I] = R->rp[I];
    for (int i = 0; i < n; ++i)
        for (int64_t k = P->rp[i]; k < P->rp[i + 1]; ++k) {
            int64_t o = pos[P->ci[k]]++;
            R->ci[o] = i;
            R->v[o] = P->v[k];
        }
    free(pos);
}

static int cmp_int(const void *a, const void *b) { int x = *(const int *)a, y = *(const int *)b; return (x > y) - (x < y); }

/* Galerkin product A_c = R A P (Section 2). Entry (I, J) accumulates the terms
 * (p_iI * a_ij) * p_jJ in the order: fine i ascending (row I of R), then j
 * ascending (row i of A), then J (row j of P); every structural term is kept,
 * so the pattern does not depend on cancellation. */
static void galerkin(const Mat *R, const Mat *A, const Mat *P, Mat *Ac)
{
    int m = R->n;
    int64_t *marker = xmalloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int J = 0; J < m; ++J) marker[J] = -1;
    /* symbolic pass */
    int64_t *rp = xcalloc((size_t)m + 1, sizeof(int64_t));
    for (int I = 0; I < m; ++I) {
        int64_t c = 0;
        for (int64_t a = R->rp[I]; a < R->rp[I + 1]; ++a) {
            int i = R->ci[a];
            for (int64_t b = A->rp[i]; b < A->rp[i + 1]; ++b) {
                int j = A->ci[b];
                for (int64_t d = P->rp[j]; d < P->rp[j + 1]; ++d) {
                    int J = P->ci[d];
                    if (marker[J] != I) { marker[J] = I; ++c; }
                }
            }
        }
        rp[I + 1] = rp[I] + c;
    }
    int *ci = xmalloc(sizeof(int) * (size_t)(rp[m] > 0 ? rp[m] : 1));
    double *v = xmalloc(sizeof(double) * (size_t)(rp[m] > 0 ? rp[m] : 1));
    double *acc = xcalloc((size_t)(m > 0 ? m : 1), sizeof(double));
    for (int J = 0; J < m; ++J) marker[J] = -1;
    for (int I = 0; I < m; ++I) {
        int64_t c = rp[I];
        for (int64_t a = R->rp[I]; a < R->rp[I + 1]; ++a) {
            int i = R->ci[a];
            double piI = R->v[a];
            for (int64_t b = A->rp[i]; b < A->rp[i + 1]; ++b) {
                int j = A->ci[b];
                double t = piI * A->v[b];
                for (int64_t d = P->rp[j]; d < P->rp[j + 1]; ++d) {
                    int J = P->ci[d];
                    double term = t * P->v[d];
                    if (marker[J] != I) { marker[J] = I; ci[c++] = J; acc[J] = 0.0; }
                    acc[J] = acc[J] + term;
                }
            }
        }
        qsort(ci + rp[I], (size_t)(rp[I + 1] - rp[I]), sizeof(int), cmp_int);
        for (int64_t k = rp[I]; k < rp[I + 1]; ++k) v[k] = acc[ci[k]];
    }
    free(acc);
    free(marker);
    Ac->n = m;
    Ac->m = m;
    Ac->rp = rp;
    Ac->ci = ci;
    Ac->v = v;
}

/* l1 row norms, summed over ascending column index. */
static double *l1_inverse(const Mat *A)
{
    double *o = xmalloc(sizeof(double) * (size_t)(A->n > 0 ? A->n : 1));
    for (int i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s = s + fabs(A->v[k]);
        o[i] = 1.0 / s;
    }
    return o;
}

/* Explicit inverse of the coarsest matrix by Gauss-Jordan elimination with
 * partial pivoting (first largest |pivot|). Returns 0 on success. */
static int gauss_jordan_inverse(const Mat *A, double *X)
{
    int n = A->n;
    double *M = xcalloc((size_t)n * (size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) M[(size_t)i * n + A->ci[k]] = A->v[k];
    memset(X, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(M[(size_t)i * n + k]) > best) { best = fabs(M[(size_t)i * n + k]); p = i; }
        if (best == 0.0) { free(M); return 1; }
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = M[(size_t)k * n + j]; M[(size_t)k * n + j] = M[(size_t)p * n + j]; M[(size_t)p * n + j] = t;
                t = X[(size_t)k * n + j]; X[(size_t)k * n + j] = X[(size_t)p * n + j]; X[(size_t)p * n + j] = t;
            }
        double piv = M[(size_t)k * n + k];
        for (int j = 0; j < n; ++j) {
            M[(size_t)k * n + j] = M[(size_t)k * n + j] / piv;
            X[(size_t)k * n + j] = X[(size_t)k * n + j] / piv;
        }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            double f = M[(size_t)i * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                M[(size_t)i * n + j] = M[(size_t)i * n + j] - f * M[(size_t)k * n + j];
                X[(size_t)i * n + j] = X[(size_t)i * n + j] - f * X[(size_t)k * n + j];
            }
        }
    }
    free(M);
    return 0;
}

static void mat_copy_in(Mat *M, int n, const int64_t *rp, const int *ci, const double *v)
{
    M->n = n;
    M->m = n;
    M->rp = xmalloc(sizeof(int64_t) * ((size_t)n + 1));
    memcpy(M->rp, rp, sizeof(int64_t) * ((size_t)n + 1));
    int64_t nnz = rp[n];
    M->ci = xmalloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    M->v = xmalloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    memcpy(M->ci, ci, sizeof(int) * (size_t)nnz);
    memcpy(M->v, v, sizeof(double) * (size_t)nnz);
}

/* Build the hierarchy: repeat C/F splitting, P_l, R_l = P_l^T and
 * A_{l+1} = R_l A_l P_l until n_l <= max_coarse, max_levels levels exist, or
 * the split keeps more than 90% of the points (Section 2). */
void *orc_hier_build(int n, const int64_t *rp, const int *ci, const double *v, double theta,
                     int max_coarse, int max_levels, int interp, int pmax, int coarsen, const int *part)
{
    Hier *H = xcalloc(1, sizeof(Hier));
    if (max_levels > ORC_MAXLEV) max_levels = ORC_MAXLEV;
    mat_copy_in(&H->A[0], n, rp, ci, v);
    /* subdomain of every point of the current level (HMIS): level 0 from
     * part, a C point keeps the subdomain of the fine point it comes from */
    int *sub = xmalloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) sub[i] = part ? part[i] : 0;
    int l = 0;
    for (;;) {
        Mat *A = &H->A[l];
        H->l1inv[l] = l1_inverse(A);
        if (l + 1 >= max_levels || A->n <= max_coarse) break;
        int64_t *srp;
        int *sci;
        strength(A, theta, &srp, &sci);
        int *state = coarsen == 1 ? hmis_coarsen(A->n, srp, sci, sub, l) : rs_coarsen(A->n, srp, sci);
        int nc = 0;
        for (int i = 0; i < A->n; ++i) nc += (state[i] == 1);
        if (nc == 0 || (int64_t)nc * 10 > (int64_t)A->n * 9) {
            free(srp); free(sci); free(state);
            break;
        }
        int *cf = xmalloc(sizeof(int) * (size_t)A->n);
        int *cmap = xmalloc(sizeof(int) * (size_t)A->n);
        int c = 0;
        for (int i = 0; i < A->n; ++i) {
            cf[i] = (state[i] == 1);
            cmap[i] = cf[i] ? c++ : -1;
        }
        if (interp == 1) exti_interp(A, srp, sci, state, cmap, nc, pmax, &H->P[l]);
        else direct_interp(A, srp, sci, state, cmap, nc, &H->P[l]);
        transpose(&H->P[l], &H->R[l]);
        galerkin(&H->R[l], A, &H->P[l], &H->A[l + 1]);
        int *subc = xmalloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
        for (int i = 0; i < A->n; ++i)
            if (cf[i]) subc[cmap[i]] = sub[i];
        free(sub);
        sub = subc;
        H->cf[l] = cf;
        H->cmap[l] = cmap;
        free(srp); free(sci); free(state);
        ++l;
    }
    free(sub);
    H->nlev = l + 1;
    int nL = H->A[l].n;
    if (nL > ORC_MAX_COARSE_DENSE) {     /* a dense inverse would not fit */
        H->ainv = xcalloc(1, sizeof(double));
        H->status = 2;
        return H;
    }
    H->ainv = xmalloc(sizeof(double) * (size_t)nL * (size_t)nL + 8);
    H->status = gauss_jordan_inverse(&H->A[l], H->ainv);
    return H;
}

void orc_hier_free(void *h)
{
    Hier *H = h;
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) {
        mat_free(&H->A[l]); mat_free(&H->P[l]); mat_free(&H->R[l]);
        free(H->cf[l]); free(H->cmap[l]); free(H->l1inv[l]);
    }
    free(H->ainv);
    free(H);
}

int orc_hier_status(void *h) { return ((Hier *)h)->status; }
int orc_hier_nlev(void *h) { return ((Hier *)h)->nlev; }
int orc_hier_n(void *h, int l) { return ((Hier *)h)->A[l].n; }

static const Mat *pick(Hier *H, int l, int which)
{
    return which == 0 ? &H->A[l] : which == 1 ? &H->P[l] : &H->R[l];
}

int64_t orc_hier_nnz(void *h, int l, int which) { const Mat *M = pick(h, l, which); return M->rp ? M->rp[M->n] : 0; }
int orc_hier_rows(void *h, int l, int which) { return pick(h, l, which)->n; }
int orc_hier_cols(void *h, int l, int which) { return pick(h, l, which)->m; }

void orc_hier_get(void *h, int l, int which, int64_t *rp, int *ci, double *v)
{
    const Mat *M = pick(h, l, which);
    memcpy(rp, M->rp, sizeof(int64_t) * ((size_t)M->n + 1));
    memcpy(ci, M->ci, sizeof(int) * (size_t)M->rp[M->n]);
    memcpy(v, M->v, sizeof(double) * (size_t)M->rp[M->n]);
}

void orc_hier_get_cf(void *h, int l, int *cf) { Hier *H = h; memcpy(cf, H->cf[l], sizeof(int) * (size_t)H->A[l].n); }
void orc_hier_get_l1inv(void *h, int l, double *o) { Hier *H = h; memcpy(o, H->l1inv[l], sizeof(double) * (size_t)H->A[l].n); }
void orc_hier_get_ainv(void *h, double *o)
{
    Hier *H = h;
    int nL = H->A[H->nlev - 1].n;
    memcpy(o, H->ainv, sizeof(double) * (size_t)nL * (size_t)nL);
}

/* ------------------------------------------------------------------ */
/* Composite grids (Section 3, Fig. 1; eq. (1))                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int nreal, nghost, nowned;
    int *real, *ghost, *owned;    /* ascending global indices of the level */
} CLevel;

typedef struct {
    int nsub, nlev;
    CLevel *lv;                   /* [p * nlev + l] */
    int64_t violations;           /* grid-level pairs that break the connectivity assumption */
    unsigned char *vflag;         /* [p * nlev + l]: 1 where pair (p, l) breaks it */
} Comp;

/* Multi-source breadth-first search to distance eta through the graph of A
 * (structural off-diagonal entries). dist[] must be -1 on entry for every
 * point; the visited points are returned ascending and dist[] is restored. */
static int *bfs_ball(const Mat *A, const int *seeds, int ns, int eta, int *dist, int *nout)
{
    int cap = ns > 16 ? ns * 4 : 64;
    int *q = xmalloc(sizeof(int) * (size_t)cap);
    int qn = 0;
    for (int s = 0; s < ns; ++s)
        if (dist[seeds[s]] < 0) { dist[seeds[s]] = 0; q[qn++] = seeds[s]; }
    for (int h = 0; h < qn; ++h) {
        int i = q[h];
        if (dist[i] >= eta) continue;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (dist[j] >= 0) continue;
            dist[j] = dist[i] + 1;
            if (qn == cap) { cap *= 2; q = realloc(q, sizeof(int) * (size_t)cap); if (!q) abort(); }
            q[qn++] = j;
        }
    }
    for (int h = 0; h < qn; ++h) dist[q[h]] = -1;
    qsort(q, (size_t)qn, sizeof(int), cmp_int);
    *nout = qn;
    return q;
}

/* Neighbours of D (graph of A) that are not in D, ascending. inD[] is a
 * scratch byte array of length n, zero on entry and on exit. */
static int *ghost_layer(const Mat *A, const int *D, int nd, unsigned char *inD, int *nout)
{
    for (int s = 0; s < nd; ++s) inD[D[s]] = 1;
    int cap = 64, c = 0;
    int *g = xmalloc(sizeof(int) * (size_t)cap);
    for (int s = 0; s < nd; ++s) {
        int i = D[s];
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (inD[j]) continue;
            inD[j] = 2;
            if (c == cap) { cap *= 2; g = realloc(g, sizeof(int) * (size_t)cap); if (!g) abort(); }
            g[c++] = j;
        }
    }
    for (int s = 0; s < nd; ++s) inD[D[s]] = 0;
    for (int s = 0; s < c; ++s) inD[g[s]] = 0;
    qsort(g, (size_t)c, sizeof(int), cmp_int);
    *nout = c;
    return g;
}

/* Composite grid of every subdomain p (Section 3): D_0 = points within
 * distance eta_0 of the owned set in graph(A_0); D_{l+1} = points within
 * eta_{l+1} of the C points of D_l in graph(A_{l+1}); the coarsest level is
 * stored whole. Dbar_l = D_l plus its neighbours (eq. (1)). The owned set on
 * level l+1 is the C points of the owned set on level l. */
void *orc_comp_build(void *h, const int *part, int nsub, const int *padding)
{
    Hier *H = h;
    int L = H->nlev - 1;
    Comp *C = xcalloc(1, sizeof(Comp));
    C->nsub = nsub;
    C->nlev = H->nlev;
    C->lv = xcalloc((size_t)nsub * (size_t)H->nlev, sizeof(CLevel));
    C->vflag = xcalloc((size_t)nsub * (size_t)H->nlev, 1);
    int n0 = H->A[0].n;
    /* owned sets on level 0 */
    int *cnt = xcalloc((size_t)nsub + 1, sizeof(int));
    for (int i = 0; i < n0; ++i) cnt[part[i] + 1]++;
    for (int p = 0; p < nsub; ++p) cnt[p + 1] += cnt[p];
    int *own0 = xmalloc(sizeof(int) * (size_t)(n0 > 0 ? n0 : 1));
    int *pos = xmalloc(sizeof(int) * (size_t)nsub + 4);
    for (int p = 0; p < nsub; ++p) pos[p] = cnt[p];
    for (int i = 0; i < n0; ++i) own0[pos[part[i]]++] = i;
    free(pos);
#pragma omp parallel
    {
        int nmax = 0;
        for (int l = 0; l <= L; ++l) if (H->A[l].n > nmax) nmax = H->A[l].n;
        int *dist = xmalloc(sizeof(int) * (size_t)(nmax > 0 ? nmax : 1));
        for (int i = 0; i < nmax; ++i) dist[i] = -1;
        unsigned char *mark = xcalloc((size_t)(nmax > 0 ? nmax : 1), 1);
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < nsub; ++p) {
            int no = cnt[p + 1] - cnt[p];
            int *owned = xmalloc(sizeof(int) * (size_t)(no > 0 ? no : 1));
            memcpy(owned, own0 + cnt[p], sizeof(int) * (size_t)no);
            int *seeds = xmalloc(sizeof(int) * (size_t)(no > 0 ? no : 1));
            memcpy(seeds, owned, sizeof(int) * (size_t)no);
            int ns = no;
            for (int l = 0; l <= L; ++l) {
                CLevel *cl = &C->lv[(size_t)p * C->nlev + l];
                cl->owned = owned;
                cl->nowned = no;
                if (l < L) {
                    cl->real = bfs_ball(&H->A[l], seeds, ns, padding[l], dist, &cl->nreal);
                    cl->ghost = ghost_layer(&H->A[l], cl->real, cl->nreal, mark, &cl->nghost);
                } else {
                    int nL = H->A[l].n;
                    cl->real = xmalloc(sizeof(int) * (size_t)(nL > 0 ? nL : 1));
                    for (int i = 0; i < nL; ++i) cl->real[i] = i;
                    cl->nreal = nL;
                    cl->ghost = xmalloc(sizeof(int));
                    cl->nghost = 0;
                }
                free(seeds);
                if (l == L) { seeds = NULL; break; }
                /* C points of D_l and of the owned set, as level l+1 indices */
                int *nxt = xmalloc(sizeof(int) * (size_t)(cl->nreal > 0 ? cl->nreal : 1));
                ns = 0;
                for (int s = 0; s < cl->nreal; ++s)
                    if (H->cf[l][cl->real[s]]) nxt[ns++] = H->cmap[l][cl->real[s]];
                seeds = nxt;
                int *ow = xmalloc(sizeof(int) * (size_t)(no > 0 ? no : 1));
                int c2 = 0;
                for (int s = 0; s < no; ++s)
                    if (H->cf[l][owned[s]]) ow[c2++] = H->cmap[l][owned[s]];
                owned = ow;
                no = c2;
            }
        }
        free(dist);
        free(mark);
    }
    free(cnt);
    free(own0);

    /* Connectivity assumption (Sections 4.2 and 4.5): a coarse point reached
     * from Dbar_l through P_l (equivalently through the columns of
     * R_l = P_l^T) that is not in Dbar_{l+1} must not reach a real point on
     * any coarser level through the interpolatory sets. */
    int64_t viol = 0;
#pragma omp parallel reduction(+ : viol)
    {
        int nmax = 0;
        for (int l = 0; l <= L; ++l) if (H->A[l].n > nmax) nmax = H->A[l].n;
        unsigned char *inbar = xcalloc((size_t)(nmax > 0 ? nmax : 1), 1);
        unsigned char *inreal = xcalloc((size_t)(nmax > 0 ? nmax : 1), 1);
        unsigned char *seen = xcalloc((size_t)(nmax > 0 ? nmax : 1), 1);
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < nsub; ++p) {
            for (int l = 0; l < L; ++l) {
                CLevel *a = &C->lv[(size_t)p * C->nlev + l];
                CLevel *b = &C->lv[(size_t)p * C->nlev + l + 1];
                for (int s = 0; s < b->nreal; ++s) inbar[b->real[s]] = 1;
                for (int s = 0; s < b->nghost; ++s) inbar[b->ghost[s]] = 1;
                /* frontier of points outside Dbar_{l+1} */
                int cap = 64, fn = 0;
                int *fr = xmalloc(sizeof(int) * (size_t)cap);
                for (int pass = 0; pass < 2; ++pass) {
                    const int *set = pass ? a->ghost : a->real;
                    int ns = pass ? a->nghost : a->nreal;
                    for (int s = 0; s < ns; ++s) {
                        int i = set[s];
                        for (int64_t k = H->P[l].rp[i]; k < H->P[l].rp[i + 1]; ++k) {
                            int J = H->P[l].ci[k];
                            if (inbar[J] || seen[J]) continue;
                            seen[J] = 1;
                            if (fn == cap) { cap *= 2; fr = realloc(fr, sizeof(int) * (size_t)cap); if (!fr) abort(); }
                            fr[fn++] = J;
                        }
                    }
                }
                for (int s = 0; s < b->nreal; ++s) inbar[b->real[s]] = 0;
                for (int s = 0; s < b->nghost; ++s) inbar[b->ghost[s]] = 0;
                for (int s = 0; s < fn; ++s) seen[fr[s]] = 0;
                /* follow the interpolatory sets down to the coarsest level */
                int bad = 0;
                for (int m = l + 1; m <= L && fn > 0 && !bad; ++m) {
                    CLevel *cm = &C->lv[(size_t)p * C->nlev + m];
                    for (int s = 0; s < cm->nreal; ++s) inreal[cm->real[s]] = 1;
                    for (int s = 0; s < fn; ++s) if (inreal[fr[s]]) { bad = 1; break; }
                    for (int s = 0; s < cm->nreal; ++s) inreal[cm->real[s]] = 0;
                    if (bad || m == L) break;
                    int cap2 = 64, gn = 0;
                    int *nx = xmalloc(sizeof(int) * (size_t)cap2);
                    for (int s = 0; s < fn; ++s) {
                        int i = fr[s];
                        for (int64_t k = H->P[m].rp[i]; k < H->P[m].rp[i + 1]; ++k) {
                            int J = H->P[m].ci[k];
                            if (seen[J]) continue;
                            seen[J] = 1;
                            if (gn == cap2) { cap2 *= 2; nx = realloc(nx, sizeof(int) * (size_t)cap2); if (!nx) abort(); }
                            nx[gn++] = J;
                        }
                    }
                    for (int s = 0; s < gn; ++s) seen[nx[s]] = 0;
                    free(fr);
                    fr = nx;
                    fn = gn;
                }
                viol += bad;
                C->vflag[(size_t)p * C->nlev + l] = (unsigned char)bad;
                free(fr);
            }
        }
        free(inbar); free(inreal); free(seen);
    }
    C->violations = viol;
    return C;
}

void orc_comp_free(void *c)
{
    Comp *C = c;
    if (!C) return;
    for (size_t k = 0; k < (size_t)C->nsub * C->nlev; ++k) {
        free(C->lv[k].real); free(C->lv[k].ghost); free(C->lv[k].owned);
    }
    free(C->lv);
    free(C->vflag);
    free(C);
}

int64_t orc_comp_violations(void *c) { return ((Comp *)c)->violations; }

/* 1 when composite grid p breaks the connectivity assumption between levels
 * l and l+1 (a point of P_l(Dbar_l) outside Dbar_{l+1} whose interpolatory
 * sets reach a real point of a coarser level), else 0. */
int orc_comp_violation_flag(void *c, int p, int l)
{
    Comp *C = c;
    return C->vflag[(size_t)p * C->nlev + l];
}

/* what: 0 = |D_l|, 1 = |Dbar_l \ D_l|, 2 = owned count */
int orc_comp_count(void *c, int p, int l, int what)
{
    Comp *C = c;
    CLevel *cl = &C->lv[(size_t)p * C->nlev + l];
    return what == 0 ? cl->nreal : what == 1 ? cl->nghost : cl->nowned;
}

/* Local order of a composite level: owned points of D_l ascending, the other
 * real points ascending, then the ghost points ascending.
 * kind: 0 owned, 1 real not owned, 2 ghost. */
void orc_comp_get_map(void *c, int p, int l, int *gidx, unsigned char *kind)
{
    Comp *C = c;
    CLevel *cl = &C->lv[(size_t)p * C->nlev + l];
    int o = 0, a = 0;
    for (int s = 0; s < cl->nowned; ++s) { gidx[o] = cl->owned[s]; kind[o] = 0; ++o; }
    for (int s = 0; s < cl->nreal; ++s) {
        int g = cl->real[s];
        while (a < cl->nowned && cl->owned[a] < g) ++a;
        if (a < cl->nowned && cl->owned[a] == g) continue;
        gidx[o] = g; kind[o] = 1; ++o;
    }
    for (int s = 0; s < cl->nghost; ++s) { gidx[o] = cl->ghost[s]; kind[o] = 2; ++o; }
}

/* Composite-grid overhead (Section 6.1): nonzeros of A_l in the real rows of
 * every composite grid, summed over grids and levels, divided by the
 * nonzeros of all A_l. */
double orc_comp_overhead(void *h, void *c)
{
    Hier *H = h;
    Comp *C = c;
    double num = 0.0, den = 0.0;
    for (int l = 0; l < H->nlev; ++l) den += (double)H->A[l].rp[H->A[l].n];
    for (int p = 0; p < C->nsub; ++p)
        for (int l = 0; l < H->nlev; ++l) {
            CLevel *cl = &C->lv[(size_t)p * C->nlev + l];
            for (int s = 0; s < cl->nreal; ++s) {
                int i = cl->real[s];
                num += (double)(H->A[l].rp[i + 1] - H->A[l].rp[i]);
            }
        }
    return num / den;
}

/* ------------------------------------------------------------------ */
/* Solve phase                                                         */
/* ------------------------------------------------------------------ */

/* One CF l1-Jacobi pass: every listed point i with cf flag `which` (or every
 * listed point when cf is NULL) takes delta_i = (f_i - (A u)_i) / l1_i computed
 * from the u before the pass; then u_i += delta_i (and t_i += delta_i). */
static void relax_pass(const Mat *A, const double *l1inv, const int *cf, int which,
                       const int *pts, int npts, const double *f, double *u, double *t, double *d)
{
    for (int s = 0; s < npts; ++s) {
        int i = pts ? pts[s] : s;
        if (cf && cf[i] != which) continue;
        d[i] = (f[i] - rowdot(A, i, u)) * l1inv[i];
    }
    for (int s = 0; s < npts; ++s) {
        int i = pts ? pts[s] : s;
        if (cf && cf[i] != which) continue;
        u[i] = u[i] + d[i];
        if (t) t[i] = t[i] + d[i];
    }
}

/* Coarsest solve u_L = A_L^{-1} f_L (Algorithm 1 and 4). */
static void coarse_solve(const Hier *H, const double *f, double *u)
{
    int nL = H->A[H->nlev - 1].n;
    for (int I = 0; I < nL; ++I) {
        double s = 0.0;
        for (int J = 0; J < nL; ++J) s = fma(H->ainv[(size_t)I * nL + J], f[J], s);
        u[I] = s;
    }
}

/* r = b - A x (Algorithm 2, first step). */
void orc_residual(void *h, const double *b, const double *x, double *r)
{
    Hier *H = h;
    const Mat *A = &H->A[0];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; ++i) r[i] = b[i] - rowdot(A, i, x);
}

/* r_{l+1} = R_l r_l for every level (Algorithm 2, second step). rl holds the
 * levels back to back; level 0 is the input. */
void orc_restrict_all(void *h, double *rl)
{
    Hier *H = h;
    int64_t off = 0;
    for (int l = 0; l + 1 < H->nlev; ++l) {
        const Mat *R = &H->R[l];
        double *src = rl + off;
        double *dst = rl + off + H->A[l].n;
#pragma omp parallel for schedule(static)
        for (int I = 0; I < R->n; ++I) dst[I] = rowdot(R, I, src);
        off += H->A[l].n;
    }
}

int64_t orc_levels_total(void *h)
{
    Hier *H = h;
    int64_t t = 0;
    for (int l = 0; l < H->nlev; ++l) t += H->A[l].n;
    return t;
}

/* One AMG V(1,1)-cycle in place (Algorithm 1): u_0 holds the iterate on
 * entry and exit, f_0 the right-hand side. Work vectors: levels back to back. */
static void vcycle(const Hier *H, double *u0, const double *f0, double *U, double *F, double *W)
{
    int L = H->nlev - 1;
    int64_t off[ORC_MAXLEV + 1];
    off[0] = 0;
    for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + H->A[l].n;
    double *u[ORC_MAXLEV], *f[ORC_MAXLEV];
    u[0] = u0;
    f[0] = (double *)f0;
    for (int l = 1; l <= L; ++l) { u[l] = U + off[l]; f[l] = F + off[l]; }
    for (int l = 0; l < L; ++l) {
        const Mat *A = &H->A[l];
        double *d = W;
        relax_pass(A, H->l1inv[l], H->cf[l], 1, NULL, A->n, f[l], u[l], NULL, d);
        relax_pass(A, H->l1inv[l], H->cf[l], 0, NULL, A->n, f[l], u[l], NULL, d);
        double *res = W;
        for (int i = 0; i < A->n; ++i) res[i] = f[l][i] - rowdot(A, i, u[l]);
        for (int I = 0; I < H->R[l].n; ++I) f[l + 1][I] = rowdot(&H->R[l], I, res);
        for (int I = 0; I < H->A[l + 1].n; ++I) u[l + 1][I] = 0.0;
    }
    coarse_solve(H, f[L], u[L]);
    for (int l = L - 1; l >= 0; --l) {
        const Mat *A = &H->A[l];
        for (int i = 0; i < A->n; ++i) u[l][i] = u[l][i] + rowdot(&H->P[l], i, u[l + 1]);
        relax_pass(A, H->l1inv[l], H->cf[l], 0, NULL, A->n, f[l], u[l], NULL, W);
        relax_pass(A, H->l1inv[l], H->cf[l], 1, NULL, A->n, f[l], u[l], NULL, W);
    }
}

/* One V-cycle applied to (u, f) in place; used to check the cycle's symmetry. */
void orc_vcycle_apply(void *h, const double *f, double *u)
{
    Hier *H = h;
    int64_t tot = orc_levels_total(h);
    double *U = xcalloc((size_t)tot, sizeof(double));
    double *F = xcalloc((size_t)tot, sizeof(double));
    double *W = xcalloc((size_t)H->A[0].n, sizeof(double));
    vcycle(H, u, f, U, F, W);
    free(U); free(F); free(W);
}

static double norm2(const double *r, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = s + r[i] * r[i];
    return sqrt(s);
}

/* V-cycle solver: iterate x <- Vcycle(x, b) until ||b - A x|| / ||b|| <= tol.
 * Returns the number of cycles; hist[k] = relative residual before cycle k+1. */
int orc_vcycle_solve(void *h, const double *b, double *x, double tol, int maxit, double *hist)
{
    Hier *H = h;
    int n = H->A[0].n;
    int64_t tot = orc_levels_total(h);
    double *U = xcalloc((size_t)tot, sizeof(double));
    double *F = xcalloc((size_t)tot, sizeof(double));
    double *W = xcalloc((size_t)n, sizeof(double));
    double *r = xcalloc((size_t)n, sizeof(double));
    double ref = norm2(b, n);
    int k = 0;
    for (;;) {
        orc_residual(h, b, x, r);
        double nr = norm2(r, n);
        if (k == 0 && ref == 0.0) ref = nr;
        double rel = ref > 0.0 ? nr / ref : 0.0;
        hist[k] = rel;
        if (rel <= tol || k >= maxit) break;
        vcycle(H, x, b, U, F, W);
        ++k;
    }
    free(U); free(F); free(W); free(r);
    return k;
}

/* Work space for one composite-grid solve with vectors indexed by the
 * global index of each level (zero outside the composite grid). */
typedef struct {
    int64_t off[ORC_MAXLEV + 1];
    double *u, *f, *t, *s, *w, *d;
} FacWork;

static void facwork_init(const Hier *H, FacWork *W)
{
    W->off[0] = 0;
    for (int l = 0; l < H->nlev; ++l) W->off[l + 1] = W->off[l] + H->A[l].n;
    size_t tot = (size_t)W->off[H->nlev];
    W->u = xcalloc(tot, sizeof(double));
    W->f = xcalloc(tot, sizeof(double));
    W->t = xcalloc(tot, sizeof(double));
    W->s = xcalloc(tot, sizeof(double));
    W->w = xcalloc(tot, sizeof(double));
    W->d = xcalloc(tot, sizeof(double));
}

static void facwork_free(FacWork *W) { free(W->u); free(W->f); free(W->t); free(W->s); free(W->w); free(W->d); }

/* AlgFAC V(1,1)-cycles on the composite grid of subdomain p (Algorithm 4).
 * rl: restricted residuals of every level (levels back to back); they are the
 * right-hand sides at the real points. On return W->u / W->f hold the cycle's
 * u_l on Dbar_l and f_l on D_l; the caller clears them with facwork_clear. */
static void algfac(const Hier *H, const Comp *C, int p, const double *rl, int nfac, FacWork *W)
{
    int L = H->nlev - 1;
    const CLevel *cl = &C->lv[(size_t)p * C->nlev];
    for (int l = 0; l <= L; ++l) {
        double *f = W->f + W->off[l];
        const double *r = rl + W->off[l];
        for (int s = 0; s < cl[l].nreal; ++s) f[cl[l].real[s]] = r[cl[l].real[s]];
    }
    for (int c = 1; c <= nfac; ++c) {
        for (int l = 0; l < L; ++l) {
            const Mat *A = &H->A[l];
            double *u = W->u + W->off[l], *f = W->f + W->off[l], *t = W->t + W->off[l];
            double *s = W->s + W->off[l], *w = W->w + W->off[l], *d = W->d + W->off[l];
            const CLevel *a = &cl[l], *b = &cl[l + 1];
            if (l != 0) {                                   /* u_l <- 0 */
                for (int q = 0; q < a->nreal; ++q) u[a->real[q]] = 0.0;
                for (int q = 0; q < a->nghost; ++q) u[a->ghost[q]] = 0.0;
            }
            /* relax (C then F points) and accumulate the update in t_l */
            relax_pass(A, H->l1inv[l], H->cf[l], 1, a->real, a->nreal, f, u, t, d);
            relax_pass(A, H->l1inv[l], H->cf[l], 0, a->real, a->nreal, f, u, t, d);
            /* s_{l+1} <- R_l (s_l + A_l t_l), with s_l + A_l t_l kept on Dbar_l */
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; w[i] = s[i] + rowdot(A, i, t); }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; w[i] = s[i] + rowdot(A, i, t); }
            double *s1 = W->s + W->off[l + 1], *f1 = W->f + W->off[l + 1], *u1 = W->u + W->off[l + 1];
            for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; s1[I] = rowdot(&H->R[l], I, w); }
            for (int q = 0; q < b->nghost; ++q) { int I = b->ghost[q]; s1[I] = rowdot(&H->R[l], I, w); }
            /* f_{l+1} <- f_{l+1} - A_{l+1} u_{l+1} (not needed while u_{l+1} = 0) */
            if (c > 1)
                for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; f1[I] = f1[I] - rowdot(&H->A[l + 1], I, u1); }
            /* f_{l+1} <- f_{l+1} - s_{l+1} */
            for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; f1[I] = f1[I] - s1[I]; }
            /* t_l <- 0, s_l <- 0; w_l is scratch and is cleared with them */
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; t[i] = 0.0; s[i] = 0.0; w[i] = 0.0; }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; t[i] = 0.0; s[i] = 0.0; w[i] = 0.0; }
        }
        coarse_solve(H, W->f + W->off[L], W->u + W->off[L]);
        for (int l = L - 1; l >= 0; --l) {
            const Mat *A = &H->A[l];
            double *u = W->u + W->off[l], *f = W->f + W->off[l], *t = W->t + W->off[l], *d = W->d + W->off[l];
            const double *u1 = W->u + W->off[l + 1];
            const CLevel *a = &cl[l];
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; u[i] = u[i] + rowdot(&H->P[l], i, u1); }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; u[i] = u[i] + rowdot(&H->P[l], i, u1); }
            relax_pass(A, H->l1inv[l], H->cf[l], 0, a->real, a->nreal, f, u, t, d);
            relax_pass(A, H->l1inv[l], H->cf[l], 1, a->real, a->nreal, f, u, t, d);
        }
    }
}

static void facwork_clear(const Hier *H, const Comp *C, int p, FacWork *W)
{
    const CLevel *cl = &C->lv[(size_t)p * C->nlev];
    for (int l = 0; l < H->nlev; ++l) {
        int64_t o = W->off[l];
        for (int pass = 0; pass < 2; ++pass) {
            const int *set = pass ? cl[l].ghost : cl[l].real;
            int ns = pass ? cl[l].nghost : cl[l].nreal;
            for (int q = 0; q < ns; ++q) {
                int64_t i = o + set[q];
                W->u[i] = 0.0; W->f[i] = 0.0; W->t[i] = 0.0; W->s[i] = 0.0; W->w[i] = 0.0; W->d[i] = 0.0;
            }
        }
    }
}

/* AlgFAC on one composite grid; u_out and f_out are levels back to back,
 * indexed globally, zero outside the grid. */
void orc_algfac(void *h, void *c, int p, const double *rl, int nfac, double *u_out, double *f_out)
{
    Hier *H = h;
    FacWork W;
    facwork_init(H, &W);
    algfac(H, c, p, rl, nfac, &W);
    int64_t tot = W.off[H->nlev];
    memcpy(u_out, W.u, sizeof(double) * (size_t)tot);
    memcpy(f_out, W.f, sizeof(double) * (size_t)tot);
    facwork_free(&W);
}

/* The global cycle that AlgFAC must reproduce (Section 4): nfac V(1,1)-cycles
 * on the whole hierarchy for A_0 e = r_0 from e = 0, with relaxation only at
 * the real points D_l of subdomain p and the usual restriction
 * f_{l+1} = R_l (f_l - A_l u_l). u_out, f_out: levels back to back. */
void orc_masked_fac(void *h, void *c, int p, const double *r0, int nfac, double *u_out, double *f_out)
{
    Hier *H = h;
    Comp *C = c;
    int L = H->nlev - 1;
    const CLevel *cl = &C->lv[(size_t)p * C->nlev];
    int64_t off[ORC_MAXLEV + 1];
    off[0] = 0;
    for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + H->A[l].n;
    memset(u_out, 0, sizeof(double) * (size_t)off[L + 1]);
    memset(f_out, 0, sizeof(double) * (size_t)off[L + 1]);
    memcpy(f_out, r0, sizeof(double) * (size_t)H->A[0].n);
    double *d = xcalloc((size_t)H->A[0].n, sizeof(double));
    double *res = xcalloc((size_t)H->A[0].n, sizeof(double));
    for (int cyc = 1; cyc <= nfac; ++cyc) {
        for (int l = 0; l < L; ++l) {
            const Mat *A = &H->A[l];
            double *u = u_out + off[l], *f = f_out + off[l];
            relax_pass(A, H->l1inv[l], H->cf[l], 1, cl[l].real, cl[l].nreal, f, u, NULL, d);
            relax_pass(A, H->l1inv[l], H->cf[l], 0, cl[l].real, cl[l].nreal, f, u, NULL, d);
            for (int i = 0; i < A->n; ++i) res[i] = f[i] - rowdot(A, i, u);
            double *f1 = f_out + off[l + 1], *u1 = u_out + off[l + 1];
            for (int I = 0; I < H->R[l].n; ++I) f1[I] = rowdot(&H->R[l], I, res);
            for (int I = 0; I < H->A[l + 1].n; ++I) u1[I] = 0.0;
        }
        coarse_solve(H, f_out + off[L], u_out + off[L]);
        for (int l = L - 1; l >= 0; --l) {
            const Mat *A = &H->A[l];
            double *u = u_out + off[l], *f = f_out + off[l];
            const double *u1 = u_out + off[l + 1];
            for (int i = 0; i < A->n; ++i) u[i] = u[i] + rowdot(&H->P[l], i, u1);
            relax_pass(A, H->l1inv[l], H->cf[l], 0, cl[l].real, cl[l].nreal, f, u, NULL, d);
            relax_pass(A, H->l1inv[l], H->cf[l], 1, cl[l].real, cl[l].nreal, f, u, NULL, d);
        }
    }
    free(d);
    free(res);
}

/* One AMG-DD iteration (Algorithm 2) restricted to a list of subdomains
 * (all subdomains when nsel < 0): r_0 = b - A x, r_{l+1} = R_l r_l, AlgFAC on
 * each composite grid, x += u_0 on the owned points. rl: scratch of
 * orc_levels_total doubles. */
void orc_amgdd_iteration(void *h, void *c, const double *b, double *x, int nfac, const int *sel,
                         int nsel, double *rl)
{
    Hier *H = h;
    Comp *C = c;
    orc_residual(h, b, x, rl);
    orc_restrict_all(h, rl);
    int np = nsel < 0 ? C->nsub : nsel;
#pragma omp parallel
    {
        FacWork W;
        facwork_init(H, &W);
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < np; ++q) {
            int p = nsel < 0 ? q : sel[q];
            algfac(H, C, p, rl, nfac, &W);
            const CLevel *c0 = &C->lv[(size_t)p * C->nlev];
            for (int s = 0; s < c0->nowned; ++s) {
                int i = c0->owned[s];
                x[i] = x[i] + W.u[i];
            }
            facwork_clear(H, C, p, &W);
        }
        facwork_free(&W);
    }
}

/* ------------------------------------------------------------------ */
/* Mixed precision: AlgFAC in FP32 inside FP64 iterative refinement     */
/* ------------------------------------------------------------------ */
/* The composite-grid cycle of Algorithm 4 with every composite vector and
 * every operator value rounded to float (round to nearest), fmaf chains over
 * ascending columns, and the coarsest solve in FP64 on the float right-hand
 * side (result rounded to float). The global residual, the restriction, the
 * gather f_l = (float) r_l and the update x += (double) u_0 stay FP64, so the
 * outer iteration of Algorithm 2 is an iterative refinement whose correction
 * comes from the FP32 cycles. */

static inline float rowdot32(const Mat *A, int i, const float *x)
{
    float s = 0.0f;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
        s = fmaf((float)A->v[k], x[A->ci[k]], s);
    return s;
}

typedef struct {
    int64_t off[ORC_MAXLEV + 1];
    float *u, *f, *t, *s, *w, *d;
} FacWork32;

static void facwork32_init(const Hier *H, FacWork32 *W)
{
    W->off[0] = 0;
    for (int l = 0; l < H->nlev; ++l) W->off[l + 1] = W->off[l] + H->A[l].n;
    size_t tot = (size_t)W->off[H->nlev];
    W->u = xcalloc(tot, sizeof(float));
    W->f = xcalloc(tot, sizeof(float));
    W->t = xcalloc(tot, sizeof(float));
    W->s = xcalloc(tot, sizeof(float));
    W->w = xcalloc(tot, sizeof(float));
    W->d = xcalloc(tot, sizeof(float));
}

static void facwork32_free(FacWork32 *W) { free(W->u); free(W->f); free(W->t); free(W->s); free(W->w); free(W->d); }

static void relax_pass32(const Mat *A, const double *l1inv, const int *cf, int which, const int *pts, int npts,
                         const float *f, float *u, float *t, float *d)
{
    for (int q = 0; q < npts; ++q) {
        int i = pts[q];
        if (cf[i] != which) continue;
        d[i] = (f[i] - rowdot32(A, i, u)) * (float)l1inv[i];
    }
    for (int q = 0; q < npts; ++q) {
        int i = pts[q];
        if (cf[i] != which) continue;
        u[i] = u[i] + d[i];
        t[i] = t[i] + d[i];
    }
}

static void algfac32(const Hier *H, const Comp *C, int p, const double *rl, int nfac, FacWork32 *W)
{
    int L = H->nlev - 1;
    int nL = H->A[L].n;
    const CLevel *cl = &C->lv[(size_t)p * C->nlev];
    for (int l = 0; l <= L; ++l) {
        float *f = W->f + W->off[l];
        const double *r = rl + W->off[l];
        for (int q = 0; q < cl[l].nreal; ++q) f[cl[l].real[q]] = (float)r[cl[l].real[q]];
    }
    for (int c = 1; c <= nfac; ++c) {
        for (int l = 0; l < L; ++l) {
            const Mat *A = &H->A[l];
            float *u = W->u + W->off[l], *f = W->f + W->off[l], *t = W->t + W->off[l];
            float *s = W->s + W->off[l], *w = W->w + W->off[l], *d = W->d + W->off[l];
            const CLevel *a = &cl[l], *b = &cl[l + 1];
            if (l != 0) {
                for (int q = 0; q < a->nreal; ++q) u[a->real[q]] = 0.0f;
                for (int q = 0; q < a->nghost; ++q) u[a->ghost[q]] = 0.0f;
            }
            relax_pass32(A, H->l1inv[l], H->cf[l], 1, a->real, a->nreal, f, u, t, d);
            relax_pass32(A, H->l1inv[l], H->cf[l], 0, a->real, a->nreal, f, u, t, d);
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; w[i] = s[i] + rowdot32(A, i, t); }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; w[i] = s[i] + rowdot32(A, i, t); }
            float *s1 = W->s + W->off[l + 1], *f1 = W->f + W->off[l + 1], *u1 = W->u + W->off[l + 1];
            for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; s1[I] = rowdot32(&H->R[l], I, w); }
            for (int q = 0; q < b->nghost; ++q) { int I = b->ghost[q]; s1[I] = rowdot32(&H->R[l], I, w); }
            if (c > 1)
                for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; f1[I] = f1[I] - rowdot32(&H->A[l + 1], I, u1); }
            for (int q = 0; q < b->nreal; ++q) { int I = b->real[q]; f1[I] = f1[I] - s1[I]; }
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; t[i] = 0.0f; s[i] = 0.0f; w[i] = 0.0f; }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; t[i] = 0.0f; s[i] = 0.0f; w[i] = 0.0f; }
        }
        {
            const float *f = W->f + W->off[L];
            float *u = W->u + W->off[L];
            for (int I = 0; I < nL; ++I) {
                double acc = 0.0;
                for (int J = 0; J < nL; ++J) acc = fma(H->ainv[(size_t)I * nL + J], (double)f[J], acc);
                u[I] = (float)acc;
            }
        }
        for (int l = L - 1; l >= 0; --l) {
            const Mat *A = &H->A[l];
            float *u = W->u + W->off[l], *f = W->f + W->off[l], *t = W->t + W->off[l], *d = W->d + W->off[l];
            const float *u1 = W->u + W->off[l + 1];
            const CLevel *a = &cl[l];
            for (int q = 0; q < a->nreal; ++q) { int i = a->real[q]; u[i] = u[i] + rowdot32(&H->P[l], i, u1); }
            for (int q = 0; q < a->nghost; ++q) { int i = a->ghost[q]; u[i] = u[i] + rowdot32(&H->P[l], i, u1); }
            relax_pass32(A, H->l1inv[l], H->cf[l], 0, a->real, a->nreal, f, u, t, d);
            relax_pass32(A, H->l1inv[l], H->cf[l], 1, a->real, a->nreal, f, u, t, d);
        }
    }
}

static void facwork32_clear(const Hier *H, const Comp *C, int p, FacWork32 *W)
{
    const CLevel *cl = &C->lv[(size_t)p * C->nlev];
    for (int l = 0; l < H->nlev; ++l) {
        int64_t o = W->off[l];
        for (int pass = 0; pass < 2; ++pass) {
            const int *set = pass ? cl[l].ghost : cl[l].real;
            int ns = pass ? cl[l].nghost : cl[l].nreal;
            for (int q = 0; q < ns; ++q) {
                int64_t i = o + set[q];
                W->u[i] = 0.0f; W->f[i] = 0.0f; W->t[i] = 0.0f; W->s[i] = 0.0f; W->w[i] = 0.0f; W->d[i] = 0.0f;
            }
        }
    }
}

/* FP32 AlgFAC on one composite grid; outputs widened to double, levels back
 * to back, global indexing, zero outside the grid. */
void orc_algfac32(void *h, void *c, int p, const double *rl, int nfac, double *u_out, double *f_out)
{
    Hier *H = h;
    FacWork32 W;
    facwork32_init(H, &W);
    algfac32(H, c, p, rl, nfac, &W);
    int64_t tot = W.off[H->nlev];
    for (int64_t i = 0; i < tot; ++i) { u_out[i] = W.u[i]; f_out[i] = W.f[i]; }
    facwork32_free(&W);
}

/* One mixed-precision AMG-DD iteration (Algorithm 2 with FP32 AlgFAC). */
void orc_amgdd_iteration32(void *h, void *c, const double *b, double *x, int nfac, double *rl)
{
    Hier *H = h;
    Comp *C = c;
    orc_residual(h, b, x, rl);
    orc_restrict_all(h, rl);
#pragma omp parallel
    {
        FacWork32 W;
        facwork32_init(H, &W);
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < C->nsub; ++p) {
            algfac32(H, C, p, rl, nfac, &W);
            const CLevel *c0 = &C->lv[(size_t)p * C->nlev];
            for (int q = 0; q < c0->nowned; ++q) {
                int i = c0->owned[q];
                x[i] = x[i] + (double)W.u[i];
            }
            facwork32_clear(H, C, p, &W);
        }
        facwork32_free(&W);
    }
}

/* ------------------------------------------------------------------ */
/* Hybrid AMG-DD (Algorithm 3)                                          */
/* ------------------------------------------------------------------ */

/* The hierarchy from level lev0 down, sharing the operators of h (a view:
 * orc_hier_sub_free releases only the view). */
void *orc_hier_sub(void *h, int lev0)
{
    Hier *H = h;
    Hier *S = xcalloc(1, sizeof(Hier));
    S->nlev = H->nlev - lev0;
    for (int l = 0; l < S->nlev; ++l) {
        S->A[l] = H->A[lev0 + l];
        S->P[l] = H->P[lev0 + l];
        S->R[l] = H->R[lev0 + l];
        S->cf[l] = H->cf[lev0 + l];
        S->cmap[l] = H->cmap[lev0 + l];
        S->l1inv[l] = H->l1inv[lev0 + l];
    }
    S->ainv = H->ainv;
    return S;
}

void orc_hier_sub_free(void *s) { free(s); }

/* Subdomain of every point of level lev0: each C point carries the subdomain
 * of the fine point it comes from. part_out: n_lev0 entries. */
void orc_part_on_level(void *h, const int *part, int lev0, int *part_out)
{
    Hier *H = h;
    int n = H->A[0].n;
    int *cur = xmalloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    memcpy(cur, part, sizeof(int) * (size_t)n);
    for (int l = 0; l < lev0; ++l) {
        int nc = H->A[l + 1].n;
        int *nx = xmalloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
        for (int i = 0; i < H->A[l].n; ++i)
            if (H->cf[l][i]) nx[H->cmap[l][i]] = cur[i];
        free(cur);
        cur = nx;
    }
    memcpy(part_out, cur, sizeof(int) * (size_t)H->A[lev0].n);
    free(cur);
}

/* One hybrid V(1,1)-cycle (Algorithm 3) in place on (u_0, f_0): V-cycle
 * relaxation / restriction on levels 0 .. lev0-1, then one AMG-DD cycle on
 * level lev0 in place of the coarse solve (r = f - A u on that level, its
 * restrictions through the sub-hierarchy, AlgFAC on every composite grid of
 * the sub-hierarchy, owned corrections added into u_lev0), then the upsweep.
 * hs: the sub-hierarchy view from lev0; cs: its composite grids. */
void orc_hybrid_apply(void *h, void *hs, void *cs, int lev0, int nfac, const double *f0, double *u0)
{
    Hier *H = h;
    Hier *HS = hs;
    Comp *CS = cs;
    int L = H->nlev - 1;
    int64_t off[ORC_MAXLEV + 1];
    off[0] = 0;
    for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + H->A[l].n;
    double *U = xcalloc((size_t)off[L + 1], sizeof(double));
    double *F = xcalloc((size_t)off[L + 1], sizeof(double));
    double *W = xcalloc((size_t)H->A[0].n, sizeof(double));
    double *u[ORC_MAXLEV], *f[ORC_MAXLEV];
    u[0] = u0;
    f[0] = (double *)f0;
    for (int l = 1; l <= L; ++l) { u[l] = U + off[l]; f[l] = F + off[l]; }
    for (int l = 0; l < lev0; ++l) {
        const Mat *A = &H->A[l];
        relax_pass(A, H->l1inv[l], H->cf[l], 1, NULL, A->n, f[l], u[l], NULL, W);
        relax_pass(A, H->l1inv[l], H->cf[l], 0, NULL, A->n, f[l], u[l], NULL, W);
        for (int i = 0; i < A->n; ++i) W[i] = f[l][i] - rowdot(A, i, u[l]);
        for (int I = 0; I < H->R[l].n; ++I) f[l + 1][I] = rowdot(&H->R[l], I, W);
        for (int I = 0; I < H->A[l + 1].n; ++I) u[l + 1][I] = 0.0;
    }
    /* AMG-DD cycle on level lev0 (Algorithm 2 on A_lev0 u = f_lev0) */
    {
        int64_t tot = 0;
        for (int l = 0; l < HS->nlev; ++l) tot += HS->A[l].n;
        double *rl = xcalloc((size_t)tot, sizeof(double));
        const Mat *A = &HS->A[0];
        for (int i = 0; i < A->n; ++i) rl[i] = f[lev0][i] - rowdot(A, i, u[lev0]);
        orc_restrict_all(HS, rl);
        FacWork FW;
        facwork_init(HS, &FW);
        for (int p = 0; p < CS->nsub; ++p) {
            algfac(HS, CS, p, rl, nfac, &FW);
            const CLevel *c0 = &CS->lv[(size_t)p * CS->nlev];
            for (int q = 0; q < c0->nowned; ++q) {
                int i = c0->owned[q];
                u[lev0][i] = u[lev0][i] + FW.u[i];
            }
            facwork_clear(HS, CS, p, &FW);
        }
        facwork_free(&FW);
        free(rl);
    }
    for (int l = lev0 - 1; l >= 0; --l) {
        const Mat *A = &H->A[l];
        for (int i = 0; i < A->n; ++i) u[l][i] = u[l][i] + rowdot(&H->P[l], i, u[l + 1]);
        relax_pass(A, H->l1inv[l], H->cf[l], 0, NULL, A->n, f[l], u[l], NULL, W);
        relax_pass(A, H->l1inv[l], H->cf[l], 1, NULL, A->n, f[l], u[l], NULL, W);
    }
    free(U); free(F); free(W);
}

int orc_hybrid_solve(void *h, void *hs, void *cs, int lev0, int nfac, const double *b, double *x, double tol,
                     int maxit, double *hist)
{
    Hier *H = h;
    int n = H->A[0].n;
    double *r = xcalloc((size_t)n, sizeof(double));
    double ref = norm2(b, n);
    int k = 0;
    for (;;) {
        orc_residual(h, b, x, r);
        double nr = norm2(r, n);
        if (k == 0 && ref == 0.0) ref = nr;
        double rel = ref > 0.0 ? nr / ref : 0.0;
        hist[k] = rel;
        if (rel <= tol || k >= maxit) break;
        orc_hybrid_apply(h, hs, cs, lev0, nfac, b, x);
        ++k;
    }
    free(r);
    return k;
}

/* AMG-DD solver: iterations of Algorithm 2 until ||b - A x|| / ||b|| <= tol. */
int orc_amgdd_solve(void *h, void *c, const double *b, double *x, double tol, int maxit, int nfac, int mixed,
                    double *hist)
{
    Hier *H = h;
    int n = H->A[0].n;
    double *rl = xcalloc((size_t)orc_levels_total(h), sizeof(double));
    double *r = xcalloc((size_t)n, sizeof(double));
    double ref = norm2(b, n);
    int k = 0;
    for (;;) {
        orc_residual(h, b, x, r);
        double nr = norm2(r, n);
        if (k == 0 && ref == 0.0) ref = nr;
        double rel = ref > 0.0 ? nr / ref : 0.0;
        hist[k] = rel;
        if (rel <= tol || k >= maxit) break;
        if (mixed) orc_amgdd_iteration32(h, c, b, x, nfac, rl);
        else orc_amgdd_iteration(h, c, b, x, nfac, NULL, -1, rl);
        ++k;
    }
    free(rl);
    free(r);
    return k;
}

/* Threads of the OpenMP loops over subdomains (timing of the CPU baseline at
 * one thread and at all cores); returns the count now in effect. */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
