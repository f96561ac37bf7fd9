// C ABI of the AMG-DD solve-phase library (declared in include/amgdd.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/amgdd.h"
#include "amgdd_internal.hpp"

using namespace amgdd;

namespace {

thread_local std::string g_last_error;

struct DevLevel {             // device copy of one global level
    SellView A{}, P{}, R{};
    int64_t n = 0;
    int64_t nC = 0;
    const double *l1inv = nullptr;
    double *u = nullptr, *f = nullptr, *d = nullptr;   // V-cycle vectors (level >= 1: u, f)
};

}  // namespace

namespace amgdd {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace amgdd

struct amgdd_handle_s {
    std::string err;
    amgdd_options opt{};
    Hierarchy H;
    Composite C;
    std::vector<FacLevelDesc> desc;     // host copy of the FAC descriptors
    std::vector<int32_t> dev2map;       // device order -> map order, per row
    std::vector<int64_t> level_off;     // offsets of the levels in r_all
    amgdd_setup_stats stats{};
    bool on_device = false;
    // device memory
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    std::vector<DevLevel> lev;
    const double *ainv = nullptr;
    const int32_t *ainv_ptr = nullptr, *ainv_col = nullptr;   // its nonzeros, by row
    const double *ainv_val = nullptr;
    int nL = 0;
    FacParams fac{};
    double *r_all = nullptr;            // sum_l n_l
    double *res = nullptr;              // n_0 scratch
    double *partial = nullptr;          // reduction partials
    double *scal = nullptr;             // device scalars
    double *h_scal = nullptr;           // pinned host scalars
    int nred = 0;                       // reduction blocks
    int threads = 512;
    int64_t launches = 0;
    cudaStream_t last_stream = nullptr;
    // one solver iteration captured as a CUDA graph, per method, keyed by the
    // vectors it was captured with
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        const double *b = nullptr;
        double *x = nullptr;
        int64_t launches = 0;
    };
    cudaStream_t cap_stream = nullptr;
    // a whole solve per method as one graph (iterations in a while node),
    // keyed by its vectors, tolerance and iteration limit
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        const double *b = nullptr;
        double *x = nullptr;
        double tol = 0.0;
        int32_t max_iter = -1;
        int64_t pre_launches = 0, body_launches = 0;
    } solve_graph[3];
    cudaStream_t cap_stream2 = nullptr;     // captures the while node's body
    ConvState *conv = nullptr, *h_conv = nullptr;   // device / pinned
    double *hist = nullptr, *h_hist = nullptr;      // device / pinned, hist_cap doubles
    int64_t hist_cap = 0;
    // work space of the several-right-hand-side path, per width (2 or 4)
    struct Multi {
        int R = 0;
        void *ws[6] = {};
        double *r_all = nullptr, *partial = nullptr, *scal = nullptr, *h_scal = nullptr;
        Graph graph;
    } multi[2];
    int64_t fac_rows = 0;
    FacParams fac_base{};
    // hybrid AMG-DD (Algorithm 3): composite grids of the hierarchy from level
    // hyb_level down, the residual of that level and its restrictions
    // FAC kernel candidate per column count (index 0: 1 column, 1: 2, 2: 4),
    // numbered as in amgdd_autotune; and the lanes per row of each level that
    // the group-per-row candidate uses (chosen from the level sizes at setup)
    int fac_cand[3] = {15, 15, 15};
    int8_t grp_level[kMaxLevels + 1] = {};
    const int32_t *one_bin_off = nullptr;   // {0, nsub}: every grid in one bin (global queue)
    int hyb_level = -1;
    FacParams fac_hyb{};
    double *r_hyb = nullptr;
    std::vector<int64_t> hyb_off;
};

namespace {

amgdd_status fail(amgdd_handle h, amgdd_status st, const std::string &msg)
{
    if (h) h->err = msg;
    g_last_error = msg;
    return st;
}

amgdd_status cuda_fail(amgdd_handle h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? AMGDD_ERR_OOM : AMGDD_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr, what)                                                  \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) return cuda_fail(h, _e, what);           \
    } while (0)

// Allocation fault injection (for tests of the failure paths): while
// amgdd_setup runs with AMGDD_FAULT_ALLOC=k (k >= 1) in the environment, its
// k-th device or pinned host allocation fails as if memory were exhausted,
// without allocating. Counted per calling thread; off outside amgdd_setup.
thread_local int64_t t_fault_at = 0;
thread_local int64_t t_alloc_seq = 0;

bool inject_alloc_fault()
{
    return t_fault_at > 0 && ++t_alloc_seq == t_fault_at;
}

cudaError_t dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes);
}

// Arms the injection for one amgdd_setup call and disarms it on every return.
struct FaultScope {
    FaultScope()
    {
        const char *v = std::getenv("AMGDD_FAULT_ALLOC");
        t_fault_at = v ? std::atoll(v) : 0;
        t_alloc_seq = 0;
    }
    ~FaultScope() { t_fault_at = 0; }
};

template <class T>
cudaError_t upload(amgdd_handle h, const std::vector<T> &v, T **out, cudaStream_t st)
{
    *out = nullptr;
    const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, bytes);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(p);
    h->dev_bytes += (int64_t)bytes;
    if (!v.empty()) {
        e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    *out = static_cast<T *>(p);
    return cudaSuccess;
}

template <class T>
cudaError_t alloc(amgdd_handle h, size_t count, T **out)
{
    *out = nullptr;
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = dev_malloc(&p, bytes);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(p);
    h->dev_bytes += (int64_t)bytes;
    *out = static_cast<T *>(p);
    return cudaSuccess;
}

cudaError_t upload_sell(amgdd_handle h, Sell &S, const std::vector<int32_t> *rowid, SellView &v, cudaStream_t st)
{
    int64_t *soff;
    uint16_t *rlen;
    int32_t *col, *rid = nullptr;
    double *val;
    cudaError_t e;
    if ((e = upload(h, S.soff, &soff, st)) != cudaSuccess) return e;
    if ((e = upload(h, S.rlen, &rlen, st)) != cudaSuccess) return e;
    if ((e = upload(h, S.col, &col, st)) != cudaSuccess) return e;
    if ((e = upload(h, S.val, &val, st)) != cudaSuccess) return e;
    if (rowid && (e = upload(h, *rowid, &rid, st)) != cudaSuccess) return e;
    v.rows = S.rows;
    v.soff = soff;
    v.rlen = rlen;
    v.col = col;
    v.val = val;
    v.rowid = rid;
    return cudaSuccess;
}

std::string validate(const amgdd_csr *A, const int32_t *part, int32_t nsub, const int32_t *padding,
                     int32_t npadding, amgdd_status &st)
{
    st = AMGDD_ERR_INVALID_ARG;
    if (!A || !A->rowptr || !A->col || !A->val) return "null matrix pointer";
    if (A->n <= 0) return "matrix has no rows";
    if (!part) return "null partition";
    if (nsub <= 0) return "nsub must be positive";
    if (!padding || npadding < 1) return "padding needs at least one entry";
    for (int i = 0; i < npadding; ++i)
        if (padding[i] < 0) return "padding must be >= 0";
    const int32_t n = A->n;
    if (A->rowptr[0] != 0 || (int64_t)A->rowptr[n] != A->nnz) return "rowptr[0] must be 0 and rowptr[n] = nnz";
    for (int32_t i = 0; i < n; ++i) {
        if (A->rowptr[i + 1] < A->rowptr[i]) return "rowptr is not non-decreasing";
        bool diag = false;
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
            const int32_t j = A->col[k];
            if (j < 0 || j >= n) return "column index out of range in row " + std::to_string(i);
            if (k > A->rowptr[i] && A->col[k - 1] >= j) return "columns not strictly ascending in row " + std::to_string(i);
            if (!std::isfinite(A->val[k])) return "non-finite value in row " + std::to_string(i);
            if (j == i) {
                diag = true;
                if (!(A->val[k] > 0.0)) return "non-positive diagonal in row " + std::to_string(i);
            }
        }
        if (!diag) return "missing diagonal in row " + std::to_string(i);
    }
    std::vector<int64_t> cnt((size_t)nsub, 0);
    for (int32_t i = 0; i < n; ++i) {
        if (part[i] < 0 || part[i] >= nsub) return "part[" + std::to_string(i) + "] out of range";
        cnt[part[i]]++;
    }
    for (int32_t p = 0; p < nsub; ++p)
        if (cnt[p] == 0) return "subdomain " + std::to_string(p) + " owns no unknowns";
    // symmetry: every (i, j) has a matching (j, i) of nearly equal value
    st = AMGDD_ERR_NOT_SYMMETRIC;
    std::vector<int32_t> pos(A->rowptr, A->rowptr + n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
            const int32_t j = A->col[k];
            if (j < i) continue;
            // find (j, i) by scanning row j from its cursor
            int32_t q = pos[j];
            while (q < A->rowptr[j + 1] && A->col[q] < i) ++q;
            if (q >= A->rowptr[j + 1] || A->col[q] != i)
                return "entry (" + std::to_string(i) + "," + std::to_string(j) + ") has no transpose";
            const double a = A->val[k], b = A->val[q];
            if (std::fabs(a - b) > 1e-12 * std::max(std::fabs(a), std::fabs(b)))
                return "values (" + std::to_string(i) + "," + std::to_string(j) + ") not symmetric";
        }
    st = AMGDD_OK;
    return "";
}

int host_threads()
{
    unsigned t = std::thread::hardware_concurrency();
    return t == 0 ? 4 : (int)std::min(t, 64u);
}

amgdd_status require_device(amgdd_handle h)
{
    if (!h) return fail(nullptr, AMGDD_ERR_INVALID_ARG, "null handle");
    if (!h->on_device) return fail(h, AMGDD_ERR_NOT_ON_DEVICE, "handle was set up with host_only");
    return AMGDD_OK;
}

// A device array appended to from the host; its capacity doubles, the old
// contents moving by a device-to-device copy.
struct DevGrow {
    char *d = nullptr;
    size_t n = 0, cap = 0;
};

// The large arrays of a composite-grid layout (five views, the map to level
// indices and the l1 weights), filled on the device chunk by chunk while the
// layout is packed: each chunk is range-checked, appended and dropped on the
// host, so the host holds one chunk of the layout at a time.
struct FacStream {
    DevGrow soff[5], rlen[5], col[5], val[5], gmap, l1inv;
    bool fp32 = false;
    bool host = false;              // check and drop only (no device)
    cudaError_t err = cudaSuccess;
    const char *what = "";
    std::vector<float> l1f;

    DevGrow *all(int k)
    {
        if (k < 5) return &soff[k];
        if (k < 10) return &rlen[k - 5];
        if (k < 15) return &col[k - 10];
        if (k < 20) return &val[k - 15];
        return k == 20 ? &gmap : &l1inv;
    }
    ~FacStream()
    {
        for (int k = 0; k < 22; ++k)
            if (all(k)->d) cudaFree(all(k)->d);
    }
    cudaError_t append(DevGrow &g, const void *src, size_t bytes, cudaStream_t st)
    {
        cudaError_t e;
        if (g.n + bytes > g.cap) {
            const size_t nc = std::max({g.cap * 2, g.n + bytes, (size_t)1 << 20});
            void *p = nullptr;
            if ((e = dev_malloc(&p, nc)) != cudaSuccess) return e;
            if (g.n && (e = cudaMemcpyAsync(p, g.d, g.n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) {
                cudaFree(p);
                return e;
            }
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
                cudaFree(p);
                return e;
            }
            if (g.d) cudaFree(g.d);
            g.d = static_cast<char *>(p);
            g.cap = nc;
        }
        if (bytes && (e = cudaMemcpyAsync(g.d + g.n, src, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
        g.n += bytes;
        return cudaSuccess;
    }
    template <class T>
    cudaError_t app(DevGrow &g, const std::vector<T> &v, cudaStream_t st)
    {
        return append(g, v.data(), v.size() * sizeof(T), st);
    }
    // Sink body: check grids [p0, p0 + pn), append what F holds, drop it.
    std::string consume(const Hierarchy &H, FacLayout &F, int p0, int pn, cudaStream_t st)
    {
        std::string bad = validate_fac_grids(H, F, p0, pn);
        if (!bad.empty()) return bad;
        FacView *views[5] = {&F.A, &F.At, &F.AFc, &F.P, &F.R};
        cudaError_t e = cudaSuccess;
        for (int v = 0; v < 5 && e == cudaSuccess && !host; ++v) {
            FacView &V = *views[v];
            what = "upload view slices";
            if ((e = app(soff[v], V.soff, st)) != cudaSuccess) break;
            what = "upload view rows";
            if ((e = app(rlen[v], V.rlen, st)) != cudaSuccess) break;
            what = "upload view columns";
            if ((e = V.c16 ? app(col[v], V.col16, st) : app(col[v], V.col32, st)) != cudaSuccess) break;
            what = "upload view values";
            if ((e = V.v32 ? app(val[v], V.val32, st) : app(val[v], V.val64, st)) != cudaSuccess) break;
        }
        if (e == cudaSuccess && !host) {
            what = "upload gmap";
            e = app(gmap, F.gmap, st);
        }
        if (e == cudaSuccess && !host) {
            what = "upload l1inv";
            if (fp32) {
                l1f.assign(F.l1inv.begin(), F.l1inv.end());
                e = app(l1inv, l1f, st);
            } else {
                e = app(l1inv, F.l1inv, st);
            }
        }
        // the host vectors are reused by the next chunk
        if (e == cudaSuccess && !host) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            err = e;
            return std::string(what) + ": " + cudaGetErrorString(e);
        }
        for (FacView *V : views) V->flush();
        F.row_base += (int64_t)F.gmap.size();
        F.gmap.clear();
        F.l1inv.clear();
        return "";
    }
};

// Moves a grown array into an exact-size allocation owned by the handle.
cudaError_t settle(amgdd_handle h, DevGrow &g, cudaStream_t st, void **out)
{
    *out = nullptr;
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(g.n, 16);
    cudaError_t e = dev_malloc(&p, bytes);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(p);
    h->dev_bytes += (int64_t)bytes;
    if (g.n && (e = cudaMemcpyAsync(p, g.d, g.n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    cudaFree(g.d);
    g = DevGrow();
    *out = p;
    return cudaSuccess;
}

}  // namespace

// Team plan of the team-partitioned FAC kernel over nblocks blocks of 32
// warps (at most 15 teams per block). Up to two grids per block on average:
// one grid per team, its warps in proportion to its work. The smallest
// per-warp work T for which every grid's ceil(work / T) warps (2 to 32)
// pack into the blocks, first fit by decreasing need, is found by bisection;
// each block's warps left over then go one at a time to its team with the
// most work per warp. More grids: two teams of 16 warps per block, each grid
// (largest first) to the team with the least work so far.
struct TeamPlan {
    std::vector<int32_t> block_off, w0, nw, grid_off, grid;
};

static TeamPlan plan_teams(const std::vector<int64_t> &work_in, int nblocks)
{
    const int nsub = (int)work_in.size();
    std::vector<double> w((size_t)nsub);
    for (int g = 0; g < nsub; ++g) w[g] = (double)std::max<int64_t>(work_in[g], 1);
    std::vector<int32_t> ord((size_t)nsub);
    for (int g = 0; g < nsub; ++g) ord[g] = g;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return w[a] > w[b]; });
    // per block: its teams as (grids, warps)
    std::vector<std::vector<std::pair<std::vector<int32_t>, int>>> blk((size_t)nblocks);
    if (nsub <= 2 * nblocks) {
        auto pack = [&](double T, bool keep) {
            std::vector<int> used((size_t)nblocks, 0), cnt((size_t)nblocks, 0);
            if (keep)
                for (auto &b : blk) b.clear();
            for (int32_t g : ord) {   // decreasing work = decreasing need
                const int need = (int)std::min(32.0, std::max(2.0, std::ceil(w[g] / T)));
                int b = 0;
                while (b < nblocks && (used[b] + need > 32 || cnt[b] >= 15)) ++b;
                if (b == nblocks) return false;
                used[b] += need;
                ++cnt[b];
                if (keep) blk[b].push_back({{g}, need});
            }
            return true;
        };
        double W = 0.0;
        for (double x : w) W += x;
        double lo = W / (32.0 * nblocks), hi = std::max(w[ord[0]], lo) * 2.0;
        while (!pack(hi, false)) hi *= 2.0;
        for (int it = 0; it < 60; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (pack(mid, false)) hi = mid;
            else lo = mid;
        }
        pack(hi, true);
        for (auto &b : blk) {
            int used = 0;
            for (auto &t : b) used += t.second;
            while (used < 32 && !b.empty()) {
                size_t best = 0;
                for (size_t k = 1; k < b.size(); ++k)
                    if (w[b[k].first[0]] / b[k].second > w[b[best].first[0]] / b[best].second) best = k;
                ++b[best].second;
                ++used;
            }
        }
    } else {
        std::vector<double> load((size_t)2 * nblocks, 0.0);
        for (int b = 0; b < nblocks; ++b) {
            blk[b].push_back({{}, 16});
            blk[b].push_back({{}, 16});
        }
        for (int32_t g : ord) {
            size_t best = 0;
            for (size_t k = 1; k < load.size(); ++k)
                if (load[k] < load[best]) best = k;
            blk[best / 2][best % 2].first.push_back(g);
            load[best] += w[g];
        }
    }
    TeamPlan T;
    T.block_off.push_back(0);
    T.grid_off.push_back(0);
    for (auto &b : blk) {
        int w0 = 0;
        for (auto &t : b) {
            T.w0.push_back(w0);
            T.nw.push_back(t.second);
            w0 += t.second;
            T.grid.insert(T.grid.end(), t.first.begin(), t.first.end());
            T.grid_off.push_back((int32_t)T.grid.size());
        }
        T.block_off.push_back((int32_t)T.w0.size());
    }
    return T;
}

// Fills the FAC kernel parameters of one composite-grid layout (all grids,
// all levels of its hierarchy): the views, map and l1 weights already streamed
// to the device by S, the small per-grid tables, the per-SM bins and the
// work space.
static cudaError_t upload_fac(amgdd_handle h, FacLayout &F, FacStream &S, int nlev, int nsub,
                              const std::vector<int64_t> &level_off, bool fp32, cudaStream_t st_, FacParams &P,
                              const char **what)
{
    cudaError_t e;
#define UP(x, y, msg)                                           \
    do {                                                        \
        if ((e = upload(h, x, y, st_)) != cudaSuccess) {        \
            *what = msg;                                        \
            return e;                                           \
        }                                                       \
    } while (0)
    P.nlev = nlev;
    P.nsub = nsub;
    P.nfac = h->opt.n_fac;
    P.nL = h->nL;
    FacLevelDesc *dd;
    int32_t *ord, *own;
    int64_t *o0;
    UP(F.desc, &dd, "upload desc");
    UP(F.order, &ord, "upload order");
    P.fp32 = fp32 ? 1 : 0;
    UP(F.owned, &own, "upload owned");
    UP(F.owned0, &o0, "upload owned0");
    P.col16 = F.A.c16 ? 1 : 0;
    P.schedule = h->opt.schedule >= 1 && h->opt.schedule <= 9 ? h->opt.schedule : 8;
    for (int l = 0; l <= kMaxLevels; ++l) P.grp[l] = 1;
    // lanes per row for the group-per-row candidate, per level: double g
    // (up to 32) while the level's mean slices per grid times g stay below
    // the 16 warps of a block and 2g entries still fit the mean real row
    if (&P == &h->fac) {
        // a single-column schedule asked for in the options, else candidate 15
        // (two operator entries in flight, four blocks per SM, L2 prefetch)
        h->fac_cand[0] = h->opt.schedule >= 1 && h->opt.schedule <= 9 ? P.schedule - 1 : 15;
        {
            std::vector<int32_t> ob{0, nsub};
            int32_t *dob;
            UP(ob, &dob, "upload queue bounds");
            h->one_bin_off = dob;
        }
        for (int l = 0; l < nlev && l <= kMaxLevels; ++l) {
            double slices = 0.0, rows = 0.0;
            for (int p = 0; p < nsub; ++p) {
                const FacLevelDesc &d = F.desc[(size_t)p * nlev + l];
                slices += (double)((d.nBar + 31) / 32);
                rows += (double)d.nReal;
            }
            slices /= std::max(nsub, 1);
            const double width = rows > 0 ? (double)F.lvA[l] / rows : 0.0;
            int g = 1;
            while (g < 32 && slices * g < 16.0 && 2.0 * g <= width) g *= 2;
            h->grp_level[l] = (int8_t)g;
        }
    }
    FacViewDev *dviews[5] = {&P.A, &P.At, &P.AFc, &P.P, &P.R};
    void *gm = nullptr, *l1 = nullptr;
    *what = "settle layout";
    for (int v = 0; v < 5; ++v) {
        void *so, *rl, *co, *va;
        if ((e = settle(h, S.soff[v], st_, &so)) != cudaSuccess) return e;
        if ((e = settle(h, S.rlen[v], st_, &rl)) != cudaSuccess) return e;
        if ((e = settle(h, S.col[v], st_, &co)) != cudaSuccess) return e;
        if ((e = settle(h, S.val[v], st_, &va)) != cudaSuccess) return e;
        dviews[v]->soff = static_cast<const int64_t *>(so);
        dviews[v]->rlen = static_cast<const uint16_t *>(rl);
        dviews[v]->col = co;
        dviews[v]->val = va;
    }
    if ((e = settle(h, S.gmap, st_, &gm)) != cudaSuccess) return e;
    if ((e = settle(h, S.l1inv, st_, &l1)) != cudaSuccess) return e;
    P.l1inv = l1;
    // one bin per SM; grids by decreasing work into the lightest bin
    {
        int dev = 0, nsm = 1;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int nb = std::max(1, nsm);
        std::vector<std::vector<int32_t>> bins((size_t)nb);
        std::vector<int64_t> load((size_t)nb, 0);
        for (int32_t g : F.order) {  // F.order: decreasing work
            int best = 0;
            for (int b = 1; b < nb; ++b)
                if (load[b] < load[best]) best = b;
            bins[best].push_back(g);
            load[best] += F.work[g] > 0 ? F.work[g] : 1;
        }
        std::vector<int32_t> off(1, 0), grid;
        for (auto &bv : bins) {
            grid.insert(grid.end(), bv.begin(), bv.end());
            off.push_back((int32_t)grid.size());
        }
        int32_t *doff, *dgrid, *dctr;
        UP(off, &doff, "upload bins");
        UP(grid, &dgrid, "upload bins");
        if ((e = alloc(h, (size_t)nb, &dctr)) != cudaSuccess) {
            *what = "alloc bin counters";
            return e;
        }
        if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return e;
        P.nbins = nb;
        P.bin_off = doff;
        P.bin_grid = dgrid;
        P.ctr = dctr;
        // teams for two blocks of 1024 threads per SM; the kernel's named
        // barriers allow at most 15 teams per block (ids 1..15), each of
        // 1..32 whole warps within the block's 32, and every grid must be
        // cycled exactly once
        const TeamPlan TP = plan_teams(F.work, 2 * nb);
        {
            bool ok = (int)TP.block_off.size() == 2 * nb + 1 && TP.grid_off.size() == TP.w0.size() + 1 &&
                      (int)TP.grid.size() == nsub;
            for (int b = 0; ok && b < 2 * nb; ++b) {
                const int k0 = TP.block_off[b], k1 = TP.block_off[b + 1];
                ok = k1 - k0 <= 15;
                for (int k = k0; ok && k < k1; ++k)
                    ok = TP.nw[k] >= 1 && TP.w0[k] >= 0 && TP.w0[k] + TP.nw[k] <= 32 &&
                         (k == k0 || TP.w0[k] >= TP.w0[k - 1] + TP.nw[k - 1]);
            }
            std::vector<char> seen((size_t)nsub, 0);
            for (int32_t g : TP.grid) {
                ok = ok && g >= 0 && g < nsub && !seen[g];
                if (ok) seen[g] = 1;
            }
            if (!ok) {
                *what = "team plan of the FAC kernel";
                return cudaErrorInvalidValue;
            }
        }
        int32_t *tb, *tw0, *tnw, *tgo, *tg;
        UP(TP.block_off, &tb, "upload teams");
        UP(TP.w0, &tw0, "upload teams");
        UP(TP.nw, &tnw, "upload teams");
        UP(TP.grid_off, &tgo, "upload teams");
        UP(TP.grid, &tg, "upload teams");
        if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return e;
        P.teams = FacTeams{2 * nb, tb, tw0, tnw, tgo, tg};
    }
    P.max_grid_rows = 0;
    for (int p = 0; p < nsub; ++p) {
        const FacLevelDesc &a = F.desc[(size_t)p * nlev], &z = F.desc[(size_t)p * nlev + nlev - 1];
        P.max_grid_rows = std::max<int64_t>(P.max_grid_rows, z.row0 + z.nBar - a.row0);
    }
    P.vsm_bytes = 0;
    P.desc = dd;
    P.order = ord;
    P.gmap = static_cast<const int32_t *>(gm);
    P.owned = own;
    P.owned0 = o0;
    P.ainv = h->ainv;
    P.ainv_ptr = h->ainv_ptr;
    P.ainv_col = h->ainv_col;
    P.ainv_val = h->ainv_val;
    for (int l = 0; l <= kMaxLevels; ++l) P.level_off[l] = l <= nlev ? level_off[l] : 0;
    void *ws[6];
    for (int k = 0; k < 6; ++k) {
        if (fp32) {
            float *w;
            if ((e = alloc(h, (size_t)F.rows_total, &w)) != cudaSuccess) {
                *what = "alloc FAC workspace";
                return e;
            }
            ws[k] = w;
        } else {
            double *w;
            if ((e = alloc(h, (size_t)F.rows_total, &w)) != cudaSuccess) {
                *what = "alloc FAC workspace";
                return e;
            }
            ws[k] = w;
        }
    }
    P.u = ws[0]; P.f = ws[1]; P.t = ws[2]; P.s = ws[3]; P.w = ws[4]; P.d = ws[5];
#undef UP
    return cudaSuccess;
}

extern "C" {

amgdd_status amgdd_options_default(amgdd_options *o)
{
    if (!o) return fail(nullptr, AMGDD_ERR_INVALID_ARG, "null options");
    std::memset(o, 0, sizeof *o);
    o->theta = 0.25;
    o->max_coarse = 16;
    o->max_levels = 25;
    o->n_fac = 2;
    o->strict_assumption = 0;
    o->host_only = 0;
    o->threads = 0;
    o->schedule = 0;
    o->precision = 0;
    o->interp = 0;
    o->p_max = 4;
    o->hybrid_level = 0;
    o->coarsen = 0;
    return AMGDD_OK;
}

amgdd_status amgdd_box_partition(int32_t nx, int32_t ny, int32_t nz, int32_t bx, int32_t by, int32_t bz,
                                 int32_t *part, int32_t *nsub)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || bx <= 0 || by <= 0 || bz <= 0 || !part)
        return fail(nullptr, AMGDD_ERR_INVALID_ARG, "box partition: sizes must be positive");
    const int64_t mx = (nx + bx - 1) / bx, my = (ny + by - 1) / by, mz = (nz + bz - 1) / bz;
    if (mx * my * mz > INT32_MAX) return fail(nullptr, AMGDD_ERR_INVALID_ARG, "too many boxes");
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                part[i + nx * (j + ny * k)] = (int32_t)((i / bx) + mx * ((j / by) + my * (k / bz)));
    if (nsub) *nsub = (int32_t)(mx * my * mz);
    return AMGDD_OK;
}

const char *amgdd_last_error(amgdd_handle h)
{
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

void amgdd_destroy(amgdd_handle h)
{
    if (!h) return;
    if (h->on_device) {
        cudaStreamSynchronize(h->last_stream);
        for (auto &m : h->multi) {
            if (m.graph.exec) cudaGraphExecDestroy(m.graph.exec);
            if (m.h_scal) cudaFreeHost(m.h_scal);
        }
        for (auto &g : h->solve_graph)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
        if (h->hist) cudaFree(h->hist);
        if (h->h_hist) cudaFreeHost(h->h_hist);
        if (h->h_conv) cudaFreeHost(h->h_conv);
        for (void *p : h->allocs) cudaFree(p);
        if (h->h_scal) cudaFreeHost(h->h_scal);
    }
    delete h;
}

amgdd_status amgdd_setup(const amgdd_csr *A, const int32_t *part, int32_t nsub, const int32_t *padding,
                         int32_t npadding, const amgdd_options *opts, void *stream, amgdd_handle *out)
{
    if (!out) return fail(nullptr, AMGDD_ERR_INVALID_ARG, "null output handle pointer");
    *out = nullptr;
    const FaultScope fault_scope;
    const auto t0 = std::chrono::steady_clock::now();
    amgdd_status st;
    std::string why = validate(A, part, nsub, padding, npadding, st);
    if (st != AMGDD_OK) return fail(nullptr, st, why);
    amgdd_handle h = new (std::nothrow) amgdd_handle_s();
    if (!h) return fail(nullptr, AMGDD_ERR_OOM, "host allocation failed");
    if (opts) h->opt = *opts;
    else amgdd_options_default(&h->opt);
    if (h->opt.n_fac < 1 || h->opt.max_levels < 1 || h->opt.max_coarse < 1 || !(h->opt.theta > 0.0) ||
        !(h->opt.theta <= 1.0) || h->opt.precision < 0 || h->opt.precision > 1 || h->opt.interp < 0 ||
        h->opt.interp > 1 || h->opt.p_max < 0 || h->opt.coarsen < 0 || h->opt.coarsen > 1) {
        delete h;
        return fail(nullptr, AMGDD_ERR_INVALID_ARG, "options out of range");
    }
    h->threads = h->opt.threads > 0 ? h->opt.threads : 512;
    if (h->threads % 32 != 0 || h->threads > 512) {
        delete h;
        return fail(nullptr, AMGDD_ERR_INVALID_ARG, "threads must be a multiple of 32 up to 512");
    }
    try {
        Csr A0;
        A0.rows = A0.cols = A->n;
        A0.ptr.assign(A->rowptr, A->rowptr + A->n + 1);
        A0.idx.assign(A->col, A->col + A->nnz);
        A0.val.assign(A->val, A->val + A->nnz);
        HierarchyParams prm;
        prm.theta = h->opt.theta;
        prm.max_coarse = h->opt.max_coarse;
        prm.max_levels = std::min(h->opt.max_levels, (int32_t)AMGDD_MAX_LEVELS);
        prm.interp = h->opt.interp;
        prm.p_max = h->opt.p_max;
        prm.coarsen = h->opt.coarsen;
        prm.part = part;
        int hst = 0;
        why = build_hierarchy(A0, prm, h->H, hst);
        if (hst != 0) {
            delete h;
            return fail(nullptr, hst == 1 ? AMGDD_ERR_SINGULAR : AMGDD_ERR_INVALID_ARG, why);
        }
        const int nlev = (int)h->H.lv.size();
        if (h->opt.hybrid_level < 0 || h->opt.hybrid_level >= nlev) {
            delete h;
            return fail(nullptr, AMGDD_ERR_INVALID_ARG,
                        "hybrid_level must be in [0, number of levels - 1] (" + std::to_string(nlev) + " levels)");
        }
        std::vector<int> eta((size_t)nlev);
        for (int l = 0; l < nlev; ++l) eta[l] = padding[std::min(l, npadding - 1)];
        const int nth = host_threads();
        build_composite(h->H, part, nsub, eta, h->C, nth);
        if (h->opt.strict_assumption && h->C.violations > 0) {
            delete h;
            return fail(nullptr, AMGDD_ERR_HIERARCHY_ASSUMPTION,
                        "composite grids break the connectivity assumption");
        }
        // statistics
        amgdd_setup_stats &S = h->stats;
        S.num_levels = nlev;
        S.nsub = nsub;
        double nnz_sum = 0, n_sum = 0, real_nnz = 0;
        for (int l = 0; l < nlev; ++l) {
            S.n[l] = h->H.lv[l].A.rows;
            S.nnz[l] = h->H.lv[l].A.nnz();
            S.nnz_P[l] = l + 1 < nlev ? h->H.lv[l].P.nnz() : 0;
            nnz_sum += (double)S.nnz[l];
            n_sum += S.n[l];
            const Csr &Al = h->H.lv[l].A;
            for (int p = 0; p < nsub; ++p) {
                const CompLevel &cl = h->C.at(p, l);
                S.comp_real[l] += (int64_t)cl.real.size();
                S.comp_ghost[l] += (int64_t)cl.ghost.size();
                for (int32_t i : cl.real) S.comp_nnz_real[l] += Al.ptr[i + 1] - Al.ptr[i];
            }
            real_nnz += (double)S.comp_nnz_real[l];
        }
        S.operator_complexity = nnz_sum / (double)S.nnz[0];
        S.grid_complexity = n_sum / (double)S.n[0];
        S.composite_overhead = real_nnz / nnz_sum;
        S.assumption_violations = h->C.violations;
        h->level_off.assign((size_t)nlev + 1, 0);
        for (int l = 0; l < nlev; ++l) h->level_off[l + 1] = h->level_off[l] + S.n[l];

        if (h->opt.host_only != 1) {
            cudaStream_t st_ = (cudaStream_t)stream;
            h->last_stream = st_;
            // with a device, the layout goes to it chunk by chunk as it is
            // packed; host_only = 3 packs, checks and drops it the same way
            const bool to_dev = h->opt.host_only == 0 || h->opt.host_only == 3;
            FacLayout F;
            FacStream FS;
            FS.fp32 = h->opt.precision == 1;
            FS.host = h->opt.host_only == 3;
            FacSink sink;
            if (to_dev) sink = [&](FacLayout &Lf, int p0, int pn) { return FS.consume(h->H, Lf, p0, pn, st_); };
            std::string badf = build_fac_layout(h->H, h->C, F, nth, h->opt.precision == 1, sink);
            if (badf.empty()) badf = to_dev ? validate_fac_totals(F) : validate_layouts(h->H, {}, F);
            if (!badf.empty()) {
                const cudaError_t fe = FS.err;
                delete h;
                if (fe != cudaSuccess) return cuda_fail(nullptr, fe, "composite layout upload");
                return fail(nullptr, AMGDD_ERR_INVALID_ARG, "internal layout check failed: " + badf);
            }
            S.fac_fma = 0;
            for (int p = 0; p < nsub; ++p)
                S.fac_fma += F.work1[p] + (int64_t)(h->opt.n_fac - 1) * F.work[p];
            S.fac_entry_bytes = (h->opt.precision == 1 ? 4 : 8) + (F.A.c16 ? 2 : 4);
            // stored entries of the local operators (padding excluded)
            for (int l = 0; l < nlev; ++l) {
                S.comp_nnz_A[l] = F.lvA[l];
                S.comp_nnz_P[l] = F.lvP[l];
                if (l > 0) S.comp_nnz_R[l - 1] = F.lvR[l];
            }
            std::vector<GlobalLevelDev> G;
            build_global_dev(h->H, G);
            const std::string bad = validate_global(h->H, G);
            if (!bad.empty()) {
                delete h;
                return fail(nullptr, AMGDD_ERR_INVALID_ARG, "internal layout check failed: " + bad);
            }
            // hybrid AMG-DD: composite grids of the hierarchy from level Lt down
            FacLayout Fs;
            FacStream FSs;
            int32_t hyb_ns = 0;
            if (h->opt.hybrid_level > 0) {
                // subdomains of level Lt: each C point keeps the subdomain of
                // the point it comes from; subdomains left without points drop out
                const int Lt = h->opt.hybrid_level;
                std::vector<int32_t> pl(part, part + h->H.lv[0].A.rows);
                for (int l = 0; l < Lt; ++l) {
                    std::vector<int32_t> nx((size_t)h->H.lv[l + 1].A.rows);
                    for (int32_t i = 0; i < h->H.lv[l].A.rows; ++i)
                        if (h->H.lv[l].isC[i]) nx[h->H.lv[l].coarse[i]] = pl[i];
                    pl.swap(nx);
                }
                std::vector<int32_t> remap((size_t)nsub, -1);
                for (int32_t q : pl) remap[q] = 0;
                for (int32_t p2 = 0; p2 < nsub; ++p2)
                    if (remap[p2] == 0) remap[p2] = hyb_ns++;
                for (int32_t &q : pl) q = remap[q];
                Hierarchy Hs;
                Hs.lv.assign(h->H.lv.begin() + Lt, h->H.lv.end());
                Hs.ainv = h->H.ainv;
                Composite Cs;
                std::vector<int> etas(eta.begin() + Lt, eta.end());
                build_composite(Hs, pl.data(), hyb_ns, etas, Cs, nth);
                FSs.host = h->opt.host_only == 3;
                FacSink sinks;
                if (to_dev) sinks = [&](FacLayout &Lf, int p0, int pn) { return FSs.consume(Hs, Lf, p0, pn, st_); };
                std::string bad2 = build_fac_layout(Hs, Cs, Fs, nth, false, sinks);
                if (bad2.empty()) bad2 = to_dev ? validate_fac_totals(Fs) : validate_layouts(Hs, {}, Fs);
                if (!bad2.empty()) {
                    const cudaError_t fe = FSs.err;
                    delete h;
                    if (fe != cudaSuccess) return cuda_fail(nullptr, fe, "hybrid layout upload");
                    return fail(nullptr, AMGDD_ERR_INVALID_ARG, "internal hybrid layout check failed: " + bad2);
                }
                const int nls = nlev - Lt;
                h->hyb_off.assign((size_t)nls + 1, 0);
                for (int l = 0; l < nls; ++l) h->hyb_off[l + 1] = h->hyb_off[l] + Hs.lv[l].A.rows;
            }
            if (h->opt.host_only >= 2) goto done;
            auto bail = [&](cudaError_t e, const char *what) {
                amgdd_status s2 = cuda_fail(nullptr, e, what);
                for (void *p : h->allocs) cudaFree(p);
                h->allocs.clear();
                if (h->h_scal) cudaFreeHost(h->h_scal);
                delete h;
                return s2;
            };
            cudaError_t e;
            h->lev.assign((size_t)nlev, DevLevel{});
            size_t maxn = 0;
            for (int l = 0; l < nlev; ++l) {
                DevLevel &D = h->lev[l];
                D.n = h->H.lv[l].A.rows;
                D.nC = G[l].nC;
                maxn = std::max(maxn, (size_t)D.n);
                if ((e = upload_sell(h, G[l].A, &G[l].rowid, D.A, st_)) != cudaSuccess) return bail(e, "upload A_l");
                if (l + 1 < nlev) {
                    if ((e = upload_sell(h, G[l].P, nullptr, D.P, st_)) != cudaSuccess) return bail(e, "upload P_l");
                    if ((e = upload_sell(h, G[l].R, nullptr, D.R, st_)) != cudaSuccess) return bail(e, "upload R_l");
                }
                double *l1;
                if ((e = upload(h, h->H.lv[l].l1inv, &l1, st_)) != cudaSuccess) return bail(e, "upload l1");
                D.l1inv = l1;
                if (l > 0) {
                    if ((e = alloc(h, (size_t)D.n, &D.u)) != cudaSuccess) return bail(e, "alloc u_l");
                    if ((e = alloc(h, (size_t)D.n, &D.f)) != cudaSuccess) return bail(e, "alloc f_l");
                }
                if ((e = alloc(h, (size_t)D.n, &D.d)) != cudaSuccess) return bail(e, "alloc d_l");
                // the host copies of the device layout are no longer needed
                G[l] = GlobalLevelDev();
            }
            double *ainv;
            if ((e = upload(h, h->H.ainv, &ainv, st_)) != cudaSuccess) return bail(e, "upload coarse inverse");
            h->ainv = ainv;
            {
                const int64_t nL = h->H.lv.back().A.rows;
                std::vector<int32_t> cp(1, 0), cc;
                std::vector<double> cv;
                for (int64_t I = 0; I < nL; ++I) {
                    for (int64_t J = 0; J < nL; ++J) {
                        const double a = h->H.ainv[(size_t)(I * nL + J)];
                        if (a != 0.0) {
                            cc.push_back((int32_t)J);
                            cv.push_back(a);
                        }
                    }
                    cp.push_back((int32_t)cc.size());
                }
                int32_t *dp, *dc;
                double *dv;
                if ((e = upload(h, cp, &dp, st_)) != cudaSuccess) return bail(e, "upload coarse inverse");
                if ((e = upload(h, cc, &dc, st_)) != cudaSuccess) return bail(e, "upload coarse inverse");
                if ((e = upload(h, cv, &dv, st_)) != cudaSuccess) return bail(e, "upload coarse inverse");
                if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return bail(e, "upload coarse inverse");
                h->ainv_ptr = dp;
                h->ainv_col = dc;
                h->ainv_val = dv;
            }
            h->nL = h->H.lv.back().A.rows;
            if ((e = alloc(h, (size_t)h->level_off.back(), &h->r_all)) != cudaSuccess) return bail(e, "alloc r");
            if ((e = alloc(h, maxn, &h->res)) != cudaSuccess) return bail(e, "alloc res");
            h->nred = 152 * 8;
            if ((e = alloc(h, (size_t)h->nred, &h->partial)) != cudaSuccess) return bail(e, "alloc partial");
            if ((e = alloc(h, 8, &h->scal)) != cudaSuccess) return bail(e, "alloc scalars");
            if ((e = pinned_malloc((void **)&h->h_scal, 8 * sizeof(double))) != cudaSuccess)
                return bail(e, "alloc pinned");
            // composite-grid layout
            {
                const char *what = "";
                if ((e = upload_fac(h, F, FS, nlev, nsub, h->level_off, h->opt.precision == 1, st_, h->fac, &what)) !=
                    cudaSuccess)
                    return bail(e, what);
            }
            if (hyb_ns > 0) {
                const int nls = nlev - h->opt.hybrid_level;
                const char *what = "";
                if ((e = upload_fac(h, Fs, FSs, nls, hyb_ns, h->hyb_off, false, st_, h->fac_hyb, &what)) != cudaSuccess)
                    return bail(e, what);
                if ((e = alloc(h, (size_t)h->hyb_off.back(), &h->r_hyb)) != cudaSuccess)
                    return bail(e, "alloc hybrid residual");
                h->hyb_level = h->opt.hybrid_level;
            }
            if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return bail(e, "setup upload");
            h->desc = F.desc;
            h->dev2map = F.dev2map;
            h->fac_rows = F.rows_total;
            h->on_device = true;
        }
    done:
        h->stats.device_bytes = h->dev_bytes;
    } catch (const std::bad_alloc &) {
        for (void *p : h->allocs) cudaFree(p);
        if (h->h_scal) cudaFreeHost(h->h_scal);
        delete h;
        return fail(nullptr, AMGDD_ERR_OOM, "host allocation failed during setup");
    }
    h->stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return AMGDD_OK;
}

amgdd_status amgdd_get_stats(amgdd_handle h, amgdd_setup_stats *s)
{
    if (!h || !s) return fail(h, AMGDD_ERR_INVALID_ARG, "null argument");
    *s = h->stats;
    return AMGDD_OK;
}

amgdd_status amgdd_get_maps(amgdd_handle h, int32_t sub, int32_t level, int32_t *global_idx, uint8_t *kind,
                            int32_t *count)
{
    if (!h || !count) return fail(h, AMGDD_ERR_INVALID_ARG, "null argument");
    if (sub < 0 || sub >= h->C.nsub || level < 0 || level >= h->C.nlev)
        return fail(h, AMGDD_ERR_INVALID_ARG, "subdomain or level out of range");
    const CompLevel &cl = h->C.at(sub, level);
    const int32_t n = (int32_t)(cl.real.size() + cl.ghost.size());
    *count = n;
    if (!global_idx) return AMGDD_OK;
    int32_t o = 0;
    for (int32_t i : cl.owned) { global_idx[o] = i; if (kind) kind[o] = 0; ++o; }
    size_t a = 0;
    for (int32_t i : cl.real) {
        while (a < cl.owned.size() && cl.owned[a] < i) ++a;
        if (a < cl.owned.size() && cl.owned[a] == i) continue;
        global_idx[o] = i;
        if (kind) kind[o] = 1;
        ++o;
    }
    for (int32_t i : cl.ghost) { global_idx[o] = i; if (kind) kind[o] = 2; ++o; }
    return AMGDD_OK;
}

amgdd_status amgdd_get_operator(amgdd_handle h, int32_t level, int32_t which, int32_t *rows, int32_t *cols,
                                int64_t *nnz, int64_t *rowptr, int32_t *col, double *val)
{
    if (!h) return fail(h, AMGDD_ERR_INVALID_ARG, "null handle");
    const int nlev = (int)h->H.lv.size();
    if (level < 0 || level >= nlev || which < 0 || which > 2 || (which > 0 && level == nlev - 1))
        return fail(h, AMGDD_ERR_INVALID_ARG, "level/operator out of range");
    const Csr &M = which == 0 ? h->H.lv[level].A : which == 1 ? h->H.lv[level].P : h->H.lv[level].R;
    if (rows) *rows = M.rows;
    if (cols) *cols = M.cols;
    if (nnz) *nnz = M.nnz();
    if (rowptr) {
        std::copy(M.ptr.begin(), M.ptr.end(), rowptr);
        if (col) std::copy(M.idx.begin(), M.idx.end(), col);
        if (val) std::copy(M.val.begin(), M.val.end(), val);
    }
    return AMGDD_OK;
}

amgdd_status amgdd_get_cf(amgdd_handle h, int32_t level, int32_t *cf, double *l1inv)
{
    if (!h) return fail(h, AMGDD_ERR_INVALID_ARG, "null handle");
    const int nlev = (int)h->H.lv.size();
    if (level < 0 || level >= nlev) return fail(h, AMGDD_ERR_INVALID_ARG, "level out of range");
    const HLevel &lv = h->H.lv[level];
    if (cf) {
        if (level == nlev - 1) return fail(h, AMGDD_ERR_INVALID_ARG, "the coarsest level has no C/F split");
        for (size_t i = 0; i < lv.isC.size(); ++i) cf[i] = lv.isC[i];
    }
    if (l1inv) std::copy(lv.l1inv.begin(), lv.l1inv.end(), l1inv);
    return AMGDD_OK;
}

amgdd_status amgdd_plan_teams(const int64_t *work, int32_t nsub, int32_t nblocks, int32_t *block_off,
                              int32_t *w0, int32_t *nw, int32_t *grid_off, int32_t *grid, int32_t *nteams)
{
    if (!work || nsub < 1 || nblocks < 1 || !block_off || !w0 || !nw || !grid_off || !grid || !nteams)
        return fail(nullptr, AMGDD_ERR_INVALID_ARG, "bad team plan arguments");
    std::vector<int64_t> wv(work, work + nsub);
    for (int64_t x : wv)
        if (x < 0) return fail(nullptr, AMGDD_ERR_INVALID_ARG, "negative work");
    const TeamPlan T = plan_teams(wv, nblocks);
    std::copy(T.block_off.begin(), T.block_off.end(), block_off);
    std::copy(T.w0.begin(), T.w0.end(), w0);
    std::copy(T.nw.begin(), T.nw.end(), nw);
    std::copy(T.grid_off.begin(), T.grid_off.end(), grid_off);
    std::copy(T.grid.begin(), T.grid.end(), grid);
    *nteams = (int32_t)T.w0.size();
    return AMGDD_OK;
}

amgdd_status amgdd_get_coarse_inverse(amgdd_handle h, double *ainv)
{
    if (!h || !ainv) return fail(h, AMGDD_ERR_INVALID_ARG, "null argument");
    std::copy(h->H.ainv.begin(), h->H.ainv.end(), ainv);
    return AMGDD_OK;
}

// ---------------------------------------------------------------------------
// Solve phase.

static amgdd_status residual_norm(amgdd_handle h, const double *b, const double *x, double *r, cudaStream_t st,
                                  double *nrm2)
{
    CK(launch_residual(h->lev[0].A, b, x, r, h->partial, h->nred, h->scal, st), "residual kernel");
    h->launches += 2;
    if (nrm2) {
        CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st), "norm copy");
        CK(cudaStreamSynchronize(st), "residual");
        *nrm2 = h->h_scal[0];
    }
    return AMGDD_OK;
}

// Levels whose restriction has at most this many rows are restricted by one
// cluster of blocks (k_chain) instead of one grid-wide launch each; a fine
// level of at most this many rows also has its residual computed there.
static constexpr int64_t kChainRows = 4096;

// First level l whose restriction R_l and all coarser ones have at most
// kChainRows rows (n_{l+1} <= kChainRows); the number of levels - 1 if none.
static int chain_first(amgdd_handle h)
{
    const int nlev = (int)h->lev.size();
    int lt = nlev - 1;
    while (lt > 0 && h->lev[lt].n <= kChainRows) --lt;
    return lt;
}

// r_{l+1} = R_l r_l for l = l0 .. L-1 as chain steps.
static void chain_steps(amgdd_handle h, double *r_all, int l0, ChainParams &C)
{
    const int nlev = (int)h->lev.size();
    C.nsteps = 0;
    for (int l = l0; l + 1 < nlev; ++l)
        C.step[C.nsteps++] = ChainStep{h->lev[l].R, r_all + h->level_off[l], r_all + h->level_off[l + 1]};
}

static amgdd_status restrict_all(amgdd_handle h, double *r_all, cudaStream_t st)
{
    const int nlev = (int)h->lev.size();
    const int lt = chain_first(h);
    for (int l = 0; l < lt; ++l) {
        const DevLevel &D = h->lev[l];
        CK(launch_spmv(D.R, 0, D.R.rows, r_all + h->level_off[l], r_all + h->level_off[l + 1], 0, st),
           "restriction kernel");
        h->launches += 1;
    }
    if (lt + 1 < nlev) {
        ChainParams C{};
        chain_steps(h, r_all, lt, C);
        CK(launch_chain(C, st), "restriction chain kernel");
        h->launches += 1;
    }
    return AMGDD_OK;
}

// The right-hand sides of an AMG-DD iteration: r = b - A x (its squared
// norm in h->scal[0]) and r_l = R_{l-1} r_{l-1} on every level, into r_all.
// A fine level of at most kChainRows rows does all of it in one block.
// chk (may be null): the convergence check of a solve graph, done by the
// single chain launch when the fine level is small enough for it; *checked
// says whether it was (else the caller launches the check itself).
static amgdd_status residual_restrict(amgdd_handle h, const double *b, const double *x, cudaStream_t st,
                                      const ChainCheck *chk = nullptr, bool *checked = nullptr)
{
    if (checked) *checked = false;
    if (h->lev[0].n > kChainRows) {
        CK(launch_residual(h->lev[0].A, b, x, h->r_all, h->partial, h->nred, h->scal, st), "residual kernel");
        h->launches += 2;
        return restrict_all(h, h->r_all, st);
    }
    ChainParams C{};
    if (chk) {
        C.check = *chk;
        C.check.on = 1;
        if (checked) *checked = true;
    }
    C.residual = 1;
    C.A = h->lev[0].A;
    C.b = b;
    C.x = x;
    C.r = h->r_all;
    C.nrm2 = h->scal;
    C.partial = h->partial;
    chain_steps(h, h->r_all, 0, C);
    CK(launch_chain(C, st), "residual and restriction chain kernel");
    h->launches += 1;
    return AMGDD_OK;
}

// FAC launch of candidate k (see amgdd_autotune) for nrhs columns with the
// inputs, outputs and work space already set in P.
static cudaError_t launch_candidate(amgdd_handle h, FacParams P, int nrhs, int k, cudaStream_t st)
{
    for (int l = 0; l <= kMaxLevels; ++l) P.grp[l] = 1;
    if (k < 9) {
        P.schedule = k + 1;
        return launch_fac_all_grids(P, P.nsub, h->threads, st);
    }
    if (k < 18) return launch_fac_multi(P, P.nsub, nrhs, k - 8, st);
    if (k == 31) return launch_fac_multi(P, P.nsub, nrhs, 16, st);      // teams sized by work
    if (k >= 25) {   // one queue, largest grid first
        P.nbins = 1;
        P.bin_off = h->one_bin_off;
        P.bin_grid = P.order;
        if (k == 25) return launch_fac_multi(P, P.nsub, nrhs, 7, st);
        if (k <= 27) return launch_fac_vsm(P, P.nsub, nrhs, k - 25, st);
        return launch_fac_cluster(P, P.nsub, nrhs, 1 << (k - 27), st);   // clusters of 2, 4, 8 blocks
    }
    if (k >= 20) return launch_fac_multi(P, P.nsub, nrhs, k - 9, st);   // variants 11-15
    for (int l = 0; l <= kMaxLevels; ++l) P.grp[l] = k == 18 ? h->grp_level[l] : (int8_t)32;
    return launch_fac_multi(P, P.nsub, nrhs, 10, st);
}

static amgdd_status fac(amgdd_handle h, const double *r_all, double *x, cudaStream_t st)
{
    FacParams P = h->fac;
    P.r_all = r_all;
    P.x = x;
    CK(launch_candidate(h, P, 1, h->fac_cand[0], st), "FAC kernel");
    h->launches += 1;
    return AMGDD_OK;
}

static amgdd_status relax(amgdd_handle h, int l, bool cpass, double *u, const double *f, cudaStream_t st)
{
    const DevLevel &D = h->lev[l];
    const int64_t r0 = cpass ? 0 : D.nC, r1 = cpass ? D.nC : D.n;
    CK(launch_relax_compute(D.A, r0, r1, f, u, D.l1inv, D.d, 0, st), "relax kernel");
    CK(launch_relax_apply(D.A.rowid, r0, r1, D.d, u, st), "relax apply kernel");
    h->launches += 2;
    return AMGDD_OK;
}

static amgdd_status vcycle(amgdd_handle h, const double *b, double *x, cudaStream_t st)
{
    const int L = (int)h->lev.size() - 1;
    amgdd_status s;
    for (int l = 0; l < L; ++l) {
        DevLevel &D = h->lev[l];
        double *u = l == 0 ? x : D.u;
        const double *f = l == 0 ? b : D.f;
        if ((s = relax(h, l, true, u, f, st)) != AMGDD_OK) return s;
        if ((s = relax(h, l, false, u, f, st)) != AMGDD_OK) return s;
        CK(launch_relax_compute(D.A, 0, D.n, f, u, D.l1inv, h->res, 1, st), "residual kernel");
        CK(launch_spmv(D.R, 0, D.R.rows, h->res, h->lev[l + 1].f, 0, st), "restriction kernel");
        CK(cudaMemsetAsync(h->lev[l + 1].u, 0, sizeof(double) * (size_t)h->lev[l + 1].n, st), "memset");
        h->launches += 2;
    }
    CK(launch_coarse_solve(h->ainv, h->nL, L == 0 ? b : h->lev[L].f, L == 0 ? x : h->lev[L].u, st), "coarse solve");
    h->launches += 1;
    for (int l = L - 1; l >= 0; --l) {
        DevLevel &D = h->lev[l];
        double *u = l == 0 ? x : D.u;
        const double *f = l == 0 ? b : D.f;
        CK(launch_spmv(D.P, 0, D.P.rows, h->lev[l + 1].u, u, 1, st), "interpolation kernel");
        h->launches += 1;
        if ((s = relax(h, l, false, u, f, st)) != AMGDD_OK) return s;
        if ((s = relax(h, l, true, u, f, st)) != AMGDD_OK) return s;
    }
    return AMGDD_OK;
}

// Hybrid AMG-DD V(1,1)-cycle (Algorithm 3): the V-cycle's downsweep on levels
// 0 .. Lt-1, one AMG-DD cycle on level Lt in place of the coarse solve, then
// the V-cycle's upsweep.
static amgdd_status vcycle_hybrid(amgdd_handle h, const double *b, double *x, cudaStream_t st)
{
    const int L = (int)h->lev.size() - 1;
    const int Lt = h->hyb_level;
    amgdd_status s;
    for (int l = 0; l < Lt; ++l) {
        DevLevel &D = h->lev[l];
        double *u = l == 0 ? x : D.u;
        const double *f = l == 0 ? b : D.f;
        if ((s = relax(h, l, true, u, f, st)) != AMGDD_OK) return s;
        if ((s = relax(h, l, false, u, f, st)) != AMGDD_OK) return s;
        CK(launch_relax_compute(D.A, 0, D.n, f, u, D.l1inv, h->res, 1, st), "residual kernel");
        CK(launch_spmv(D.R, 0, D.R.rows, h->res, h->lev[l + 1].f, 0, st), "restriction kernel");
        CK(cudaMemsetAsync(h->lev[l + 1].u, 0, sizeof(double) * (size_t)h->lev[l + 1].n, st), "memset");
        h->launches += 2;
    }
    {
        // AMG-DD cycle on level Lt: r = f - A u, restrictions, AlgFAC on the
        // composite grids of the sub-hierarchy, owned corrections into u
        DevLevel &D = h->lev[Lt];
        double *u = Lt == 0 ? x : D.u;
        const double *f = Lt == 0 ? b : D.f;
        CK(launch_relax_compute(D.A, 0, D.n, f, u, D.l1inv, h->r_hyb, 1, st), "residual kernel");
        h->launches += 1;
        for (int l = Lt; l < L; ++l) {
            CK(launch_spmv(h->lev[l].R, 0, h->lev[l].R.rows, h->r_hyb + h->hyb_off[l - Lt],
                           h->r_hyb + h->hyb_off[l - Lt + 1], 0, st), "restriction kernel");
            h->launches += 1;
        }
        FacParams P = h->fac_hyb;
        P.r_all = h->r_hyb;
        P.x = u;
        CK(launch_fac_all_grids(P, P.nsub, h->threads, st), "FAC kernel");
        h->launches += 1;
    }
    for (int l = Lt - 1; l >= 0; --l) {
        DevLevel &D = h->lev[l];
        double *u = l == 0 ? x : D.u;
        const double *f = l == 0 ? b : D.f;
        CK(launch_spmv(D.P, 0, D.P.rows, h->lev[l + 1].u, u, 1, st), "interpolation kernel");
        h->launches += 1;
        if ((s = relax(h, l, false, u, f, st)) != AMGDD_OK) return s;
        if ((s = relax(h, l, true, u, f, st)) != AMGDD_OK) return s;
    }
    return AMGDD_OK;
}

amgdd_status amgdd_residual(amgdd_handle h, const double *b, const double *x, double *r, double *nrm2, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x || !r) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    h->last_stream = (cudaStream_t)stream;
    return residual_norm(h, b, x, r, (cudaStream_t)stream, nrm2);
}

amgdd_status amgdd_restrict(amgdd_handle h, double *r_all, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!r_all) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    h->last_stream = (cudaStream_t)stream;
    return restrict_all(h, r_all, (cudaStream_t)stream);
}

amgdd_status amgdd_fac(amgdd_handle h, const double *r_all, double *x, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!r_all || !x) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    h->last_stream = (cudaStream_t)stream;
    return fac(h, r_all, x, (cudaStream_t)stream);
}

amgdd_status amgdd_get_fac_state(amgdd_handle h, int32_t sub, int32_t level, double *u, double *f)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (sub < 0 || sub >= h->C.nsub || level < 0 || level >= h->C.nlev)
        return fail(h, AMGDD_ERR_INVALID_ARG, "subdomain or level out of range");
    const FacLevelDesc &d = h->desc[(size_t)sub * h->C.nlev + level];
    std::vector<double> hu((size_t)d.nBar), hf((size_t)d.nBar);
    cudaStream_t st = h->last_stream;
    CK(cudaStreamSynchronize(st), "sync");
    if (h->fac.fp32) {
        std::vector<float> fu((size_t)d.nBar), ff((size_t)d.nBar);
        CK(cudaMemcpy(fu.data(), static_cast<float *>(h->fac.u) + d.row0, sizeof(float) * (size_t)d.nBar,
                      cudaMemcpyDeviceToHost), "copy u");
        CK(cudaMemcpy(ff.data(), static_cast<float *>(h->fac.f) + d.row0, sizeof(float) * (size_t)d.nBar,
                      cudaMemcpyDeviceToHost), "copy f");
        hu.assign(fu.begin(), fu.end());
        hf.assign(ff.begin(), ff.end());
    } else {
        CK(cudaMemcpy(hu.data(), static_cast<double *>(h->fac.u) + d.row0, sizeof(double) * (size_t)d.nBar,
                      cudaMemcpyDeviceToHost), "copy u");
        CK(cudaMemcpy(hf.data(), static_cast<double *>(h->fac.f) + d.row0, sizeof(double) * (size_t)d.nBar,
                      cudaMemcpyDeviceToHost), "copy f");
    }
    for (int32_t r = 0; r < d.nBar; ++r) {
        const int32_t m = h->dev2map[d.row0 + r];
        if (u) u[m] = hu[r];
        if (f) f[m] = r < d.nReal ? hf[r] : 0.0;
    }
    return AMGDD_OK;
}

amgdd_status amgdd_iterate(amgdd_handle h, const double *b, double *x, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    if ((s = residual_restrict(h, b, x, st)) != AMGDD_OK) return s;
    return fac(h, h->r_all, x, st);
}

amgdd_status amg_vcycle(amgdd_handle h, const double *b, double *x, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    h->last_stream = (cudaStream_t)stream;
    return vcycle(h, b, x, (cudaStream_t)stream);
}

// The whole solve of a method as one graph: |b|^2, the residual of x_0 (and,
// for AMG-DD, its restriction to every level) and the first convergence
// check, then a while node whose body is one iteration (Algorithm 2, or the
// V-cycle, or the hybrid cycle) followed by the residual of the new iterate
// and the check; the check sets the node's condition, so the iterations run
// back to back on the device with no host round trip between them.
static amgdd_status capture_solve(amgdd_handle h, int method, const double *b, double *x, double tol,
                                  int32_t max_iter)
{
    auto &G = h->solve_graph[method];
    if (G.exec && G.b == b && G.x == x && G.tol == tol && G.max_iter == max_iter) return AMGDD_OK;
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G = amgdd_handle_s::SolveGraph();
    }
    if ((int64_t)max_iter + 1 > h->hist_cap) {
        if (h->hist) cudaFree(h->hist);
        if (h->h_hist) cudaFreeHost(h->h_hist);
        h->hist = nullptr;
        h->h_hist = nullptr;
        h->hist_cap = 0;
        const int64_t cap = std::max<int64_t>((int64_t)max_iter + 1, 256);
        CK(dev_malloc((void **)&h->hist, sizeof(double) * (size_t)cap), "alloc solve history");
        CK(cudaMallocHost((void **)&h->h_hist, sizeof(double) * (size_t)cap), "alloc solve history");
        h->hist_cap = cap;
    }
    if (!h->conv) {
        CK(alloc(h, 1, &h->conv), "alloc convergence state");
        CK(cudaMallocHost((void **)&h->h_conv, sizeof(ConvState)), "alloc convergence state");
    }
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (!h->cap_stream2) CK(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking), "capture stream");
    cudaStream_t cs = h->cap_stream, cs2 = h->cap_stream2;
    const bool amgdd = method == 0;
    const int64_t l0 = h->launches;
    amgdd_status s = AMGDD_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle hc = 0;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    auto step = [&](cudaError_t r, const char *what) {
        if (s == AMGDD_OK && r != cudaSuccess) s = cuda_fail(h, r, what);
        return s == AMGDD_OK;
    };
    cudaStreamCaptureStatus cst;
    // the check of the first residual (first = 1) and of every iteration's
    ChainCheck chk{};
    chk.first = 1;
    chk.max_iter = max_iter;
    chk.tol = tol;
    chk.ref2 = h->scal + 1;
    chk.cs = h->conv;
    chk.hist = h->hist;
    bool folded = false;
    if (step(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph), "capture info") &&
        step(cudaGraphConditionalHandleCreate(&hc, graph, 0, 0), "conditional handle")) {
        chk.hc = hc;
        if (step(launch_sumsq(b, h->lev[0].n, h->partial, h->nred, h->scal + 1, cs), "norm kernel")) {
            h->launches += 2;
            if (amgdd) {
                s = residual_restrict(h, b, x, cs, &chk, &folded);
            } else {
                step(launch_residual(h->lev[0].A, b, x, h->r_all, h->partial, h->nred, h->scal, cs),
                     "residual kernel");
                h->launches += 2;
            }
        }
    }
    if (s == AMGDD_OK && !folded &&
        step(launch_converge(hc, h->scal, h->scal + 1, h->conv, h->hist, tol, max_iter, 1, cs), "check kernel"))
        h->launches += 1;
    G.pre_launches = h->launches - l0;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphNode_t wnode = nullptr;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (step(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps), "capture info") &&
        step(cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &cp), "while node") &&
        step(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies),
             "capture dependencies") &&
        step(cudaStreamBeginCaptureToGraph(cs2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal),
             "begin body capture")) {
        const int64_t l1 = h->launches;
        s = amgdd ? fac(h, h->r_all, x, cs2) : method == 1 ? vcycle(h, b, x, cs2) : vcycle_hybrid(h, b, x, cs2);
        chk.first = 0;
        bool folded_body = false;
        if (s == AMGDD_OK && amgdd) s = residual_restrict(h, b, x, cs2, &chk, &folded_body);
        if (s == AMGDD_OK && !amgdd) {
            step(launch_residual(h->lev[0].A, b, x, h->r_all, h->partial, h->nred, h->scal, cs2), "residual kernel");
            h->launches += 2;
        }
        if (s == AMGDD_OK && !folded_body &&
            step(launch_converge(hc, h->scal, h->scal + 1, h->conv, h->hist, tol, max_iter, 0, cs2), "check kernel"))
            h->launches += 1;
        G.body_launches = h->launches - l1;
        cudaGraph_t body = nullptr;
        const cudaError_t eb = cudaStreamEndCapture(cs2, &body);
        step(eb, "end body capture");
    }
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs, &out);
    h->launches = l0;
    if (s != AMGDD_OK) {
        if (out) cudaGraphDestroy(out);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    e = cudaGraphInstantiate(&G.exec, out, 0);
    cudaGraphDestroy(out);
    if (e != cudaSuccess) {
        G = amgdd_handle_s::SolveGraph();
        return cuda_fail(h, e, "graph instantiate");
    }
    G.b = b;
    G.x = x;
    G.tol = tol;
    G.max_iter = max_iter;
    return AMGDD_OK;
}

static amgdd_status solve_loop(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter,
                               cudaStream_t st, amgdd_solve_info *info, int method)
{
    const auto t0 = std::chrono::steady_clock::now();
    amgdd_status s;
    if (max_iter < 0) return fail(h, AMGDD_ERR_INVALID_ARG, "max_iter < 0");
    if ((s = capture_solve(h, method, b, x, tol, max_iter)) != AMGDD_OK) return s;
    const auto &G = h->solve_graph[method];
    CK(cudaGraphLaunch(G.exec, st), "graph launch");
    CK(cudaMemcpyAsync(h->h_conv, h->conv, sizeof(ConvState), cudaMemcpyDeviceToHost, st), "iteration count copy");
    CK(cudaStreamSynchronize(st), "solve");
    const int32_t k = h->h_conv->k;
    if (k < 0 || k > max_iter) return fail(h, AMGDD_ERR_CUDA, "iteration count out of range");
    CK(cudaMemcpyAsync(h->h_hist, h->hist, sizeof(double) * ((size_t)k + 1), cudaMemcpyDeviceToHost, st),
       "history copy");
    CK(cudaStreamSynchronize(st), "history copy");
    const double rel = h->h_hist[k];
    h->launches += G.pre_launches + (int64_t)k * G.body_launches;
    if (info) {
        if (info->history) std::copy(h->h_hist, h->h_hist + k + 1, info->history);
        info->iterations = k;
        info->converged = rel <= tol;
        info->final_relres = rel;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->kernel_launches = G.pre_launches + (int64_t)k * G.body_launches;
    }
    if (!(rel <= tol)) return fail(h, AMGDD_ERR_NO_CONVERGENCE, "max_iter reached before tol");
    return AMGDD_OK;
}

// ---------------------------------------------------------------------------
// Several right-hand sides.

static amgdd_status multi_space(amgdd_handle h, int R, amgdd_handle_s::Multi **out)
{
    auto &m = h->multi[R == 2 ? 0 : 1];
    if (m.R != R) {
        const size_t elt = h->fac.fp32 ? sizeof(float) : sizeof(double);
        for (int k = 0; k < 6; ++k) {
            void *p = nullptr;
            CK(cudaMalloc(&p, std::max<size_t>(1, (size_t)h->fac_rows * R * elt)), "alloc multi work space");
            h->allocs.push_back(p);
            h->dev_bytes += (int64_t)h->fac_rows * R * (int64_t)elt;
            m.ws[k] = p;
        }
        CK(alloc(h, (size_t)h->level_off.back() * R, &m.r_all), "alloc multi residual");
        CK(alloc(h, (size_t)h->nred * R, &m.partial), "alloc multi partial sums");
        CK(alloc(h, (size_t)2 * R, &m.scal), "alloc multi scalars");
        CK(cudaMallocHost((void **)&m.h_scal, sizeof(double) * 2 * R), "alloc multi pinned");
        m.R = R;
    }
    *out = &m;
    return AMGDD_OK;
}

static amgdd_status iterate_multi(amgdd_handle h, amgdd_handle_s::Multi &m, const double *B, double *X, bool fresh_residual,
                                  cudaStream_t st)
{
    const int R = m.R;
    if (fresh_residual) {
        CK(launch_residual_multi(h->lev[0].A, B, X, m.r_all, m.partial, h->nred, m.scal, R, st), "residual kernel");
        h->launches += 2;
    }
    const int nlev = (int)h->lev.size();
    for (int l = 0; l + 1 < nlev; ++l) {
        CK(launch_spmv_multi(h->lev[l].R, m.r_all + h->level_off[l] * R, m.r_all + h->level_off[l + 1] * R, R, st),
           "restriction kernel");
        h->launches += 1;
    }
    FacParams P = h->fac;
    P.u = m.ws[0]; P.f = m.ws[1]; P.t = m.ws[2]; P.s = m.ws[3]; P.w = m.ws[4]; P.d = m.ws[5];
    P.r_all = m.r_all;
    P.x = X;
    CK(launch_candidate(h, P, R, h->fac_cand[R == 2 ? 1 : 2], st), "FAC kernel");
    h->launches += 1;
    return AMGDD_OK;
}

amgdd_status amgdd_iterate_multi(amgdd_handle h, const double *B, double *X, int32_t nrhs, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!B || !X || (nrhs != 2 && nrhs != 4)) return fail(h, AMGDD_ERR_INVALID_ARG, "nrhs must be 2 or 4");
    amgdd_handle_s::Multi *m;
    if ((s = multi_space(h, nrhs, &m)) != AMGDD_OK) return s;
    h->last_stream = (cudaStream_t)stream;
    return iterate_multi(h, *m, B, X, true, (cudaStream_t)stream);
}

amgdd_status amgdd_fac_multi(amgdd_handle h, const double *R_all, double *X, int32_t nrhs, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!R_all || !X || (nrhs != 2 && nrhs != 4)) return fail(h, AMGDD_ERR_INVALID_ARG, "nrhs must be 2 or 4");
    amgdd_handle_s::Multi *m;
    if ((s = multi_space(h, nrhs, &m)) != AMGDD_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    FacParams P = h->fac;
    P.u = m->ws[0]; P.f = m->ws[1]; P.t = m->ws[2]; P.s = m->ws[3]; P.w = m->ws[4]; P.d = m->ws[5];
    P.r_all = R_all;
    P.x = X;
    CK(launch_candidate(h, P, nrhs, h->fac_cand[nrhs == 2 ? 1 : 2], st), "FAC kernel");
    h->launches += 1;
    return AMGDD_OK;
}

amgdd_status amgdd_solve_multi(amgdd_handle h, const double *B, double *X, int32_t nrhs, double tol, int32_t max_iter,
                               void *stream, amgdd_solve_info *info)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!B || !X || (nrhs != 2 && nrhs != 4) || max_iter < 0 || !(tol >= 0.0))
        return fail(h, AMGDD_ERR_INVALID_ARG, "bad multi-column solve arguments");
    amgdd_handle_s::Multi *mp;
    if ((s = multi_space(h, nrhs, &mp)) != AMGDD_OK) return s;
    auto &m = *mp;
    const int R = nrhs;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = h->launches;
    // one iteration = restriction + FAC + residual of the new iterate + the
    // copy of the squared column norms, captured once per (B, X)
    if (!(m.graph.exec && m.graph.b == B && m.graph.x == X)) {
        if (m.graph.exec) {
            cudaGraphExecDestroy(m.graph.exec);
            m.graph.exec = nullptr;
        }
        if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
        const int64_t c0 = h->launches;
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        amgdd_status cs = iterate_multi(h, m, B, X, false, h->cap_stream);
        if (cs == AMGDD_OK) {
            cudaError_t e = launch_residual_multi(h->lev[0].A, B, X, m.r_all, m.partial, h->nred, m.scal, R,
                                                  h->cap_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(m.h_scal, m.scal, sizeof(double) * R, cudaMemcpyDeviceToHost, h->cap_stream);
            h->launches += 2;
            if (e != cudaSuccess) cs = cuda_fail(h, e, "capture residual");
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (cs != AMGDD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cs;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
        e = cudaGraphInstantiate(&m.graph.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
        m.graph.b = B;
        m.graph.x = X;
        m.graph.launches = h->launches - c0;
        h->launches = c0;
    }
    CK(launch_sumsq_multi(B, h->lev[0].n, m.partial, h->nred, m.scal + R, R, st), "norm kernel");
    CK(launch_residual_multi(h->lev[0].A, B, X, m.r_all, m.partial, h->nred, m.scal, R, st), "residual kernel");
    h->launches += 4;
    CK(cudaMemcpyAsync(m.h_scal, m.scal, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st), "norm copy");
    CK(cudaStreamSynchronize(st), "residual");
    double ref[4], rel[4];
    for (int j = 0; j < R; ++j) ref[j] = std::sqrt(m.h_scal[R + j]);
    int32_t k = 0;
    double worst = 0.0;
    for (;;) {
        worst = 0.0;
        for (int j = 0; j < R; ++j) {
            const double nr = std::sqrt(m.h_scal[j]);
            if (k == 0 && ref[j] == 0.0) ref[j] = nr;
            rel[j] = ref[j] > 0.0 ? nr / ref[j] : 0.0;
            if (info && info->history) info->history[(size_t)j * (max_iter + 1) + k] = rel[j];
            worst = std::max(worst, rel[j]);
        }
        if (worst <= tol || k >= max_iter) break;
        CK(cudaGraphLaunch(m.graph.exec, st), "graph launch");
        CK(cudaStreamSynchronize(st), "iteration");
        h->launches += m.graph.launches;
        ++k;
    }
    if (info) {
        info->iterations = k;
        info->converged = worst <= tol;
        info->final_relres = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->kernel_launches = h->launches - l0;
    }
    if (!(worst <= tol)) return fail(h, AMGDD_ERR_NO_CONVERGENCE, "max_iter reached before tol");
    return AMGDD_OK;
}

amgdd_status amgdd_solve(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter, void *stream,
                         amgdd_solve_info *info)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x || max_iter < 0 || !(tol >= 0.0)) return fail(h, AMGDD_ERR_INVALID_ARG, "bad solve arguments");
    h->last_stream = (cudaStream_t)stream;
    return solve_loop(h, b, x, tol, max_iter, (cudaStream_t)stream, info, 0);
}

amgdd_status amg_vcycle_solve(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter,
                              void *stream, amgdd_solve_info *info)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x || max_iter < 0 || !(tol >= 0.0)) return fail(h, AMGDD_ERR_INVALID_ARG, "bad solve arguments");
    h->last_stream = (cudaStream_t)stream;
    return solve_loop(h, b, x, tol, max_iter, (cudaStream_t)stream, info, 1);
}

amgdd_status amg_hybrid_cycle(amgdd_handle h, const double *b, double *x, void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x) return fail(h, AMGDD_ERR_INVALID_ARG, "null vector");
    if (h->hyb_level < 0) return fail(h, AMGDD_ERR_INVALID_ARG, "handle was set up without hybrid_level");
    h->last_stream = (cudaStream_t)stream;
    return vcycle_hybrid(h, b, x, (cudaStream_t)stream);
}

amgdd_status amg_hybrid_solve(amgdd_handle h, const double *b, double *x, double tol, int32_t max_iter,
                              void *stream, amgdd_solve_info *info)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (!b || !x || max_iter < 0 || !(tol >= 0.0)) return fail(h, AMGDD_ERR_INVALID_ARG, "bad solve arguments");
    if (h->hyb_level < 0) return fail(h, AMGDD_ERR_INVALID_ARG, "handle was set up without hybrid_level");
    h->last_stream = (cudaStream_t)stream;
    return solve_loop(h, b, x, tol, max_iter, (cudaStream_t)stream, info, 2);
}

// ---------------------------------------------------------------------------
// FAC kernel choice.

// Candidate k of amgdd_autotune / amgdd_set_fac_kernel: k < 9 is the
// single-column kernel with schedule k + 1 (one column only; FP32 composite
// grids have schedules 1 and 8), 9 <= k < 18 the several-column kernel's
// variant k - 8, 18 and 19 its group-per-row variant (lanes per row by level
// size, or 32 on every level), whose row sums are not the ascending chain,
// 20-24 its variants 11-15 (L1 prefetch, shared-memory staging), 25 its
// variant 7 with every grid in one queue (largest first) instead of per-SM
// bins, 26 and 27 the kernel that keeps each grid's work vectors in shared
// memory (two entries in flight and two blocks per SM, or four and one) on
// that queue, 28-30 the kernel that cycles each grid with a cluster of 2, 4
// or 8 blocks, on that queue, 31 variant 7 in work-sized teams of warps
// (blocks of 1024 threads).
static bool candidate_applies(amgdd_handle h, int nrhs, int k)
{
    if (k < 0 || k >= AMGDD_FAC_CANDIDATES) return false;
    if (k < 9) return nrhs == 1 && (!h->fac.fp32 || k == 0 || k == 7);
    if (k >= 18) return h->fac.col16 != 0;
    return true;
}

static bool candidate_reorders(int k) { return k == 18 || k == 19; }

static void drop_graphs(amgdd_handle h)
{
    for (auto &g : h->solve_graph)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g = amgdd_handle_s::SolveGraph();
        }
    for (auto &m : h->multi)
        if (m.graph.exec) {
            cudaGraphExecDestroy(m.graph.exec);
            m.graph = amgdd_handle_s::Graph();
        }
}

static void apply_candidate(amgdd_handle h, int nrhs, int k)
{
    h->fac_cand[nrhs == 1 ? 0 : nrhs == 2 ? 1 : 2] = k;
}

amgdd_status amgdd_set_fac_kernel(amgdd_handle h, int32_t nrhs, int32_t candidate)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (nrhs != 1 && nrhs != 2 && nrhs != 4) return fail(h, AMGDD_ERR_INVALID_ARG, "nrhs must be 1, 2 or 4");
    if (!candidate_applies(h, nrhs, candidate))
        return fail(h, AMGDD_ERR_INVALID_ARG, "candidate does not apply to this handle and column count");
    CK(cudaStreamSynchronize(h->last_stream), "sync");
    drop_graphs(h);
    apply_candidate(h, nrhs, candidate);
    return AMGDD_OK;
}

amgdd_status amgdd_autotune(amgdd_handle h, int32_t nrhs, int32_t reps, int32_t flags, double *ms, int32_t *best,
                            void *stream)
{
    amgdd_status s = require_device(h);
    if (s != AMGDD_OK) return s;
    if (nrhs != 1 && nrhs != 2 && nrhs != 4) return fail(h, AMGDD_ERR_INVALID_ARG, "nrhs must be 1, 2 or 4");
    if (reps < 1) return fail(h, AMGDD_ERR_INVALID_ARG, "reps must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    // inputs: zero restricted residuals; output: a scratch x
    FacParams P = h->fac;
    double *r_all = h->r_all;
    if (nrhs > 1) {
        amgdd_handle_s::Multi *m;
        if ((s = multi_space(h, nrhs, &m)) != AMGDD_OK) return s;
        P.u = m->ws[0]; P.f = m->ws[1]; P.t = m->ws[2]; P.s = m->ws[3]; P.w = m->ws[4]; P.d = m->ws[5];
        r_all = m->r_all;
    }
    CK(cudaMemsetAsync(r_all, 0, sizeof(double) * (size_t)h->level_off.back() * nrhs, st), "clear residuals");
    double *xs = nullptr;
    CK(cudaMalloc(&xs, sizeof(double) * (size_t)h->lev[0].n * nrhs), "alloc scratch x");
    P.r_all = r_all;
    P.x = xs;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int bk = -1;
    double bms = 0.0;
    double times[AMGDD_FAC_CANDIDATES];
    for (double &t : times) t = -1.0;
    for (int k = 0; k < AMGDD_FAC_CANDIDATES && e == cudaSuccess; ++k) {
        if (ms) ms[k] = -1.0;
        if (!candidate_applies(h, nrhs, k)) continue;
        if (candidate_reorders(k) && !(flags & AMGDD_TUNE_ALLOW_REORDERED)) continue;
        auto launch = [&]() -> cudaError_t { return launch_candidate(h, P, nrhs, k, st); };
        if ((e = launch()) != cudaSuccess) {                // warm-up
            // a cluster shape this device cannot schedule is refused before
            // anything runs: that candidate does not apply here
            if (k >= 28 && (e == cudaErrorInvalidConfiguration || e == cudaErrorInvalidClusterSize ||
                            e == cudaErrorLaunchOutOfResources)) {
                cudaGetLastError();
                e = cudaSuccess;
                continue;
            }
            break;
        }
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
        const double per = (double)t / reps;
        if (ms) ms[k] = per;
        times[k] = per;
        if (bk < 0 || per < bms) {
            bk = k;
            bms = per;
        }
        h->launches += 1 + reps;
    }
    // candidates within 1 % of the fastest are ties: keep the lowest-numbered,
    // so repeated tuning of the same workload settles on the same kernel
    if (e == cudaSuccess && bk >= 0)
        for (int k = 0; k < bk; ++k)
            if (times[k] >= 0.0 && times[k] <= 1.01 * bms) {
                bk = k;
                break;
            }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(xs);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    drop_graphs(h);
    apply_candidate(h, nrhs, bk);
    if (best) *best = bk;
    return AMGDD_OK;
}

}  // extern "C"

