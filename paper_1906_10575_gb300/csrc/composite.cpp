// Composite grids of the virtual subdomains (Section 3, Fig. 1; eq. (1)) and
// their packing into the device layouts used by the solve-phase kernels.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>

#include "amgdd_internal.hpp"

namespace amgdd {
namespace {

template <class F>
void parallel_for(int n, int nthreads, F &&fn)
{
    if (nthreads <= 1 || n <= 1) {
        for (int i = 0; i < n; ++i) fn(i, 0);
        return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    int nt = std::min(nthreads, n);
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
            for (;;) {
                int i = next.fetch_add(1);
                if (i >= n) break;
                fn(i, t);
            }
        });
    for (auto &th : pool) th.join();
}

// Points within graph distance eta of `seeds` in graph(A) (structural
// entries), returned ascending. `level` is a scratch array of -1s.
std::vector<int32_t> ball(const Csr &A, const std::vector<int32_t> &seeds, int eta,
                          std::vector<int32_t> &level)
{
    std::vector<int32_t> out;
    out.reserve(seeds.size() * 2);
    for (int32_t s : seeds)
        if (level[s] < 0) { level[s] = 0; out.push_back(s); }
    size_t begin = 0;
    for (int d = 0; d < eta; ++d) {
        const size_t end = out.size();
        for (size_t h = begin; h < end; ++h) {
            const int32_t i = out[h];
            for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                const int32_t j = A.idx[k];
                if (level[j] < 0) { level[j] = d + 1; out.push_back(j); }
            }
        }
        begin = end;
    }
    for (int32_t i : out) level[i] = -1;
    std::sort(out.begin(), out.end());
    return out;
}

// Neighbours of the sorted set D that are not in D, ascending.
std::vector<int32_t> halo(const Csr &A, const std::vector<int32_t> &D, std::vector<uint8_t> &flag)
{
    std::vector<int32_t> out;
    for (int32_t i : D) flag[i] = 1;
    for (int32_t i : D)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int32_t j = A.idx[k];
            if (!flag[j]) { flag[j] = 2; out.push_back(j); }
        }
    for (int32_t i : D) flag[i] = 0;
    for (int32_t i : out) flag[i] = 0;
    std::sort(out.begin(), out.end());
    return out;
}

}  // namespace

void build_composite(const Hierarchy &H, const int32_t *part, int nsub, const std::vector<int> &eta,
                     Composite &C, int nthreads)
{
    const int L = H.L();
    C.nsub = nsub;
    C.nlev = L + 1;
    C.g.assign((size_t)nsub * (L + 1), CompLevel{});
    const int32_t n0 = H.lv[0].A.rows;
    std::vector<std::vector<int32_t>> own((size_t)nsub);
    for (int32_t i = 0; i < n0; ++i) own[part[i]].push_back(i);
    int32_t nmax = 0;
    for (const auto &lv : H.lv) nmax = std::max(nmax, lv.A.rows);
    std::vector<std::vector<int32_t>> scratch_lvl((size_t)std::max(nthreads, 1));
    std::vector<std::vector<uint8_t>> scratch_flag((size_t)std::max(nthreads, 1));
    parallel_for(nsub, nthreads, [&](int p, int t) {
        auto &lvl = scratch_lvl[t];
        auto &flag = scratch_flag[t];
        if ((int32_t)lvl.size() < nmax) { lvl.assign((size_t)nmax, -1); flag.assign((size_t)nmax, 0); }
        std::vector<int32_t> seeds = own[p];
        std::vector<int32_t> owned = own[p];
        for (int l = 0; l <= L; ++l) {
            CompLevel &cl = C.at(p, l);
            cl.owned = owned;
            if (l < L) {
                cl.real = ball(H.lv[l].A, seeds, eta[l], lvl);
                cl.ghost = halo(H.lv[l].A, cl.real, flag);
                // the C points of D_l and of the owned set seed level l+1
                std::vector<int32_t> ns, no;
                for (int32_t i : cl.real)
                    if (H.lv[l].isC[i]) ns.push_back(H.lv[l].coarse[i]);
                for (int32_t i : owned)
                    if (H.lv[l].isC[i]) no.push_back(H.lv[l].coarse[i]);
                seeds.swap(ns);
                owned.swap(no);
            } else {
                cl.real.resize((size_t)H.lv[l].A.rows);
                std::iota(cl.real.begin(), cl.real.end(), 0);
                cl.ghost.clear();
            }
        }
    });

    // Connectivity assumption (Sections 4.2 and 4.5): a level-(l+1) point that
    // Dbar_l reaches through P_l (the columns of R_l = P_l^T) but that lies
    // outside Dbar_{l+1} must reach no real point of any coarser level through
    // the interpolation stencils; otherwise dropping it changes the cycle.
    std::vector<int64_t> bad((size_t)nsub, 0);
    parallel_for(nsub, nthreads, [&](int p, int t) {
        auto &flag = scratch_flag[t];
        if ((int32_t)flag.size() < nmax) flag.assign((size_t)nmax, 0);
        for (int l = 0; l < L; ++l) {
            const CompLevel &a = C.at(p, l);
            const CompLevel &b = C.at(p, l + 1);
            for (int32_t i : b.real) flag[i] = 1;
            for (int32_t i : b.ghost) flag[i] = 1;
            std::vector<int32_t> front;
            const Csr &P = H.lv[l].P;
            for (const auto *set : {&a.real, &a.ghost})
                for (int32_t i : *set)
                    for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k)
                        if (!flag[P.idx[k]]) { flag[P.idx[k]] = 2; front.push_back(P.idx[k]); }
            for (int32_t i : b.real) flag[i] = 0;
            for (int32_t i : b.ghost) flag[i] = 0;
            for (int32_t i : front) flag[i] = 0;
            bool violated = false;
            for (int m = l + 1; m <= L && !front.empty() && !violated; ++m) {
                const CompLevel &cm = C.at(p, m);
                for (int32_t i : cm.real) flag[i] = 1;
                for (int32_t i : front) if (flag[i] == 1) { violated = true; break; }
                for (int32_t i : cm.real) flag[i] = 0;
                if (violated || m == L) break;
                std::vector<int32_t> nxt;
                const Csr &Pm = H.lv[m].P;
                for (int32_t i : front)
                    for (int64_t k = Pm.ptr[i]; k < Pm.ptr[i + 1]; ++k)
                        if (!flag[Pm.idx[k]]) { flag[Pm.idx[k]] = 3; nxt.push_back(Pm.idx[k]); }
                for (int32_t i : nxt) flag[i] = 0;
                front.swap(nxt);
            }
            bad[p] += violated ? 1 : 0;
        }
    });
    C.violations = std::accumulate(bad.begin(), bad.end(), (int64_t)0);
}

// ---------------------------------------------------------------------------

namespace {

// Append rows (each a list of (column, value) in ascending global column
// order) as SELL-32 slices.
struct RowList {
    std::vector<int64_t> ptr{0};
    std::vector<int32_t> col;
    std::vector<double> val;
    void add_entry(int32_t c, double v) { col.push_back(c); val.push_back(v); }
    void end_row() { ptr.push_back((int64_t)col.size()); }
    int32_t rows() const { return (int32_t)ptr.size() - 1; }
};

void append_sell(const RowList &rl, std::vector<int64_t> &soff, std::vector<uint16_t> &rlen,
                 std::vector<int32_t> &col, std::vector<double> &val)
{
    const int32_t n = rl.rows();
    for (int32_t s = 0; s * 32 < n; ++s) {
        int64_t width = 0;
        for (int32_t r = s * 32; r < std::min(n, s * 32 + 32); ++r)
            width = std::max(width, rl.ptr[r + 1] - rl.ptr[r]);
        const int64_t base = (int64_t)col.size();
        soff.push_back(base);
        col.resize((size_t)(base + 32 * width), 0);
        val.resize((size_t)(base + 32 * width), 0.0);
        for (int32_t r = s * 32; r < std::min(n, s * 32 + 32); ++r) {
            const int lane = r - s * 32;
            for (int64_t k = rl.ptr[r]; k < rl.ptr[r + 1]; ++k) {
                col[(size_t)(base + 32 * (k - rl.ptr[r]) + lane)] = rl.col[k];
                val[(size_t)(base + 32 * (k - rl.ptr[r]) + lane)] = rl.val[k];
            }
        }
    }
    for (int32_t r = 0; r < n; ++r) rlen.push_back((uint16_t)(rl.ptr[r + 1] - rl.ptr[r]));
}

void finish_sell(Sell &S, const RowList &rl)
{
    S.rows = rl.rows();
    S.soff.clear();
    append_sell(rl, S.soff, S.rlen, S.col, S.val);
    S.soff.push_back((int64_t)S.col.size());
}

}  // namespace

void build_global_dev(const Hierarchy &H, std::vector<GlobalLevelDev> &G)
{
    const int L = H.L();
    G.assign((size_t)L + 1, GlobalLevelDev{});
    for (int l = 0; l <= L; ++l) {
        const HLevel &lv = H.lv[l];
        GlobalLevelDev &g = G[l];
        g.rowid.clear();
        if (l < L) {
            for (int32_t i = 0; i < lv.A.rows; ++i) if (lv.isC[i]) g.rowid.push_back(i);
            g.nC = (int32_t)g.rowid.size();
            for (int32_t i = 0; i < lv.A.rows; ++i) if (!lv.isC[i]) g.rowid.push_back(i);
        } else {
            g.rowid.resize((size_t)lv.A.rows);
            std::iota(g.rowid.begin(), g.rowid.end(), 0);
            g.nC = 0;
        }
        RowList ra;
        for (int32_t i : g.rowid) {
            for (int64_t k = lv.A.ptr[i]; k < lv.A.ptr[i + 1]; ++k) ra.add_entry(lv.A.idx[k], lv.A.val[k]);
            ra.end_row();
        }
        finish_sell(g.A, ra);
        if (l < L) {
            RowList rp, rr;
            for (int32_t i = 0; i < lv.P.rows; ++i) {
                for (int64_t k = lv.P.ptr[i]; k < lv.P.ptr[i + 1]; ++k) rp.add_entry(lv.P.idx[k], lv.P.val[k]);
                rp.end_row();
            }
            for (int32_t I = 0; I < lv.R.rows; ++I) {
                for (int64_t k = lv.R.ptr[I]; k < lv.R.ptr[I + 1]; ++k) rr.add_entry(lv.R.idx[k], lv.R.val[k]);
                rr.end_row();
            }
            finish_sell(g.P, rp);
            finish_sell(g.R, rr);
        }
    }
}

// Device order of a composite level: [real C | real F | ghost] for l < L, each
// group by decreasing row length of A_l (real rows: full length; ghost rows:
// real columns only) and then ascending global index; the coarsest level is
// whole and keeps ascending global order.
//
// Views per level (all entries of a row in ascending global column order, so
// every row product is the same fma chain as over the full global row: the
// entries a view omits multiply values that are exactly zero at that point of
// Algorithm 4):
//   A   : real rows, all columns            (smoothing, coarse recomputation)
//   At  : all rows, real columns only       (s_l + A_l t_l; t_l = 0 off D_l)
//   AFc : real F rows, real C columns only  (downsweep F half-sweep on l >= 1,
//                                            where u_l = 0 except at C points)
//   P   : rows Dbar_l, columns in Dbar_{l+1}
//   R   : R_{l-1} rows Dbar_l, columns in Dbar_{l-1}
namespace {

struct GridBuild {
    std::vector<std::vector<int32_t>> dev;
    std::vector<int32_t> nC, nReal;
    RowList A[kMaxLevels], At[kMaxLevels], AFc[kMaxLevels], P[kMaxLevels], R[kMaxLevels];
    std::vector<int32_t> owned_local;
    std::vector<std::vector<int32_t>> d2m;
    int64_t work = 0, work1 = 0;
};

void emit_view(RowList &rl, int32_t first_row, int32_t rows_total_level, FacView &V)
{
    // rows of the view are local rows [first_row, first_row + rl.rows());
    // rlen is written for every local row of the level (zero outside the view)
    const int32_t n = rl.rows();
    for (int32_t s = 0; s * 32 < n; ++s) {
        int64_t width = 0;
        for (int32_t r = s * 32; r < std::min(n, s * 32 + 32); ++r) width = std::max(width, rl.ptr[r + 1] - rl.ptr[r]);
        const int64_t base = (int64_t)V.size();   // held entries; soff is absolute
        const size_t end = (size_t)(base + 32 * width);
        V.soff.push_back(V.base + base);
        if (V.c16) V.col16.resize(end, 0); else V.col32.resize(end, 0);
        if (V.v32) V.val32.resize(end, 0.0f); else V.val64.resize(end, 0.0);
        for (int32_t r = s * 32; r < std::min(n, s * 32 + 32); ++r) {
            const int lane = r - s * 32;
            for (int64_t k = rl.ptr[r]; k < rl.ptr[r + 1]; ++k) {
                const size_t o = (size_t)(base + 32 * (k - rl.ptr[r]) + lane);
                if (V.c16) V.col16[o] = (uint16_t)rl.col[k]; else V.col32[o] = rl.col[k];
                if (V.v32) V.val32[o] = (float)rl.val[k]; else V.val64[o] = rl.val[k];
            }
        }
    }
    V.soff.push_back(V.total());
    for (int32_t r = 0; r < rows_total_level; ++r) {
        const int32_t v = r - first_row;
        V.rlen.push_back(v >= 0 && v < n ? (uint16_t)(rl.ptr[v + 1] - rl.ptr[v]) : (uint16_t)0);
    }
    V.entries += rl.ptr.back();
    rl = RowList();
}

}  // namespace

std::string build_fac_layout(const Hierarchy &H, const Composite &C, FacLayout &F, int nthreads, bool fp32,
                             const FacSink &sink)
{
    const int L = H.L();
    const int nlev = L + 1;
    const int nsub = C.nsub;
    F.nlev = nlev;
    F.nsub = nsub;
    F.desc.assign((size_t)nsub * nlev, FacLevelDesc{});
    // column width and value type are fixed before packing
    int64_t maxbar = 0;
    for (const CompLevel &cl : C.g) maxbar = std::max<int64_t>(maxbar, (int64_t)(cl.real.size() + cl.ghost.size()));
    for (FacView *V : {&F.A, &F.At, &F.AFc, &F.P, &F.R}) {
        V->c16 = maxbar < 65536;
        V->v32 = fp32;
    }
    // grids are built in chunks (in parallel) and packed (in order) before
    // the next chunk, so only one chunk's row lists exist at a time
    const int chunk = std::max(64, 4 * std::max(nthreads, 1));
    std::vector<GridBuild> grids((size_t)std::min(chunk, std::max(nsub, 1)));
    int32_t nmax = 0;
    for (const auto &lv : H.lv) nmax = std::max(nmax, lv.A.rows);
    const int nt = std::max(nthreads, 1);
    std::vector<std::vector<int32_t>> g2l_s((size_t)nt), g2l_n((size_t)nt), g2l_p((size_t)nt);
    std::vector<std::vector<uint8_t>> realf((size_t)nt), cflag((size_t)nt);

    F.gmap.clear();
    F.owned.clear();
    F.owned0.assign((size_t)nsub + 1, 0);
    F.work.assign((size_t)nsub, 0);
    F.work1.assign((size_t)nsub, 0);
    F.lvA.assign(nlev, 0); F.lvAt.assign(nlev, 0); F.lvAFc.assign(nlev, 0);
    F.lvP.assign(nlev, 0); F.lvR.assign(nlev, 0);
    int64_t row0 = 0;
    for (int p0 = 0; p0 < nsub; p0 += chunk) {
    const int pn = std::min(chunk, nsub - p0);
    parallel_for(pn, nthreads, [&](int pi, int t) {
        const int p = p0 + pi;
        GridBuild &G = grids[pi];
        G = GridBuild();
        G.dev.resize(nlev);
        G.nC.assign(nlev, 0);
        G.nReal.assign(nlev, 0);
        G.d2m.resize(nlev);
        auto &g2l = g2l_s[t];
        auto &g2ln = g2l_n[t];
        auto &g2lp = g2l_p[t];
        auto &isreal = realf[t];
        auto &isC = cflag[t];
        if ((int32_t)g2l.size() < nmax) {
            g2l.assign((size_t)nmax, -1);
            g2ln.assign((size_t)nmax, -1);
            g2lp.assign((size_t)nmax, -1);
            isreal.assign((size_t)nmax, 0);
            isC.assign((size_t)nmax, 0);
        }
        for (int l = 0; l <= L; ++l) {
            const CompLevel &cl = C.at(p, l);
            const Csr &A = H.lv[l].A;
            std::vector<int32_t> &dev = G.dev[l];
            dev.clear();
            if (l == L) {
                dev = cl.real;
                G.nC[l] = 0;
                G.nReal[l] = (int32_t)cl.real.size();
            } else {
                for (int32_t i : cl.real) isreal[i] = 1;
                auto arow_len = [&](int32_t i) -> int64_t {
                    if (isreal[i]) return A.ptr[i + 1] - A.ptr[i];
                    int64_t c = 0;
                    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) c += isreal[A.idx[k]];
                    return c;
                };
                std::vector<std::pair<int64_t, int32_t>> cset, fset, gset;
                for (int32_t i : cl.real) (H.lv[l].isC[i] ? cset : fset).emplace_back(-arow_len(i), i);
                for (int32_t i : cl.ghost) gset.emplace_back(-arow_len(i), i);
                std::sort(cset.begin(), cset.end());
                std::sort(fset.begin(), fset.end());
                std::sort(gset.begin(), gset.end());
                for (auto &e : cset) dev.push_back(e.second);
                for (auto &e : fset) dev.push_back(e.second);
                for (auto &e : gset) dev.push_back(e.second);
                G.nC[l] = (int32_t)cset.size();
                G.nReal[l] = (int32_t)(cset.size() + fset.size());
                for (int32_t i : cl.real) isreal[i] = 0;
            }
            // device -> map order (owned asc, other real asc, ghost asc)
            std::vector<int32_t> mapord = cl.owned;
            {
                size_t a = 0;
                for (int32_t i : cl.real) {
                    while (a < cl.owned.size() && cl.owned[a] < i) ++a;
                    if (a < cl.owned.size() && cl.owned[a] == i) continue;
                    mapord.push_back(i);
                }
                mapord.insert(mapord.end(), cl.ghost.begin(), cl.ghost.end());
            }
            for (size_t k = 0; k < mapord.size(); ++k) g2l[mapord[k]] = (int32_t)k;
            G.d2m[l].resize(dev.size());
            for (size_t k = 0; k < dev.size(); ++k) G.d2m[l][k] = g2l[dev[k]];
            for (int32_t i : mapord) g2l[i] = -1;
        }
        for (int l = 0; l <= L; ++l) {
            const Csr &A = H.lv[l].A;
            const std::vector<int32_t> &dev = G.dev[l];
            for (size_t k = 0; k < dev.size(); ++k) g2l[dev[k]] = (int32_t)k;
            const int32_t nReal = G.nReal[l], nC = G.nC[l];
            for (size_t r = 0; r < dev.size(); ++r) {
                const int32_t i = dev[r];
                const bool realrow = (int32_t)r < nReal;
                const bool frow = realrow && (int32_t)r >= nC;
                for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                    const int32_t lc = g2l[A.idx[k]];
                    if (realrow) G.A[l].add_entry(lc, A.val[k]);
                    if (lc >= 0 && lc < nReal) G.At[l].add_entry(lc, A.val[k]);
                    if (frow && lc >= 0 && lc < nC) G.AFc[l].add_entry(lc, A.val[k]);
                }
                if (realrow) G.A[l].end_row();
                G.At[l].end_row();
                if (frow) G.AFc[l].end_row();
            }
            if (l < L) {
                const Csr &P = H.lv[l].P;
                const std::vector<int32_t> &devn = G.dev[l + 1];
                for (size_t k = 0; k < devn.size(); ++k) g2ln[devn[k]] = (int32_t)k;
                for (size_t r = 0; r < dev.size(); ++r) {
                    const int32_t i = dev[r];
                    for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
                        const int32_t lc = g2ln[P.idx[k]];
                        if (lc >= 0) G.P[l].add_entry(lc, P.val[k]);
                    }
                    G.P[l].end_row();
                }
                for (size_t k = 0; k < devn.size(); ++k) g2ln[devn[k]] = -1;
            }
            if (l > 0) {
                const Csr &R = H.lv[l - 1].R;
                const std::vector<int32_t> &devp = G.dev[l - 1];
                for (size_t k = 0; k < devp.size(); ++k) g2lp[devp[k]] = (int32_t)k;
                for (size_t r = 0; r < dev.size(); ++r) {
                    const int32_t I = dev[r];
                    for (int64_t k = R.ptr[I]; k < R.ptr[I + 1]; ++k) {
                        const int32_t lc = g2lp[R.idx[k]];
                        if (lc >= 0) G.R[l].add_entry(lc, R.val[k]);
                    }
                    G.R[l].end_row();
                }
                for (size_t k = 0; k < devp.size(); ++k) g2lp[devp[k]] = -1;
            }
            if (l == 0)
                for (int32_t i : C.at(p, 0).owned) G.owned_local.push_back(g2l[i]);
            for (size_t k = 0; k < dev.size(); ++k) g2l[dev[k]] = -1;
        }
        // FMAs of one cycle after the first (the coarse recomputation included)
        // executed fma: downsweep half-sweeps (full rows on level 0, C columns
        // of the F rows above it), s + A t, R, the upsweep P and half-sweeps,
        // the coarse recomputation (not in the first cycle) and the dense
        // coarsest product
        const int64_t nL = (int64_t)G.dev[L].size();
        for (int l = 0; l < L; ++l) {
            const int64_t a = G.A[l].ptr.back(), at = G.At[l].ptr.back(), afc = G.AFc[l].ptr.back();
            const int64_t base = (l == 0 ? a : afc) + a + at + G.P[l].ptr.back() + G.R[l + 1].ptr.back();
            G.work1 += base;
            G.work += base + G.A[l + 1].ptr.back();
        }
        G.work1 += nL * nL;
        G.work += nL * nL;
    });

    for (int pi = 0; pi < pn; ++pi) {
        const int p = p0 + pi;
        GridBuild &G = grids[pi];
        for (int l = 0; l <= L; ++l) {
            FacLevelDesc &d = F.desc[(size_t)p * nlev + l];
            const int32_t nbar = (int32_t)G.dev[l].size();
            d.nC = G.nC[l];
            d.nReal = G.nReal[l];
            d.nBar = nbar;
            d.row0 = row0;
            F.max_bar = std::max(F.max_bar, nbar);
            const HLevel &lv = H.lv[l];
            for (int32_t i : G.dev[l]) {
                F.gmap.push_back(i);
                F.l1inv.push_back(lv.l1inv[i]);
            }
            F.dev2map.insert(F.dev2map.end(), G.d2m[l].begin(), G.d2m[l].end());
            F.lvA[l] += G.A[l].ptr.back();
            F.lvAt[l] += G.At[l].ptr.back();
            F.lvAFc[l] += G.AFc[l].ptr.back();
            F.lvP[l] += G.P[l].ptr.back();
            F.lvR[l] += G.R[l].ptr.back();
            d.sA = F.A.sbase + (int64_t)F.A.soff.size();
            emit_view(G.A[l], 0, nbar, F.A);
            d.sAt = F.At.sbase + (int64_t)F.At.soff.size();
            emit_view(G.At[l], 0, nbar, F.At);
            d.sAFc = F.AFc.sbase + (int64_t)F.AFc.soff.size();
            emit_view(G.AFc[l], d.nC, nbar, F.AFc);
            d.sP = F.P.sbase + (int64_t)F.P.soff.size();
            emit_view(G.P[l], 0, nbar, F.P);
            d.sR = F.R.sbase + (int64_t)F.R.soff.size();
            emit_view(G.R[l], 0, nbar, F.R);
            row0 += nbar;
        }
        F.owned.insert(F.owned.end(), G.owned_local.begin(), G.owned_local.end());
        F.owned0[p + 1] = (int64_t)F.owned.size();
        F.work[p] = G.work;
        F.work1[p] = G.work1;
        G = GridBuild();
    }
    F.rows_total = row0;
    if (sink) {
        const std::string e = sink(F, p0, pn);
        if (!e.empty()) return e;
    }
    }
    F.rows_total = row0;
    F.order.resize((size_t)nsub);
    std::iota(F.order.begin(), F.order.end(), 0);
    std::stable_sort(F.order.begin(), F.order.end(),
                     [&](int32_t a, int32_t b) { return F.work[a] > F.work[b]; });
    return "";
}

}  // namespace amgdd

namespace amgdd {

namespace {

// Checks one SELL block: slices cover exactly `rows` rows, every row length
// fits its slice width, and every stored column lies in [0, ncols). Slice
// offsets are absolute; `lo` is the first entry still held and `hi` one past
// the last, and colat takes an absolute entry index.
template <class ColAt>
std::string check_sell_g(const std::vector<int64_t> &soff, int64_t s0, const std::vector<uint16_t> &rlen, int64_t r0,
                         int64_t rows, int64_t lo, int64_t hi, ColAt colat, int64_t ncols, const char *what)
{
    const int64_t nsl = (rows + 31) / 32;
    if (s0 < 0 || r0 < 0) return std::string(what) + ": slices or rows no longer held";
    if (s0 + nsl >= (int64_t)soff.size() + (rows == 0 ? 1 : 0)) return std::string(what) + ": slice table too short";
    for (int64_t q = 0; q < nsl; ++q) {
        const int64_t a = soff[s0 + q], b = soff[s0 + q + 1];
        if (a < lo || b < a || b > hi || (b - a) % 32) return std::string(what) + ": bad slice offsets";
        const int64_t width = (b - a) / 32;
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t r = q * 32 + lane;
            if (r >= rows) break;
            if (r0 + r >= (int64_t)rlen.size()) return std::string(what) + ": row length table too short";
            const int64_t len = rlen[r0 + r];
            if (len > width) return std::string(what) + ": row longer than its slice";
            for (int64_t k = 0; k < len; ++k) {
                const int32_t c = colat(a + 32 * k + lane);
                if (c < 0 || c >= ncols) return std::string(what) + ": column out of range";
            }
        }
    }
    return "";
}

std::string check_view(const FacView &V, int64_t s0, int64_t r0, int64_t rows, int64_t ncols, const char *what)
{
    if ((V.v32 ? V.val32.size() : V.val64.size()) != V.size()) return std::string(what) + ": value array size";
    return check_sell_g(V.soff, s0 - V.sbase, V.rlen, r0 - V.rbase, rows, V.base, V.total(),
                        [&](int64_t i) { return V.col((size_t)(i - V.base)); }, ncols, what);
}

std::string check_sell(const std::vector<int64_t> &soff, int64_t s0, const std::vector<uint16_t> &rlen, int64_t r0,
                       int64_t rows, const std::vector<int32_t> &col, int64_t ncols, const char *what)
{
    return check_sell_g(soff, s0, rlen, r0, rows, 0, (int64_t)col.size(), [&](int64_t i) { return col[(size_t)i]; },
                        ncols, what);
}

}  // namespace

std::string validate_global(const Hierarchy &H, const std::vector<GlobalLevelDev> &G)
{
    const int L = H.L();
    std::string e;
    for (int l = 0; l <= L && !G.empty(); ++l) {
        const GlobalLevelDev &g = G[l];
        const int64_t n = H.lv[l].A.rows;
        if ((int64_t)g.rowid.size() != n) return "global rowid size";
        for (int32_t i : g.rowid) if (i < 0 || i >= n) return "global rowid out of range";
        if (!(e = check_sell(g.A.soff, 0, g.A.rlen, 0, g.A.rows, g.A.col, n, "global A")).empty()) return e;
        if (l < L) {
            const int64_t nc = H.lv[l + 1].A.rows;
            if (!(e = check_sell(g.P.soff, 0, g.P.rlen, 0, g.P.rows, g.P.col, nc, "global P")).empty()) return e;
            if (!(e = check_sell(g.R.soff, 0, g.R.rlen, 0, g.R.rows, g.R.col, n, "global R")).empty()) return e;
            if (g.P.rows != n || g.R.rows != nc) return "global P/R row counts";
        }
    }
    return "";
}

std::string validate_fac_grids(const Hierarchy &H, const FacLayout &F, int p0, int pn)
{
    const int L = H.L();
    std::string e;
    for (int p = p0; p < p0 + pn; ++p) {
        for (int l = 0; l <= L; ++l) {
            const FacLevelDesc &d = F.desc[(size_t)p * F.nlev + l];
            if (d.nC < 0 || d.nC > d.nReal || d.nReal > d.nBar) return "composite counts";
            if (d.row0 < F.row_base || d.row0 + d.nBar > F.rows_total ||
                d.row0 + d.nBar - F.row_base > (int64_t)F.gmap.size())
                return "composite row range";
            for (int32_t r = 0; r < d.nBar; ++r) {
                const int32_t gi = F.gmap[(size_t)(d.row0 - F.row_base + r)];
                if (gi < 0 || gi >= H.lv[l].A.rows) return "composite map out of range";
            }
            const int64_t nup = l < L ? F.desc[(size_t)p * F.nlev + l + 1].nBar : 0;
            const int64_t ndn = l > 0 ? F.desc[(size_t)p * F.nlev + l - 1].nBar : 0;
            if (!(e = check_view(F.A, d.sA, d.row0, d.nReal, d.nBar, "local A")).empty()) return e;
            if (!(e = check_view(F.At, d.sAt, d.row0, d.nBar, d.nReal, "local At")).empty()) return e;
            if (!(e = check_view(F.AFc, d.sAFc, d.row0 + d.nC, d.nReal - d.nC, d.nC, "local AFc")).empty()) return e;
            if (!(e = check_view(F.P, d.sP, d.row0, l < L ? d.nBar : 0, nup, "local P")).empty()) return e;
            if (!(e = check_view(F.R, d.sR, d.row0, l > 0 ? d.nBar : 0, ndn, "local R")).empty()) return e;
            if (l == L && d.nBar != H.lv[L].A.rows) return "coarsest composite level is not whole";
            if (l == L && d.nReal != d.nBar) return "coarsest composite level has ghosts";
        }
        const FacLevelDesc &d0 = F.desc[(size_t)p * F.nlev];
        for (int64_t k = F.owned0[p]; k < F.owned0[p + 1]; ++k)
            if (F.owned[k] < 0 || F.owned[k] >= d0.nReal) return "owned index out of range";
    }
    return "";
}

std::string validate_fac_totals(const FacLayout &F)
{
    for (const FacView *V : {&F.A, &F.At, &F.AFc, &F.P, &F.R})
        if (V->rbase + (int64_t)V->rlen.size() != F.rows_total) return "view row-length table size";
    if (F.row_base + (int64_t)F.gmap.size() != F.rows_total || F.row_base + (int64_t)F.l1inv.size() != F.rows_total)
        return "composite row count";
    std::vector<uint8_t> seen((size_t)F.nsub, 0);
    if (F.order.size() != (size_t)F.nsub) return "grid order is not a permutation";
    for (int32_t p : F.order) {
        if (p < 0 || p >= F.nsub || seen[p]) return "grid order is not a permutation";
        seen[p] = 1;
    }
    return "";
}

std::string validate_layouts(const Hierarchy &H, const std::vector<GlobalLevelDev> &G, const FacLayout &F)
{
    std::string e = validate_global(H, G);
    if (!e.empty() || F.nsub == 0) return e;
    if (!(e = validate_fac_totals(F)).empty()) return e;
    return validate_fac_grids(H, F, 0, F.nsub);
}

}  // namespace amgdd
