// Internal host-side structures of the AMG-DD library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <functional>
#include <vector>

#include "kernels.cuh"

namespace amgdd {

// Host CSR: ascending unique columns per row.
struct Csr {
    int32_t rows = 0, cols = 0;
    std::vector<int64_t> ptr;   // rows+1
    std::vector<int32_t> idx;
    std::vector<double> val;
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// One level of the classical AMG hierarchy (Section 2).
struct HLevel {
    Csr A;                        // A_l
    Csr P;                        // P_l : n_l x n_{l+1} (l < L)
    Csr R;                        // R_l = P_l^T (l < L)
    std::vector<uint8_t> isC;     // l < L: 1 for C points
    std::vector<int32_t> coarse;  // l < L: coarse index of a C point, -1 otherwise
    std::vector<double> l1inv;    // 1 / sum_j |a_ij|
};

struct Hierarchy {
    std::vector<HLevel> lv;       // levels 0..L
    std::vector<double> ainv;     // row-major inverse of A_L
    int L() const { return (int)lv.size() - 1; }
};

struct HierarchyParams {
    double theta = 0.25;
    int max_coarse = 16;
    int max_levels = 25;
    int interp = 0;       // 0 direct, 1 extended+i
    int p_max = 4;        // extended+i truncation (0 = none)
    int coarsen = 0;      // 0 Ruge-Stueben first pass, 1 HMIS over the subdomains
    const int32_t *part = nullptr;   // subdomain of every level-0 point (HMIS)
};

// Returns an empty string on success, else the reason.
std::string build_hierarchy(const Csr &A0, const HierarchyParams &prm, Hierarchy &H, int &status);

// Composite grid of one subdomain on one level (Section 3, eq. (1)); all sets
// hold ascending global indices of the level.
struct CompLevel {
    std::vector<int32_t> owned;   // Omega_l^p
    std::vector<int32_t> real;    // D_l^p
    std::vector<int32_t> ghost;   // Dbar_l^p \ D_l^p
};

struct Composite {
    int nsub = 0, nlev = 0;
    std::vector<CompLevel> g;     // [p * nlev + l]
    int64_t violations = 0;
    const CompLevel &at(int p, int l) const { return g[(size_t)p * nlev + l]; }
    CompLevel &at(int p, int l) { return g[(size_t)p * nlev + l]; }
};

void build_composite(const Hierarchy &H, const int32_t *part, int nsub,
                     const std::vector<int> &eta, Composite &C, int nthreads);

// ---------------------------------------------------------------------------
// Device-side layouts (filled on the host, uploaded as flat arrays).
//
// SELL-32: rows grouped in slices of 32 consecutive (device-order) rows; the
// k-th entry of row 32*s + lane is stored at soff[s] + 32*k + lane, entries of
// a row in ascending column order of the level's global numbering. rlen holds
// each row's length; a slice's width is (soff[s+1]-soff[s])/32.
struct Sell {
    int32_t rows = 0;
    std::vector<int64_t> soff;    // slices+1
    std::vector<uint16_t> rlen;   // rows
    std::vector<int32_t> col;
    std::vector<double> val;
};

// Row order [C rows ascending | F rows ascending] of a global level; rowid maps
// a device row to the level index.
struct GlobalLevelDev {
    Sell A;                       // rows in C|F order (all rows for l = L)
    std::vector<int32_t> rowid;   // device row -> level index
    int32_t nC = 0;
    Sell P;                       // natural row order (l < L)
    Sell R;                       // natural row order (l < L)
};

// One SELL family of the composite-grid layout (see FacViewDev). Columns are
// stored as 16-bit or 32-bit local indices and values as FP64 or FP32, chosen
// before packing (only one of each pair is filled).
struct FacView {
    std::vector<int64_t> soff;            // per slice, plus a sentinel per grid-level
    std::vector<uint16_t> rlen;           // per row (row0 + local row)
    std::vector<uint16_t> col16;
    std::vector<int32_t> col32;
    std::vector<double> val64;
    std::vector<float> val32;
    bool c16 = true, v32 = false;
    int64_t entries = 0;                  // stored (non-padding) entries
    // A streamed layout hands each packed chunk on and drops it: base, sbase
    // and rbase count the entries, slice offsets and rows already handed on,
    // so soff values, desc slice indices and row indices stay absolute.
    int64_t base = 0, sbase = 0, rbase = 0;
    size_t size() const { return c16 ? col16.size() : col32.size(); }   // entries held
    int64_t total() const { return base + (int64_t)size(); }
    int32_t col(size_t i) const { return c16 ? (int32_t)col16[i] : col32[i]; }   // held index
    void flush()
    {
        base = total();
        sbase += (int64_t)soff.size();
        rbase += (int64_t)rlen.size();
        soff.clear(); rlen.clear(); col16.clear(); col32.clear(); val64.clear(); val32.clear();
    }
};
struct FacLayout {
    int nlev = 0, nsub = 0;
    std::vector<FacLevelDesc> desc;       // [p * nlev + l]
    std::vector<int32_t> gmap;            // local -> level index
    std::vector<double> l1inv;            // per row (real rows used)
    int64_t row_base = 0;                 // rows of gmap / l1inv already handed on
    FacView A, At, AFc, P, R;
    std::vector<int32_t> owned;           // level-0 local indices of owned points
    std::vector<int64_t> owned0;          // per grid offset into owned (nsub+1)
    std::vector<int32_t> order;           // grids in launch order (largest first)
    std::vector<int64_t> work;            // per grid FMA count of one cycle after the first
    std::vector<int64_t> work1;           // per grid FMA count of the first cycle
    // local device order -> position in the map order (owned, real, ghost)
    std::vector<int32_t> dev2map;         // per row
    int64_t rows_total = 0;
    int32_t max_bar = 0;                  // largest composite level
    // per level: stored entries of each view over all grids
    std::vector<int64_t> lvA, lvAt, lvAFc, lvP, lvR;
};

// Called after each chunk of grids [p0, p0 + pn) has been packed into F; a
// consumer that streams the layout checks the chunk, copies it away and calls
// flush() on the views (and advances row_base). A non-empty return aborts the
// build with that message.
using FacSink = std::function<std::string(FacLayout &F, int p0, int pn)>;

// Packs the composite-grid layout; without a sink F ends up holding all of it.
// Returns the sink's error, or an empty string.
std::string build_fac_layout(const Hierarchy &H, const Composite &C, FacLayout &F, int nthreads, bool fp32,
                             const FacSink &sink = FacSink());
void build_global_dev(const Hierarchy &H, std::vector<GlobalLevelDev> &G);

// Range checks of every index the kernels will dereference; empty if valid.
std::string validate_global(const Hierarchy &H, const std::vector<GlobalLevelDev> &G);
// the grids [p0, p0 + pn) of F, whose rows and slices F still holds
std::string validate_fac_grids(const Hierarchy &H, const FacLayout &F, int p0, int pn);
// row totals of the views and the launch order, once all grids are packed
std::string validate_fac_totals(const FacLayout &F);
// all of the above for a layout held whole
std::string validate_layouts(const Hierarchy &H, const std::vector<GlobalLevelDev> &G, const FacLayout &F);

}  // namespace amgdd
