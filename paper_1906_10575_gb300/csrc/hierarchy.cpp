// Classical AMG setup on the host (Section 2 of the AMG-DD paper): strength of
// connection, Ruge-Stueben first-pass C/F splitting, direct interpolation,
// R = P^T, Galerkin coarse operators and the explicit coarsest inverse.
//
// Arithmetic is defined so that results are reproducible bit for bit on any
// IEEE host (this file is compiled with -ffp-contract=off):
//   * strength  : j in S_i  iff  j != i and -a_ij >= theta * max_{k != i}(-a_ik),
//                 with no strong connection when that maximum is <= 0;
//   * splitting : repeatedly take the undecided point of largest measure
//                 lambda_i = |S_i^T n U| + 2 |S_i^T n F| (smallest index on a
//                 tie), make it C and the undecided points depending on it F;
//                 points with no strong connection either way start as F;
//                 or (option) HMIS over the subdomains, stated at hmis_split;
//   * interp.   : F point i, strong C neighbours C_i, ascending sums
//                 alpha = sum_{j != i, a_ij < 0} a_ij / sum_{k in C_i} a_ik,
//                 d = a_ii + sum_{j != i, a_ij > 0} a_ij,  w_ik = (-alpha a_ik) / d;
//   * ext.+i    : (option) distance-two interpolation; its sums and their
//                 order are stated at extended_i_interpolation below;
//   * Galerkin  : entry (I,J) of R A P sums (p_iI * a_ij) * p_jJ, fine i
//                 ascending, then j ascending, then J; the pattern keeps every
//                 structural term;
//   * inverse   : Gauss-Jordan with partial pivoting (first largest |pivot|).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "amgdd_internal.hpp"

namespace amgdd {
namespace {

constexpr int kMaxDenseCoarse = 8192;

struct Pattern {
    std::vector<int64_t> ptr;
    std::vector<int32_t> idx;
};

Pattern strong_connections(const Csr &A, double theta)
{
    Pattern S;
    S.ptr.assign((size_t)A.rows + 1, 0);
    S.idx.reserve((size_t)A.nnz());
    for (int32_t i = 0; i < A.rows; ++i) {
        bool have = false;
        double big = 0.0;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            if (A.idx[k] == i) continue;
            const double neg = -A.val[k];
            if (!have || neg > big) { big = neg; have = true; }
        }
        if (have && big > 0.0) {
            const double cut = theta * big;
            for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
                if (A.idx[k] != i && -A.val[k] >= cut) S.idx.push_back(A.idx[k]);
        }
        S.ptr[i + 1] = (int64_t)S.idx.size();
    }
    return S;
}

Pattern transpose_pattern(const Pattern &S, int32_t n)
{
    Pattern T;
    T.ptr.assign((size_t)n + 1, 0);
    T.idx.resize(S.idx.size());
    for (int32_t j : S.idx) T.ptr[j + 1]++;
    std::partial_sum(T.ptr.begin(), T.ptr.end(), T.ptr.begin());
    std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t k = S.ptr[i]; k < S.ptr[i + 1]; ++k) T.idx[fill[S.idx[k]]++] = i;
    return T;
}

// Tournament tree over the points: every internal node keeps the winner of
// its subtree (largest key, then smallest index). Decided points carry key -1.
class Tournament {
public:
    Tournament(const std::vector<int64_t> &key) : key_(key)
    {
        n_ = (int32_t)key.size();
        size_ = 1;
        while (size_ < n_) size_ <<= 1;
        win_.assign(2 * (size_t)size_, -1);
        for (int32_t i = 0; i < n_; ++i) win_[size_ + i] = i;
        for (int64_t v = size_ - 1; v >= 1; --v) win_[v] = pick(win_[2 * v], win_[2 * v + 1]);
    }
    int32_t best() const { return win_[1]; }
    void refresh(int32_t i)
    {
        for (int64_t v = (size_ + i) >> 1; v >= 1; v >>= 1) win_[v] = pick(win_[2 * v], win_[2 * v + 1]);
    }

private:
    int32_t pick(int32_t a, int32_t b) const
    {
        if (a < 0) return b;
        if (b < 0) return a;
        if (key_[a] != key_[b]) return key_[a] > key_[b] ? a : b;
        return a < b ? a : b;
    }
    const std::vector<int64_t> &key_;
    int32_t n_;
    int64_t size_;
    std::vector<int32_t> win_;
};

// Ruge-Stueben first pass; returns 1 for C, 0 for F.
std::vector<uint8_t> first_pass_split(const Pattern &S, const Pattern &St, int32_t n)
{
    enum : int8_t { kU = 0, kC = 1, kF = 2 };
    std::vector<int8_t> st((size_t)n, kU);
    std::vector<int64_t> key((size_t)n, -1);
    for (int32_t i = 0; i < n; ++i) {
        const int64_t infl = St.ptr[i + 1] - St.ptr[i];
        const int64_t dep = S.ptr[i + 1] - S.ptr[i];
        if (infl == 0 && dep == 0) st[i] = kF;   // isolated: F, empty P row
        else key[i] = infl;                       // |S_i^T|, all undecided
    }
    Tournament T(key);
    for (;;) {
        const int32_t i = T.best();
        if (i < 0 || key[i] < 0) break;
        st[i] = kC;
        key[i] = -1;
        T.refresh(i);
        for (int64_t a = St.ptr[i]; a < St.ptr[i + 1]; ++a) {
            const int32_t j = St.idx[a];
            if (st[j] != kU) continue;
            st[j] = kF;
            key[j] = -1;
            T.refresh(j);
            for (int64_t b = S.ptr[j]; b < S.ptr[j + 1]; ++b) {
                const int32_t m = S.idx[b];
                if (st[m] == kU) { key[m] += 1; T.refresh(m); }
            }
        }
        for (int64_t a = S.ptr[i]; a < S.ptr[i + 1]; ++a) {
            const int32_t j = S.idx[a];
            if (st[j] == kU) { key[j] -= 1; T.refresh(j); }
        }
    }
    std::vector<uint8_t> isC((size_t)n);
    for (int32_t i = 0; i < n; ++i) isC[i] = (st[i] == kC);
    return isC;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output for counter x; the
// reproducible stand-in for the random part of the PMIS measure.
uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// HMIS splitting (De Sterck, Yang and Heys 2006; the coarsening of the hypre
// defaults the paper runs with) with the subdomains as the processors: the
// first pass on each subdomain's own strong connections; its C points at
// interior points (every strong connection, either direction, inside the
// subdomain) start PMIS on the whole strength graph, whose measure |S_i^T| is
// tie-broken by splitmix64((level << 40) + i), then by the smaller index.
// Returns 1 for C, 0 for F.
std::vector<uint8_t> hmis_split(const Pattern &S, const Pattern &St, int32_t n, const std::vector<int32_t> &sub,
                                int level)
{
    Pattern Sl;
    Sl.ptr.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t k = S.ptr[i]; k < S.ptr[i + 1]; ++k)
            if (sub[S.idx[k]] == sub[i]) Sl.idx.push_back(S.idx[k]);
        Sl.ptr[i + 1] = (int64_t)Sl.idx.size();
    }
    const std::vector<uint8_t> first = first_pass_split(Sl, transpose_pattern(Sl, n), n);
    enum : int8_t { kU = 0, kC = 1, kF = 2 };
    std::vector<int8_t> st((size_t)n, kU);
    for (int32_t i = 0; i < n; ++i) {
        bool interior = true;
        for (int64_t k = S.ptr[i]; k < S.ptr[i + 1] && interior; ++k) interior = sub[S.idx[k]] == sub[i];
        for (int64_t k = St.ptr[i]; k < St.ptr[i + 1] && interior; ++k) interior = sub[St.idx[k]] == sub[i];
        if (interior && first[i]) st[i] = kC;
    }
    std::vector<uint64_t> draw((size_t)n);
    for (int32_t i = 0; i < n; ++i) draw[i] = splitmix64(((uint64_t)level << 40) + (uint64_t)i);
    auto before = [&](int32_t i, int32_t j) {   // i ahead of j in the PMIS order
        const int64_t ci = St.ptr[i + 1] - St.ptr[i], cj = St.ptr[j + 1] - St.ptr[j];
        if (ci != cj) return ci > cj;
        if (draw[i] != draw[j]) return draw[i] > draw[j];
        return i < j;
    };
    for (int32_t i = 0; i < n; ++i)
        if (st[i] == kU && St.ptr[i + 1] == St.ptr[i]) st[i] = kF;
    std::vector<uint8_t> pick((size_t)n, 0);
    for (;;) {
        int64_t left = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (st[i] != kU) continue;
            for (int64_t k = S.ptr[i]; k < S.ptr[i + 1]; ++k)
                if (st[S.idx[k]] == kC) {
                    st[i] = kF;
                    break;
                }
            left += st[i] == kU;
        }
        if (left == 0) break;
        for (int32_t i = 0; i < n; ++i) {
            pick[i] = 0;
            if (st[i] != kU) continue;
            bool ahead = true;
            for (int64_t k = S.ptr[i]; k < S.ptr[i + 1] && ahead; ++k) {
                const int32_t j = S.idx[k];
                if (j != i && st[j] == kU && before(j, i)) ahead = false;
            }
            for (int64_t k = St.ptr[i]; k < St.ptr[i + 1] && ahead; ++k) {
                const int32_t j = St.idx[k];
                if (j != i && st[j] == kU && before(j, i)) ahead = false;
            }
            pick[i] = ahead;
        }
        for (int32_t i = 0; i < n; ++i)
            if (pick[i]) st[i] = kC;
    }
    std::vector<uint8_t> isC((size_t)n);
    for (int32_t i = 0; i < n; ++i) isC[i] = (st[i] == kC);
    return isC;
}

Csr direct_interpolation(const Csr &A, const Pattern &S, const std::vector<uint8_t> &isC,
                         const std::vector<int32_t> &coarse, int32_t nc)
{
    Csr P;
    P.rows = A.rows;
    P.cols = nc;
    P.ptr.assign((size_t)A.rows + 1, 0);
    for (int32_t i = 0; i < A.rows; ++i) {
        if (isC[i]) {
            P.idx.push_back(coarse[i]);
            P.val.push_back(1.0);
            P.ptr[i + 1] = (int64_t)P.idx.size();
            continue;
        }
        // strong C neighbours with their matrix entries, ascending column
        std::vector<std::pair<int32_t, double>> cs;
        int64_t k = A.ptr[i];
        for (int64_t q = S.ptr[i]; q < S.ptr[i + 1]; ++q) {
            const int32_t j = S.idx[q];
            while (A.idx[k] < j) ++k;
            if (isC[j]) cs.emplace_back(j, A.val[k]);
        }
        if (!cs.empty()) {
            double diag = 0.0;
            for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
                if (A.idx[q] == i) diag = A.val[q];
            double neg_sum = 0.0;
            double d = diag;
            for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
                if (A.idx[q] == i) continue;
                const double a = A.val[q];
                if (a < 0.0) neg_sum = neg_sum + a;
                else if (a > 0.0) d = d + a;
            }
            double c_sum = 0.0;
            for (const auto &e : cs) c_sum = c_sum + e.second;
            const double alpha = neg_sum / c_sum;
            for (const auto &e : cs) {
                P.idx.push_back(coarse[e.first]);
                P.val.push_back((-alpha * e.second) / d);
            }
        }
        P.ptr[i + 1] = (int64_t)P.idx.size();
    }
    return P;
}

// Entry (r, c) of A, 0 when it is not stored (columns ascend within a row).
double entry_of(const Csr &A, int32_t r, int32_t c)
{
    const auto b = A.idx.begin() + A.ptr[r], e = A.idx.begin() + A.ptr[r + 1];
    const auto it = std::lower_bound(b, e, c);
    return (it != e && *it == c) ? A.val[(size_t)(it - A.idx.begin())] : 0.0;
}

// Extended+i interpolation. F point i, strong set S_i (ascending):
//   F_i = strong F neighbours; H_i = strong C neighbours, and the strong C
//   neighbours of every k in F_i, ascending;
//   ab(k, l) = a_kl when a_kl and a_kk have opposite signs, else 0;
//   D_k = sum of ab(k, l) over row k's entries l in H_i or l = i, ascending;
//   d = a_ii, then over row i's other entries n ascending: n in F_i adds
//       (a_in * ab(n, i)) / D_n (or a_in when D_n = 0); n outside H_i and F_i
//       adds a_in; n in H_i adds nothing;
//   num_j = a_ij (0 if absent), then for k in F_i ascending with D_k != 0:
//       + (a_ik * ab(k, j)) / D_k;   w_ij = (-num_j) / d, j in H_i.
// With p_max > 0 a row longer than p_max keeps its p_max largest |w| (the
// smaller column first on equal |w|), scaled by sum(all w) / sum(kept w)
// (ascending sums) when the kept sum is not zero. C points inject; an F point
// with empty H_i has an empty row.
Csr extended_i_interpolation(const Csr &A, const Pattern &S, const std::vector<uint8_t> &isC,
                             const std::vector<int32_t> &coarse, int32_t nc, int p_max)
{
    const int32_t n = A.rows;
    Csr P;
    P.rows = n;
    P.cols = nc;
    P.ptr.assign((size_t)n + 1, 0);
    std::vector<int32_t> tagH((size_t)n, -1), tagF((size_t)n, -1);
    std::vector<double> D((size_t)n, 0.0);
    std::vector<int32_t> H;
    std::vector<double> w;
    auto ab = [&](int32_t k, int32_t l) {
        const double a = entry_of(A, k, l);
        return a * entry_of(A, k, k) < 0.0 ? a : 0.0;
    };
    for (int32_t i = 0; i < n; ++i) {
        if (isC[i]) {
            P.idx.push_back(coarse[i]);
            P.val.push_back(1.0);
            P.ptr[i + 1] = (int64_t)P.idx.size();
            continue;
        }
        H.clear();
        for (int64_t q = S.ptr[i]; q < S.ptr[i + 1]; ++q) {
            const int32_t j = S.idx[q];
            if (isC[j]) {
                if (tagH[j] != i) { tagH[j] = i; H.push_back(j); }
                continue;
            }
            tagF[j] = i;
            for (int64_t q2 = S.ptr[j]; q2 < S.ptr[j + 1]; ++q2) {
                const int32_t m = S.idx[q2];
                if (isC[m] && tagH[m] != i) { tagH[m] = i; H.push_back(m); }
            }
        }
        if (H.empty()) {
            P.ptr[i + 1] = (int64_t)P.idx.size();
            continue;
        }
        std::sort(H.begin(), H.end());
        for (int64_t q = S.ptr[i]; q < S.ptr[i + 1]; ++q) {
            const int32_t k = S.idx[q];
            if (tagF[k] != i) continue;
            const double akk = entry_of(A, k, k);
            double s = 0.0;
            for (int64_t e = A.ptr[k]; e < A.ptr[k + 1]; ++e) {
                const int32_t l = A.idx[e];
                if (l == i || tagH[l] == i)
                    if (A.val[e] * akk < 0.0) s = s + A.val[e];
            }
            D[k] = s;
        }
        double d = entry_of(A, i, i);
        for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const int32_t nn = A.idx[e];
            if (nn == i) continue;
            if (tagF[nn] == i) d = D[nn] != 0.0 ? d + (A.val[e] * ab(nn, i)) / D[nn] : d + A.val[e];
            else if (tagH[nn] != i) d = d + A.val[e];
        }
        w.assign(H.size(), 0.0);
        for (size_t t = 0; t < H.size(); ++t) {
            const int32_t j = H[t];
            double num = entry_of(A, i, j);
            for (int64_t q = S.ptr[i]; q < S.ptr[i + 1]; ++q) {
                const int32_t k = S.idx[q];
                if (tagF[k] != i || D[k] == 0.0) continue;
                num = num + (entry_of(A, i, k) * ab(k, j)) / D[k];
            }
            w[t] = (-num) / d;
        }
        std::vector<uint8_t> keep(H.size(), 1);
        if (p_max > 0 && (int)H.size() > p_max) {
            std::vector<int32_t> byw(H.size());
            std::iota(byw.begin(), byw.end(), 0);
            std::sort(byw.begin(), byw.end(), [&](int32_t a, int32_t b) {
                const double fa = std::fabs(w[a]), fb = std::fabs(w[b]);
                return fa != fb ? fa > fb : H[a] < H[b];
            });
            std::fill(keep.begin(), keep.end(), 0);
            for (int t = 0; t < p_max; ++t) keep[byw[t]] = 1;
            double all = 0.0, kept = 0.0;
            for (size_t t = 0; t < H.size(); ++t) all = all + w[t];
            for (size_t t = 0; t < H.size(); ++t)
                if (keep[t]) kept = kept + w[t];
            if (kept != 0.0)
                for (size_t t = 0; t < H.size(); ++t)
                    if (keep[t]) w[t] = w[t] * (all / kept);
        }
        for (size_t t = 0; t < H.size(); ++t)
            if (keep[t]) {
                P.idx.push_back(coarse[H[t]]);
                P.val.push_back(w[t]);
            }
        P.ptr[i + 1] = (int64_t)P.idx.size();
    }
    return P;
}

Csr transpose(const Csr &P)
{
    Csr R;
    R.rows = P.cols;
    R.cols = P.rows;
    R.ptr.assign((size_t)R.rows + 1, 0);
    for (int32_t J : P.idx) R.ptr[J + 1]++;
    std::partial_sum(R.ptr.begin(), R.ptr.end(), R.ptr.begin());
    R.idx.resize(P.idx.size());
    R.val.resize(P.val.size());
    std::vector<int64_t> fill(R.ptr.begin(), R.ptr.end() - 1);
    for (int32_t i = 0; i < P.rows; ++i)
        for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
            const int64_t o = fill[P.idx[k]]++;
            R.idx[o] = i;
            R.val[o] = P.val[k];
        }
    return R;
}

Csr galerkin_product(const Csr &R, const Csr &A, const Csr &P)
{
    const int32_t m = R.rows;
    Csr C;
    C.rows = m;
    C.cols = m;
    C.ptr.assign((size_t)m + 1, 0);
    std::vector<double> acc((size_t)m, 0.0);
    std::vector<int32_t> seen((size_t)m, -1);
    std::vector<int32_t> touched;
    for (int32_t I = 0; I < m; ++I) {
        touched.clear();
        for (int64_t a = R.ptr[I]; a < R.ptr[I + 1]; ++a) {
            const int32_t i = R.idx[a];
            const double p_iI = R.val[a];
            for (int64_t b = A.ptr[i]; b < A.ptr[i + 1]; ++b) {
                const int32_t j = A.idx[b];
                const double t = p_iI * A.val[b];
                for (int64_t c = P.ptr[j]; c < P.ptr[j + 1]; ++c) {
                    const int32_t J = P.idx[c];
                    const double term = t * P.val[c];
                    if (seen[J] != I) { seen[J] = I; acc[J] = 0.0; touched.push_back(J); }
                    acc[J] = acc[J] + term;
                }
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int32_t J : touched) {
            C.idx.push_back(J);
            C.val.push_back(acc[J]);
        }
        C.ptr[I + 1] = (int64_t)C.idx.size();
    }
    return C;
}

std::vector<double> l1_inverse(const Csr &A)
{
    std::vector<double> out((size_t)A.rows);
    for (int32_t i = 0; i < A.rows; ++i) {
        double s = 0.0;
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s = s + std::fabs(A.val[k]);
        out[i] = 1.0 / s;
    }
    return out;
}

bool dense_inverse(const Csr &A, std::vector<double> &X)
{
    const int n = A.rows;
    std::vector<double> M((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) M[(size_t)i * n + A.idx[k]] = A.val[k];
    X.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    auto m = [&](int r, int c) -> double & { return M[(size_t)r * n + c]; };
    auto x = [&](int r, int c) -> double & { return X[(size_t)r * n + c]; };
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double pmag = std::fabs(m(col, col));
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(m(r, col)) > pmag) { pmag = std::fabs(m(r, col)); piv = r; }
        if (pmag == 0.0) return false;
        if (piv != col)
            for (int c = 0; c < n; ++c) { std::swap(m(col, c), m(piv, c)); std::swap(x(col, c), x(piv, c)); }
        const double p = m(col, col);
        for (int c = 0; c < n; ++c) { m(col, c) = m(col, c) / p; x(col, c) = x(col, c) / p; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = m(r, col);
            if (f == 0.0) continue;
            for (int c = 0; c < n; ++c) {
                m(r, c) = m(r, c) - f * m(col, c);
                x(r, c) = x(r, c) - f * x(col, c);
            }
        }
    }
    return true;
}

}  // namespace

std::string build_hierarchy(const Csr &A0, const HierarchyParams &prm, Hierarchy &H, int &status)
{
    status = 0;
    H.lv.clear();
    H.lv.emplace_back();
    H.lv[0].A = A0;
    const int max_levels = std::min(prm.max_levels, 40);
    // subdomain of every point of the current level (HMIS): level 0 from the
    // partition, a C point keeps the subdomain of the fine point it comes from
    std::vector<int32_t> sub((size_t)A0.rows, 0);
    if (prm.part) sub.assign(prm.part, prm.part + A0.rows);
    for (int l = 0;; ++l) {
        HLevel &cur = H.lv[l];
        cur.l1inv = l1_inverse(cur.A);
        if (l + 1 >= max_levels || cur.A.rows <= prm.max_coarse) break;
        Pattern S = strong_connections(cur.A, prm.theta);
        Pattern St = transpose_pattern(S, cur.A.rows);
        std::vector<uint8_t> isC = prm.coarsen == 1 ? hmis_split(S, St, cur.A.rows, sub, l)
                                                    : first_pass_split(S, St, cur.A.rows);
        int64_t nc = 0;
        for (uint8_t c : isC) nc += c;
        if (nc == 0 || nc * 10 > (int64_t)cur.A.rows * 9) break;
        std::vector<int32_t> coarse((size_t)cur.A.rows, -1);
        int32_t next = 0;
        for (int32_t i = 0; i < cur.A.rows; ++i)
            if (isC[i]) coarse[i] = next++;
        HLevel nxt;
        cur.P = prm.interp == 1 ? extended_i_interpolation(cur.A, S, isC, coarse, (int32_t)nc, prm.p_max)
                                : direct_interpolation(cur.A, S, isC, coarse, (int32_t)nc);
        cur.R = transpose(cur.P);
        nxt.A = galerkin_product(cur.R, cur.A, cur.P);
        std::vector<int32_t> subc((size_t)nc);
        for (int32_t i = 0; i < cur.A.rows; ++i)
            if (isC[i]) subc[coarse[i]] = sub[i];
        sub.swap(subc);
        cur.isC = std::move(isC);
        cur.coarse = std::move(coarse);
        H.lv.push_back(std::move(nxt));
    }
    const Csr &AL = H.lv.back().A;
    if (AL.rows > kMaxDenseCoarse) {
        status = 2;
        return "coarsest level has " + std::to_string(AL.rows) +
               " points, too many for a dense inverse (raise max_levels or lower max_coarse)";
    }
    if (!dense_inverse(AL, H.ainv)) {
        status = 1;
        return "coarsest matrix is singular";
    }
    return "";
}

}  // namespace amgdd
