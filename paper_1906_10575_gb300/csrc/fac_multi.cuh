// Composite-grid FAC kernel for several right-hand sides at once (R = 1, 2
// or 4): every vector is stored row by row with its R values side by side
// (v[i * R + j]), and one load of an operator entry feeds R independent fma
// chains. Column j's chain is exactly the single-right-hand-side chain (same
// entries, same ascending order), so each column reproduces the
// one-at-a-time result bit for bit. Instantiated per R in fac_multi_r*.cu.
#pragma once

#include <cstdint>

#include "fac_device.cuh"
#include "kernels.cuh"

namespace amgdd {
namespace dev {

template <class T, int R>
struct VecR {
    T v[R];
};

// R consecutive values of the gathered vector (16- or 32-byte aligned groups
// are loaded as vectors).
template <class T, int R>
__device__ __forceinline__ VecR<T, R> load_r(const T *__restrict__ p)
{
    VecR<T, R> o;
    if constexpr (sizeof(T) == 4 && R == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        o.v[0] = q.x; o.v[1] = q.y; o.v[2] = q.z; o.v[3] = q.w;
    } else if constexpr (sizeof(T) == 8 && R == 2) {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        o.v[0] = q.x; o.v[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && R == 4) {
        const double2 q0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 q1 = reinterpret_cast<const double2 *>(p)[1];
        o.v[0] = q0.x; o.v[1] = q0.y; o.v[2] = q1.x; o.v[3] = q1.y;
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) o.v[j] = p[j];
    }
    return o;
}

// Hint that the line holding p is wanted soon: fetched into L2 (or into L1
// and L2), no register is held and nothing waits for it.
template <bool TO_L1>
__device__ __forceinline__ void prefetch_line(const void *p)
{
    if constexpr (TO_L1) asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    else asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Where a pass reads a gathered level vector. One: local row c at x + c R.
// Two: local row c at (c < split ? a : b) + c R, for a pass that reads the
// rows below `split` from the buffer the previous half-sweep wrote them to
// and the others from the buffer that still holds their current values.
template <class T_, int R_>
struct One {
    using T = T_;
    static constexpr int R = R_;
    const T *x;
    __device__ __forceinline__ const T *at(int64_t c) const { return x + c * R; }
    __device__ __forceinline__ static One onchip(const T *p) { return One{p}; }
};

template <class T_, int R_>
struct Two {
    using T = T_;
    static constexpr int R = R_;
    const T *a, *b;
    int split;
    __device__ __forceinline__ const T *at(int64_t c) const { return (c < split ? a : b) + c * R; }
    __device__ __forceinline__ static Two onchip(const T *p) { return Two{p, p, 0}; }
};

// s_j = sum_k a_k x[c_k * R + j] for the lane's row, one fma chain per column.
// UNR entries are loaded before any of them is used (UNR operator loads and
// UNR gathers in flight per lane); the fmas stay in ascending entry order.
// PF != 0: each step first asks L2 (PF > 0) or L1 (PF < 0) for the operator
// entries |PF| steps ahead, so their loads find them there instead of in HBM
// (entries past the row's length are not touched).
template <class CI, class T, int R, int UNR, int PF, class SV, bool STREAM = true, class G>
__device__ __forceinline__ VecR<T, R> sell_dot_g(const int64_t *soff, const uint16_t *rlen, const CI *col,
                                                 const SV *val, int64_t slice, int lane, int64_t row,
                                                 const G &x)
{
    const int64_t base = __ldg(soff + slice) + lane;
    const int len = __ldg(rlen + row);
    VecR<T, R> s;
#pragma unroll
    for (int j = 0; j < R; ++j) s.v[j] = T(0);
    int k = 0;
    if constexpr (PF != 0) {
        constexpr int D = PF > 0 ? PF : -PF;
#pragma unroll 1
        for (; k + UNR <= len; k += UNR) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int kp = k + D * UNR + u;
                if (kp < len) {
                    prefetch_line<(PF < 0)>(col + base + 32 * kp);
                    prefetch_line<(PF < 0)>(val + base + 32 * kp);
                }
            }
            int c[UNR];
            T a[UNR];
            VecR<T, R> xv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) c[u] = ld_op<STREAM>(col + base + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < UNR; ++u) a[u] = (T)ld_op<STREAM>(val + base + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < UNR; ++u) xv[u] = load_r<T, R>(x.at(c[u]));
#pragma unroll
            for (int u = 0; u < UNR; ++u)
#pragma unroll
                for (int j = 0; j < R; ++j) s.v[j] = fma(a[u], xv[u].v[j], s.v[j]);
        }
    }
    if constexpr (UNR > 1) {
#pragma unroll 1
        for (; k + UNR <= len; k += UNR) {
            int c[UNR];
            T a[UNR];
            VecR<T, R> xv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) c[u] = ld_op<STREAM>(col + base + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < UNR; ++u) a[u] = (T)ld_op<STREAM>(val + base + 32 * (k + u));
#pragma unroll
            for (int u = 0; u < UNR; ++u) xv[u] = load_r<T, R>(x.at(c[u]));
#pragma unroll
            for (int u = 0; u < UNR; ++u)
#pragma unroll
                for (int j = 0; j < R; ++j) s.v[j] = fma(a[u], xv[u].v[j], s.v[j]);
        }
    }
#pragma unroll 1
    for (; k < len; ++k) {
        const int c = ld_op<STREAM>(col + base + 32 * k);
        const T a = (T)ld_op<STREAM>(val + base + 32 * k);
        const VecR<T, R> xv = load_r<T, R>(x.at(c));
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = fma(a, xv.v[j], s.v[j]);
    }
    return s;
}

// sell_dot_g over one plain vector x.
template <class CI, class T, int R, int UNR, int PF = 0, class SV>
__device__ __forceinline__ VecR<T, R> sell_dot_r(const int64_t *soff, const uint16_t *rlen, const CI *col,
                                                 const SV *val, int64_t slice, int lane, int64_t row,
                                                 const T *__restrict__ x)
{
    return sell_dot_g<CI, T, R, UNR, PF, SV>(soff, rlen, col, val, slice, lane, row, One<T, R>{x});
}

// ---- composite grids ------------------------------------------------------

template <class CI, class T, int R, int UNR, int PF, bool STREAM = true, class G>
__device__ __forceinline__ VecR<T, R> view_dot_r(const FacViewDev &V, int64_t slice0, int64_t row0, int first,
                                                 int r, const G &x)
{
    const int v = r - first;
    return sell_dot_g<CI, T, R, UNR, PF, T, STREAM>(V.soff, V.rlen, static_cast<const CI *>(V.col),
                                                    static_cast<const T *>(V.val), slice0 + (v >> 5), v & 31,
                                                    row0 + r, x);
}

// Row products V_r . x of local rows [r0, r1) of a view whose slices start at
// local row `first`; fn(r, s) is called once per row (by one lane).
// g == 1 (tile): one row per lane of a SELL-32 slice, the single-column chain.
// g > 1 (GRP builds only): g lanes per row, lane j of the group sums entries
// j, j + g, j + 2g, ... of the row, then the group adds its g partial sums by
// an xor butterfly. The warp covers 32 / g consecutive rows of one slice per
// pass, so rows of small levels spread over all warps and each lane's chain
// is g times shorter; the rounding order is not the ascending chain's.
template <class CI, class T, int R, int UNR, int PF, bool GRP, bool STREAM = true, class G, class Fn>
__device__ __forceinline__ void rows_dot(const Block &B, int g, const FacViewDev &V, int64_t s0, int64_t row0,
                                         int first, int r0, int r1, const G &x, Fn &&fn)
{
    if (!GRP || g <= 1) {
        for_rows(B, first, r0, r1,
                 [&](int r) { fn(r, view_dot_r<CI, T, R, UNR, PF, STREAM>(V, s0, row0, first, r, x)); });
        return;
    }
    if (r1 <= r0) return;
    const int rpw = 32 / g;
    const int sub = B.lane / g, j = B.lane & (g - 1);
    const int u0 = (r0 - first) / rpw, u1 = (r1 - first + rpw - 1) / rpw;
    const CI *__restrict__ col = static_cast<const CI *>(V.col);
    const T *__restrict__ val = static_cast<const T *>(V.val);
    for (int uu = u0 + B.warp; uu < u1; uu += B.nw) {
        const int r = first + uu * rpw + sub;
        const bool on = r >= r0 && r < r1;
        VecR<T, R> acc;
#pragma unroll
        for (int q = 0; q < R; ++q) acc.v[q] = T(0);
        if (on) {
            const int v = r - first;
            const int64_t base = __ldg(V.soff + s0 + (v >> 5)) + (v & 31);
            const int len = __ldg(V.rlen + row0 + r);
            int k = j;
#pragma unroll 1
            for (; k + g < len; k += 2 * g) {
                const int c0 = ld_op<true>(col + base + 32 * k), c1 = ld_op<true>(col + base + 32 * (k + g));
                const T a0 = ld_op<true>(val + base + 32 * k), a1 = ld_op<true>(val + base + 32 * (k + g));
                const VecR<T, R> x0 = load_r<T, R>(x.at(c0)), x1 = load_r<T, R>(x.at(c1));
#pragma unroll
                for (int q = 0; q < R; ++q) acc.v[q] = fma(a0, x0.v[q], acc.v[q]);
#pragma unroll
                for (int q = 0; q < R; ++q) acc.v[q] = fma(a1, x1.v[q], acc.v[q]);
            }
            if (k < len) {
                const int c0 = ld_op<true>(col + base + 32 * k);
                const T a0 = ld_op<true>(val + base + 32 * k);
                const VecR<T, R> x0 = load_r<T, R>(x.at(c0));
#pragma unroll
                for (int q = 0; q < R; ++q) acc.v[q] = fma(a0, x0.v[q], acc.v[q]);
            }
        }
        for (int m = 1; m < g; m <<= 1)
#pragma unroll
            for (int q = 0; q < R; ++q) acc.v[q] = acc.v[q] + __shfl_xor_sync(0xffffffffu, acc.v[q], m);
        if (on && j == 0) fn(r, acc);
    }
}

// Shared-memory staging of a gathered vector: when the nrows rows of the
// level vector x fit the block's SB-byte buffer, the block copies them there
// and the pass's gathers read the copy (the pass writes other rows or other
// vectors only, and the previous pass ended at a barrier). Called by every
// thread of the block; the condition is the same for all of them.
template <int SB, class G>
__device__ __forceinline__ G stage(const Block &B, const G &x, int64_t nrows, unsigned char *buf)
{
    using T = typename G::T;
    constexpr int R = G::R;
    if constexpr (SB > 0) {
        if (nrows * R * (int64_t)sizeof(T) <= SB) {
            T *sb = reinterpret_cast<T *>(buf);
            for (int64_t i = B.tid; i < nrows * R; i += B.nt) sb[i] = x.at(i / R)[i % R];
            B.sync();
            return G::onchip(sb);
        }
    }
    return x;
}

// How a half-sweep updates t with its correction v: t += v, t = v (t_l holds
// nothing of this iteration yet), or not at all (the last cycle's upsweep,
// whose t nothing reads).
constexpr int kTAdd = 0, kTAssign = 1, kTNone = 2;

// One Jacobi half-sweep over the rows [r0, r1) of one set (C or F points):
// v = (f - V u) * (1/l1) with u gathered through `src`; the row's new value
// own + v goes to dst, and t is updated by t_mode. dst is either the row's own buffer (in place:
// the pass reads u only at rows outside the set) or the other buffer of the
// pair, which the pass reads only outside the set; either way every read of
// the pass sees the values from before it, as Jacobi needs, without a
// scratch vector or a barrier between computing and applying.
// The work vectors of the grid being cycled: u in two buffers (u, u2), f, t
// and s, R values per row. Row i of the composite layout (row0 + local row)
// is entry i - rb: rb = 0 where they are the global arrays, rb = the grid's
// first row where they sit in the block's shared memory.
template <class T>
struct WorkVecs {
    T *u, *u2, *f, *t, *s;
    int64_t rb;
};

template <class CI, class T, int R, int UNR, int PF, bool GRP, int SB, bool STREAM, class G>
__device__ __forceinline__ void relax_pass_r(const FacParams &P, const WorkVecs<T> &W, const Block &B,
                                             const FacLevelDesc &d, int g, const FacViewDev &V, int64_t s0,
                                             int first, int r0, int r1, const G &src, const T *own, T *dst,
                                             int t_mode, unsigned char *buf)
{
    T *__restrict__ t = W.t + (d.row0 - W.rb) * R;
    const T *__restrict__ f = W.f + (d.row0 - W.rb) * R;
    const T *__restrict__ l1 = static_cast<const T *>(P.l1inv) + d.row0;
    const G x = stage<SB>(B, src, (int64_t)d.nBar, buf);
    rows_dot<CI, T, R, UNR, PF, GRP, STREAM>(B, g, V, s0, d.row0, first, r0, r1, x,
                                             [&](int r, const VecR<T, R> &s) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const T v = (f[r * R + j] - s.v[j]) * l1[r];
            dst[r * R + j] = own[r * R + j] + v;
            if (t_mode == kTAssign) t[r * R + j] = v;
            else if (t_mode == kTAdd) t[r * R + j] = t[r * R + j] + v;
        }
    });
    B.sync();
}

// The composite-grid FAC launch (Algorithm 4 on every composite grid, the
// owned corrections added to x as in Algorithm 2). u_l lives in two buffers,
// U0 = P.u and U1 = P.d: a grid's level is either wholly in U0, or its real
// rows are in U1 while its ghost rows stay in U0 (ghost rows are never
// relaxed). Every level starts each AlgFAC cycle and ends the launch in U0:
//   downsweep, l = 0: C half-sweep U0 -> U1, F half-sweep (C rows from U1)
//     -> U1 (first cycle: u_0 = 0, so the C half-sweep is f / l1 and the F
//     half-sweep reads the C columns only);
//   downsweep, l >= 1: u_l = 0 with the first C half-sweep folded in, into
//     U1, done row by row by the restriction pass from level l - 1 as soon
//     as a row's f_l is final, then the in-place F half-sweep on U1;
//   upsweep: u_l += P_l u_{l+1} (u_{l+1} in U0; on the ghost rows of
//     l >= 1, which are zero until then, 0 + P_l u_{l+1} into U0), then F
//     half-sweep U1 -> U0 (ghost columns from U0), C half-sweep (F and ghost
//     columns from U0) U1 -> U0.
// t_l is never cleared: the first write of each of its phases assigns, and
// the s_l + A_l t_l product reads t only at real rows, which every half-sweep
// pair writes; the last cycle's upsweep does not write t at all (nothing
// reads it before the next launch assigns it again). s_l + A_l t_l overwrites s_l, which nothing reads again
// before the restriction from level l - 1 writes it in the next cycle (s_0
// is zero in Algorithm 4, so on level 0 the product alone is stored).
template <class CI, class T, int R, int UNR, int PF, bool GRP, int SB, bool STREAM = true>
__device__ __forceinline__ void fac_grid_r(const FacParams &P, const Block &B, int p, const WorkVecs<T> &W,
                                           unsigned char *fac_stage)
{
    T *__restrict__ U0 = W.u;
    T *__restrict__ U1 = W.u2;
    T *__restrict__ Pf = W.f;
    T *__restrict__ Pt = W.t;
    T *__restrict__ Ps = W.s;
    const int64_t rb = W.rb;
    const T *__restrict__ Pl1 = static_cast<const T *>(P.l1inv);
    // one half-sweep of level d over rows [r0, r1) of view V (slices from `first`)
    auto relax = [&](const FacLevelDesc &d, int g, const FacViewDev &V, int64_t s0, int first, int r0, int r1,
                     const auto &src, const T *own, T *dst, int t_mode) {
        relax_pass_r<CI, T, R, UNR, PF, GRP, SB, STREAM>(P, W, B, d, g, V, s0, first, r0, r1, src, own, dst, t_mode,
                                                         fac_stage);
    };
    {
        const FacLevelDesc *D = P.desc + (int64_t)p * P.nlev;
        const int L = P.nlev - 1;

        // f_l = r_l on the real rows of every level; u_0 = 0 (all its rows,
        // in U0). Nothing else needs a start value: u_l (l >= 1) and s_l are
        // written before they are read, t_l is assigned on first use.
        for (int l = 0; l <= L; ++l) {
            const FacLevelDesc d = D[l];
            const double *__restrict__ rl = P.r_all + P.level_off[l] * R;
            const int nr = l == 0 ? d.nBar : d.nReal;
            for (int r = B.tid; r < nr; r += B.nt) {
                const int64_t i = d.row0 + r;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (l == 0) U0[(i - rb) * R + j] = T(0);
                    if (r < d.nReal) Pf[(i - rb) * R + j] = (T)rl[P.gmap[i] * R + j];
                }
            }
        }
        B.sync();

        for (int c = 1; c <= P.nfac; ++c) {
            const bool first_cycle = c == 1;
            // t in the downsweep: assigned in the first cycle, else added to
            // the previous upsweep's; in the upsweep: assigned, or not kept
            // at all in the last cycle
            const int tdown = first_cycle ? kTAssign : kTAdd;
            const int tup = c == P.nfac ? kTNone : kTAssign;
            for (int l = 0; l < L; ++l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                const int gl = GRP ? P.grp[l] : 1, gn = GRP ? P.grp[l + 1] : 1;
                T *__restrict__ u0 = U0 + (d.row0 - rb) * R;
                T *__restrict__ u1 = U1 + (d.row0 - rb) * R;
                if (l > 0) {
                    // u_l = 0 and its first C half-sweep were done row by row
                    // by the restriction pass from level l - 1 (below)
                    relax(d, gl, P.AFc, d.sAFc, d.nC, d.nC, d.nReal, One<T, R>{u1}, u1, u1, tdown);
                } else if (first_cycle) {
                    // u_0 = 0 (prologue): every product of the C half-sweep is
                    // +0, so its correction is f / l1 with no row product, and
                    // the F half-sweep sees nonzero u only at C columns (view
                    // AFc; the omitted products are exact zeros)
                    T *__restrict__ t = Pt + (d.row0 - rb) * R;
                    const T *__restrict__ f = Pf + (d.row0 - rb) * R;
                    const T *__restrict__ l1 = Pl1 + d.row0;
                    for (int r = B.tid; r < d.nC; r += B.nt) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            const T v = f[r * R + j] * l1[r];
                            u1[r * R + j] = T(0) + v;
                            t[r * R + j] = v;
                        }
                    }
                    B.sync();
                    relax(d, gl, P.AFc, d.sAFc, d.nC, d.nC, d.nReal, One<T, R>{u1}, u0, u1, kTAssign);
                } else {
                    relax(d, gl, P.A, d.sA, 0, 0, d.nC, One<T, R>{u0}, u0, u1, tdown);
                    relax(d, gl, P.A, d.sA, 0, d.nC, d.nReal, Two<T, R>{u1, u0, d.nC}, u0, u1, tdown);
                }
                {
                    // s_l <- s_l + A_l t_l (s_0 = 0)
                    T *__restrict__ s = Ps + (d.row0 - rb) * R;
                    const One<T, R> t = stage<SB>(B, One<T, R>{Pt + (d.row0 - rb) * R}, (int64_t)d.nBar, fac_stage);
                    rows_dot<CI, T, R, UNR, PF, GRP, STREAM>(B, gl, P.At, d.sAt, d.row0, 0, 0, d.nBar, t,
                                                     [&](int r, const VecR<T, R> &at) {
#pragma unroll
                        for (int j = 0; j < R; ++j) s[r * R + j] = l == 0 ? at.v[j] : s[r * R + j] + at.v[j];
                    });
                }
                B.sync();
                {
                    const One<T, R> w = stage<SB>(B, One<T, R>{Ps + (d.row0 - rb) * R}, (int64_t)d.nBar, fac_stage);
                    const One<T, R> un{U0 + (dn.row0 - rb) * R};
                    T *__restrict__ s1 = Ps + (dn.row0 - rb) * R;
                    T *__restrict__ f1 = Pf + (dn.row0 - rb) * R;
                    T *__restrict__ t1 = Pt + (dn.row0 - rb) * R;
                    T *__restrict__ v1 = U1 + (dn.row0 - rb) * R;
                    const T *__restrict__ l1n = Pl1 + dn.row0;
                    const bool relaxed = l + 1 < L;
                    // the downsweep start of level l+1 < L for a real row whose
                    // f_{l+1} is final: u_{l+1} = 0 in U1, then on a C row the
                    // first half-sweep's correction f / l1 (u_{l+1} = 0 makes
                    // its row product +0). Ghost rows of U0 are not touched
                    // (this pass still reads u_{l+1} there); the upsweep
                    // assigns them.
                    auto start = [&](int r) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (r < dn.nC) {
                                const T v = f1[r * R + j] * l1n[r];
                                v1[r * R + j] = T(0) + v;
                                t1[r * R + j] = first_cycle ? v : t1[r * R + j] + v;
                            } else {
                                v1[r * R + j] = T(0);
                            }
                        }
                    };
                    // s_{l+1} = R_l w_l on every row of level l+1; then, on its
                    // real rows, f_{l+1} -= A_{l+1} u_{l+1} (cycles after the
                    // first; u_{l+1} is in U0 from the previous upsweep) and
                    // f_{l+1} -= s_{l+1}
                    if (!GRP || gn <= 1) {
                        for_rows(B, 0, 0, dn.nBar, [&](int r) {
                            const VecR<T, R> sv = view_dot_r<CI, T, R, UNR, PF, STREAM>(P.R, dn.sR, dn.row0, 0, r, w);
#pragma unroll
                            for (int j = 0; j < R; ++j) s1[r * R + j] = sv.v[j];
                            if (r < dn.nReal) {
                                if (!first_cycle) {
                                    const VecR<T, R> au =
                                        view_dot_r<CI, T, R, UNR, PF, STREAM>(P.A, dn.sA, dn.row0, 0, r, un);
#pragma unroll
                                    for (int j = 0; j < R; ++j)
                                        f1[r * R + j] = (f1[r * R + j] - au.v[j]) - sv.v[j];
                                } else {
#pragma unroll
                                    for (int j = 0; j < R; ++j) f1[r * R + j] = f1[r * R + j] - sv.v[j];
                                }
                                if (relaxed) start(r);
                            }
                        });
                    } else {
                        // groups: two traversals; row r has the same owning
                        // lane in both, which reads back its own s_{l+1}
                        rows_dot<CI, T, R, UNR, PF, GRP, STREAM>(B, gn, P.R, dn.sR, dn.row0, 0, 0, dn.nBar, w,
                                                         [&](int r, const VecR<T, R> &sv) {
#pragma unroll
                            for (int j = 0; j < R; ++j) s1[r * R + j] = sv.v[j];
                            if (first_cycle && r < dn.nReal) {
#pragma unroll
                                for (int j = 0; j < R; ++j) f1[r * R + j] = f1[r * R + j] - sv.v[j];
                                if (relaxed) start(r);
                            }
                        });
                        if (!first_cycle)
                            rows_dot<CI, T, R, UNR, PF, GRP, STREAM>(B, gn, P.A, dn.sA, dn.row0, 0, 0, dn.nReal, un,
                                                             [&](int r, const VecR<T, R> &au) {
#pragma unroll
                                for (int j = 0; j < R; ++j)
                                    f1[r * R + j] = (f1[r * R + j] - au.v[j]) - s1[r * R + j];
                                if (relaxed) start(r);
                            });
                    }
                }
                B.sync();
            }
            {
                const FacLevelDesc d = D[L];
                const T *__restrict__ f = Pf + (d.row0 - rb) * R;
                T *__restrict__ u = U0 + (d.row0 - rb) * R;
                // u_L = A_L^{-1} f_L in FP64 over the nonzeros of the inverse:
                // the chain starts at +0 and never returns to -0, so each
                // skipped fma(0, f_J, s) would have left s unchanged (finite f)
                for (int e = B.tid; e < P.nL * R; e += B.nt) {
                    const int I = e / R, j = e % R;
                    double s = 0.0;
                    const int32_t k1 = __ldg(P.ainv_ptr + I + 1);
                    for (int32_t k = __ldg(P.ainv_ptr + I); k < k1; ++k)
                        s = fma(__ldg(P.ainv_val + k), (double)f[__ldg(P.ainv_col + k) * R + j], s);
                    u[I * R + j] = (T)s;
                }
            }
            B.sync();
            for (int l = L - 1; l >= 0; --l) {
                const FacLevelDesc d = D[l];
                const FacLevelDesc dn = D[l + 1];
                T *__restrict__ u0 = U0 + (d.row0 - rb) * R;
                T *__restrict__ u1 = U1 + (d.row0 - rb) * R;
                const One<T, R> un = stage<SB>(B, One<T, R>{U0 + (dn.row0 - rb) * R}, (int64_t)dn.nBar, fac_stage);
                const int gl = GRP ? P.grp[l] : 1;
                // u_l += P_l u_{l+1}: real rows in U1, ghost rows in U0; on
                // l >= 1 the ghost rows, zero since this cycle's downsweep and
                // never relaxed, are written 0 + P_l u_{l+1} (u_0 keeps its
                // ghost values from cycle to cycle)
                rows_dot<CI, T, R, UNR, PF, GRP, STREAM>(B, gl, P.P, d.sP, d.row0, 0, 0, d.nBar, un,
                                                 [&](int r, const VecR<T, R> &pu) {
                    if (r < d.nReal) {
#pragma unroll
                        for (int j = 0; j < R; ++j) u1[r * R + j] = u1[r * R + j] + pu.v[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < R; ++j) u0[r * R + j] = (l > 0 ? T(0) : u0[r * R + j]) + pu.v[j];
                    }
                });
                B.sync();
                relax(d, gl, P.A, d.sA, 0, d.nC, d.nReal, Two<T, R>{u1, u0, d.nReal}, u1, u0, tup);
                relax(d, gl, P.A, d.sA, 0, 0, d.nC, Two<T, R>{u1, u0, d.nC}, u1, u0, tup);
            }
        }

        const FacLevelDesc d0 = D[0];
        const int64_t o0 = P.owned0[p], o1 = P.owned0[p + 1];
        for (int64_t k = o0 + B.tid; k < o1; k += B.nt) {
            const int64_t i = d0.row0 + P.owned[k];
            const int64_t g = P.gmap[i];
#pragma unroll
            for (int j = 0; j < R; ++j) P.x[g * R + j] = P.x[g * R + j] + (double)U0[(i - rb) * R + j];
        }
    }
}

// The work vectors in the global arrays of P (u2 is P.d).
template <class T>
__device__ __forceinline__ WorkVecs<T> global_vecs(const FacParams &P)
{
    return WorkVecs<T>{static_cast<T *>(P.u), static_cast<T *>(P.d), static_cast<T *>(P.f), static_cast<T *>(P.t),
                       static_cast<T *>(P.s), 0};
}

// One block of 512 threads per composite grid at a time; a block claims its
// grids from the bin of the SM it runs on, then from the other bins.
template <class CI, class T, int R, int UNR, int MINB, int PF, bool GRP, int SB>
__global__ void __launch_bounds__(512, MINB) k_fac_all_grids_r(FacParams P)
{
    extern __shared__ __align__(16) unsigned char fac_stage[];
    Block B;
    B.tid = threadIdx.x;
    B.nt = blockDim.x;
    B.lane = threadIdx.x & 31;
    B.warp = threadIdx.x >> 5;
    B.nw = blockDim.x >> 5;
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
        fac_grid_r<CI, T, R, UNR, PF, GRP, SB>(P, B, p, global_vecs<T>(P), fac_stage);
    }
}

// Teams: blocks of 1024 threads (two per SM), each split by the host into up
// to 15 teams of whole warps; team k of a block cycles the grids of its list
// in order, waiting only on its own named barrier (k + 1). The host sizes each
// team by the work of its grids, so that the teams of the whole launch finish
// together instead of the largest grids' blocks ending it alone.
template <class CI, class T, int R, int UNR, int PF>
__global__ void __launch_bounds__(1024, 2) k_fac_teams(FacParams P, FacTeams TT)
{
    const int w = threadIdx.x >> 5;
    const int k0 = TT.block_off[blockIdx.x], k1 = TT.block_off[blockIdx.x + 1];
    int k = k0;
    while (k < k1 && !(w >= TT.w0[k] && w < TT.w0[k] + TT.nw[k])) ++k;
    if (k >= k1) return;   // a warp of no team
    Block B;
    B.lane = threadIdx.x & 31;
    B.warp = w - TT.w0[k];
    B.nw = TT.nw[k];
    B.tid = (int)threadIdx.x - 32 * TT.w0[k];
    B.nt = 32 * TT.nw[k];
    B.bar = k - k0 + 1;
    for (int j = TT.grid_off[k]; j < TT.grid_off[k + 1]; ++j)
        fac_grid_r<CI, T, R, UNR, PF, false, 0>(P, B, TT.grid[j], global_vecs<T>(P), nullptr);
}

}  // namespace dev

// Variant v of the composite-grid kernel for R columns: entries in flight per
// row (UNR), resident blocks per SM (MINB) of 512 threads, and the L2
// prefetch distance in steps (PF, 0 = none).
//   1: UNR 1, 2 blocks    2: UNR 2, 2 blocks    3: UNR 2, 3 blocks
//   4: UNR 4, 2 blocks    5: UNR 1, 4 blocks    6: UNR 2, 4 blocks
//   7: UNR 2, 4 blocks, PF 2    8: UNR 2, 3 blocks, PF 2
//   9: UNR 2, 4 blocks, PF 4
//  10: UNR 2, 3 blocks, PF 2, with g lanes per row on level l where
//      P.grp[l] = g > 1
//  11: UNR 2, 4 blocks, 2 steps ahead into L1   12: same, 4 steps ahead
//  13-15: as 7, with gathered level vectors of up to 16, 32 or 44 KB staged
//      in shared memory (with the block's static shared memory, the total
//      stays within the 48 KB a launch gets without an opt-in attribute)
//  16: UNR 2, PF 2 in the team-partitioned kernel (blocks of 1024 threads,
//      two per SM, split into teams sized by their grids' work; the plan is
//      P.teams)
// 32-bit local columns (composite levels above 65,535 points) use variant 1.
constexpr int kMultiVariants = 16;

template <class CI, class T, int R, int UNR, int MINB, int PF = 0, bool GRP = false, int SB = 0>
cudaError_t launch_fac_r_variant(const FacParams &P, int nsub, cudaStream_t st)
{
    static_assert(SB % 16 == 0 && SB <= 44 * 1024, "staging buffer plus static shared memory within 48 KB");
    auto kern = dev::k_fac_all_grids_r<CI, T, R, UNR, MINB, PF, GRP, SB>;
    int per_sm = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, SB);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // every block that fits at once (the bins only say where blocks look first)
    int ctas = (per_sm < 1 ? 1 : per_sm) * (nsm < 1 ? 1 : nsm);
    if (ctas > nsub) ctas = nsub;
    if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(int32_t) * (size_t)P.nbins, st)) != cudaSuccess) return e;
    kern<<<ctas, 512, SB, st>>>(P);
    return cudaGetLastError();
}

template <class CI, class T, int R>
cudaError_t launch_fac_teams_variant(const FacParams &P, cudaStream_t st)
{
    const FacTeams &TT = P.teams;
    if (TT.nblocks < 1 || !TT.block_off || !TT.w0 || !TT.nw || !TT.grid_off || !TT.grid) return cudaErrorInvalidValue;
    dev::k_fac_teams<CI, T, R, 2, 2><<<TT.nblocks, 1024, 0, st>>>(P, TT);
    return cudaGetLastError();
}

template <class T, int R>
cudaError_t launch_fac_r_typed(const FacParams &P, int nsub, int variant, cudaStream_t st)
{
    if (!P.col16) return launch_fac_r_variant<int32_t, T, R, 1, 2>(P, nsub, st);
    switch (variant) {
    case 16: return launch_fac_teams_variant<uint16_t, T, R>(P, st);
    case 2: return launch_fac_r_variant<uint16_t, T, R, 2, 2>(P, nsub, st);
    case 3: return launch_fac_r_variant<uint16_t, T, R, 2, 3>(P, nsub, st);
    case 4: return launch_fac_r_variant<uint16_t, T, R, 4, 2>(P, nsub, st);
    case 5: return launch_fac_r_variant<uint16_t, T, R, 1, 4>(P, nsub, st);
    case 6: return launch_fac_r_variant<uint16_t, T, R, 2, 4>(P, nsub, st);
    case 7: return launch_fac_r_variant<uint16_t, T, R, 2, 4, 2>(P, nsub, st);
    case 8: return launch_fac_r_variant<uint16_t, T, R, 2, 3, 2>(P, nsub, st);
    case 9: return launch_fac_r_variant<uint16_t, T, R, 2, 4, 4>(P, nsub, st);
    case 10: return launch_fac_r_variant<uint16_t, T, R, 2, 3, 2, true>(P, nsub, st);
    case 11: return launch_fac_r_variant<uint16_t, T, R, 2, 4, -2>(P, nsub, st);
    case 12: return launch_fac_r_variant<uint16_t, T, R, 2, 4, -4>(P, nsub, st);
    case 13: return launch_fac_r_variant<uint16_t, T, R, 2, 4, 2, false, 16384>(P, nsub, st);
    case 14: return launch_fac_r_variant<uint16_t, T, R, 2, 4, 2, false, 32768>(P, nsub, st);
    case 15: return launch_fac_r_variant<uint16_t, T, R, 2, 4, 2, false, 45056>(P, nsub, st);
    default: return launch_fac_r_variant<uint16_t, T, R, 1, 2>(P, nsub, st);
    }
}

}  // namespace amgdd
