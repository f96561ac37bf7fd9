// Device helpers shared by the composite-grid (FAC) kernels.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace amgdd {
namespace dev {

// The threads that cycle one composite grid: a whole block (bar = 0), or a
// team of whole warps inside a block that waits on its own named barrier
// (bar = 1..15) and never on the other teams.
struct Block {
    int lane, warp, nw, tid, nt;
    int bar = 0;
    __device__ __forceinline__ void sync() const
    {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

// Loads of operator entries, which every launch streams once: evict-first
// (ld.global.cs) when STREAM is set, so they do not push the composite-grid
// vectors out of L2; read-only path (ld.global.nc) otherwise.
template <bool STREAM, class X>
__device__ __forceinline__ X ld_op(const X *p)
{
    if constexpr (STREAM) return __ldcs(p);
    else return __ldg(p);
}

// Local rows [r0, r1) of a view whose slices start at local row `first`
// (r0 >= first), thread-per-row, warp-per-slice.
template <class Fn>
__device__ __forceinline__ void for_rows(const Block &B, int first, int r0, int r1, Fn &&fn)
{
    if (r1 <= r0) return;
    const int q0 = (r0 - first) >> 5, q1 = (r1 - first + 31) >> 5;
    for (int q = q0 + B.warp; q < q1; q += B.nw) {
        const int r = first + (q << 5) + B.lane;
        if (r >= r0 && r < r1) fn(r);
    }
}

// Warp-uniform traversal of the slices covering local rows [r0, r1) of a view
// whose slices start at `first`; fn(q, r, active) is called by every lane.
template <class Fn>
__device__ __forceinline__ void for_slices(const Block &B, int first, int r0, int r1, Fn &&fn)
{
    if (r1 <= r0) return;
    const int q0 = (r0 - first) >> 5, q1 = (r1 - first + 31) >> 5;
    for (int q = q0 + B.warp; q < q1; q += B.nw) {
        const int r = first + (q << 5) + B.lane;
        fn(q, r, r >= r0 && r < r1);
    }
}

}  // namespace dev
}  // namespace amgdd
