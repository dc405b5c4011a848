// kx_traverse_impl.cuh -- device helpers shared by the traversal of
// kx_exchange (kx_traverse.cu) and the allocation-free level step
// (kx_noalloc.cu), so that both apply exactly the same Eq. 8 query and the
// same deterministic compaction.
#pragma once

#include "kx_internal.cuh"

namespace kx {

// A shard of the K rows: only row blocks A whose tree positions meet
// [r0, r1) are traversed; lo/hi give the tree-position range [lo, hi) of
// every node of the level the children live on.  lo == nullptr: all rows.
struct RowRange {
    const int32_t* lo;
    const int32_t* hi;
    int r0, r1;
    __device__ bool keeps(int node) const { return !lo || (lo[node] < r1 && hi[node] > r0); }
};

// Survivor mask of the up to 16 children of task t = (A,B,C,D) one level
// down (Eq. 7): bit ((iA*2 + iB)*2 + iC)*2 + iD is set iff
//     beta = (||Q_{A'B'}|| * ||P_{B'D'}||) * ||Q_{C'D'}|| > tau
// (Eq. 8, IEEE products without fused multiply-add).  The next level's norm
// tables of the task's system hold entry (X,Y) at t0 + X * nn + Y.  With
// diag (a symmetric build and A == C) only the children with iA <= iC are
// tested: every child of a node left of another lies left of all of the
// other's children, so the K blocks (A',C') with A' <= C' are exactly these.
// Children whose row block A' lies outside `rows` are dropped.
__device__ __forceinline__ unsigned task_child_mask(const Task t, const int32_t* __restrict__ child,
                                                    const int32_t* __restrict__ nchild,
                                                    const double* __restrict__ S, const double* __restrict__ Pn,
                                                    int64_t t0, int nn, double tau, bool diag,
                                                    const RowRange rows) {
    const int ca = child[t.a], na = nchild[t.a];
    const int cb = child[t.b], nb = nchild[t.b];
    const int cc = child[t.c], nc = nchild[t.c];
    const int cd = child[t.d], nd = nchild[t.d];
    unsigned m = 0;
    for (int ia = 0; ia < na; ++ia) {
        if (!rows.keeps(ca + ia)) continue;
        for (int ib = 0; ib < nb; ++ib) {
            const double sab = S[t0 + (int64_t)(ca + ia) * nn + (cb + ib)];
            for (int id = 0; id < nd; ++id) {
                const double x = __dmul_rn(sab, Pn[t0 + (int64_t)(cb + ib) * nn + (cd + id)]);
                for (int ic = diag ? ia : 0; ic < nc; ++ic) {
                    const double beta = __dmul_rn(x, S[t0 + (int64_t)(cc + ic) * nn + (cd + id)]);
                    if (beta > tau) m |= 1u << (((ia * 2 + ib) * 2 + ic) * 2 + id);
                }
            }
        }
    }
    return m;
}

// The children of task t selected by mask m, in bit order ((iA, iB, iC, iD),
// A most significant), written at out[pos], out[pos+1], ...; positions at
// or beyond cap are skipped.  Returns the position after the last child.
__device__ __forceinline__ int64_t write_children(const Task t, unsigned m, const int32_t* __restrict__ child,
                                                  Task* __restrict__ out, int64_t pos, int64_t cap) {
    const int ca = child[t.a], cb = child[t.b], cc = child[t.c], cd = child[t.d];
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        if (pos < cap)
            out[pos] = Task{(uint16_t)(ca + ((bit >> 3) & 1)), (uint16_t)(cb + ((bit >> 2) & 1)),
                            (uint16_t)(cc + ((bit >> 1) & 1)), (uint16_t)(cd + (bit & 1))};
        ++pos;
    }
    return pos;
}

// Exclusive prefix sum of v over the block (blockDim.x a multiple of 32, at
// most 1024 threads; sh holds 32 entries); *total = the block's sum.
__device__ __forceinline__ int64_t block_excl_scan64(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int64_t ex = x - v + (w > 0 ? sh[w - 1] : 0);
    *total = sh[nw - 1];
    __syncthreads();
    return ex;
}

}  // namespace kx
