// The k passes of the 1D box filter (Sec. 3.1) over one row held by one warp.
//
// Lane l owns the contiguous cells [l*C, (l+1)*C) of a row of 32*C cells in
// registers (R = the radius r, a template parameter so that every window index is a
// compile-time register). A pass first fetches the R+1 cells on one side of the
// chunk and the R on the other from the neighbouring lanes by warp shuffles; lane 0
// and lane 31 take the half-sample reflection of their own cells instead (cell -1-i
// is cell i, cell n+i is cell n-1-i). R < C keeps every border within one
// neighbour's chunk and every reflected cell within the edge lane's own chunk. Each
// output is a running window sum: one addition of the cell entering the window and
// one subtraction of the cell leaving it, in unsigned arithmetic (wrap-around
// cancels). The first window is summed as a balanced tree.
//
// Passes alternate direction so that no pass moves its outputs back into place:
//  - left to right: the chunk at E[R+1 .. R+C] (cell c at E[c+R+1], c in [-R-1, C+R));
//    output c is written over cell c-R-1, the one that just left the window, so the
//    outputs land at E[0 .. C-1];
//  - right to left: the chunk at E[0 .. C-1] (cell c at E[c] for c in [0, C+R], cell
//    -j at E[C+R+j] for j in [1, R]); output c is written over cell c+R+1, the one
//    that just left, so the outputs land at E[R+1 .. R+C] again.
#pragma once

namespace heb {

// E[A] + ... + E[A+M-1] as a balanced tree.
template <int A, int M, typename TS, int N>
__device__ __forceinline__ TS tree_sum(const TS (&E)[N]) {
    if constexpr (M == 1) {
        return E[A];
    } else {
        return tree_sum<A, M / 2>(E) + tree_sum<A + M / 2, M - M / 2>(E);
    }
}

template <typename TS, int C, int R>
__device__ __forceinline__ void box_pass_lr(TS (&E)[C + 2 * R + 1], int lane) {
    // cells -R-1 .. -1: the previous lane's C-R-1 .. C-1; lane 0 reflects its 0 .. R
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        const TS left = __shfl_up_sync(0xffffffffu, E[C + m], 1);
        E[m] = lane == 0 ? E[2 * R + 1 - m] : left;
    }
    // cells C .. C+R-1: the next lane's 0 .. R-1; lane 31 reflects its C-1 .. C-R
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const TS right = __shfl_down_sync(0xffffffffu, E[R + 1 + m], 1);
        E[R + 1 + C + m] = lane == 31 ? E[R + C - m] : right;
    }
    TS s = tree_sum<0, 2 * R + 1>(E);  // cells -R-1 .. R-1
#pragma unroll
    for (int q = 0; q < C; ++q) {
        s += E[q + 2 * R + 1] - E[q];  // cell q+R enters, cell q-R-1 leaves
        E[q] = s;
    }
}

template <typename TS, int C, int R>
__device__ __forceinline__ void box_pass_rl(TS (&E)[C + 2 * R + 1], int lane) {
    // cells C .. C+R: the next lane's 0 .. R; lane 31 reflects its C-1 .. C-1-R
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        const TS right = __shfl_down_sync(0xffffffffu, E[m], 1);
        E[C + m] = lane == 31 ? E[C - 1 - m] : right;
    }
    // cells -1 .. -R (at E[C+R+1 ..]): the previous lane's C-1 .. C-R; lane 0 reflects 0 .. R-1
#pragma unroll
    for (int j = 1; j <= R; ++j) {
        const TS left = __shfl_up_sync(0xffffffffu, E[C - j], 1);
        E[C + R + j] = lane == 0 ? E[j - 1] : left;
    }
    TS s = tree_sum<C - 1 - R, 2 * R + 1>(E);  // cells C-1-R .. C-1+R
    E[C + R] = s;                              // output C-1 over cell C+R
#pragma unroll
    for (int x = C - 2; x >= 0; --x) {
        // cell x-R enters (at E[x-R], or E[C+2R-x] left of the chunk), cell x+R+1 leaves
        s += E[x - R >= 0 ? x - R : C + 2 * R - x] - E[x + R + 1];
        E[x + R + 1] = s;
    }
}

// k passes; the outputs end at E[R+1 .. R+C] (where the input was).
template <typename TS, int C, int R>
__device__ __forceinline__ void box_passes_shfl(TS (&E)[C + 2 * R + 1], int lane, int passes) {
    static_assert(R >= 1 && R < C, "the border must come from one neighbour");
    int p = 0;
    for (; p + 1 < passes; p += 2) {
        box_pass_lr<TS, C, R>(E, lane);
        box_pass_rl<TS, C, R>(E, lane);
    }
    if (p < passes) {
        box_pass_lr<TS, C, R>(E, lane);
#pragma unroll
        for (int q = C - 1; q >= 0; --q) E[R + 1 + q] = E[q];
    }
}

}  // namespace heb
