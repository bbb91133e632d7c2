// The row of the fused SELL-32 step (sliced layout with column indices or
// with offset patterns): the slot loop and the epilogue, shared by the
// single-system step kernels (nc_sell.cu) and the batched engine's explicit-
// matrix slots (nc_batch.cu).
#pragma once

#include <type_traits>

#include "nc_step.cuh"

namespace nc {

constexpr int kSellGroup = 8;

// One row: the slot loop and the epilogue; returns the row's dot term.
// PAT: the slice's columns are row + its pattern's offsets (clamped to the
// matrix, for padded slots whose offset leaves it; their value is 0), not
// loaded from `col`.
template <typename VT, typename XT, typename YT, int DOT, bool PAT, bool UNIT>
__device__ __forceinline__ double sell_row(const int row, const int n, const int32_t* __restrict__ slice_ptr,
                                           const int32_t* __restrict__ col, const SellPat& pat,
                                           const VT* __restrict__ val, const XT* __restrict__ u,
                                           const XT* __restrict__ w, const XT* __restrict__ r, YT* __restrict__ y,
                                           const StepCoef<typename AccOf<XT>::type>& c,
                                           const double* __restrict__ rdot) {
    using AT = typename AccOf<XT>::type;
    // float32 values: r and x_{k-2} depend on nothing, so their loads go out
    // first and their latency overlaps the slot loop's instead of following
    // it (the float32 step of the 128^3 system 25.6 -> 21.8 us); with
    // float64 or bfloat16 values the same order measured slower (41.9 ->
    // 43.5 and 25.4 -> 31.7 us), so those load them in the epilogue
    constexpr bool kEarly = std::is_same<VT, float>::value;
    AT rv = AT(0), wv = AT(0);
    if constexpr (kEarly) {
        if (c.terms & kTermR) rv = (AT)r[row];
        if (c.terms & kTermW) wv = (AT)w[row];
    }
    const int s = row >> 5;
    const int beg = slice_ptr[s];
    const int len = (slice_ptr[s + 1] - beg) >> 5;   // warp-uniform
    const VT* vp = val + beg + (row & 31);
    const int32_t* cp = nullptr;   // plain: the slot's column indices
    const int32_t* op = nullptr;   // PAT: the slice's offsets
    if constexpr (PAT) op = pat.poff + __ldg(pat.pstart + s);
    else cp = col + beg + (row & 31);
    // column of slot t of the current group
    auto colt = [&](int t) -> int {
        if constexpr (PAT) return min(max(row + __ldg(op + t), 0), n - 1);
        else return ld_stream(cp + 32 * t);
    };
    auto advance = [&](int g) {
        vp += 32 * g;
        if constexpr (PAT) op += g;
        else cp += 32 * g;
    };
    AT acc = AT(0);
    if constexpr (sizeof(AT) == 8) {
        // float64: the fma chain itself is long-latency on GB300's narrow
        // FP64 pipe, so occupancy matters most: a 4-slot unroll keeps the
        // kernel at 32 registers and 8 CTAs (2048 threads) per SM.
        int j = 0;
        for (; j + 4 <= len; j += 4) {
            const int c0 = colt(0), c1 = colt(1), c2 = colt(2), c3 = colt(3);
            const AT v0 = (AT)ld_stream(vp), v1 = (AT)ld_stream(vp + 32), v2 = (AT)ld_stream(vp + 64),
                     v3 = (AT)ld_stream(vp + 96);
            const AT x0 = (AT)__ldg(u + c0), x1 = (AT)__ldg(u + c1), x2 = (AT)__ldg(u + c2),
                     x3 = (AT)__ldg(u + c3);
            acc = fma(v0, x0, acc);
            acc = fma(v1, x1, acc);
            acc = fma(v2, x2, acc);
            acc = fma(v3, x3, acc);
            advance(4);
        }
        for (; j < len; ++j) {
            const int c0 = colt(0);
            acc = fma((AT)ld_stream(vp), (AT)__ldg(u + c0), acc);
            advance(1);
        }
    } else {
        // float: memory latency is the limit, so every column and value
        // load of a group of 8 slots is issued before the gathers, and all
        // gathers before the fma chain: a grid row (<= 8 slots) costs two
        // memory latencies in total.  The guards are warp-uniform.
        constexpr int G = kSellGroup;
        for (int j0 = 0; j0 < len; j0 += G) {
            int cc_[G];
            AT vv[G], xx[G];
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) {
                    cc_[t] = colt(t);
                    vv[t] = (AT)ld_stream(vp + 32 * t);
                }
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) xx[t] = (AT)__ldg(u + cc_[t]);
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) acc = fma(vv[t], xx[t], acc);
            advance(G);
        }
    }
    if constexpr (kEarly) return sell_row_out<XT, YT, DOT, AT, UNIT>(row, acc, c, rv, wv, u, y, rdot);
    else return step_row_out<XT, YT, DOT, AT, UNIT>(row, acc, c, u, w, r, y, rdot);
}

}  // namespace nc
