// SELL-32: sliced ELLPACK layout of a CSR matrix for the fused step kernel.
//
// Rows are grouped in slices of 32 consecutive rows (one warp).  Inside a
// slice the nonzeros are stored slot-major: slot j of row 32s + l sits at
// slice_ptr[s] + 32 j + l, and every row of the slice is padded to the
// slice's longest row with (value 0, column = the row itself).  A warp then
// reads slot j of its 32 rows with one coalesced load, no shared-memory
// staging and no barrier is needed, and all slot loads of a row are
// independent, so many of them are in flight at once.  For grid operators
// the columns of slot j are consecutive across the slice, which makes the
// gathers of x_{k-1} coalesced as well.  Slots are filled in CSR order and a
// padded slot adds fma(0, u_row, acc) = acc, so each row's sum is the same
// fma chain, in the same order, as the CSR kernel's.
//
// The layout is built once at solver setup from the CSR arrays; it is chosen
// when its padding is small (grid and finite-element matrices), otherwise
// the CSR kernel runs.  Its offset-pattern form (below, PAT) drops the column
// indices where the slices' columns are row + a few repeated offsets.  The
// solver stores the shifted operator A - theta' I
// (only diagonal entries change): the p_k recursion of Sec. 3 applies
// 2 sigma (1 - A/theta') = -(2/delta)(A - theta' I), so with the shift every
// Chebyshev step after the first needs no separate x_{k-1} term, one FP64
// instruction less per row on GB300's narrow FP64 pipe; the outer products
// add theta' u back (q = A' p + theta' p).
#include <climits>
#include <type_traits>

#include "nc_sell.cuh"

namespace nc {
namespace {

// Two rows per thread (rows row0 and row0 + 256: slices w and w + 8 of a
// 512-row tile for warp w), no dot product: every load of both rows is
// issued before either fma chain, so twice the loads are in flight per warp
// (the float step is latency-bound).  Each row's arithmetic is sell_row's.
template <typename VT, typename XT, typename YT, bool PAT, bool UNIT>
__device__ __forceinline__ void sell_rows2(const int row0, const int n, const int32_t* __restrict__ slice_ptr,
                                           const int32_t* __restrict__ col, const SellPat& pat,
                                           const VT* __restrict__ val, const XT* __restrict__ u,
                                           const XT* __restrict__ w, const XT* __restrict__ r, YT* __restrict__ y,
                                           const StepCoef<typename AccOf<XT>::type>& c) {
    using AT = typename AccOf<XT>::type;
    constexpr int Q = 2;
    const int nslices = (n + 31) >> 5;
    int row[Q], len[Q];
    bool act[Q];
    const VT* vp[Q];
    const int32_t* cp[Q];
    AT rv[Q], wv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        row[q] = row0 + kBlock * q;
        act[q] = row[q] < n;
        rv[q] = (act[q] && (c.terms & kTermR)) ? (AT)r[row[q]] : AT(0);
        wv[q] = (act[q] && (c.terms & kTermW)) ? (AT)w[row[q]] : AT(0);
        const int s = row[q] >> 5;
        len[q] = 0;
        vp[q] = val;
        cp[q] = col;
        if (s < nslices) {   // warp-uniform; lanes past n read padded slots (clamped columns)
            const int beg = slice_ptr[s];
            len[q] = (slice_ptr[s + 1] - beg) >> 5;
            vp[q] = val + beg + (row[q] & 31);
            if constexpr (PAT) cp[q] = pat.poff + __ldg(pat.pstart + s);
            else cp[q] = col + beg + (row[q] & 31);
        }
    }
    auto colt = [&](int q, int t) -> int {
        if constexpr (PAT) return min(max(row[q] + __ldg(cp[q] + t), 0), n - 1);
        else return ld_stream(cp[q] + 32 * t);
    };
    constexpr int G = sizeof(AT) == 8 ? 4 : kSellGroup;
    const int maxlen = max(len[0], len[1]);
    AT acc[Q] = {AT(0), AT(0)};
    for (int j0 = 0; j0 < maxlen; j0 += G) {
        int cc_[Q][G];
        AT vv[Q][G], xx[Q][G];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len[q]) {
                    cc_[q][t] = colt(q, j0 + t);
                    vv[q][t] = (AT)ld_stream(vp[q] + 32 * (j0 + t));
                }
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len[q]) xx[q][t] = (AT)__ldg(u + cc_[q][t]);
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len[q]) acc[q] = fma(vv[q][t], xx[q][t], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (act[q]) sell_row_out<XT, YT, 0, AT, UNIT>(row[q], acc[q], c, rv[q], wv[q], u, y, nullptr);
}

// Resident CTAs per SM the register budget aims at: plain steps 8 with
// float64 values (32 registers), 5 with float32 (48), 4 with bfloat16 (64),
// 3 with two rows per thread; dot-product variants 8 in float64 (32: they fit
// without spilling, so a persistent grid of 8 per SM is one wave) and 4 in
// float (64).
template <typename VT, typename XT, int DOT, int RPT>
constexpr int sell_min_ctas() {
    constexpr bool f64 = sizeof(typename AccOf<XT>::type) == 8;
    return DOT != 0 ? (f64 ? 8 : 4) : (RPT == 2 ? 3 : (f64 ? 8 : (sizeof(VT) == 4 ? 5 : 4)));
}

template <typename VT, typename XT, typename YT, int DOT, bool PAT, bool UNIT, int RPT = 1>
__global__ void __launch_bounds__(kBlock, sell_min_ctas<VT, XT, DOT, RPT>())
sell_step_kernel(const int n, const int32_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                 const SellPat pat, const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                 const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                 const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done, const int ahead) {
    if (done != nullptr && *done) return;
    if constexpr (DOT == 0 && RPT == 2) {
        // one 512-row tile (two 256-row tiles) per CTA
        if constexpr (sizeof(typename AccOf<XT>::type) == 4)
            if (threadIdx.x < 2 && ahead > 0)
                prefetch_sell_tile(2 * ((int)blockIdx.x + ahead) + (int)threadIdx.x, n, slice_ptr, PAT ? nullptr : col,
                                   val);
        sell_rows2<VT, XT, YT, PAT, UNIT>(2 * (int)blockIdx.x * kBlock + (int)threadIdx.x, n, slice_ptr, col, pat, val,
                                          u, w, r, y, c);
    } else if constexpr (DOT == 0) {
        // one 256-row tile per CTA
        if constexpr (sizeof(typename AccOf<XT>::type) == 4)
            if (threadIdx.x == 0 && ahead > 0)
                prefetch_sell_tile((int)blockIdx.x + ahead, n, slice_ptr, PAT ? nullptr : col, val);
        const int row = blockIdx.x * kBlock + threadIdx.x;
        if (row < n) sell_row<VT, XT, YT, 0, PAT, UNIT>(row, n, slice_ptr, col, pat, val, u, w, r, y, c, rdot);
    } else {
        // with a dot product: a persistent grid loops over the tiles and
        // reduces once per CTA
        double dv = 0.0;
        const int ntiles = (n + kBlock - 1) / kBlock;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if constexpr (sizeof(typename AccOf<XT>::type) == 4)
                if (threadIdx.x == 0 && ahead > 0)
                    prefetch_sell_tile(tile + (int)gridDim.x, n, slice_ptr, PAT ? nullptr : col, val);
            const int row = tile * kBlock + threadIdx.x;
            if (row < n)
                dv += sell_row<VT, XT, YT, DOT, PAT, UNIT>(row, n, slice_ptr, col, pat, val, u, w, r, y, c, rdot);
        }
        grid_reduce<kBlock>(dv, R);
    }
}

// longest row of each slice
__global__ void sell_len_kernel(int n, const int32_t* __restrict__ rowptr, int32_t* __restrict__ slice_len) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int nslices = (n + 31) >> 5;
    int len = 0;
    if (row < n) len = rowptr[row + 1] - rowptr[row];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && (row >> 5) < nslices) slice_len[row >> 5] = len;
}

__device__ __forceinline__ void put_val(double* p, double v) { *p = v; }
__device__ __forceinline__ void put_val(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void put_val(__nv_bfloat16* p, double v) { *p = __double2bfloat16(v); }

// Slot-major fill.  The diagonal entry of every row is stored shifted,
// a_ii - shift (shift = 0 stores A itself); *nodiag is set if some row has
// no stored diagonal entry to shift.
template <typename VT>
__global__ void sell_fill_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const int32_t* __restrict__ slice_ptr,
                                 double shift, int32_t* __restrict__ scol, VT* __restrict__ sval,
                                 int* __restrict__ nodiag) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int nslices = (n + 31) >> 5;
    if ((row >> 5) >= nslices) return;
    const int s = row >> 5;
    const int beg = slice_ptr[s] + (row & 31);
    const int len = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    int rs = 0, rl = 0;
    if (row < n) {
        rs = rowptr[row];
        rl = rowptr[row + 1] - rs;
    }
    const int self = row < n ? row : n - 1;
    bool has_diag = false;
    for (int j = 0; j < len; ++j) {
        const int idx = beg + 32 * j;
        if (j < rl) {
            const int cj = col[rs + j];
            scol[idx] = cj;
            double v = val[rs + j];
            if (cj == row) {
                v -= shift;
                has_diag = true;
            }
            put_val(&sval[idx], v);
        } else {
            scol[idx] = self;
            put_val(&sval[idx], 0.0);
        }
    }
    if (row < n && !has_diag && shift != 0.0 && nodiag != nullptr) atomicOr(nodiag, 1);
}

// Offset patterns.  The columns of a row of a regularly numbered grid are
// row + a few fixed offsets; a slice of 32 such rows shares one sorted set of
// offsets (col - row), and all interior slices share the same set.  The
// pattern layout stores each distinct set once and per slice only where its
// set starts, so a step reads no column indices: 4 bytes less per stored
// entry and no dependent column load before the gathers.  Rows that lack an
// offset of their slice's set (faces of the grid) hold a 0 there.

// Merge of one slice's 32 sorted rows of offsets into its set, one warp per
// slice: each round takes the warp's smallest pending offset (an offset a row
// repeats counts once per repetition), so a slice holding L entries ends
// after at most L rounds.  Counting pass (off null): cnt[s].  Writing pass:
// off[opos[s] + j].  *bad is set if a row's columns do not increase or a
// slice needs more than kPatMaxSlots offsets.  skip_diag: the diagonal
// entries are left out (a constant diagonal applied by the step's u term).
constexpr int kPatMaxSlots = 64;

__global__ void psell_merge_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ opos, int32_t* __restrict__ cnt,
                                   int32_t* __restrict__ off, int* __restrict__ bad, const int skip_diag) {
    const int s = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nslices = (n + 31) >> 5;
    if (s >= nslices) return;   // warp-uniform
    const int row = s * 32 + lane;
    int pos = 0, end = 0;
    if (row < n) {
        pos = rowptr[row];
        end = rowptr[row + 1];
    }
    const int base = off != nullptr ? opos[s] : 0;
    int last = INT_MIN, c = 0;
    bool fail = false;
    while (true) {
        if (skip_diag && pos < end && col[pos] == row) ++pos;   // at most once: the columns increase
        const int my = pos < end ? col[pos] - row : INT_MAX;
        int m = my;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (m == INT_MAX) break;
        if (c >= kPatMaxSlots) {
            fail = true;
            break;
        }
        if (off != nullptr && lane == 0) off[base + c] = m;
        if (my == m) {
            if (my < last) fail = true;
            last = my;
            ++pos;
        }
        ++c;
    }
    if (__any_sync(0xffffffffu, fail) && lane == 0) atomicOr(bad, 1);
    if (off == nullptr && lane == 0) cnt[s] = c;
}

// Slot-major fill of the pattern layout: slot j of a row holds its entry at
// column row + offset j, or 0; diagonal entries stored as a_ii - shift, or
// not at all (skip_diag: the pattern has no offset 0 for them).
template <typename VT>
__global__ void psell_fill_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, const int32_t* __restrict__ slice_ptr,
                                  const int32_t* __restrict__ pstart, const int32_t* __restrict__ poff, double shift,
                                  VT* __restrict__ sval, int* __restrict__ nodiag, const int skip_diag) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int nslices = (n + 31) >> 5;
    if ((row >> 5) >= nslices) return;
    const int s = row >> 5;
    const int beg = slice_ptr[s] + (row & 31);
    const int len = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    const int32_t* op = poff + pstart[s];
    int pos = 0, end = 0;
    if (row < n) {
        pos = rowptr[row];
        end = rowptr[row + 1];
    }
    bool has_diag = false;
    for (int j = 0; j < len; ++j) {
        const int o = op[j];
        double v = 0.0;
        if (skip_diag && pos < end && col[pos] == row) {
            ++pos;
            has_diag = true;
        }
        if (pos < end && col[pos] - row == o) {
            v = val[pos];
            if (o == 0) {
                v -= shift;
                has_diag = true;
            }
            ++pos;
        }
        put_val(&sval[beg + 32 * j], v);
    }
    if (skip_diag && pos < end && col[pos] == row) has_diag = true;   // after the row's last stored offset
    if (row < n && !has_diag && shift != 0.0 && nodiag != nullptr) atomicOr(nodiag, 1);
}

template <typename VT, typename XT, typename YT, bool PAT, bool UNIT>
cudaError_t sell_dispatch_pu(int n, const int32_t* sptr, const int32_t* col, const SellPat& pat, const void* val,
                             const void* u, const void* w, const void* r, void* y, double ca, double cb, double cc,
                             double cd, int dot, const double* rdot, const Reduce& R, const int* done,
                             cudaStream_t st, const StepTune& tune) {
    using AT = typename AccOf<XT>::type;
    const int tiles = (n + kBlock - 1) / kBlock;
    const int red = num_sms() * (tune.red_ctas_per_sm > 0 ? tune.red_ctas_per_sm : kCtasPerSm);
    const int grid = (dot == 0 || tiles < red) ? tiles : red;
    const int ahead = tune.lookahead < 0 ? default_lookahead() : tune.lookahead;
    const StepCoef<AT> c = make_coef<AT>(ca, cb, cc, cd);
    const VT* v = static_cast<const VT*>(val);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
#define NC_SELL_KARGS n, sptr, col, pat, v, uu, ww, rr, yy, c, rdot, R, done, ahead
    switch (dot) {
    case 0:
        if (tune.rpt == 2)
            sell_step_kernel<VT, XT, YT, 0, PAT, UNIT, 2><<<(tiles + 1) / 2, kBlock, 0, st>>>(NC_SELL_KARGS);
        else
            sell_step_kernel<VT, XT, YT, 0, PAT, UNIT><<<grid, kBlock, 0, st>>>(NC_SELL_KARGS);
        break;
    case 1: sell_step_kernel<VT, XT, YT, 1, PAT, UNIT><<<grid, kBlock, 0, st>>>(NC_SELL_KARGS); break;
    default: sell_step_kernel<VT, XT, YT, 2, PAT, UNIT><<<grid, kBlock, 0, st>>>(NC_SELL_KARGS); break;
    }
#undef NC_SELL_KARGS
    return cudaGetLastError();
}

// float64 steps whose product coefficient is exactly 1 (the scaled iterates,
// q = A p) run a kernel without the multiply
template <typename VT, typename XT, typename YT, bool PAT>
cudaError_t sell_dispatch_p(int n, const int32_t* sptr, const int32_t* col, const SellPat& pat, const void* val,
                            const void* u, const void* w, const void* r, void* y, double ca, double cb, double cc,
                            double cd, int dot, const double* rdot, const Reduce& R, const int* done,
                            cudaStream_t st, const StepTune& tune) {
    if constexpr (sizeof(typename AccOf<XT>::type) == 8) {
        if (cd == 1.0)
            return sell_dispatch_pu<VT, XT, YT, PAT, true>(n, sptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                           rdot, R, done, st, tune);
    }
    return sell_dispatch_pu<VT, XT, YT, PAT, false>(n, sptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R,
                                                    done, st, tune);
}

template <typename VT, typename XT, typename YT>
cudaError_t sell_dispatch(int n, const int32_t* sptr, const int32_t* col, const SellPat& pat, const void* val,
                          const void* u, const void* w, const void* r, void* y, double ca, double cb, double cc,
                          double cd, int dot, const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                          const StepTune& tune) {
    if (pat.pstart != nullptr)
        return sell_dispatch_p<VT, XT, YT, true>(n, sptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R,
                                                 done, st, tune);
    return sell_dispatch_p<VT, XT, YT, false>(n, sptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done,
                                              st, tune);
}

}  // namespace

cudaError_t launch_sell_step(int n, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                             const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                             const void* r, void* y, double ca, double cb, double cc, double cd, int dot,
                             const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                             const StepTune& tune) {
    if (n <= 0) return cudaSuccess;
    if (dot != 0 && tune.dot_variant == STEP_SPLIT) {
        // the step without its dot product, then (rdot, y), (u, y) or (y, y)
        // over the finished vectors (the dot steps write y in float64)
        cudaError_t e = launch_sell_step(n, slice_ptr, col, pat, val, vdt, x_f32, y_f64, u, w, r, y, ca, cb, cc, cd,
                                         0, nullptr, R, done, st, tune);
        if (e != cudaSuccess) return e;
        if (!y_f64) return cudaErrorInvalidValue;
        const double* yd = static_cast<const double*>(y);
        const double* a = dot == 1 ? rdot : (dot == 2 ? static_cast<const double*>(u) : yd);
        if (dot == 2 && x_f32) return cudaErrorInvalidValue;
        return launch_dot_fast(n, a, yd, R, done, st);
    }
    if ((dot == 0 ? tune.variant : tune.dot_variant) == STEP_STAGED) {
        const cudaError_t e = launch_sell_staged(n, slice_ptr, col, pat, val, vdt, x_f32, y_f64, u, w, r, y, ca, cb,
                                                 cc, cd, dot, rdot, R, done, st, tune);
        if (e != cudaErrorNotSupported) return e;
    }
#define NC_SELL_ARGS n, slice_ptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done, st, tune
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        return sell_dispatch<double, double, double>(NC_SELL_ARGS);
    }
    if (vdt == NC_F32)
        return y_f64 ? sell_dispatch<float, float, double>(NC_SELL_ARGS)
                     : sell_dispatch<float, float, float>(NC_SELL_ARGS);
    if (vdt == NC_BF16)
        return y_f64 ? sell_dispatch<__nv_bfloat16, float, double>(NC_SELL_ARGS)
                     : sell_dispatch<__nv_bfloat16, float, float>(NC_SELL_ARGS);
#undef NC_SELL_ARGS
    return cudaErrorInvalidValue;
}

cudaError_t launch_sell_lengths(int n, const int32_t* rowptr, int32_t* slice_len, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int nslices = (n + 31) / 32;
    const int threads = nslices * 32;
    sell_len_kernel<<<(threads + 255) / 256, 256, 0, st>>>(n, rowptr, slice_len);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                             const int32_t* slice_ptr, int vdt, double shift, int32_t* scol, void* sval,
                             int* nodiag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = ((n + 31) / 32) * 32;
    const int grid = (threads + 255) / 256;
    if (vdt == NC_F64)
        sell_fill_kernel<double><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, shift, scol,
                                                       static_cast<double*>(sval), nodiag);
    else if (vdt == NC_F32)
        sell_fill_kernel<float><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, shift, scol,
                                                      static_cast<float*>(sval), nodiag);
    else if (vdt == NC_BF16)
        sell_fill_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, shift, scol,
                                                              static_cast<__nv_bfloat16*>(sval), nodiag);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_psell_merge(int n, const int32_t* rowptr, const int32_t* col, const int32_t* opos, int32_t* cnt,
                               int32_t* off, int* bad, int skip_diag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long threads = (long long)((n + 31) / 32) * 32;
    psell_merge_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rowptr, col, opos, cnt, off, bad,
                                                                           skip_diag);
    return cudaGetLastError();
}

cudaError_t launch_psell_fill(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                              const int32_t* slice_ptr, const int32_t* pstart, const int32_t* poff, int vdt,
                              double shift, void* sval, int* nodiag, int skip_diag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = ((n + 31) / 32) * 32;
    const int grid = (threads + 255) / 256;
    if (vdt == NC_F64)
        psell_fill_kernel<double><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, pstart, poff, shift,
                                                        static_cast<double*>(sval), nodiag, skip_diag);
    else if (vdt == NC_F32)
        psell_fill_kernel<float><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, pstart, poff, shift,
                                                       static_cast<float*>(sval), nodiag, skip_diag);
    else if (vdt == NC_BF16)
        psell_fill_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(n, rowptr, col, val, slice_ptr, pstart, poff, shift,
                                                               static_cast<__nv_bfloat16*>(sval), nodiag,
                                                               skip_diag);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace nc
