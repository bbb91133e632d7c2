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
// the CSR kernel runs.  The solver stores the shifted operator A - theta' I
// (only diagonal entries change): the p_k recursion of Sec. 3 applies
// 2 sigma (1 - A/theta') = -(2/delta)(A - theta' I), so with the shift every
// Chebyshev step after the first needs no separate x_{k-1} term, one FP64
// instruction less per row on GB300's narrow FP64 pipe; the outer products
// add theta' u back (q = A' p + theta' p).
#include "nc_step.cuh"

namespace nc {
namespace {

constexpr int kSellGroup = 8;

// One row: the slot loop and the epilogue; returns the row's dot term.
template <typename VT, typename XT, typename YT, int DOT>
__device__ __forceinline__ double sell_row(const int row, const int32_t* __restrict__ slice_ptr,
                                           const int32_t* __restrict__ col, const VT* __restrict__ val,
                                           const XT* __restrict__ u, const XT* __restrict__ w,
                                           const XT* __restrict__ r, YT* __restrict__ y,
                                           const StepCoef<typename AccOf<XT>::type>& c,
                                           const double* __restrict__ rdot) {
    using AT = typename AccOf<XT>::type;
    const int s = row >> 5;
    const int beg = slice_ptr[s];
    const int len = (slice_ptr[s + 1] - beg) >> 5;   // warp-uniform
    const VT* vp = val + beg + (row & 31);
    const int32_t* cp = col + beg + (row & 31);
    AT acc = AT(0);
    if constexpr (sizeof(AT) == 8) {
        // float64: the fma chain itself is long-latency on GB300's narrow
        // FP64 pipe, so occupancy matters most: a 4-slot unroll keeps the
        // kernel at 32 registers and 8 CTAs (2048 threads) per SM.
        int j = 0;
        for (; j + 4 <= len; j += 4) {
            const int c0 = ld_stream(cp), c1 = ld_stream(cp + 32), c2 = ld_stream(cp + 64),
                      c3 = ld_stream(cp + 96);
            const AT v0 = (AT)ld_stream(vp), v1 = (AT)ld_stream(vp + 32), v2 = (AT)ld_stream(vp + 64),
                     v3 = (AT)ld_stream(vp + 96);
            const AT x0 = (AT)__ldg(u + c0), x1 = (AT)__ldg(u + c1), x2 = (AT)__ldg(u + c2),
                     x3 = (AT)__ldg(u + c3);
            acc = fma(v0, x0, acc);
            acc = fma(v1, x1, acc);
            acc = fma(v2, x2, acc);
            acc = fma(v3, x3, acc);
            vp += 128;
            cp += 128;
        }
        for (; j < len; ++j) {
            const int c0 = ld_stream(cp);
            acc = fma((AT)ld_stream(vp), (AT)__ldg(u + c0), acc);
            vp += 32;
            cp += 32;
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
                    cc_[t] = ld_stream(cp + 32 * t);
                    vv[t] = (AT)ld_stream(vp + 32 * t);
                }
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) xx[t] = (AT)__ldg(u + cc_[t]);
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) acc = fma(vv[t], xx[t], acc);
            vp += 32 * G;
            cp += 32 * G;
        }
    }
    return step_row_out<XT, YT, DOT, AT>(row, acc, c, u, w, r, y, rdot);
}

template <typename VT, typename XT, typename YT, int DOT>
__global__ void __launch_bounds__(kBlock)
sell_step_kernel(const int n, const int32_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                 const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                 const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                 const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    if constexpr (DOT == 0) {
        // one 256-row tile per CTA
        if constexpr (sizeof(typename AccOf<XT>::type) == 4)
            if (threadIdx.x == 0) prefetch_sell_tile((int)blockIdx.x + kPrefetchAhead, n, slice_ptr, col, val);
        const int row = blockIdx.x * kBlock + threadIdx.x;
        if (row < n) sell_row<VT, XT, YT, 0>(row, slice_ptr, col, val, u, w, r, y, c, rdot);
    } else {
        // with a dot product: a persistent grid loops over the tiles and
        // reduces once per CTA
        double dv = 0.0;
        const int ntiles = (n + kBlock - 1) / kBlock;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if constexpr (sizeof(typename AccOf<XT>::type) == 4)
                if (threadIdx.x == 0) prefetch_sell_tile(tile + (int)gridDim.x, n, slice_ptr, col, val);
            const int row = tile * kBlock + threadIdx.x;
            if (row < n) dv += sell_row<VT, XT, YT, DOT>(row, slice_ptr, col, val, u, w, r, y, c, rdot);
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

template <typename VT, typename XT, typename YT>
cudaError_t sell_dispatch(int n, const int32_t* sptr, const int32_t* col, const void* val, const void* u,
                          const void* w, const void* r, void* y, double ca, double cb, double cc, double cd,
                          int dot, const double* rdot, const Reduce& R, const int* done, cudaStream_t st) {
    using AT = typename AccOf<XT>::type;
    const int tiles = (n + kBlock - 1) / kBlock;
    const int grid = (dot == 0 || tiles < kRedGrid) ? tiles : kRedGrid;
    const StepCoef<AT> c = make_coef<AT>(ca, cb, cc, cd);
    const VT* v = static_cast<const VT*>(val);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
    switch (dot) {
    case 0:
        sell_step_kernel<VT, XT, YT, 0><<<grid, kBlock, 0, st>>>(n, sptr, col, v, uu, ww, rr, yy, c, rdot, R, done);
        break;
    case 1:
        sell_step_kernel<VT, XT, YT, 1><<<grid, kBlock, 0, st>>>(n, sptr, col, v, uu, ww, rr, yy, c, rdot, R, done);
        break;
    default:
        sell_step_kernel<VT, XT, YT, 2><<<grid, kBlock, 0, st>>>(n, sptr, col, v, uu, ww, rr, yy, c, rdot, R, done);
        break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sell_step(int n, const int32_t* slice_ptr, const int32_t* col, const void* val, int vdt,
                             bool x_f32, bool y_f64, const void* u, const void* w, const void* r, void* y,
                             double ca, double cb, double cc, double cd, int dot, const double* rdot,
                             const Reduce& R, const int* done, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        return sell_dispatch<double, double, double>(n, slice_ptr, col, val, u, w, r, y, ca, cb, cc, cd, dot, rdot,
                                                     R, done, st);
    }
    if (vdt == NC_F32) {
        if (y_f64)
            return sell_dispatch<float, float, double>(n, slice_ptr, col, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                       rdot, R, done, st);
        return sell_dispatch<float, float, float>(n, slice_ptr, col, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R,
                                                  done, st);
    }
    if (vdt == NC_BF16) {
        if (y_f64)
            return sell_dispatch<__nv_bfloat16, float, double>(n, slice_ptr, col, val, u, w, r, y, ca, cb, cc, cd,
                                                               dot, rdot, R, done, st);
        return sell_dispatch<__nv_bfloat16, float, float>(n, slice_ptr, col, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                          rdot, R, done, st);
    }
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

}  // namespace nc
