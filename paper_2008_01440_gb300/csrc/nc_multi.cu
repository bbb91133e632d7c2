// Multi-right-hand-side fused step: the Chebyshev step of Algorithm 2 (and
// q = A p) for m independent PCG recurrences that share the matrix:
//     Y[:, c] = ca U[:, c] + cb W[:, c] + cc R[:, c] + cd (A U[:, c]),  c < m,
// the coefficients being the same for every column (same polynomial).  The
// m columns are stored one after the other (column c at offset c * ld), so
// the per-column vector kernels of the outer loop run unchanged on them.
//
// One thread per row of the SELL-32 layout: each slot's column index and
// value are loaded once and applied to all m columns -- the matrix, the
// dominant stream of a step, is read once per step instead of m times (a
// sparse times dense-block product).  The gathers of U stay per column.
#include "nc_step.cuh"

namespace nc {
namespace {

constexpr int kMaxRhs = 8;

__device__ __forceinline__ bool all_done(const PcgScalars* Sm, int m) {
    for (int c = 0; c < m; ++c)
        if (!Sm[c].done) return false;
    return true;
}

// The column count is a template parameter: with a runtime count the guard
// between columns keeps the compiler from issuing the next column's gathers
// before this column's FMAs, one memory latency per column (measured: the
// 8-column float step of the 128^3 system at 30 % of DRAM bandwidth, stalled
// on loads).  G slots per group, so that about 16 gathers are in flight.
// UNIT: the product's coefficient is exactly 1 (float64 scaled iterates), a
// compile-time case so that no multiply is issued.
template <typename VT, typename XT, typename YT, int M, bool PAT, bool UNIT>
__global__ void __launch_bounds__(kBlock)
sell_mstep_kernel(const int n, const int ld, const int32_t* __restrict__ slice_ptr,
                  const int32_t* __restrict__ col, const SellPat pat, const VT* __restrict__ val,
                  const XT* __restrict__ u, const XT* __restrict__ w, const XT* __restrict__ r, YT* __restrict__ y,
                  const StepCoef<typename AccOf<XT>::type> cf, const PcgScalars* __restrict__ Sm, const int ahead) {
    using AT = typename AccOf<XT>::type;
    constexpr int G = M >= 8 ? 2 : (M >= 4 ? 4 : 8);
    if (Sm != nullptr && all_done(Sm, M)) return;
    if constexpr (sizeof(AT) == 4)
        if (threadIdx.x == 0 && ahead > 0)
            prefetch_sell_tile((int)blockIdx.x + ahead, n, slice_ptr, PAT ? nullptr : col, val);
    const int row = blockIdx.x * kBlock + threadIdx.x;
    if (row >= n) return;
    const int s = row >> 5;
    const int beg = slice_ptr[s];
    const int len = (slice_ptr[s + 1] - beg) >> 5;   // warp-uniform
    const VT* vp = val + beg + (row & 31);
    const int32_t* cp = nullptr;
    const int32_t* op = nullptr;   // PAT: columns row + op[j] (clamped; padded slots have value 0)
    if constexpr (PAT) op = pat.poff + __ldg(pat.pstart + s);
    else cp = col + beg + (row & 31);
    AT acc[M];
#pragma unroll
    for (int c = 0; c < M; ++c) acc[c] = AT(0);
    for (int j0 = 0; j0 < len; j0 += G) {
        int cj[G];
        AT vj[G];
#pragma unroll
        for (int t = 0; t < G; ++t) {
            cj[t] = row;   // padding of a short group: a valid address, weight 0
            vj[t] = AT(0);
            if (j0 + t < len) {
                if constexpr (PAT) cj[t] = min(max(row + __ldg(op + j0 + t), 0), n - 1);
                else cj[t] = ld_stream(cp + 32 * t);
                vj[t] = (AT)ld_stream(vp + 32 * t);
            }
        }
        AT xv[M][G];
#pragma unroll
        for (int c = 0; c < M; ++c)
#pragma unroll
            for (int t = 0; t < G; ++t) xv[c][t] = (AT)__ldg(u + (size_t)c * ld + cj[t]);
#pragma unroll
        for (int c = 0; c < M; ++c)
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) acc[c] = fma(vj[t], xv[c][t], acc[c]);
        vp += 32 * G;
        if constexpr (!PAT) cp += 32 * G;
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
        const size_t o = (size_t)c * ld;
        AT v;
        if constexpr (UNIT) v = acc[c];
        else v = cf.cd * acc[c];
        if (cf.terms & kTermR) v = fma(cf.cc, (AT)r[o + row], v);
        if (cf.terms & kTermW) v = fma(cf.cb, (AT)w[o + row], v);
        if (cf.terms & kTermU) v = fma(cf.ca, (AT)u[o + row], v);
        y[o + row] = (YT)v;
    }
}

// Graph loop condition of a multi-right-hand-side solve: any column still running.
__global__ void any_active_kernel(const PcgScalars* __restrict__ Sm, int m, cudaGraphConditionalHandle h,
                                  int use_cond, int* __restrict__ active) {
    int a = 0;
    for (int c = 0; c < m; ++c) a |= Sm[c].done ? 0 : 1;
    if (active) *active = a;
    if (use_cond) cudaGraphSetConditional(h, a ? 1u : 0u);
}

template <typename VT, typename XT, typename YT, int M>
cudaError_t mstep_launch_m(int n, int ld, const int32_t* sptr, const int32_t* col, const SellPat& pat,
                           const void* val, const void* u, const void* w, const void* r, void* y, double ca,
                           double cb, double cc, double cd, const PcgScalars* Sm, cudaStream_t st) {
    using AT = typename AccOf<XT>::type;
    const StepCoef<AT> c = make_coef<AT>(ca, cb, cc, cd);
    const unsigned grid = (unsigned)((n + kBlock - 1) / kBlock);
    const int ahead = default_lookahead();
    const VT* v = static_cast<const VT*>(val);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
    if constexpr (sizeof(AT) == 8) {
        if (cd == 1.0) {
            if (pat.pstart != nullptr)
                sell_mstep_kernel<VT, XT, YT, M, true, true><<<grid, kBlock, 0, st>>>(n, ld, sptr, col, pat, v, uu,
                                                                                      ww, rr, yy, c, Sm, ahead);
            else
                sell_mstep_kernel<VT, XT, YT, M, false, true><<<grid, kBlock, 0, st>>>(n, ld, sptr, col, pat, v, uu,
                                                                                       ww, rr, yy, c, Sm, ahead);
            return cudaGetLastError();
        }
    }
    if (pat.pstart != nullptr)
        sell_mstep_kernel<VT, XT, YT, M, true, false><<<grid, kBlock, 0, st>>>(n, ld, sptr, col, pat, v, uu, ww, rr,
                                                                               yy, c, Sm, ahead);
    else
        sell_mstep_kernel<VT, XT, YT, M, false, false><<<grid, kBlock, 0, st>>>(n, ld, sptr, col, pat, v, uu, ww, rr,
                                                                                yy, c, Sm, ahead);
    return cudaGetLastError();
}

template <typename VT, typename XT, typename YT>
cudaError_t mstep_launch(int n, int m, int ld, const int32_t* sptr, const int32_t* col, const SellPat& pat,
                         const void* val,
                         const void* u, const void* w, const void* r, void* y, double ca, double cb, double cc,
                         double cd, const PcgScalars* Sm, cudaStream_t st) {
#define NC_MSTEP(MM) \
    case MM: return mstep_launch_m<VT, XT, YT, MM>(n, ld, sptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, Sm, st);
    switch (m) {
        NC_MSTEP(1) NC_MSTEP(2) NC_MSTEP(3) NC_MSTEP(4) NC_MSTEP(5) NC_MSTEP(6) NC_MSTEP(7) NC_MSTEP(8)
    default: return cudaErrorInvalidValue;
    }
#undef NC_MSTEP
}

}  // namespace

int max_rhs() { return kMaxRhs; }

cudaError_t launch_sell_mstep(int n, int m, int ld, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                              const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                              const void* r, void* y, double ca, double cb, double cc, double cd,
                              const PcgScalars* Sm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (m < 1 || m > kMaxRhs) return cudaErrorInvalidValue;
#define NC_MSTEP_ARGS n, m, ld, slice_ptr, col, pat, val, u, w, r, y, ca, cb, cc, cd, Sm, st
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        return mstep_launch<double, double, double>(NC_MSTEP_ARGS);
    }
    if (vdt == NC_F32)
        return y_f64 ? mstep_launch<float, float, double>(NC_MSTEP_ARGS)
                     : mstep_launch<float, float, float>(NC_MSTEP_ARGS);
    if (vdt == NC_BF16)
        return y_f64 ? mstep_launch<__nv_bfloat16, float, double>(NC_MSTEP_ARGS)
                     : mstep_launch<__nv_bfloat16, float, float>(NC_MSTEP_ARGS);
#undef NC_MSTEP_ARGS
    return cudaErrorInvalidValue;
}

cudaError_t launch_any_active(const PcgScalars* Sm, int m, cudaGraphConditionalHandle h, int use_cond, int* active,
                              cudaStream_t st) {
    any_active_kernel<<<1, 1, 0, st>>>(Sm, m, h, use_cond, active);
    return cudaGetLastError();
}

}  // namespace nc
