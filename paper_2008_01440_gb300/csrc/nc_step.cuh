// Epilogue shared by the fused step kernels of every matrix format:
//     y = ca*u + cb*w + cc*r + cd*(A u)   (one Chebyshev step of Algorithm 2)
// plus an optional dot product finished by the last CTA (DOT: 0 none,
// 1 (rdot, y), 2 (u, y), 3 (y, y)).
#pragma once

#include "nc_common.cuh"

namespace nc {

constexpr int kTermU = 1, kTermW = 2, kTermR = 4;
constexpr int kUnitD = 8;   // cd == 1: the product is taken as it is

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ double ld_val(const double* p) { return *p; }
__device__ __forceinline__ float ld_val(const float* p) { return *p; }
__device__ __forceinline__ float ld_val(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Streaming (evict-first) loads for matrix data that is read exactly once.
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const __nv_bfloat16* p) {
    const unsigned short b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(((unsigned int)b) << 16);
}
__device__ __forceinline__ int ld_stream(const int32_t* p) { return __ldcs(p); }

// L2 prefetch of the SELL-32 slices (columns, unless null, and values) of 256-row tile t,
// issued by one thread: cp.async.bulk.prefetch is a hint that holds no
// registers and has nothing to wait for.  Slice offsets are multiples of 32
// entries, so both ranges start and end on 16-byte boundaries.  The float
// step kernels take the tile `ahead` tiles ahead of their own (by default
// two CTAs per SM later, default_lookahead()): its loads then hit L2, which
// brought the float step of the 128^3 system from 26.5 to 25.0 us (0.95 of
// the copy bandwidth).  The float64 kernels, latency-bound at full
// occupancy, ran slower with it.
inline int default_lookahead() { return 2 * num_sms(); }

template <typename VT>
__device__ __forceinline__ void prefetch_sell_tile(int t, int n, const int32_t* __restrict__ slice_ptr,
                                                   const int32_t* __restrict__ col, const VT* __restrict__ val) {
    const int nslices = (n + 31) >> 5;
    const int s0 = t * (kBlock / 32);
    if (t < 0 || s0 >= nslices) return;
    const int b = slice_ptr[s0], e = slice_ptr[min(s0 + kBlock / 32, nslices)];
    if (e <= b) return;
    if (col != nullptr)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(col + b),
                     "r"((uint32_t)(e - b) * (uint32_t)sizeof(int32_t)) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(val + b),
                 "r"((uint32_t)(e - b) * (uint32_t)sizeof(VT)) : "memory");
}

// Coefficients of one step in the accumulation type (float coefficients for
// the float path: a double->float conversion per thread would run on the
// scarce FP64 pipe).  `terms` says which optional terms are present.
template <typename AT>
struct StepCoef {
    AT ca, cb, cc, cd;
    int terms;
};

template <typename AT>
inline StepCoef<AT> make_coef(double ca, double cb, double cc, double cd) {
    StepCoef<AT> c;
    c.ca = (AT)ca;
    c.cb = (AT)cb;
    c.cc = (AT)cc;
    c.cd = (AT)cd;
    c.terms = (ca != 0.0 ? kTermU : 0) | (cb != 0.0 ? kTermW : 0) | (cc != 0.0 ? kTermR : 0) |
              (cd == 1.0 ? kUnitD : 0);
    return c;
}

// Row epilogue: returns the dot-product contribution of this row (DOT: 0
// none, 1 (rdot, y), 2 (u, y)).  UNIT: cd == 1, the product taken as it is
// -- a compile-time case, since a runtime test of kUnitD is if-converted and
// the multiply issued anyway.
template <typename XT, typename YT, int DOT, typename AT, bool UNIT = false>
__device__ __forceinline__ double step_row_out(int row, AT acc, const StepCoef<AT>& c,
                                               const XT* __restrict__ u, const XT* __restrict__ w,
                                               const XT* __restrict__ r, YT* __restrict__ y,
                                               const double* __restrict__ rdot) {
    AT o;
    if constexpr (UNIT) o = acc;
    else o = (c.terms & kUnitD) ? acc : c.cd * acc;
    if (c.terms & kTermR) o = fma(c.cc, (AT)r[row], o);
    if (c.terms & kTermW) o = fma(c.cb, (AT)w[row], o);
    if (c.terms & kTermU) o = fma(c.ca, (AT)u[row], o);
    const YT yo = (YT)o;
    y[row] = yo;
    if (DOT == 1) return rdot[row] * (double)yo;
    if (DOT == 2) return (double)u[row] * (double)yo;
    if (DOT == 3) return (double)yo * (double)yo;
    return 0.0;
}

// The same epilogue with r[row] and w[row] already loaded (rv, wv; zero
// when their term is absent), in the same order of operations.
template <typename XT, typename YT, int DOT, typename AT, bool UNIT = false>
__device__ __forceinline__ double sell_row_out(int row, AT acc, const StepCoef<AT>& c, AT rv, AT wv,
                                               const XT* __restrict__ u, YT* __restrict__ y,
                                               const double* __restrict__ rdot) {
    AT o;
    if constexpr (UNIT) o = acc;
    else o = (c.terms & kUnitD) ? acc : c.cd * acc;
    if (c.terms & kTermR) o = fma(c.cc, rv, o);
    if (c.terms & kTermW) o = fma(c.cb, wv, o);
    if (c.terms & kTermU) o = fma(c.ca, (AT)u[row], o);
    const YT yo = (YT)o;
    y[row] = yo;
    if (DOT == 1) return rdot[row] * (double)yo;
    if (DOT == 2) return (double)u[row] * (double)yo;
    if (DOT == 3) return (double)yo * (double)yo;
    return 0.0;
}

}  // namespace nc
