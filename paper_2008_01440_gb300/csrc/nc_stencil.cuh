// Device-side 7-point stencil tile: the fused Chebyshev step over one
// 32 x 8 tile of (x, y) and a chunk of z planes (see nc_stencil.cu for the
// layout).  Shared by the single-system kernel and the batched engine.
#pragma once

#include "nc_step.cuh"

namespace nc {

constexpr int kTX = 32, kTY = 8;

template <typename AT>
struct StencilCoef {
    AT e0, ex, ey, ez, cb, cc;
    int terms;   // kTermW / kTermR
};

// y = e0 u + ex (u_{i-1}+u_{i+1}) + ey (u_{j-1}+u_{j+1}) + ez (u_{k-1}+u_{k+1})
//     + cb w + cc r over planes [k0, k1) of tile (bx, by).  DOT 1: returns
// this thread's sum of rdot*y, DOT 2: u*y, DOT 3: y*y.  Must be called by all
// 32 lanes of a warp together (shuffles).
//
// The z-march works in batches of P planes: every load a batch needs (the
// next P centre values, the y- and tile-edge x-neighbours, w and r) is issued
// before any of the batch's arithmetic, so a batch costs one memory latency
// rather than one per plane.  u at the planes below and at the current plane
// stay in registers across batches.
// XU: ex == -1 exactly (the stored operator normalised by its x-weight and
// the iterates scaled so the product's coefficient is 1): the step starts
// from -(x-neighbours) and needs no multiply for the centre.
//
// PZ: planes per z-march batch.  Measured on the float32 step: 2 planes are
// best for short z-chunks (511^3, 52-plane chunks: 388 us against 410 with 4),
// 4 planes for long ones (1023^3, 341-plane chunks: 3316 us against 3481);
// float64 takes 2.
template <typename XT, typename YT, int DOT, bool XU = false, int PZ = 2>
__device__ __forceinline__ double stencil_tile(const int nx, const int ny, const int nz, const int bx, const int by,
                                               const int k0, const int k1, const XT* __restrict__ u,
                                               const XT* __restrict__ w, const XT* __restrict__ r,
                                               YT* __restrict__ y, const StencilCoef<typename AccOf<XT>::type>& c,
                                               const double* __restrict__ rdot, const int lane, const int ty) {
    using AT = typename AccOf<XT>::type;
    constexpr int P = PZ;
    const int i = bx * kTX + lane;
    const int j = by * kTY + ty;
    const bool in = i < nx && j < ny;
    const long long plane = (long long)nx * ny;
    long long idx = ((long long)k0 * ny + j) * nx + i;
    const AT zero = AT(0);
    const bool has_w = (c.terms & kTermW) != 0, has_r = (c.terms & kTermR) != 0;
    AT u_prev = (in && k0 > 0) ? (AT)__ldg(u + idx - plane) : zero;
    AT u_cur = (in && k0 < nz) ? (AT)__ldg(u + idx) : zero;
    double dv = 0.0;
    for (int k = k0; k < k1; k += P) {
        AT un[P], ym[P], yp[P], xe[P], wv[P], rv[P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const long long q = idx + t * plane;
            const bool live = in && k + t < k1;
            un[t] = (in && k + 1 + t < nz) ? (AT)__ldg(u + q + plane) : zero;
            ym[t] = (live && j > 0) ? (AT)__ldg(u + q - nx) : zero;
            yp[t] = (live && j + 1 < ny) ? (AT)__ldg(u + q + nx) : zero;
            // the neighbour across the tile edge, for lanes 0 and 31 only
            xe[t] = zero;
            if (live && lane == 0 && i > 0) xe[t] = (AT)__ldg(u + q - 1);
            if (live && lane == kTX - 1 && i + 1 < nx) xe[t] = (AT)__ldg(u + q + 1);
            wv[t] = (live && has_w) ? (AT)w[q] : zero;
            rv[t] = (live && has_r) ? (AT)r[q] : zero;
        }
#pragma unroll
        for (int t = 0; t < P; ++t) {
            if (k + t >= k1) break;   // uniform across the CTA
            const AT u_next = un[t];
            AT xm = __shfl_up_sync(0xffffffffu, u_cur, 1);
            AT xp = __shfl_down_sync(0xffffffffu, u_cur, 1);
            if (lane == 0) xm = xe[t];
            if (lane == kTX - 1) xp = xe[t];
            if (in) {
                const long long q = idx + t * plane;
                AT o;
                if constexpr (XU) {
                    o = fma(c.e0, u_cur, -(xm + xp));
                } else {
                    o = c.e0 * u_cur;
                    o = fma(c.ex, xm + xp, o);
                }
                o = fma(c.ey, ym[t] + yp[t], o);
                o = fma(c.ez, u_prev + u_next, o);
                if (has_r) o = fma(c.cc, rv[t], o);
                if (has_w) o = fma(c.cb, wv[t], o);
                const YT yo = (YT)o;
                y[q] = yo;
                if (DOT == 1) dv += rdot[q] * (double)yo;
                if (DOT == 2) dv += (double)u_cur * (double)yo;
                if (DOT == 3) dv += (double)yo * (double)yo;
            }
            u_prev = u_cur;
            u_cur = u_next;
        }
        idx += P * plane;
    }
    return dv;
}

// The same step over a flattened tile: the kFT consecutive points
// [f0, f0 + kFT) of the row-major xy-plane (thread tid owns f0 + tid), planes
// [k0, k1).  Every lane is busy whatever nx is (a 32-wide box tile leaves
// 32 ceil(nx/32) - nx lanes idle); x-neighbours come from the adjacent lane
// within a row and are loaded where the row or the warp ends.  Must be
// called by all lanes of each warp together.
constexpr int kFT = 256;

// E1: e0 == 1 exactly (the Jacobi-scaled operator itself, q = A p and
// b - A x): the centre term is u itself, no multiply (the same value).
template <typename XT, typename YT, int DOT, bool XU = false, bool E1 = false>
__device__ __forceinline__ double stencil_flat(const int nx, const int ny, const int nz, const int f0, const int k0,
                                               const int k1, const XT* __restrict__ u, const XT* __restrict__ w,
                                               const XT* __restrict__ r, YT* __restrict__ y,
                                               const StencilCoef<typename AccOf<XT>::type>& c,
                                               const double* __restrict__ rdot, const int tid) {
    using AT = typename AccOf<XT>::type;
    // planes per z-march batch (measured on the 256-system batch, float:
    // 2 planes 487 ms, 4 planes 436 ms, 8 planes 592 ms)
    constexpr int P = sizeof(AT) == 8 ? 2 : 4;
    const int lane = tid & 31;
    const int nxy = nx * ny;
    const int f = f0 + tid;
    const bool in = f < nxy;
    const int yy = in ? f / nx : 0;
    const int xx = f - yy * nx;
    const bool has_xm = in && xx > 0, has_xp = in && xx + 1 < nx;
    const bool has_ym = in && yy > 0, has_yp = in && yy + 1 < ny;
    // lane 0's left and lane 31's right neighbour live in another warp
    const bool ld_xm = has_xm && lane == 0, ld_xp = has_xp && lane == 31;
    const long long plane = nxy;
    long long idx = (long long)k0 * plane + f;
    const AT zero = AT(0);
    const bool has_w = (c.terms & kTermW) != 0, has_r = (c.terms & kTermR) != 0;
    AT u_prev = (in && k0 > 0) ? (AT)__ldg(u + idx - plane) : zero;
    AT u_cur = (in && k0 < nz) ? (AT)__ldg(u + idx) : zero;
    double dv = 0.0;
    for (int k = k0; k < k1; k += P) {
        AT un[P], ym[P], yp[P], xe[P], wv[P], rv[P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const long long q = idx + t * plane;
            const bool live = in && k + t < k1;
            un[t] = (in && k + 1 + t < nz) ? (AT)__ldg(u + q + plane) : zero;
            ym[t] = (live && has_ym) ? (AT)__ldg(u + q - nx) : zero;
            yp[t] = (live && has_yp) ? (AT)__ldg(u + q + nx) : zero;
            xe[t] = zero;
            if (live && ld_xm) xe[t] = (AT)__ldg(u + q - 1);
            if (live && ld_xp) xe[t] = (AT)__ldg(u + q + 1);
            wv[t] = (live && has_w) ? (AT)w[q] : zero;
            rv[t] = (live && has_r) ? (AT)r[q] : zero;
        }
#pragma unroll
        for (int t = 0; t < P; ++t) {
            if (k + t >= k1) break;   // uniform across the CTA
            const AT u_next = un[t];
            AT xm = __shfl_up_sync(0xffffffffu, u_cur, 1);
            AT xp = __shfl_down_sync(0xffffffffu, u_cur, 1);
            if (lane == 0) xm = xe[t];
            if (lane == 31) xp = xe[t];
            if (!has_xm) xm = zero;
            if (!has_xp) xp = zero;
            if (in) {
                const long long q = idx + t * plane;
                AT o;
                if constexpr (XU) {   // ex == -1 exactly
                    o = fma(c.e0, u_cur, -(xm + xp));
                } else {
                    o = E1 ? u_cur : c.e0 * u_cur;
                    o = fma(c.ex, xm + xp, o);
                }
                o = fma(c.ey, ym[t] + yp[t], o);
                o = fma(c.ez, u_prev + u_next, o);
                if (has_r) o = fma(c.cc, rv[t], o);
                if (has_w) o = fma(c.cb, wv[t], o);
                const YT yo = (YT)o;
                y[q] = yo;
                if (DOT == 1) dv += rdot[q] * (double)yo;
                if (DOT == 2) dv += (double)u_cur * (double)yo;
                if (DOT == 3) dv += (double)yo * (double)yo;
            }
            u_prev = u_cur;
            u_cur = u_next;
        }
        idx += P * plane;
    }
    return dv;
}

}  // namespace nc
