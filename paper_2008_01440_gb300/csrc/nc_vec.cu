// Streaming vector kernels of the outer PCG loop (Sec. 5: standard PCG with
// three dot products per iteration, Table 4), each fused with the dot product
// that follows it so that every vector is read once per update:
//   axpy2_rr : x += alpha p, r -= alpha q, ||r||^2 and the stopping test;
//   p_update : p = z + beta p, and the device-side loop condition;
// plus the copies in and out of the solver's workspace.  Grid-stride loops
// over a fixed grid (4 CTAs per SM) so the per-CTA partial sums, and hence
// every reduction, are deterministic for a given n.
#include "nc_common.cuh"

namespace nc {
namespace {

__global__ void __launch_bounds__(kBlock)
axpy2_rr_kernel(int n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                const double* __restrict__ q, float* __restrict__ r32, const Reduce R) {
    const PcgScalars* S = R.S;
    if (S->done) return;
    const double alpha = S->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        if (r32 != nullptr) r32[i] = (float)ri;
        acc = fma(ri, ri, acc);
    }
    grid_reduce<kBlock>(acc, R);
}

__global__ void __launch_bounds__(kBlock)
p_update_kernel(int n, double* __restrict__ p, const double* __restrict__ z,
                const PcgScalars* __restrict__ S, cudaGraphConditionalHandle h, int use_cond) {
    const int done = S->done;
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, done ? 0u : 1u);
    if (done) return;
    const double beta = S->beta;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        p[i] = fma(beta, p[i], z[i]);
}

__global__ void __launch_bounds__(kBlock)
scale_dot_kernel(int n, const double* __restrict__ r, double c, double* __restrict__ z,
                 const Reduce R, const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double zi = c * r[i];
        z[i] = zi;
        acc = fma(r[i], zi, acc);
    }
    if (R.fin != FIN_NONE) grid_reduce<kBlock>(acc, R);
}

__global__ void __launch_bounds__(kBlock)
dot_kernel(int n, const double* __restrict__ a, const double* __restrict__ b, const Reduce R,
           const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        acc = fma(a[i], b[i], acc);
    grid_reduce<kBlock>(acc, R);
}

// (a, b) for 16-byte-aligned vectors: each thread takes pairs of entries
// gtid, gtid + T, ... (T threads), four pairs per round with all eight
// 16-byte loads issued before the FMAs, summed in index order; the odd last
// entry goes to thread 0.  The grid is fixed by n, so the sum's order is.
__global__ void __launch_bounds__(kBlock)
dot_pairs_kernel(int n, const double* __restrict__ a, const double* __restrict__ b, const Reduce R,
                 const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const double2* b2 = reinterpret_cast<const double2*>(b);
    const int n2 = n >> 1;
    const int T = gridDim.x * kBlock;
    int i = blockIdx.x * kBlock + threadIdx.x;
    double acc = 0.0;
    for (; i + 3 * T < n2; i += 4 * T) {
        double2 x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldcs(a2 + i + u * T);
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = __ldcs(b2 + i + u * T);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc = fma(x[u].x, y[u].x, acc);
            acc = fma(x[u].y, y[u].y, acc);
        }
    }
    for (; i < n2; i += T) {
        const double2 x = __ldcs(a2 + i), y = __ldcs(b2 + i);
        acc = fma(x.x, y.x, acc);
        acc = fma(x.y, y.y, acc);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) acc = fma(a[n - 1], b[n - 1], acc);
    grid_reduce<kBlock>(acc, R);
}

__global__ void copy_kernel(int n, const double* __restrict__ x, double* __restrict__ y,
                            const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i];
}

// The scaling is a vector d^{-1/2} (dis) or, when dis is null, the constant ds
// (1 for an unscaled matrix: the copies are then exact).
__global__ void copy_in_kernel(int n, const double* __restrict__ b, const double* __restrict__ x,
                               const double* __restrict__ dis, double ds, int zero, double* __restrict__ bs,
                               double* __restrict__ xs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = dis ? dis[i] : ds;
        bs[i] = b[i] * d;
        xs[i] = zero ? 0.0 : x[i] / d;
    }
}

__global__ void copy_out_kernel(int n, const double* __restrict__ xs, const double* __restrict__ dis, double ds,
                                const PcgScalars* __restrict__ S, double* __restrict__ x) {
    const bool zero = S->bb == 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = zero ? 0.0 : xs[i] * (dis ? dis[i] : ds);
}

__global__ void __launch_bounds__(kBlock)
axpy_dot_kernel(int n, double a, const double* __restrict__ x, double* __restrict__ y, const Reduce R) {
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double yi = fma(a, x[i], y[i]);
        y[i] = yi;
        acc = fma(yi, yi, acc);
    }
    grid_reduce<kBlock>(acc, R);
}

// out = a x + b y (out may alias y); with rdot, (rdot, out) -> R.  The level
// combine of the Newton recursion, zeta_j (2 P_j u - P_j A P_j u).
__global__ void __launch_bounds__(kBlock)
axpby_dot_kernel(int n, double a, const double* __restrict__ x, double b, const double* y, double* out,
                 const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double o = fma(a, x[i], b * y[i]);
        out[i] = o;
        if (rdot != nullptr) acc = fma(rdot[i], o, acc);
    }
    if (rdot != nullptr && R.fin != FIN_NONE) grid_reduce<kBlock>(acc, R);
}

__global__ void refresh_r32_kernel(int n, const double* __restrict__ r, float* __restrict__ r32,
                                   const int* __restrict__ skip) {
    if (*skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r32[i] = (float)r[i];
}

__global__ void div_kernel(int n, const double* __restrict__ x, double d, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i] / d;
}

}  // namespace

int num_sms() {
    // one entry per device ordinal; 0 = not read yet (a benign race: every
    // thread that reads it stores the same value)
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;
    }
    int v = __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 1;
    }
    if (v > kMaxGrid / kCtasPerSm) v = kMaxGrid / kCtasPerSm;
    __atomic_store_n(&cache[dev], v, __ATOMIC_RELAXED);
    return v;
}

int vec_grid(int64_t n) {
    const int64_t want = (n + kBlock - 1) / kBlock;
    const int cap = vec_grid_max();
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_axpy2_rr(int n, double* x, double* r, const double* p, const double* q,
                            float* r32, const Reduce& R, cudaStream_t st) {
    axpy2_rr_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, x, r, p, q, r32, R);
    return cudaGetLastError();
}

cudaError_t launch_p_update(int n, double* p, const double* z, PcgScalars* S,
                            cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    p_update_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, p, z, S, h, use_cond);
    return cudaGetLastError();
}

cudaError_t launch_scale_dot(int n, const double* r, double c, double* z, const Reduce& R,
                             const int* done, cudaStream_t st) {
    scale_dot_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, r, c, z, R, done);
    return cudaGetLastError();
}

cudaError_t launch_dot(int n, const double* a, const double* b, const Reduce& R, const int* done,
                       cudaStream_t st) {
    dot_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, a, b, R, done);
    return cudaGetLastError();
}

cudaError_t launch_dot_fast(int n, const double* a, const double* b, const Reduce& R, const int* done,
                            cudaStream_t st) {
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u)
        return launch_dot(n, a, b, R, done, st);
    // about eight pairs per thread: four-pair rounds, enough CTAs to fill the device
    dot_pairs_kernel<<<vec_grid(((int64_t)n + 15) / 16), kBlock, 0, st>>>(n, a, b, R, done);
    return cudaGetLastError();
}

cudaError_t launch_copy(int n, const double* x, double* y, const int* done, cudaStream_t st) {
    copy_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, x, y, done);
    return cudaGetLastError();
}

cudaError_t launch_copy_in(int n, const double* b, const double* x, const double* dis, double ds, int zero,
                           double* bs, double* xs, cudaStream_t st) {
    copy_in_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, b, x, dis, ds, zero, bs, xs);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(int n, const double* xs, const double* dis, double ds, const PcgScalars* S,
                            double* x, cudaStream_t st) {
    copy_out_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, xs, dis, ds, S, x);
    return cudaGetLastError();
}

cudaError_t launch_axpy_dot(int n, double a, const double* x, double* y, const Reduce& R,
                            cudaStream_t st) {
    axpy_dot_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, a, x, y, R);
    return cudaGetLastError();
}

cudaError_t launch_axpby_dot(int n, double a, const double* x, double b, const double* y, double* out,
                             const double* rdot, const Reduce& R, const int* done, cudaStream_t st) {
    axpby_dot_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, a, x, b, y, out, rdot, R, done);
    return cudaGetLastError();
}

cudaError_t launch_refresh_r32(int n, const double* r, float* r32, const int* skip, cudaStream_t st) {
    refresh_r32_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, r, r32, skip);
    return cudaGetLastError();
}

cudaError_t launch_div(int n, const double* x, double d, double* y, cudaStream_t st) {
    div_kernel<<<vec_grid(n), kBlock, 0, st>>>(n, x, d, y);
    return cudaGetLastError();
}

}  // namespace nc
