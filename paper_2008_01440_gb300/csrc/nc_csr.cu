// CSR kernels: the fused matrix-vector product + Chebyshev recurrence step.
//
// One Chebyshev step of Algorithm 2 (Sec. 3), with the loop body written as
//     x_k = a_k x_{k-1} + b_k x_{k-2} + c_k r + d_k (A x_{k-1}),
//     a_k = 2 sigma rho_k, b_k = -rho_k rho_{k-1}, c_k = 2 rho_k/delta,
//     d_k = -2 rho_k/delta,
// is one kernel: the matrix is read once, x_{k-1} is gathered, x_{k-2} and
// r are read once at the row's own index and x_k is written once.  The same
// kernel with (a, b, c, d) = (0, 0, 0, 1) is the plain product q = A p of the
// outer CG, and with a dot-product epilogue it also produces (p, q) or
// (r, z) (Table 4 counts these as the only reductions).
//
// Layout: one thread per row, 256 rows per CTA.  The CTA first streams the
// nonzeros of its rows (values and column indices, contiguous in CSR) into
// shared memory with fully coalesced loads, then each thread runs the
// multiply-add chain of its row from shared memory, gathering x_{k-1}
// through the read-only cache.  Each row's sum is one fma chain in column
// order, so a float64 row costs nnz_row + 4 floating-point instructions,
// the minimum for this operation.
#include "nc_step.cuh"

namespace nc {
namespace {

template <typename VT, typename XT, typename YT, int DOT>
__global__ void __launch_bounds__(kBlock)
csr_step_kernel(const int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done) {
    using AT = typename AccOf<XT>::type;
    if (done != nullptr && *done) return;
    __shared__ VT s_val[kChunk];
    __shared__ int32_t s_col[kChunk];
    double dv = 0.0;
    const int ntiles = (n + kBlock - 1) / kBlock;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * kBlock;
    const int row = row0 + threadIdx.x;
    const int row_end = min(row0 + kBlock, n);
    const int blk_s = rowptr[row0];
    const int blk_e = rowptr[row_end];
    int my_s = 0, my_e = 0;
    if (row < n) {
        my_s = rowptr[row];
        my_e = rowptr[row + 1];
    }
    AT acc = AT(0);
    for (int cs = blk_s; cs < blk_e; cs += kChunk) {
        const int ce = min(cs + kChunk, blk_e);
        for (int j = cs + threadIdx.x; j < ce; j += kBlock) {
            s_val[j - cs] = val[j];
            s_col[j - cs] = col[j];
        }
        __syncthreads();
        const int js = max(my_s, cs), je = min(my_e, ce);
        for (int j = js; j < je; ++j)
            acc = fma((AT)ld_val(&s_val[j - cs]), (AT)__ldg(&u[s_col[j - cs]]), acc);
        __syncthreads();
    }
    if (row < n) dv += step_row_out<XT, YT, DOT, AT>(row, acc, c, u, w, r, y, rdot);
    }
    if (DOT != 0) grid_reduce<kBlock>(dv, R);
}

template <typename VT, typename XT, typename YT>
cudaError_t step_dispatch(int n, const int32_t* rowptr, const int32_t* col, const void* val,
                          const void* u, const void* w, const void* r, void* y, double ca,
                          double cb, double cc, double cd, int dot, const double* rdot,
                          const Reduce& R, const int* done, cudaStream_t st) {
    const int tiles = (n + kBlock - 1) / kBlock;
    const int red = vec_grid_max();
    const int grid = (dot == 0 || tiles < red) ? tiles : red;
    const VT* v = static_cast<const VT*>(val);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
    const StepCoef<typename AccOf<XT>::type> c = make_coef<typename AccOf<XT>::type>(ca, cb, cc, cd);
    switch (dot) {
    case 0:
        csr_step_kernel<VT, XT, YT, 0><<<grid, kBlock, 0, st>>>(n, rowptr, col, v, uu, ww, rr, yy, c,
                                                                rdot, R, done);
        break;
    case 1:
        csr_step_kernel<VT, XT, YT, 1><<<grid, kBlock, 0, st>>>(n, rowptr, col, v, uu, ww, rr, yy, c,
                                                                rdot, R, done);
        break;
    default:
        csr_step_kernel<VT, XT, YT, 2><<<grid, kBlock, 0, st>>>(n, rowptr, col, v, uu, ww, rr, yy, c,
                                                                rdot, R, done);
        break;
    }
    return cudaGetLastError();
}

// Diagonal of a CSR matrix -> d^{-1/2}; *bad is set if a diagonal entry is
// missing or not positive.
__global__ void csr_diag_kernel(int n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                double* __restrict__ dis, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
        if (col[j] == i) d = val[j];
    if (!(d > 0.0)) {
        atomicOr(bad, 1);
        dis[i] = 0.0;
    } else {
        dis[i] = 1.0 / sqrt(d);
    }
}

// a_ij -> (a_ij d_i^{-1/2}) d_j^{-1/2}; the diagonal becomes its exact
// value 1 (a_ii d_i^{-1/2} d_i^{-1/2} rounds to 1 +- an ulp otherwise), so
// that a scaled matrix has the constant diagonal the offset-pattern layout
// can fold into its step coefficients
__global__ void csr_scale_kernel(int n, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const double* __restrict__ val,
                                 const double* __restrict__ dis, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double di = dis[i];
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) out[j] = col[j] == i ? 1.0 : val[j] * di * dis[col[j]];
}

// Whether every row has a diagonal entry and all of them equal row 0's
// (bitwise): *flags bit 0 set if not.  The diagonal of row 0 is the
// reference; a row without one sets the bit as well.
__global__ void csr_diag_const_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const double* __restrict__ val, int* __restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool found = false, found0 = false;
    double d = 0.0, d0 = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
        if (col[j] == i) { d = val[j]; found = true; }
    for (int j = rowptr[0]; j < rowptr[1]; ++j)
        if (col[j] == 0) { d0 = val[j]; found0 = true; }
    if (!found || !found0 || __double_as_longlong(d) != __double_as_longlong(d0)) atomicOr(flags, 1);
}

// max_i sum_j |a_ij|; non-negative doubles order like their bit patterns.
__global__ void csr_gershgorin_kernel(int n, const int32_t* __restrict__ rowptr,
                                      const double* __restrict__ val,
                                      unsigned long long* __restrict__ out_bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n)
        for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s += fabs(val[j]);
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(s));
}

__global__ void convert_f32_kernel(int64_t count, const double* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void convert_bf16_kernel(int64_t count, const double* __restrict__ in,
                                    __nv_bfloat16* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2bfloat16(in[i]);
}

}  // namespace

cudaError_t launch_csr_step(int n, const int32_t* rowptr, const int32_t* col, const void* val,
                            int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                            const void* r, void* y, double ca, double cb, double cc, double cd,
                            int dot, const double* rdot, const Reduce& R, const int* done,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        return step_dispatch<double, double, double>(n, rowptr, col, val, u, w, r, y, ca, cb, cc, cd,
                                                     dot, rdot, R, done, st);
    }
    if (vdt == NC_F32) {
        if (y_f64)
            return step_dispatch<float, float, double>(n, rowptr, col, val, u, w, r, y, ca, cb, cc, cd,
                                                       dot, rdot, R, done, st);
        return step_dispatch<float, float, float>(n, rowptr, col, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                  rdot, R, done, st);
    }
    if (vdt == NC_BF16) {
        if (y_f64)
            return step_dispatch<__nv_bfloat16, float, double>(n, rowptr, col, val, u, w, r, y, ca, cb,
                                                               cc, cd, dot, rdot, R, done, st);
        return step_dispatch<__nv_bfloat16, float, float>(n, rowptr, col, val, u, w, r, y, ca, cb, cc,
                                                          cd, dot, rdot, R, done, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_csr_diag(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                            double* dis, int* bad, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    csr_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, col, val, dis, bad);
    return cudaGetLastError();
}

cudaError_t launch_csr_scale(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                             const double* dis, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    csr_scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, col, val, dis, out);
    return cudaGetLastError();
}

cudaError_t launch_csr_diag_const(int n, const int32_t* rowptr, const int32_t* col, const double* val, int* flags,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    csr_diag_const_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, col, val, flags);
    return cudaGetLastError();
}

cudaError_t launch_csr_gershgorin(int n, const int32_t* rowptr, const double* val,
                                  unsigned long long* out_bits, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    csr_gershgorin_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, val, out_bits);
    return cudaGetLastError();
}

cudaError_t launch_convert(int64_t count, const double* in, int out_dt, void* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int64_t want = (count + 255) / 256;
    const int grid = (int)(want < 4096 ? want : 4096);
    if (out_dt == NC_F32)
        convert_f32_kernel<<<grid, 256, 0, st>>>(count, in, static_cast<float*>(out));
    else if (out_dt == NC_BF16)
        convert_bf16_kernel<<<grid, 256, 0, st>>>(count, in, static_cast<__nv_bfloat16*>(out));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace nc
