// 3x3-block sparse matrices (three displacement dofs per node, the paper's
// finite-element structural matrices of Sec. 5): the fused Chebyshev step
//     y = ca u + cb w + cc r + cd (A u)
// with A in block CSR (row-major 3x3 blocks) or in its sliced layout BSELL-32.
//
// BSELL-32: slices of 32 consecutive block rows (one warp, one thread per
// block row); slot j of a slice holds one block of each of its 32 rows.  The
// 9 entries of the slot's blocks are stored entry-major, [entry e][lane], so
// each of the 9 value loads of a slot is one coalesced 32-wide access, and
// the block-column load is another.  For grid meshes the 32 rows of a slot
// reference 32 consecutive nodes, so the gathers of x are coalesced too.
// Rows are padded to the slice's longest block row with zero blocks whose
// column is the row itself.  As for the scalar layouts, the solver stores
// A - theta' I (the diagonal block's diagonal shifted) so the x_{k-1} term
// of every Chebyshev step after the first vanishes.
//
// One thread accumulates its block row's three outputs in three independent
// fma chains (27 blocks x 9 fma for an interior elasticity node).
#include "nc_step.cuh"

namespace nc {
namespace {

template <typename XT, typename YT, int DOT, typename AT>
__device__ __forceinline__ double bsr_rows_out(int brow, const AT (&acc)[3], const StepCoef<AT>& c,
                                               const XT* __restrict__ u, const XT* __restrict__ w,
                                               const XT* __restrict__ r, YT* __restrict__ y,
                                               const double* __restrict__ rdot) {
    double dv = 0.0;
#pragma unroll
    for (int t = 0; t < 3; ++t) dv += step_row_out<XT, YT, DOT, AT>(3 * brow + t, acc[t], c, u, w, r, y, rdot);
    return dv;
}

// Plain block CSR: one thread per block row, blocks read in place.
template <typename VT, typename XT, typename YT, int DOT>
__global__ void __launch_bounds__(kBlock)
bsr3_step_kernel(const int nb, const int32_t* __restrict__ browptr, const int32_t* __restrict__ bcol,
                 const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                 const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                 const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done) {
    using AT = typename AccOf<XT>::type;
    if (done != nullptr && *done) return;
    double dv = 0.0;
    const int ntiles = (nb + kBlock - 1) / kBlock;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int br = tile * kBlock + threadIdx.x;
    if (br < nb) {
        AT acc[3] = {AT(0), AT(0), AT(0)};
        for (int p = browptr[br]; p < browptr[br + 1]; ++p) {
            const int bc = bcol[p];
            const VT* b = val + (long long)p * 9;
            const AT x0 = (AT)__ldg(u + 3 * bc), x1 = (AT)__ldg(u + 3 * bc + 1), x2 = (AT)__ldg(u + 3 * bc + 2);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                acc[t] = fma((AT)ld_val(b + 3 * t), x0, acc[t]);
                acc[t] = fma((AT)ld_val(b + 3 * t + 1), x1, acc[t]);
                acc[t] = fma((AT)ld_val(b + 3 * t + 2), x2, acc[t]);
            }
        }
        dv += bsr_rows_out<XT, YT, DOT, AT>(br, acc, c, u, w, r, y, rdot);
    }
    }
    if (DOT != 0) grid_reduce<kBlock>(dv, R);
}

// BSELL-32: slice_ptr in blocks; block (slot j, lane l) of slice s is at
// q = slice_ptr[s] + 32 j + l; its column at bcol[q]; its entry e at
// val[(slice_ptr[s] + 32 j) * 9 + 32 e + l].
template <typename VT, typename XT, typename YT, int DOT>
__global__ void __launch_bounds__(kBlock)
bsell3_step_kernel(const int nb, const int32_t* __restrict__ slice_ptr, const int32_t* __restrict__ bcol,
                   const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                   const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                   const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done) {
    using AT = typename AccOf<XT>::type;
    if (done != nullptr && *done) return;
    double dv = 0.0;
    const int ntiles = (nb + kBlock - 1) / kBlock;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int br = tile * kBlock + threadIdx.x;
    if (br < nb) {
        const int s = br >> 5, lane = br & 31;
        const int beg = slice_ptr[s];
        const int len = (slice_ptr[s + 1] - beg) >> 5;
        const int32_t* cp = bcol + beg + lane;
        const VT* vp = val + (long long)beg * 9 + lane;
        AT acc[3] = {AT(0), AT(0), AT(0)};
#pragma unroll 2
        for (int j = 0; j < len; ++j) {
            const int bc = ld_stream(cp);
            AT v[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) v[e] = (AT)ld_stream(vp + 32 * e);
            const AT x0 = (AT)__ldg(u + 3 * bc), x1 = (AT)__ldg(u + 3 * bc + 1), x2 = (AT)__ldg(u + 3 * bc + 2);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                acc[t] = fma(v[3 * t], x0, acc[t]);
                acc[t] = fma(v[3 * t + 1], x1, acc[t]);
                acc[t] = fma(v[3 * t + 2], x2, acc[t]);
            }
            cp += 32;
            vp += 32 * 9;
        }
        dv += bsr_rows_out<XT, YT, DOT, AT>(br, acc, c, u, w, r, y, rdot);
    }
    }
    if (DOT != 0) grid_reduce<kBlock>(dv, R);
}

template <typename VT, typename XT, typename YT>
cudaError_t bsr_dispatch(bool sliced, int nb, const int32_t* ptr, const int32_t* bcol, const void* val,
                         const void* u, const void* w, const void* r, void* y, double ca, double cb, double cc,
                         double cd, int dot, const double* rdot, const Reduce& R, const int* done,
                         cudaStream_t st) {
    using AT = typename AccOf<XT>::type;
    const int tiles = (nb + kBlock - 1) / kBlock;
    const int red = vec_grid_max();
    const int grid = (dot == 0 || tiles < red) ? tiles : red;
    const StepCoef<AT> c = make_coef<AT>(ca, cb, cc, cd);
    const VT* v = static_cast<const VT*>(val);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
#define NC_BSR_LAUNCH(K, D) K<VT, XT, YT, D><<<grid, kBlock, 0, st>>>(nb, ptr, bcol, v, uu, ww, rr, yy, c, rdot, R, done)
    if (sliced) {
        if (dot == 0) NC_BSR_LAUNCH(bsell3_step_kernel, 0);
        else if (dot == 1) NC_BSR_LAUNCH(bsell3_step_kernel, 1);
        else NC_BSR_LAUNCH(bsell3_step_kernel, 2);
    } else {
        if (dot == 0) NC_BSR_LAUNCH(bsr3_step_kernel, 0);
        else if (dot == 1) NC_BSR_LAUNCH(bsr3_step_kernel, 1);
        else NC_BSR_LAUNCH(bsr3_step_kernel, 2);
    }
#undef NC_BSR_LAUNCH
    return cudaGetLastError();
}

// d^{-1/2} from the diagonal entries of each diagonal block
__global__ void bsr3_diag_kernel(int nb, const int32_t* __restrict__ browptr, const int32_t* __restrict__ bcol,
                                 const double* __restrict__ val, double* __restrict__ dis, int* __restrict__ bad) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    if (br >= nb) return;
    double d[3] = {0.0, 0.0, 0.0};
    for (int p = browptr[br]; p < browptr[br + 1]; ++p)
        if (bcol[p] == br)
            for (int t = 0; t < 3; ++t) d[t] = val[(long long)p * 9 + 4 * t];
    for (int t = 0; t < 3; ++t) {
        if (!(d[t] > 0.0)) {
            atomicOr(bad, 1);
            dis[3 * br + t] = 0.0;
        } else {
            dis[3 * br + t] = 1.0 / sqrt(d[t]);
        }
    }
}

// a -> (a d_row^{-1/2}) d_col^{-1/2}, entrywise
__global__ void bsr3_scale_kernel(int nb, const int32_t* __restrict__ browptr, const int32_t* __restrict__ bcol,
                                  const double* __restrict__ val, const double* __restrict__ dis,
                                  double* __restrict__ out) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    if (br >= nb) return;
    for (int p = browptr[br]; p < browptr[br + 1]; ++p) {
        const int bc = bcol[p];
        for (int t = 0; t < 3; ++t)
            for (int q = 0; q < 3; ++q) {
                const long long e = (long long)p * 9 + 3 * t + q;
                out[e] = val[e] * dis[3 * br + t] * dis[3 * bc + q];
            }
    }
}

// First level of the two-level variant (Sec. 6, conclusions): P_0 = W W^T
// with W = blockdiag(L_i^{-T}), A_ii = L_i L_i^T.  One thread per block row:
// the 3x3 Cholesky factor of the diagonal block and its triangular inverse
// (written out from the definitions; sqrt and division are CUDA's).  W_i and
// L_i are stored row-major; *bad is set when a block is not positive
// definite or has no diagonal block.
__global__ void bsr3_block_factor_kernel(int nb, const int32_t* __restrict__ browptr,
                                         const int32_t* __restrict__ bcol, const double* __restrict__ val,
                                         double* __restrict__ wblk, double* __restrict__ lblk,
                                         int* __restrict__ bad) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    if (br >= nb) return;
    const double* d = nullptr;
    for (int p = browptr[br]; p < browptr[br + 1]; ++p)
        if (bcol[p] == br) d = val + (long long)p * 9;
    double* W = wblk + (long long)br * 9;
    double* L = lblk + (long long)br * 9;
    for (int e = 0; e < 9; ++e) W[e] = L[e] = 0.0;
    if (d == nullptr) { atomicOr(bad, 1); return; }
    const double p0 = d[0];
    if (!(p0 > 0.0)) { atomicOr(bad, 1); return; }
    const double l00 = sqrt(p0);
    const double l10 = d[3] / l00, l20 = d[6] / l00;
    const double p1 = d[4] - l10 * l10;
    if (!(p1 > 0.0)) { atomicOr(bad, 1); return; }
    const double l11 = sqrt(p1);
    const double l21 = (d[7] - l20 * l10) / l11;
    const double p2 = d[8] - l20 * l20 - l21 * l21;
    if (!(p2 > 0.0) || !isfinite(p2)) { atomicOr(bad, 1); return; }
    const double l22 = sqrt(p2);
    // M = L^{-1} (lower): M L = I
    const double m00 = 1.0 / l00, m11 = 1.0 / l11, m22 = 1.0 / l22;
    const double m10 = -l10 * m00 / l11;
    const double m21 = -l21 * m11 / l22;
    const double m20 = -(l20 * m00 + l21 * m10) / l22;
    // W = M^T (upper)
    W[0] = m00; W[1] = m10; W[2] = m20;
    W[4] = m11; W[5] = m21;
    W[8] = m22;
    L[0] = l00;
    L[3] = l10; L[4] = l11;
    L[6] = l20; L[7] = l21; L[8] = l22;
}

// out_p = W_i^T A_p W_j for block p in row i, column j
__global__ void bsr3_block_scale_kernel(int nb, const int32_t* __restrict__ browptr,
                                        const int32_t* __restrict__ bcol, const double* __restrict__ val,
                                        const double* __restrict__ wblk, double* __restrict__ out) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    if (br >= nb) return;
    const double* Wi = wblk + (long long)br * 9;
    for (int p = browptr[br]; p < browptr[br + 1]; ++p) {
        const double* Wj = wblk + (long long)bcol[p] * 9;
        const double* a = val + (long long)p * 9;
        double t[9];   // A_p W_j
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                t[3 * r + c] = a[3 * r] * Wj[c] + a[3 * r + 1] * Wj[3 + c] + a[3 * r + 2] * Wj[6 + c];
        double* o = out + (long long)p * 9;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                o[3 * r + c] = Wi[r] * t[c] + Wi[3 + r] * t[3 + c] + Wi[6 + r] * t[6 + c];
    }
}

// Transforms between the original and the scaled system, per block row:
// copy in bs = W^T b, xs = L^T x (= W^{-1} x, or 0); copy out x = W y
// (0 when b = 0).
__global__ void bsr3_block_copy_in_kernel(int nb, const double* __restrict__ b, const double* __restrict__ x,
                                          const double* __restrict__ wblk, const double* __restrict__ lblk,
                                          int zero, double* __restrict__ bs, double* __restrict__ xs) {
    for (int br = blockIdx.x * blockDim.x + threadIdx.x; br < nb; br += gridDim.x * blockDim.x) {
        const double* W = wblk + (long long)br * 9;
        const double* L = lblk + (long long)br * 9;
        const long long o = 3LL * br;
        for (int t = 0; t < 3; ++t) {
            bs[o + t] = W[t] * b[o] + W[3 + t] * b[o + 1] + W[6 + t] * b[o + 2];
            xs[o + t] = zero ? 0.0 : L[t] * x[o] + L[3 + t] * x[o + 1] + L[6 + t] * x[o + 2];
        }
    }
}

__global__ void bsr3_block_copy_out_kernel(int nb, const double* __restrict__ ys, const double* __restrict__ wblk,
                                           const PcgScalars* __restrict__ S, double* __restrict__ x) {
    const bool zero = S->bb == 0.0;
    for (int br = blockIdx.x * blockDim.x + threadIdx.x; br < nb; br += gridDim.x * blockDim.x) {
        const double* W = wblk + (long long)br * 9;
        const long long o = 3LL * br;
        for (int t = 0; t < 3; ++t)
            x[o + t] = zero ? 0.0 : W[3 * t] * ys[o] + W[3 * t + 1] * ys[o + 1] + W[3 * t + 2] * ys[o + 2];
    }
}

__global__ void bsr3_gershgorin_kernel(int nb, const int32_t* __restrict__ browptr, const double* __restrict__ val,
                                       unsigned long long* __restrict__ out_bits) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (br < nb)
        for (int t = 0; t < 3; ++t) {
            double s = 0.0;
            for (int p = browptr[br]; p < browptr[br + 1]; ++p)
                for (int q = 0; q < 3; ++q) s += fabs(val[(long long)p * 9 + 3 * t + q]);
            m = fmax(m, s);
        }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void bsell3_len_kernel(int nb, const int32_t* __restrict__ browptr, int32_t* __restrict__ slice_len) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    const int nslices = (nb + 31) >> 5;
    int len = 0;
    if (br < nb) len = browptr[br + 1] - browptr[br];
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && (br >> 5) < nslices) slice_len[br >> 5] = len;
}

__device__ __forceinline__ void put(double* p, double v) { *p = v; }
__device__ __forceinline__ void put(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void put(__nv_bfloat16* p, double v) { *p = __double2bfloat16(v); }

template <typename VT>
__global__ void bsell3_fill_kernel(int nb, const int32_t* __restrict__ browptr, const int32_t* __restrict__ bcol,
                                   const double* __restrict__ val, const int32_t* __restrict__ slice_ptr, double shift,
                                   int32_t* __restrict__ scol, VT* __restrict__ sval, int* __restrict__ nodiag) {
    const int br = blockIdx.x * blockDim.x + threadIdx.x;
    const int nslices = (nb + 31) >> 5;
    if ((br >> 5) >= nslices) return;
    const int s = br >> 5, lane = br & 31;
    const int beg = slice_ptr[s];
    const int len = (slice_ptr[s + 1] - beg) >> 5;
    int rs = 0, rl = 0;
    if (br < nb) {
        rs = browptr[br];
        rl = browptr[br + 1] - rs;
    }
    const int self = br < nb ? br : nb - 1;
    bool has_diag = false;
    for (int j = 0; j < len; ++j) {
        const int q = beg + 32 * j + lane;
        VT* dst = sval + (long long)(beg + 32 * j) * 9 + lane;
        if (j < rl) {
            const int bc = bcol[rs + j];
            scol[q] = bc;
            const double* src = val + (long long)(rs + j) * 9;
            for (int e = 0; e < 9; ++e) {
                double v = src[e];
                if (bc == br && (e == 0 || e == 4 || e == 8)) v -= shift;
                put(dst + 32 * e, v);
            }
            if (bc == br) has_diag = true;
        } else {
            scol[q] = self;
            for (int e = 0; e < 9; ++e) put(dst + 32 * e, 0.0);
        }
    }
    if (br < nb && !has_diag && shift != 0.0 && nodiag != nullptr) atomicOr(nodiag, 1);
}

}  // namespace

cudaError_t launch_bsr3_step(bool sliced, int nb, const int32_t* ptr, const int32_t* bcol, const void* val, int vdt,
                             bool x_f32, bool y_f64, const void* u, const void* w, const void* r, void* y, double ca,
                             double cb, double cc, double cd, int dot, const double* rdot, const Reduce& R,
                             const int* done, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        return bsr_dispatch<double, double, double>(sliced, nb, ptr, bcol, val, u, w, r, y, ca, cb, cc, cd, dot, rdot,
                                                    R, done, st);
    }
    if (vdt == NC_F32) {
        if (y_f64)
            return bsr_dispatch<float, float, double>(sliced, nb, ptr, bcol, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                      rdot, R, done, st);
        return bsr_dispatch<float, float, float>(sliced, nb, ptr, bcol, val, u, w, r, y, ca, cb, cc, cd, dot, rdot, R,
                                                 done, st);
    }
    if (vdt == NC_BF16) {
        if (y_f64)
            return bsr_dispatch<__nv_bfloat16, float, double>(sliced, nb, ptr, bcol, val, u, w, r, y, ca, cb, cc, cd,
                                                              dot, rdot, R, done, st);
        return bsr_dispatch<__nv_bfloat16, float, float>(sliced, nb, ptr, bcol, val, u, w, r, y, ca, cb, cc, cd, dot,
                                                         rdot, R, done, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_bsr3_diag(int nb, const int32_t* browptr, const int32_t* bcol, const double* val, double* dis,
                             int* bad, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_diag_kernel<<<(nb + 255) / 256, 256, 0, st>>>(nb, browptr, bcol, val, dis, bad);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_scale(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                              const double* dis, double* out, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_scale_kernel<<<(nb + 255) / 256, 256, 0, st>>>(nb, browptr, bcol, val, dis, out);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_block_factor(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                                     double* wblk, double* lblk, int* bad, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_block_factor_kernel<<<(nb + 255) / 256, 256, 0, st>>>(nb, browptr, bcol, val, wblk, lblk, bad);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_block_scale(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                                    const double* wblk, double* out, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_block_scale_kernel<<<(nb + 255) / 256, 256, 0, st>>>(nb, browptr, bcol, val, wblk, out);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_block_copy_in(int nb, const double* b, const double* x, const double* wblk,
                                      const double* lblk, int zero, double* bs, double* xs, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_block_copy_in_kernel<<<vec_grid(nb), 256, 0, st>>>(nb, b, x, wblk, lblk, zero, bs, xs);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_block_copy_out(int nb, const double* ys, const double* wblk, const PcgScalars* S, double* x,
                                       cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_block_copy_out_kernel<<<vec_grid(nb), 256, 0, st>>>(nb, ys, wblk, S, x);
    return cudaGetLastError();
}

cudaError_t launch_bsr3_gershgorin(int nb, const int32_t* browptr, const double* val, unsigned long long* out_bits,
                                   cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    bsr3_gershgorin_kernel<<<(nb + 255) / 256, 256, 0, st>>>(nb, browptr, val, out_bits);
    return cudaGetLastError();
}

cudaError_t launch_bsell3_lengths(int nb, const int32_t* browptr, int32_t* slice_len, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int threads = ((nb + 31) / 32) * 32;
    bsell3_len_kernel<<<(threads + 255) / 256, 256, 0, st>>>(nb, browptr, slice_len);
    return cudaGetLastError();
}

cudaError_t launch_bsell3_fill(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                               const int32_t* slice_ptr, int vdt, double shift, int32_t* scol, void* sval,
                               int* nodiag, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int threads = ((nb + 31) / 32) * 32;
    const int grid = (threads + 255) / 256;
    if (vdt == NC_F64)
        bsell3_fill_kernel<double><<<grid, 256, 0, st>>>(nb, browptr, bcol, val, slice_ptr, shift, scol,
                                                         static_cast<double*>(sval), nodiag);
    else if (vdt == NC_F32)
        bsell3_fill_kernel<float><<<grid, 256, 0, st>>>(nb, browptr, bcol, val, slice_ptr, shift, scol,
                                                        static_cast<float*>(sval), nodiag);
    else if (vdt == NC_BF16)
        bsell3_fill_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(nb, browptr, bcol, val, slice_ptr, shift, scol,
                                                                static_cast<__nv_bfloat16*>(sval), nodiag);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace nc
