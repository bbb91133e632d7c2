// Internal declarations shared by the CUDA translation units of libncpcg.
//
// Device-side PCG state lives in one PcgScalars block so that a whole solve
// can run as a CUDA graph with no host round trip: every reduction kernel
// finishes its own dot product in the last CTA to arrive ("last block"
// pattern, no spin-wait) and that CTA derives the next PCG scalar (alpha,
// beta, the stopping test) in place.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/nc_pcg.h"

namespace nc {

constexpr int kBlock = 256;           // threads per CTA of the row kernels
constexpr int kChunk = 2048;          // nonzeros staged in shared memory per pass
constexpr int kCtasPerSm = 8;         // 2048 threads per SM at kBlock threads per CTA

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device; 152 on GB300).  Grid sizes of the persistent and
// grid-stride kernels are multiples of it.
int num_sms();
// CTAs of the grid-stride vector kernels (kCtasPerSm per SM)
inline int vec_grid_max() { return num_sms() * kCtasPerSm; }
// Upper bound of vec_grid_max() over any device (partial-sum buffers are
// sized with it so that a solver never depends on the device it was set up on)
constexpr int kMaxGrid = 1024 * kCtasPerSm;

constexpr int kRedOneTile = 64;   // CTAs per SM large enough for one tile per CTA

// Launch choices of the SELL-32 step kernels (sliced and offset-pattern
// layouts), fixed per solver at setup -- by default, or by the tuner, which
// times candidates on the solver's own operator.
enum StepVariant : int {
    STEP_DIRECT = 0,   // one row per thread, loads straight from global memory
    STEP_STAGED = 1,   // persistent CTAs; each 256-row tile's slices (and its r and
                       // x_{k-2} rows) brought into shared memory by bulk
                       // asynchronous copies, `stages` tiles ahead
    STEP_SPLIT = 2     // steps with a dot product only: the plain step's kernel
                       // (its variant and shape), then a separate dot product
                       // over the step's two vectors (launch_dot_fast)
};
struct StepTune {
    int variant = STEP_DIRECT;       // plain steps (no dot product)
    int dot_variant = STEP_DIRECT;   // steps with a dot product
    int stages = 3;         // staged: tiles in flight per CTA (2..4)
    int ctas_per_sm = 2;    // staged: resident CTAs per SM
    int rpt = 1;            // staged: rows per thread (1 or 2; tiles of 256 rpt rows)
    int contig = 0;         // staged: 1 = each CTA takes a contiguous run of tiles
    int dot_stages = 3;     // the same four for the staged steps with a dot product
    int dot_ctas_per_sm = 2;
    int dot_rpt = 1;
    int dot_contig = 0;
    int lookahead = -1;     // direct float kernels: L2 prefetch distance in tiles
                            // (-1: two waves, 2 x num_sms(); 0: off)
    int red_ctas_per_sm = kCtasPerSm;   // direct kernels with a dot product:
                                        // persistent CTAs per SM (kRedOneTile:
                                        // one 256-row tile per CTA)
    int vcap = 0;           // staged: matrix entries of the largest 256-row tile
    int vcap2 = 0;          // and of the largest 512-row tile (rpt = 2)
    int npoff = 0;          // staged: entries of the offset-pattern table
};

// What the last CTA of a reduction does with the finished sum.
enum Fin : int {
    FIN_NONE = 0,
    FIN_STORE = 1,   // *out = sum
    FIN_BB = 2,      // bb = (b, b)
    FIN_RR0 = 3,     // initial (r, r): converged before the first iteration?
    FIN_RZ0 = 4,     // initial (r, z)
    FIN_ALPHA = 5,   // (p, q): alpha = rz / pq
    FIN_RR = 6,      // (r, r) after the update: iteration count and stopping test
    FIN_BETA = 7,    // new (r, z): beta = rz_new / rz
    FIN_TRUE = 8     // ||b - A x||^2 at exit
};

struct PcgScalars {
    double rz, pq, alpha, beta, rr, bb, tol2, rr_true;
    int iter, maxit, done, status;
    int n_dot, n_prec, rr_period, rr_skip;   // residual replacement: period, and
                                             // "skip it this iteration" flag
    int n_replace;
    int fault;       // set by a kernel whose bounded wait on its own copies ran out
    int pad1, pad2;
};

struct Reduce {
    double* partials;        // >= gridDim.x doubles
    unsigned int* counter;   // 0 between reductions; reset by the last CTA
    PcgScalars* S;           // for the PCG finalize kinds
    double* out;             // FIN_STORE target
    int fin;
};

// ---- device helpers -------------------------------------------------------

// Sum over a CTA of BS threads; the result is valid in every lane of warp 0.
// A shared-memory halving tree with full warps (BS/2, BS/4, ... 32 adds),
// then a butterfly inside warp 0: every FP64 add is one warp instruction on
// GB300's narrow FP64 pipe whatever the number of active lanes, and this
// order needs about a quarter of the instructions of a per-warp shuffle tree.
// The order is fixed, so the sum is deterministic.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* sh, int tid) {
    sh[tid] = v;
    __syncthreads();
#pragma unroll
    for (int s = BS / 2; s >= 32; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    double r = 0.0;
    if (tid < 32) {
        r = sh[tid];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ void finalize(const Reduce& R, double s) {
    PcgScalars* S = R.S;
    const bool finite = isfinite(s);
    switch (R.fin) {
    case FIN_STORE:
        *R.out = s;
        break;
    case FIN_BB:
        S->bb = s;
        break;
    case FIN_RR0:
        S->rr = s;
        if (!finite) { S->status = NC_ERR_BREAKDOWN; S->done = 1; }
        else if (S->bb == 0.0 || s <= S->tol2 * S->bb) { S->status = NC_OK; S->done = 1; }
        else if (S->maxit <= 0) { S->status = NC_ERR_MAXIT; S->done = 1; }
        break;
    case FIN_RZ0:
        S->n_dot += 1; S->n_prec += 1;
        S->rz = s;
        if (!(s > 0.0)) { S->status = finite ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN; S->done = 1; }
        break;
    case FIN_ALPHA:
        S->n_dot += 1;
        S->pq = s;
        if (!(s > 0.0) || !finite) { S->status = finite ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN; S->done = 1; }
        else S->alpha = S->rz / s;
        break;
    case FIN_RR:
        S->n_dot += 1;
        S->rr = s;
        S->iter += 1;
        if (!finite) { S->status = NC_ERR_BREAKDOWN; S->done = 1; }
        else if (s <= S->tol2 * S->bb) { S->status = NC_OK; S->done = 1; }
        else if (S->iter >= S->maxit) { S->status = NC_ERR_MAXIT; S->done = 1; }
        // residual replacement r = b - A x after every rr_period-th iteration
        S->rr_skip = S->done || S->rr_period <= 0 || (S->iter % S->rr_period) != 0;
        if (!S->rr_skip) S->n_replace += 1;
        break;
    case FIN_BETA:
        S->n_dot += 1; S->n_prec += 1;
        if (!(s > 0.0) || !finite) { S->status = finite ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN; S->done = 1; }
        else { S->beta = s / S->rz; S->rz = s; }
        break;
    case FIN_TRUE:
        S->rr_true = s;
        break;
    default:
        break;
    }
}

// Each CTA contributes v (one value per thread); the last CTA to finish sums
// the per-CTA partials in a fixed order and applies R.fin.  Must be reached
// by every thread of every CTA of the grid.
template <int BS>
__device__ __forceinline__ void grid_reduce_ex(double v, const Reduce& R, int bid, int nblocks) {
    __shared__ double sh[BS];
    __shared__ int is_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    v = block_sum<BS>(v, sh, tid);
    if (tid == 0) {
        R.partials[bid] = v;
        __threadfence();
        const unsigned int t = atomicAdd(R.counter, 1u);
        is_last = (t == (unsigned int)nblocks - 1u);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s = 0.0;
        for (int i = tid; i < nblocks; i += BS) s += __ldcg(&R.partials[i]);
        s = block_sum<BS>(s, sh, tid);
        if (tid == 0) {
            finalize(R, s);
            *R.counter = 0u;
        }
    }
}

template <int BS>
__device__ __forceinline__ void grid_reduce(double v, const Reduce& R) {
    grid_reduce_ex<BS>(v, R, (int)blockIdx.x, (int)gridDim.x);
}

// ---- host-side launchers (defined in nc_csr.cu / nc_vec.cu) ---------------

enum VecKind : int { VK_F64 = 0, VK_F32 = 1 };

// y = ca*u + cb*w + cc*r + cd*(A u) for a CSR matrix with value type vdt
// (nc_dtype) and vector type given by the pointers' kinds: x_f32 selects
// float u/w/r; y_f64 selects a float64 output.  dot: 0 none, 1 (rdot, y),
// 2 (u, y); the reduction finishes with R.  Coefficients equal to zero skip
// their loads.  Kernels return at once when *done != 0 (done may be null).
cudaError_t launch_csr_step(int n, const int32_t* rowptr, const int32_t* col, const void* val,
                            int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                            const void* r, void* y, double ca, double cb, double cc, double cd,
                            int dot, const double* rdot, const Reduce& R, const int* done,
                            cudaStream_t st);

// Offset patterns of a SELL-32 layout (pstart null: plain SELL, columns in
// `col`): slice s takes the columns row + poff[pstart[s] + j], j < its slots.
struct SellPat {
    const int32_t* pstart = nullptr;
    const int32_t* poff = nullptr;
};

// Same step for the SELL-32 layout (slice_ptr: nslices+1 int32 offsets).
cudaError_t launch_sell_step(int n, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                             const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                             const void* r, void* y, double ca, double cb, double cc, double cd, int dot,
                             const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                             const StepTune& tune = StepTune());
// The staged variant (nc_sell_staged.cu).  Returns cudaErrorNotSupported when
// it does not apply (no scalar block to report a fault in, unaligned vectors
// or values, a stage larger than shared memory); the caller then runs the
// direct kernel.  *R.S->fault is set if a wait for a tile's copies ran out.
cudaError_t launch_sell_staged(int n, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                               const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                               const void* r, void* y, double ca, double cb, double cc, double cd, int dot,
                               const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                               const StepTune& tune);
// Resident CTAs per SM the staged variant would run with for this value /
// vector type, dot kind and tune (at most tune.ctas_per_sm); 0 when it cannot
// run on the current device.
int sell_staged_ctas(int vdt, bool x_f32, bool y_f64, int dot, bool unit, const StepTune& tune);
// Largest number of matrix entries of any tile of `per_tile` slices of a
// SELL-32 layout with host slice offsets hsptr[0..nslices].
int sell_max_tile_entries(const int32_t* hsptr, int nslices, int per_tile);
// Pattern layout construction from CSR: per-slice offset sets (a counting
// pass with off null, then a writing pass at opos), then the slot-major fill;
// skip_diag leaves the diagonal entries out of both.
cudaError_t launch_psell_merge(int n, const int32_t* rowptr, const int32_t* col, const int32_t* opos, int32_t* cnt,
                               int32_t* off, int* bad, int skip_diag, cudaStream_t st);
cudaError_t launch_psell_fill(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                              const int32_t* slice_ptr, const int32_t* pstart, const int32_t* poff, int vdt,
                              double shift, void* sval, int* nodiag, int skip_diag, cudaStream_t st);
// SELL-32 construction from CSR: longest row per slice, then the slot-major fill
cudaError_t launch_sell_lengths(int n, const int32_t* rowptr, int32_t* slice_len, cudaStream_t st);
// (diagonal entries stored as a_ii - shift; *nodiag set if a row lacks one)
cudaError_t launch_sell_fill(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                             const int32_t* slice_ptr, int vdt, double shift, int32_t* scol, void* sval,
                             int* nodiag, cudaStream_t st);

// Matrix-free 7-point stencil (c4 = {c0, cx, cy, cz}, host array).
struct StencilGeom {
    int nx, ny, nz;
    int zc = 0;   // plain steps: z-chunk (planes per CTA); 0 = the size policy
    int pz = 0;   // plain float steps: planes per z-march batch (2 or 4); 0 = the policy
};
// The policy z-chunk (stencil_zchunk ignores g.zc): dot-product steps always
// take it, so the partial-sum buffers sized from it hold.
int stencil_zchunk_policy(const StencilGeom& g);
int stencil_zchunk(const StencilGeom& g);
dim3 stencil_grid(const StencilGeom& g);
long long stencil_nblocks(const StencilGeom& g);
cudaError_t launch_stencil_step(const StencilGeom& g, const double* c4, bool x_f32, bool y_f64, const void* u,
                                const void* w, const void* r, void* y, double ca, double cb, double cc, double cd,
                                int dot, const double* rdot, const Reduce& R, const int* done, cudaStream_t st);

// 3x3-block matrices: plain block CSR (sliced = false, ptr = block row
// pointers) or BSELL-32 (sliced = true, ptr = slice pointers in blocks).
cudaError_t launch_bsr3_step(bool sliced, int nb, const int32_t* ptr, const int32_t* bcol, const void* val, int vdt,
                             bool x_f32, bool y_f64, const void* u, const void* w, const void* r, void* y, double ca,
                             double cb, double cc, double cd, int dot, const double* rdot, const Reduce& R,
                             const int* done, cudaStream_t st);
cudaError_t launch_bsr3_diag(int nb, const int32_t* browptr, const int32_t* bcol, const double* val, double* dis,
                             int* bad, cudaStream_t st);
cudaError_t launch_bsr3_scale(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                              const double* dis, double* out, cudaStream_t st);
// Two-level variant, first level block Jacobi: W_i = L_i^{-T}, L_i the
// Cholesky factor of diagonal block i (row-major 3x3 each); *bad set when a
// block is missing or not positive definite
cudaError_t launch_bsr3_block_factor(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                                     double* wblk, double* lblk, int* bad, cudaStream_t st);
// out_p = W_i^T A_p W_j
cudaError_t launch_bsr3_block_scale(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                                    const double* wblk, double* out, cudaStream_t st);
// bs = W^T b, xs = L^T x (or 0); and x = W ys (0 when S->bb == 0)
cudaError_t launch_bsr3_block_copy_in(int nb, const double* b, const double* x, const double* wblk,
                                      const double* lblk, int zero, double* bs, double* xs, cudaStream_t st);
cudaError_t launch_bsr3_block_copy_out(int nb, const double* ys, const double* wblk, const PcgScalars* S, double* x,
                                       cudaStream_t st);
cudaError_t launch_bsr3_gershgorin(int nb, const int32_t* browptr, const double* val, unsigned long long* out_bits,
                                   cudaStream_t st);
cudaError_t launch_bsell3_lengths(int nb, const int32_t* browptr, int32_t* slice_len, cudaStream_t st);
cudaError_t launch_bsell3_fill(int nb, const int32_t* browptr, const int32_t* bcol, const double* val,
                               const int32_t* slice_ptr, int vdt, double shift, int32_t* scol, void* sval,
                               int* nodiag, cudaStream_t st);

cudaError_t launch_csr_diag(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                            double* dis, int* bad, cudaStream_t st);
cudaError_t launch_csr_scale(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                             const double* dis, double* out, cudaStream_t st);
// *flags |= 1 unless every row has a diagonal entry equal (bitwise) to row 0's
cudaError_t launch_csr_diag_const(int n, const int32_t* rowptr, const int32_t* col, const double* val, int* flags,
                                  cudaStream_t st);
cudaError_t launch_csr_gershgorin(int n, const int32_t* rowptr, const double* val,
                                  unsigned long long* out_bits, cudaStream_t st);
cudaError_t launch_convert(int64_t count, const double* in, int out_dt, void* out, cudaStream_t st);

int vec_grid(int64_t n);

// Whole PCG solve in one kernel on one thread-block cluster, the system held
// in the cluster's shared memory (nc_cluster.cu).  C CTAs of R rows each;
// `slots` SELL entries and `smem` bytes of shared memory per CTA.
struct ClusterPlan {
    int C, R, slots;
    size_t smem;
};
// Plan for a float64 SELL-32 operator of n rows with host slice offsets
// hsptr[0..ceil(n/32)]; false when it does not fit one cluster.
bool plan_cluster_pcg(int n, const int32_t* hsptr, ClusterPlan* plan);
cudaError_t launch_cluster_pcg(const ClusterPlan& p, int n, int k, int x0_zero, int maxit, double tol2, double shift,
                               const int32_t* sptr, const int32_t* col, const double* val, const double* coef,
                               const double* b, double* x, PcgScalars* S, cudaStream_t st);

// x += alpha p; r -= alpha q; r32 = (float) r (if r32); (r, r) -> FIN_RR
cudaError_t launch_axpy2_rr(int n, double* x, double* r, const double* p, const double* q,
                            float* r32, const Reduce& R, cudaStream_t st);
// p = z + beta p; then (if use_cond) set the loop condition to !done
cudaError_t launch_p_update(int n, double* p, const double* z, PcgScalars* S,
                            cudaGraphConditionalHandle h, int use_cond, cudaStream_t st);
// z = c r and (r, z) (degree-0 preconditioner); skip if *done
cudaError_t launch_scale_dot(int n, const double* r, double c, double* z, const Reduce& R,
                             const int* done, cudaStream_t st);
// (a, b) -> R (skip if *done when done != null)
// the same sum order for every call with the same n; 16-byte-aligned vectors
// take a kernel with 16-byte loads, four pairs per round (others: launch_dot)
cudaError_t launch_dot_fast(int n, const double* a, const double* b, const Reduce& R, const int* done,
                            cudaStream_t st);
cudaError_t launch_dot(int n, const double* a, const double* b, const Reduce& R, const int* done,
                       cudaStream_t st);
// y = x (skip if *done)
cudaError_t launch_copy(int n, const double* x, double* y, const int* done, cudaStream_t st);
// b_s = d .* b; x_s = 0 if zero else x ./ d, with d = dis (vector) or ds (constant)
cudaError_t launch_copy_in(int n, const double* b, const double* x, const double* dis, double ds, int zero,
                           double* bs, double* xs, cudaStream_t st);
// x = d .* x_s; x = 0 when S->bb == 0
cudaError_t launch_copy_out(int n, const double* xs, const double* dis, double ds, const PcgScalars* S,
                            double* x, cudaStream_t st);
// y = y + a x and (y, y) -> R
cudaError_t launch_axpy_dot(int n, double a, const double* x, double* y, const Reduce& R,
                            cudaStream_t st);
// Block step for m <= max_rhs() right-hand sides stored one after the other
// (column c of u, w, r, y at offset c * ld): Y = ca U + cb W + cc R + cd A U,
// the SELL matrix read once for all columns; returns at once when every
// column's scalars (Sm[0..m)) say done.
int max_rhs();
cudaError_t launch_sell_mstep(int n, int m, int ld, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                              const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                              const void* r, void* y, double ca, double cb, double cc, double cd,
                              const PcgScalars* Sm, cudaStream_t st);
// loop condition of a multi-right-hand-side graph: some column not done
cudaError_t launch_any_active(const PcgScalars* Sm, int m, cudaGraphConditionalHandle h, int use_cond, int* active,
                              cudaStream_t st);
// out = a x + b y (out may alias y); with rdot non-null, (rdot, out) -> R;
// skipped when *done
cudaError_t launch_axpby_dot(int n, double a, const double* x, double b, const double* y, double* out,
                             const double* rdot, const Reduce& R, const int* done, cudaStream_t st);
// r32 = (float) r unless *skip
cudaError_t launch_refresh_r32(int n, const double* r, float* r32, const int* skip, cudaStream_t st);
// y = x / d
cudaError_t launch_div(int n, const double* x, double d, double* y, cudaStream_t st);

}  // namespace nc
