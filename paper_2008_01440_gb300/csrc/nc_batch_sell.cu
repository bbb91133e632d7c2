// Batched engine, explicit matrices: the kernels of single explicit-matrix
// slots and of groups (several right-hand sides of one solver sharing each
// matrix read), over their own tile lists, and their launchers; the tables
// and the host side are nc_batch.cuh and nc_batch.cu.
#include <type_traits>

#include "nc_batch.cuh"
#include "nc_sell.cuh"

namespace nc {
namespace batch {
namespace {

// ---- explicit-matrix slots: their own kernels over their own tile list
// (kSellTileRows rows per tile, walked by the CTA in 256-row blocks), so
// that the stencil kernels keep their register budgets; launched only while
// the engine holds such slots

// The dot terms of a tile's rows are summed with __dadd_rn (never fused
// into an fma with the term's product), so that the single-slot kernels and
// the group kernels round them alike whatever the compiler contracts.

// Chebyshev step j of the explicit slots whose values inside P are VT
// (double: the float64 apply; float or bfloat16: the float32 apply)
template <typename VT, typename XT, typename YT, int DOT, bool UNIT>
__device__ __forceinline__ double sell_block(int row, int n, const int32_t* sptr, const int32_t* scol,
                                             const SellPat& pat, const VT* val, const XT* u, const XT* w,
                                             const XT* r, YT* y, const StepCoef<typename AccOf<XT>::type>& c,
                                             const double* rdot) {
    if (row >= n) return 0.0;
    if (pat.pstart != nullptr)
        return sell_row<VT, XT, YT, DOT, true, UNIT>(row, n, sptr, nullptr, pat, val, u, w, r, y, c, rdot);
    return sell_row<VT, XT, YT, DOT, false, UNIT>(row, n, sptr, scol, pat, val, u, w, r, y, c, rdot);
}

__global__ void __launch_bounds__(256, 6) bk_sell_opq(const BDesc* __restrict__ D, BState* S,
                                                   const BTile* __restrict__ T, BCtl* ctl, double* partials) {
    const int tid = threadIdx.x;
    const int nt = ctl->nstiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        if (st->phase != PH_RUN) continue;
        const BDesc* dp = D + tl.pair;
        const int n = dp->n;
        const SellPat pat = dp->pat;
        const int32_t *sptr = dp->sptr, *scol = dp->scol;
        const double* val = dp->val64;
        const double* p = dp->p;
        double* q = dp->q;
        StepCoef<double> c;   // q = A' p + shift p, (p, q)
        c.ca = dp->shift; c.cb = 0.0; c.cc = 0.0; c.cd = 1.0;
        c.terms = (c.ca != 0.0 ? kTermU : 0) | kUnitD;
        const int tile0 = dp->tile0, ntl = dp->tile1 - dp->tile0;
        double dv = 0.0;
        const int f1 = min(tl.f0 + kSellTileRows, n);
#pragma unroll 1
        for (int f = tl.f0; f < f1; f += kFT)
            dv = __dadd_rn(dv, sell_block<double, double, double, 2, true>(f + tid, n, sptr, scol, pat, val, p,
                                                                            nullptr, nullptr, q, c, nullptr));
        reduce_slot(dv, partials, t, tile0, ntl, st, ctl, BF_ALPHA);
    }
}

// PART: 0 every slot (float64 apply), 1 only the slots whose last step is
// j (with (r, z)), 2 only the others -- the float kernels are split so that
// each inlines one row path and keeps its register budget
template <typename VT, int PART>
__global__ void __launch_bounds__(256, std::is_same<VT, double>::value ? 6 : 4) bk_sell_cheb(const BDesc* __restrict__ D, BState* S,
                                                    const BTile* __restrict__ T, const BCoef* __restrict__ C,
                                                    BCtl* ctl, double* partials, int j,
                                                    const int* __restrict__ ntile_step) {
    constexpr bool F64 = std::is_same<VT, double>::value;
    using XT = typename std::conditional<F64, double, float>::type;
    using AT = XT;
    const int tid = threadIdx.x;
    const int nt = ntile_step[j];   // tiles of slots with k >= j (ordered by degree)
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        const int ph = st->phase;
        if (ph != PH_RUN && ph != PH_INIT) continue;
        const BDesc* dp = D + tl.pair;
        const int k = dp->k;
        if (j > k) continue;
        if ((PART == 1 && j != k) || (PART == 2 && j == k)) continue;
        const int vdt = dp->vdtP;
        if (!F64 && (vdt == NC_BF16) != std::is_same<VT, __nv_bfloat16>::value) continue;   // the other kernel's
        // the fields this step needs, read once per tile
        const int n = dp->n;
        const int32_t* sptr = dp->sptr;
        const int32_t* scol = dp->scol;
        const SellPat pat = dp->pat;
        const VT* val = F64 ? reinterpret_cast<const VT*>(dp->val64) : static_cast<const VT*>(dp->valP);
        const double* r64 = dp->r;
        double* z = dp->z;
        XT *t0, *t1, *t2;
        const XT* r;
        if constexpr (F64) {
            t0 = dp->dt0; t1 = dp->dt1; t2 = dp->dt2;
            r = dp->r;
        } else {
            t0 = dp->t0; t1 = dp->t1; t2 = dp->t2;
            r = dp->r32;
        }
        // the rotating vectors by index, selected (not an indexed array: no local memory)
        auto tb = [&](int i) -> XT* { return i == 0 ? t0 : (i == 1 ? t1 : t2); };
        const int tile0 = dp->tile0, ntl = dp->tile1 - dp->tile0;
        const BCoef bc = C[dp->coef0 + j - 1];
        StepCoef<AT> c;
        if constexpr (F64) {
            c.ca = bc.e0d; c.cb = bc.cbd; c.cc = bc.ccd; c.cd = bc.exd;
        } else {
            c.ca = bc.e0; c.cb = bc.cb; c.cc = bc.cc; c.cd = bc.ex;
        }
        c.terms = bc.terms;
        const XT* u = (j == 1) ? r : tb((j - 1) % 3);
        const XT* w = (j >= 3) ? tb((j - 2) % 3) : nullptr;
        const int f1 = min(tl.f0 + kSellTileRows, n);
        const bool unit = F64 && bc.xu;
        if constexpr (PART != 2) {
            if (j == k) {
                double dv = 0.0;
#pragma unroll 1
                for (int f = tl.f0; f < f1; f += kFT)
                    dv = __dadd_rn(dv, unit ? sell_block<VT, XT, double, 1, F64>(f + tid, n, sptr, scol, pat, val, u,
                                                                                  w, r, z, c, r64)
                                            : sell_block<VT, XT, double, 1, false>(f + tid, n, sptr, scol, pat, val,
                                                                                    u, w, r, z, c, r64));
                reduce_slot(dv, partials, t, tile0, ntl, st, ctl, BF_RZ);
                continue;
            }
        }
        if constexpr (PART != 1) {
            XT* y = tb(j % 3);
#pragma unroll 1
            for (int f = tl.f0; f < f1; f += kFT) {
                if (unit) sell_block<VT, XT, XT, 0, F64>(f + tid, n, sptr, scol, pat, val, u, w, r, y, c, nullptr);
                else sell_block<VT, XT, XT, 0, false>(f + tid, n, sptr, scol, pat, val, u, w, r, y, c, nullptr);
            }
        }
    }
}

__global__ void __launch_bounds__(256) bk_sell_true(const BDesc* __restrict__ D, BState* S,
                                                    const BTile* __restrict__ T, BCtl* ctl, double* partials) {
    const int tid = threadIdx.x;
    const int nt = ctl->nstiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        if (st->phase != PH_FINISH) continue;
        const BDesc* dp = D + tl.pair;
        const int n = dp->n;
        const SellPat pat = dp->pat;
        const int32_t *sptr = dp->sptr, *scol = dp->scol;
        const double* val = dp->val64;
        StepCoef<double> c;   // q = b - (A' x + shift x), ||q||^2
        c.ca = -dp->shift; c.cb = 0.0; c.cc = 1.0; c.cd = -1.0;
        c.terms = (c.ca != 0.0 ? kTermU : 0) | kTermR;
        const double *x = dp->x, *b = dp->b;
        double* q = dp->q;
        const int tile0 = dp->tile0, ntl = dp->tile1 - dp->tile0;
        double dv = 0.0;
        const int f1 = min(tl.f0 + kSellTileRows, n);
#pragma unroll 1
        for (int f = tl.f0; f < f1; f += kFT)
            dv = __dadd_rn(dv, sell_block<double, double, double, 3, false>(f + tid, n, sptr, scol, pat, val, x,
                                                                             nullptr, b, q, c, nullptr));
        reduce_slot(dv, partials, t, tile0, ntl, st, ctl, BF_TRUE);
    }
}

// ---- groups: kernels over the group tile list, one instance per width M
// (2, 4 or 8 columns), each over its own segment of the list (kSellTileRows
// rows of one group per tile, all its columns)

// One row of a group of width M: the row's columns (or offsets) and values
// are loaded once per slot and applied to every column whose bit is set in
// `mask` (the others are neither gathered nor written).  Per column the
// products are summed in the single-slot kernels' order and the epilogue is
// theirs (step_row_out), so a column's result is bit-identical to the same
// right-hand side in a slot of its own.  Column q's vectors are column 0's
// plus q times their stride (32-bit: groups are formed only where 7 strides
// fit).
template <typename VT, typename XT, typename YT, int DOT, bool PAT, bool UNIT, int M>
__device__ __forceinline__ void sell_row_group(const int row, const int n, const int32_t* __restrict__ slice_ptr,
                                               const int32_t* __restrict__ col, const SellPat& pat,
                                               const VT* __restrict__ val, const XT* u, const int ldu,
                                               const XT* w, const int ldw, const XT* r, const int ldr, YT* y,
                                               const int ldy, const double* rdot, const int ldd,
                                               const StepCoef<typename AccOf<XT>::type>& c, const unsigned mask,
                                               double (&dv)[M]) {
    using AT = typename AccOf<XT>::type;
    // slots per load group: about 16 (float) or 8 (double) gathers in flight
    constexpr int G = sizeof(AT) == 8 ? (M >= 8 ? 1 : 8 / M) : (M >= 8 ? 2 : 16 / M);
    const int s = row >> 5;
    const int beg = slice_ptr[s];
    const int len = (slice_ptr[s + 1] - beg) >> 5;   // warp-uniform
    const VT* vp = val + beg + (row & 31);
    const int32_t* cp = nullptr;
    const int32_t* op = nullptr;
    if constexpr (PAT) op = pat.poff + __ldg(pat.pstart + s);
    else cp = col + beg + (row & 31);
    AT acc[M];
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] = AT(0);
    for (int j0 = 0; j0 < len; j0 += G) {
        int cj[G];
        AT vj[G];
#pragma unroll
        for (int t = 0; t < G; ++t) {
            cj[t] = row;
            vj[t] = AT(0);
            if (j0 + t < len) {
                if constexpr (PAT) cj[t] = min(max(row + __ldg(op + t), 0), n - 1);
                else cj[t] = ld_stream(cp + 32 * t);
                vj[t] = (AT)ld_stream(vp + 32 * t);
            }
        }
        AT xv[M][G];
#pragma unroll
        for (int q = 0; q < M; ++q)
#pragma unroll
            for (int t = 0; t < G; ++t)
                xv[q][t] = (((mask >> q) & 1u) && j0 + t < len) ? (AT)__ldg(u + (q * ldu + cj[t])) : AT(0);
#pragma unroll
        for (int q = 0; q < M; ++q)
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (j0 + t < len) acc[q] = fma(vj[t], xv[q][t], acc[q]);
        vp += 32 * G;
        if constexpr (PAT) op += G;
        else cp += 32 * G;
    }
#pragma unroll
    for (int q = 0; q < M; ++q)
        if ((mask >> q) & 1u) {
            const double t = step_row_out<XT, YT, DOT, AT, UNIT>(row, acc[q], c, u + q * ldu,
                                                                 w ? w + q * ldw : nullptr, r ? r + q * ldr : nullptr,
                                                                 y + q * ldy, rdot ? rdot + q * ldd : nullptr);
            if (DOT != 0) dv[q] = __dadd_rn(dv[q], t);
        }
}

// The tile's rows [f0, f1), one per thread per block of kFT rows.
template <typename VT, typename XT, typename YT, int DOT, bool UNIT, int M>
__device__ __forceinline__ void group_rows(const BGDesc* g, const int f0, const int f1, const VT* val, const XT* u,
                                           const int ldu, const XT* w, const int ldw, const XT* r, const int ldr,
                                           YT* y, const int ldy, const double* rdot,
                                           const StepCoef<typename AccOf<XT>::type>& c, const unsigned mask,
                                           double (&dv)[M]) {
    const int n = g->n;
    const int32_t *sptr = g->sptr, *scol = g->scol;
    const SellPat pat = g->pat;
    const int ldd = g->ld64;
    if (pat.pstart != nullptr) {
#pragma unroll 1
        for (int f = f0; f < f1; f += kFT) {
            const int row = f + (int)threadIdx.x;
            if (row < n)
                sell_row_group<VT, XT, YT, DOT, true, UNIT, M>(row, n, sptr, nullptr, pat, val, u, ldu, w, ldw, r,
                                                               ldr, y, ldy, rdot, ldd, c, mask, dv);
        }
    } else {
#pragma unroll 1
        for (int f = f0; f < f1; f += kFT) {
            const int row = f + (int)threadIdx.x;
            if (row < n)
                sell_row_group<VT, XT, YT, DOT, false, UNIT, M>(row, n, sptr, scol, pat, val, u, ldu, w, ldw, r,
                                                                ldr, y, ldy, rdot, ldd, c, mask, dv);
        }
    }
}

// The columns of a group whose slot is in phase ph0 or ph1.  Uniform across
// the CTA: a column's phase changes only when its last tile is reduced,
// which cannot happen before this CTA has reduced the tile it reads for.
template <int M>
__device__ __forceinline__ unsigned group_mask(const BGDesc* g, const BState* S, int ph0, int ph1) {
    unsigned m = 0;
    const int live = g->live;
#pragma unroll
    for (int q = 0; q < M; ++q)
        if ((live >> q) & 1) {
            const int ph = S[g->slot[q]].phase;
            if (ph == ph0 || ph == ph1) m |= 1u << q;
        }
    return m;
}

// Every selected column's partial of tile t into its own row of the group
// partials (column q: [q * gpstride + tile]) and its slot's reduction, all
// columns in one pass: each column's block sum takes block_sum's order and
// the last tile's total reduce_slot's, so the sums are those of single slots.
template <int M>
__device__ void group_reduce(const double (&dv)[M], double* part, const int t, const BGDesc* g, BState* S,
                             BCtl* ctl, const unsigned mask, const int kind) {
    __shared__ double sh[M][256];
    __shared__ int last[M];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < M; ++q) sh[q][tid] = dv[q];
    __syncthreads();
#pragma unroll
    for (int s = 128; s >= 32; s >>= 1) {
        if (tid < s) {
#pragma unroll
            for (int q = 0; q < M; ++q) sh[q][tid] += sh[q][tid + s];
        }
        __syncthreads();
    }
    if (tid < 32) {
#pragma unroll
        for (int q = 0; q < M; ++q) {
            double r = sh[q][tid];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (tid == 0) sh[q][0] = r;
        }
    }
    __syncthreads();
    const int gps = ctl->gpstride, tile0 = g->tile0, ntl = g->tile1 - g->tile0;
    if (tid < M) {
        int is_last = 0;
        if ((mask >> tid) & 1u) {
            part[tid * gps + t] = sh[tid][0];
            __threadfence();
            const unsigned int c = atomicAdd(&S[g->slot[tid]].counter, 1u);
            is_last = (c == (unsigned int)ntl - 1u);
        }
        last[tid] = is_last;
    }
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < M; ++q) {
        if (!last[q]) continue;   // uniform
        __threadfence();
        const int first = q * gps + tile0;
        double s = 0.0;
        for (int i = tid; i < ntl; i += 256) s += __ldcg(&part[first + i]);
        s = block_sum<256>(s, &sh[0][0], tid);
        if (tid == 0) {
            BState* st = S + g->slot[q];
            bfinalize(st, ctl, kind, s);
            st->counter = 0u;
        }
        __syncthreads();
    }
}

template <int M>
__global__ void __launch_bounds__(256, 3) bk_group_opq(const BGDesc* __restrict__ G, BState* S,
                                                       const BTile* __restrict__ T, BCtl* ctl, double* part) {
    const int t0 = ctl->gseg[M == 2 ? 0 : 1], t1 = ctl->gseg[M == 2 ? 1 : 2];
    for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
        const BTile tl = T[t];
        const BGDesc* g = G + tl.pair;
        const unsigned mask = group_mask<M>(g, S, PH_RUN, PH_RUN);
        if (mask == 0u) continue;
        StepCoef<double> c;   // q = A' p + shift p, (p, q)
        c.ca = g->shift; c.cb = 0.0; c.cc = 0.0; c.cd = 1.0;
        c.terms = (c.ca != 0.0 ? kTermU : 0) | kUnitD;
        const int ld = g->ld64;
        double dv[M];
#pragma unroll
        for (int q = 0; q < M; ++q) dv[q] = 0.0;
        group_rows<double, double, double, 2, true, M>(g, tl.f0, min(tl.f0 + kSellTileRows, g->n), g->val64, g->p,
                                                       ld, nullptr, 0, nullptr, 0, g->q, ld, nullptr, c, mask, dv);
        group_reduce<M>(dv, part, t, g, S, ctl, mask, BF_ALPHA);
    }
}

// PART 1: only the groups whose last step is j (z = P r in float64 and
// (r, z)), 2: only the others (no dot product: the most frequent kernel
// keeps more CTAs per SM)
template <typename VT, int PART, int M>
constexpr int group_min_ctas() {
    return PART != 2 ? 3 : (std::is_same<VT, double>::value ? (M >= 8 ? 4 : 5) : (M >= 8 ? 5 : 6));
}

template <typename VT, int PART, int M>
__global__ void __launch_bounds__(256, group_min_ctas<VT, PART, M>()) bk_group_cheb(const BGDesc* __restrict__ G, BState* S,
                                                                        const BTile* __restrict__ T,
                                                                        const BCoef* __restrict__ C, BCtl* ctl,
                                                                        double* part, int j,
                                                                        const int* __restrict__ ntile_step) {
    constexpr bool F64 = std::is_same<VT, double>::value;
    using XT = typename std::conditional<F64, double, float>::type;
    constexpr int seg = M == 2 ? 0 : 1;
    const int t0 = ctl->gseg[seg];
    const int t1 = t0 + ntile_step[j];   // the segment's tiles of groups with k >= j (by degree)
    for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
        const BTile tl = T[t];
        const BGDesc* g = G + tl.pair;
        const int k = g->k;
        if (j > k) continue;
        if ((PART == 1 && j != k) || (PART == 2 && j == k)) continue;
        if (!F64 && (g->vdtP == NC_BF16) != std::is_same<VT, __nv_bfloat16>::value) continue;
        const unsigned mask = group_mask<M>(g, S, PH_RUN, PH_INIT);
        if (mask == 0u) continue;
        const BCoef bc = C[g->coef0 + j - 1];
        const VT* val = F64 ? reinterpret_cast<const VT*>(g->val64) : static_cast<const VT*>(g->valP);
        const int ldP = g->ldP, ld64 = g->ld64;
        XT *v0, *v1, *v2;
        const XT* r;
        int ldr;
        if constexpr (F64) {
            v0 = g->dt0; v1 = g->dt1; v2 = g->dt2;
            r = g->r;
            ldr = ld64;
        } else {
            v0 = g->t0; v1 = g->t1; v2 = g->t2;
            r = g->r32;
            ldr = ldP;
        }
        auto tb = [&](int i) -> XT* { return i == 0 ? v0 : (i == 1 ? v1 : v2); };
        StepCoef<XT> c;
        if constexpr (F64) {
            c.ca = bc.e0d; c.cb = bc.cbd; c.cc = bc.ccd; c.cd = bc.exd;
        } else {
            c.ca = bc.e0; c.cb = bc.cb; c.cc = bc.cc; c.cd = bc.ex;
        }
        c.terms = bc.terms;
        const XT* u = (j == 1) ? r : tb((j - 1) % 3);
        const int ldu = (j == 1) ? ldr : ldP;
        const XT* w = (j >= 3) ? tb((j - 2) % 3) : nullptr;
        const int f1 = min(tl.f0 + kSellTileRows, g->n);
        const bool unit = F64 && bc.xu;
        double dv[M];
#pragma unroll
        for (int q = 0; q < M; ++q) dv[q] = 0.0;
        if constexpr (PART == 1) {
            if (unit)
                group_rows<VT, XT, double, 1, F64, M>(g, tl.f0, f1, val, u, ldu, w, ldP, r, ldr, g->z, ld64, g->r, c,
                                                      mask, dv);
            else
                group_rows<VT, XT, double, 1, false, M>(g, tl.f0, f1, val, u, ldu, w, ldP, r, ldr, g->z, ld64, g->r,
                                                        c, mask, dv);
            group_reduce<M>(dv, part, t, g, S, ctl, mask, BF_RZ);
        } else {
            XT* y = tb(j % 3);
            if (unit)
                group_rows<VT, XT, XT, 0, F64, M>(g, tl.f0, f1, val, u, ldu, w, ldP, r, ldr, y, ldP, nullptr, c, mask,
                                                  dv);
            else
                group_rows<VT, XT, XT, 0, false, M>(g, tl.f0, f1, val, u, ldu, w, ldP, r, ldr, y, ldP, nullptr, c,
                                                    mask, dv);
        }
    }
}

template <int M>
__global__ void __launch_bounds__(256, 3) bk_group_true(const BGDesc* __restrict__ G, BState* S,
                                                        const BTile* __restrict__ T, BCtl* ctl, double* part) {
    const int t0 = ctl->gseg[M == 2 ? 0 : 1], t1 = ctl->gseg[M == 2 ? 1 : 2];
    for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
        const BTile tl = T[t];
        const BGDesc* g = G + tl.pair;
        const unsigned mask = group_mask<M>(g, S, PH_FINISH, PH_FINISH);
        if (mask == 0u) continue;
        StepCoef<double> c;   // q = b - (A' x + shift x), ||q||^2
        c.ca = -g->shift; c.cb = 0.0; c.cc = 1.0; c.cd = -1.0;
        c.terms = (c.ca != 0.0 ? kTermU : 0) | kTermR;
        const int ld = g->ld64;
        double dv[M];
#pragma unroll
        for (int q = 0; q < M; ++q) dv[q] = 0.0;
        group_rows<double, double, double, 3, false, M>(g, tl.f0, min(tl.f0 + kSellTileRows, g->n), g->val64, g->x,
                                                        ld, nullptr, 0, g->b, ld, g->q, ld, nullptr, c, mask, dv);
        group_reduce<M>(dv, part, t, g, S, ctl, mask, BF_TRUE);
    }
}

}  // namespace

void launch_sell_opq(const SellLaunch& L, cudaStream_t st) {
    if (L.graph_sell & 3)
        bk_sell_opq<<<resident_grid(bk_sell_opq, 256), 256, 0, st>>>(L.desc, L.state, L.stiles, L.ctl, L.partials);
    if (L.graph_sell & 12) {
#define NB_GROUP_OPQ(M) \
    if (L.gwidths & (M)) \
        bk_group_opq<M><<<resident_grid(bk_group_opq<M>, 256, 4), 256, 0, st>>>(L.gdesc, L.state, L.gtiles, L.ctl, \
                                                                             L.gpartials)
        NB_GROUP_OPQ(2);
        NB_GROUP_OPQ(4);
#undef NB_GROUP_OPQ
    }
}

void launch_sell_cheb(const SellLaunch& L, int j, cudaStream_t st) {
    if (L.graph_sell & 3) {
#define NB_SELL_CHEB(VT, P)                                                                                   \
    bk_sell_cheb<VT, P><<<resident_grid(bk_sell_cheb<VT, P>, 256), 256, 0, st>>>(L.desc, L.state, L.stiles, L.coef, \
                                                                                L.ctl, L.partials, j, L.sntile_step)
        if (L.f64) {
            NB_SELL_CHEB(double, 0);
        } else {
            if (L.graph_sell & 1) {
                NB_SELL_CHEB(float, 1);
                NB_SELL_CHEB(float, 2);
            }
            if (L.graph_sell & 2) {
                NB_SELL_CHEB(__nv_bfloat16, 1);
                NB_SELL_CHEB(__nv_bfloat16, 2);
            }
        }
#undef NB_SELL_CHEB
    }
    if (L.graph_sell & 12) {
        // one launch per (value type, part, width) present
#define NB_GROUP_CHEB1(VT, P, M, SEG)                                                                         \
    if (L.gwidths & (M))                                                                                      \
    bk_group_cheb<VT, P, M><<<resident_grid(bk_group_cheb<VT, P, M>, 256, 4), 256, 0, st>>>(                     \
        L.gdesc, L.state, L.gtiles, L.coef, L.ctl, L.gpartials, j, L.gntile_step + (SEG) * (L.kmax + 1))
#define NB_GROUP_CHEB(VT, P) NB_GROUP_CHEB1(VT, P, 2, 0); NB_GROUP_CHEB1(VT, P, 4, 1)
        if (L.f64) {
            NB_GROUP_CHEB(double, 1);
            NB_GROUP_CHEB(double, 2);
        } else {
            if (L.graph_sell & 4) {
                NB_GROUP_CHEB(float, 1);
                NB_GROUP_CHEB(float, 2);
            }
            if (L.graph_sell & 8) {
                NB_GROUP_CHEB(__nv_bfloat16, 1);
                NB_GROUP_CHEB(__nv_bfloat16, 2);
            }
        }
#undef NB_GROUP_CHEB
#undef NB_GROUP_CHEB1
    }
}

void launch_sell_true(const SellLaunch& L, cudaStream_t st) {
    if (L.graph_sell & 3)
        bk_sell_true<<<resident_grid(bk_sell_true, 256), 256, 0, st>>>(L.desc, L.state, L.stiles, L.ctl, L.partials);
    if (L.graph_sell & 12) {
#define NB_GROUP_TRUE(M) \
    if (L.gwidths & (M)) \
        bk_group_true<M><<<resident_grid(bk_group_true<M>, 256, 4), 256, 0, st>>>(L.gdesc, L.state, L.gtiles, L.ctl, \
                                                                               L.gpartials)
        NB_GROUP_TRUE(2);
        NB_GROUP_TRUE(4);
#undef NB_GROUP_TRUE
    }
}

}  // namespace batch
}  // namespace nc
