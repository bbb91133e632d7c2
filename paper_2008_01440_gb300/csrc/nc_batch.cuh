// Batched engine: the tables the host side (nc_batch.cu) writes and the
// kernels read -- slot descriptors and states, coefficients, tiles, vector
// chunks, the control block, group descriptors -- the per-slot reduction
// shared by all its kernels, and the launchers of the explicit-matrix
// kernels (nc_batch_sell.cu).
#pragma once

#include <type_traits>

#include "nc_internal.h"
#include "nc_stencil.cuh"

namespace nc {
namespace batch {

constexpr int kVch = 8192;    // vector-chunk length
constexpr int kZC = 32;       // planes per stencil tile (32 measured 4.5% faster than 16 or 64 on the 256-system batch)
// rows per tile of an explicit-matrix slot or group: 8 blocks of 256 rows
// (one row per thread), so that a step over a few systems still has a tile
// for every CTA, while the per-tile reduction (fence + atomic) stays rare
constexpr int kSellTileRows = 8 * kFT;

enum Phase : int { PH_FREE = 0, PH_INIT = 1, PH_RUN = 2, PH_FINISH = 3, PH_DONE = 4 };

enum BFin : int { BF_ALPHA = 1, BF_RR = 2, BF_INIT = 3, BF_RZ = 4, BF_START = 5, BF_TRUE = 6 };

enum SlotKind : int { SLOT_STENCIL = 0, SLOT_SELL = 1 };

struct BDesc {
    int nx, ny, nz, n;
    int k, coef0;
    int tile0, tile1, vch0, vch1;
    double c0, cx, cy, cz;
    double *b, *x, *r, *z, *p, *q;
    float *t0, *t1, *t2, *r32;      // float32 apply (NC_BATCH_F64_APPLY unset)
    double *dt0, *dt1, *dt2;        // float64 apply: the Chebyshev vectors, r read directly
    // SLOT_SELL: an explicit matrix in a solver's SELL-32 layout (borrowed):
    // slice offsets, columns (plain) or offset patterns, the float64 values of
    // the stored operator S (A - theta' I, its constant diagonal possibly left
    // out) and the values inside P (apply precision vdtP); A u = S u + shift u
    int kind, vdtP;
    double shift;
    const int32_t *sptr, *scol;
    SellPat pat;
    const double* val64;
    const void* valP;
    const double* disv;             // d^{-1/2} per unknown (null: the slot's scalar)
};

struct BState {
    double rz, pq, alpha, beta, rr, bb, rr_true;
    int iter, phase, status, n_dot, n_prec;
    unsigned int counter;
};

struct BCoef {
    float e0, ex, ey, ez, cb, cc;
    int terms;
    int xu;                                // float64 fields: exd == -1 exactly (no centre multiply)
    double e0d, exd, eyd, ezd, cbd, ccd;   // float64 apply: the step for the scaled iterates
    // SLOT_SELL: y = ca u + cb w + cc r + cd A' u (nc_step.cuh's StepCoef),
    // float for the float32 apply, double for the float64 one; xu: cd == 1
};

struct BTile {
    int pair, f0, pad, bz;   // f0: first point of the tile in the flattened xy-plane
};

struct BVch {
    int pair, start;
};

struct BCtl {
    double tol2;
    int maxit, ntiles, nvch, active;
    int iters_this_call, iter_limit, nstiles, gpstride;   // tiles of explicit-matrix slots; a group
                                                          // column's partials: [c * gpstride + tile]
    int gseg[3];   // the group tile list's segments of widths 2 and 4: [gseg[i], gseg[i + 1])
    int pad2;
};

// A group: up to kGroupWidth slots (columns) of one solver that share every
// read of its matrix -- each step loads a row's columns and values once and
// applies them to all the group's columns (a sparse times dense-block
// product), as one solver's multi-right-hand-side block does.  Each column is
// a slot of its own (state, result, collect, release); the group only owns
// the tile list entry.  The columns' vectors lie in one pool range, column
// c's at column 0's plus c * ld64 (float64 pool) or c * ldP (apply pool).
constexpr int kMaxGroup = 8;     // right-hand sides one pcg_batch_add_solver_multi call takes
// columns of one group: a call with more forms several groups (two groups of
// 4 measured faster than one of 8 on the c4csr batch, 0.86 against 0.91 s:
// the 8-wide kernel holds too few rows in flight at its register count)
constexpr int kGroupWidth = 4;

struct BGDesc {
    int M, n, k, coef0;          // M: the kernel width (2, 4 or 8 >= columns)
    int tile0, tile1, live, vdtP;   // live: bit c set while column c is owned
    int slot[kGroupWidth];       // the engine slot of column c
    double shift;
    const int32_t *sptr, *scol;
    SellPat pat;
    const double* val64;
    const void* valP;
    double *b, *x, *r, *z, *p, *q;   // column 0
    float *t0, *t1, *t2, *r32;
    double *dt0, *dt1, *dt2;
    int ld64, ldP;
};

// What the explicit-matrix kernels of one engine iteration need: the device
// tables and which kernels the captured iteration holds.
struct SellLaunch {
    const BDesc* desc;
    BState* state;
    const BTile* stiles;         // tiles of single explicit slots
    const BGDesc* gdesc;         // groups
    const BTile* gtiles;
    const BCoef* coef;
    BCtl* ctl;
    double* partials;
    double* gpartials;
    const int* sntile_step;      // single slots' tiles with k >= j
    const int* gntile_step;      // per group segment, kmax + 1 each
    int kmax;
    int graph_sell;              // bit 0 float32 / float64 values, bit 1 bfloat16; bits 2, 3 the same for groups
    int gwidths;                 // group widths present (bits 2 and 4)
    bool f64;                    // the float64 apply
};

// Launchers (nc_batch_sell.cu), each a no-op when its kernels are absent:
// q = A p with (p, q); Chebyshev step j; the true residual of stopped slots.
void launch_sell_opq(const SellLaunch& L, cudaStream_t st);
void launch_sell_cheb(const SellLaunch& L, int j, cudaStream_t st);
void launch_sell_true(const SellLaunch& L, cudaStream_t st);

// Grid of a kernel over a work list: `waves` times as many CTAs as the
// device holds at once (per SM capped at kCtasPerSm).  One wave keeps every
// CTA resident with statically assigned tiles; several let CTAs that finish
// early be replaced (the group kernels: 4 waves, c4csr 1359 -> 1407 solves/s).
template <typename K>
inline int resident_grid(K kernel, int threads, int waves = 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (per_sm > kCtasPerSm) per_sm = kCtasPerSm;
    return waves * per_sm * num_sms();
}

namespace {   // device helpers: one copy per translation unit

__device__ void bfinalize(BState* st, BCtl* ctl, int kind, double s) {
    const bool finite = isfinite(s);
    switch (kind) {
    case BF_ALPHA:
        st->n_dot += 1;
        st->pq = s;
        if (!(s > 0.0) || !finite) {
            st->status = finite ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN;
            st->phase = PH_FINISH;
        } else {
            st->alpha = st->rz / s;
        }
        break;
    case BF_RR:
        st->n_dot += 1;
        st->rr = s;
        st->iter += 1;
        if (!finite) { st->status = NC_ERR_BREAKDOWN; st->phase = PH_FINISH; }
        else if (s <= ctl->tol2 * st->bb) { st->status = NC_OK; st->phase = PH_FINISH; }
        else if (st->iter >= ctl->maxit) { st->status = NC_ERR_MAXIT; st->phase = PH_FINISH; }
        break;
    case BF_INIT:   // r = b: ||r0||^2 = ||b||^2
        st->bb = s;
        st->rr = s;
        if (!finite) { st->status = NC_ERR_BREAKDOWN; st->phase = PH_FINISH; }
        else if (s == 0.0) { st->status = NC_OK; st->phase = PH_FINISH; }
        else if (ctl->maxit <= 0) { st->status = NC_ERR_MAXIT; st->phase = PH_FINISH; }
        break;
    case BF_RZ:
        st->n_dot += 1;
        st->n_prec += 1;
        if (!(s > 0.0) || !finite) {
            st->status = finite ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN;
            st->phase = PH_FINISH;
        } else if (st->phase == PH_INIT) {
            st->rz = s;
        } else {
            st->beta = s / st->rz;
            st->rz = s;
        }
        break;
    case BF_START:
        if (st->phase == PH_INIT) st->phase = PH_RUN;
        break;
    case BF_TRUE:
        st->rr_true = s;
        st->phase = PH_DONE;
        atomicSub(&ctl->active, 1);
        break;
    default:
        break;
    }
}

// Per-slot reduction: this CTA's partial goes to partials[slotidx]; the CTA
// completing the slot's count-th partial sums partials[first, first+count)
// in order and finalizes.  All threads of the CTA call it (uniform).
__device__ void reduce_slot(double v, double* partials, int slotidx, int first, int count, BState* st, BCtl* ctl,
                            int kind) {
    __shared__ double sh[256];
    __shared__ int is_last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    v = block_sum<256>(v, sh, tid);
    if (tid == 0) {
        partials[slotidx] = v;
        __threadfence();
        const unsigned int t = atomicAdd(&st->counter, 1u);
        is_last = (t == (unsigned int)count - 1u);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s = 0.0;
        for (int i = tid; i < count; i += 256) s += __ldcg(&partials[first + i]);
        s = block_sum<256>(s, sh, tid);
        if (tid == 0) {
            bfinalize(st, ctl, kind, s);
            st->counter = 0u;
        }
    }
    __syncthreads();
}

}  // namespace
}  // namespace batch
}  // namespace nc
