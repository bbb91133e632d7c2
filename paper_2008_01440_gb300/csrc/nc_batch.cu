// Batched / continuous-batching PCG engine for many independent matrix-free
// 7-point systems of uneven size, each with its own degree k, bounds and
// right-hand side (one "slot" per (system, right-hand side) pair).
//
// All slots advance together: one PCG iteration for every slot is a fixed
// sequence of persistent grid-stride kernels over two work lists held in
// device memory -- stencil tiles (kFT consecutive points of one slot's
// flattened xy-plane x ZC planes) and vector chunks (kVch entries of one
// slot):
//   opq      q = A p and (p, q) -> alpha              (float64, tiles)
//   axpy     x += alpha p, r -= alpha q, ||r||^2, stop? (float64, chunks);
//            slots being admitted instead start r = b, x = 0, ||b||^2
//   cheb(j)  Chebyshev step j = 1..kmax, float32 vectors, float64 z at
//            j = k_slot with (r, z) -> beta (or the initial (r, z))  (tiles)
//   pupd     p = z + beta p (or p = z for admitted slots)   (chunks)
//   true     r_true = b - A x, ||r_true||^2 for slots that just stopped
//   cond     loop condition: slots left and iterations this call < limit
// Every slot reduces its own dot products: each tile / chunk writes a
// partial sum; the CTA that completes a slot's last partial sums that slot's
// partials in order (deterministic, independent of the other slots, so a
// slot's result is the same alone and in any mix) and updates its scalars.
//
// The sequence is captured once as the body of a conditional WHILE node; the
// work lists, slot descriptors and coefficients live in device tables that
// the host rewrites between launches (admission, retirement) without
// re-capturing.  A launch runs up to `iter_limit` iterations: the whole
// batch in one launch, or a few iterations per serving tick.
//
// Memory: every slot owns 6 float64 and 4 float32 vectors of its length in
// two pools allocated once (first-fit free list on the host); a slot is
// refused when the pools have no room (the HBM budget).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <type_traits>
#include <vector>

#include "nc_batch.cuh"


namespace nc {
using namespace batch;
namespace {

__global__ void __launch_bounds__(256) bk_opq(const BDesc* __restrict__ D, BState* S, const BTile* __restrict__ T,
                                              BCtl* ctl, double* partials) {
    const int tid = threadIdx.x + kTX * threadIdx.y;   // launched as kTX x kTY
    const int nt = ctl->ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        if (st->phase != PH_RUN) continue;
        const BDesc& d = D[tl.pair];
        StencilCoef<double> c;
        c.e0 = d.c0;
        c.ex = -d.cx;
        c.ey = -d.cy;
        c.ez = -d.cz;
        c.cb = 0.0;
        c.cc = 0.0;
        c.terms = 0;
        const int k0 = tl.bz * kZC, k1 = min(k0 + kZC, d.nz);
        // (the admitted operator is Jacobi scaled: c0 == 1, the centre takes no multiply)
        const double dv = stencil_flat<double, double, 2, false, true>(d.nx, d.ny, d.nz, tl.f0, k0, k1, d.p, nullptr,
                                                                       nullptr, d.q, c, nullptr, tid);
        reduce_slot(dv, partials, t, d.tile0, d.tile1 - d.tile0, st, ctl, BF_ALPHA);
    }
}

__global__ void __launch_bounds__(256) bk_axpy(const BDesc* __restrict__ D, BState* S, const BVch* __restrict__ V,
                                               BCtl* ctl, double* partials) {
    const int nv = ctl->nvch;
    for (int c = blockIdx.x; c < nv; c += gridDim.x) {
        const BVch ch = V[c];
        BState* st = S + ch.pair;
        const int ph = st->phase;
        if (ph != PH_RUN && ph != PH_INIT) continue;
        const BDesc& d = D[ch.pair];
        const int e = min(ch.start + kVch, d.n);
        double acc = 0.0;
        if (ph == PH_RUN) {
            const double a = st->alpha;
            for (int i = ch.start + threadIdx.x; i < e; i += 256) {
                d.x[i] = fma(a, d.p[i], d.x[i]);
                const double ri = fma(-a, d.q[i], d.r[i]);
                d.r[i] = ri;
                if (d.r32) d.r32[i] = (float)ri;
                acc = fma(ri, ri, acc);
            }
        } else {
            for (int i = ch.start + threadIdx.x; i < e; i += 256) {
                const double bi = d.b[i];
                d.x[i] = 0.0;
                d.r[i] = bi;
                if (d.r32) d.r32[i] = (float)bi;
                acc = fma(bi, bi, acc);
            }
        }
        reduce_slot(acc, partials, c, d.vch0, d.vch1 - d.vch0, st, ctl, ph == PH_RUN ? BF_RR : BF_INIT);
    }
}

// F64: the float64 apply (NC_BATCH_F64_APPLY), a separate instantiation so
// that the float32 kernel keeps its register count
template <bool F64>
__global__ void __launch_bounds__(256) bk_cheb(const BDesc* __restrict__ D, BState* S, const BTile* __restrict__ T,
                                               const BCoef* __restrict__ C, BCtl* ctl, double* partials, int j,
                                               const int* __restrict__ ntile_step) {
    const int tid = threadIdx.x + kTX * threadIdx.y;   // launched as kTX x kTY
    // tiles are ordered by their slot's degree, highest first: step j only
    // visits the prefix of tiles whose slots have k >= j
    const int nt = ntile_step[j];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        const int ph = st->phase;
        if (ph != PH_RUN && ph != PH_INIT) continue;
        const BDesc& d = D[tl.pair];
        if (j > d.k) continue;
        const BCoef bc = C[d.coef0 + j - 1];
        const int k0 = tl.bz * kZC, k1 = min(k0 + kZC, d.nz);
        if constexpr (F64) {
            // float64 apply
            StencilCoef<double> c;
            c.e0 = bc.e0d;
            c.ex = bc.exd;
            c.ey = bc.eyd;
            c.ez = bc.ezd;
            c.cb = bc.cbd;
            c.cc = bc.ccd;
            c.terms = bc.terms;
            // the rotating vectors by index, selected (an indexed array would sit in local memory)
            auto tb = [&](int i) -> double* { return i == 0 ? d.dt0 : (i == 1 ? d.dt1 : d.dt2); };
            const double* u = (j == 1) ? d.r : tb((j - 1) % 3);
            const double* w = (j >= 3) ? tb((j - 2) % 3) : nullptr;
            if (j == d.k) {
                const double dv =
                    bc.xu ? stencil_flat<double, double, 1, true>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r, d.z, c,
                                                                  d.r, tid)
                          : stencil_flat<double, double, 1>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r, d.z, c, d.r,
                                                            tid);
                reduce_slot(dv, partials, t, d.tile0, d.tile1 - d.tile0, st, ctl, BF_RZ);
            } else if (bc.xu) {
                stencil_flat<double, double, 0, true>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r, tb(j % 3), c,
                                                      nullptr, tid);
            } else {
                stencil_flat<double, double, 0>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r, tb(j % 3), c, nullptr,
                                                tid);
            }
        } else {
        StencilCoef<float> c;
        c.e0 = bc.e0;
        c.ex = bc.ex;
        c.ey = bc.ey;
        c.ez = bc.ez;
        c.cb = bc.cb;
        c.cc = bc.cc;
        c.terms = bc.terms;
        auto tb = [&](int i) -> float* { return i == 0 ? d.t0 : (i == 1 ? d.t1 : d.t2); };
        const float* u = (j == 1) ? d.r32 : tb((j - 1) % 3);
        const float* w = (j >= 3) ? tb((j - 2) % 3) : nullptr;
        if (j == d.k) {
            const double dv = stencil_flat<float, double, 1>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r32, d.z, c,
                                                             d.r, tid);
            reduce_slot(dv, partials, t, d.tile0, d.tile1 - d.tile0, st, ctl, BF_RZ);
        } else {
            stencil_flat<float, float, 0>(d.nx, d.ny, d.nz, tl.f0, k0, k1, u, w, d.r32, tb(j % 3), c, nullptr, tid);
        }
        }
    }
}

__global__ void __launch_bounds__(256) bk_pupd(const BDesc* __restrict__ D, BState* S, const BVch* __restrict__ V,
                                               BCtl* ctl, double* partials) {
    const int nv = ctl->nvch;
    for (int c = blockIdx.x; c < nv; c += gridDim.x) {
        const BVch ch = V[c];
        BState* st = S + ch.pair;
        const int ph = st->phase;
        if (ph != PH_RUN && ph != PH_INIT) continue;
        const BDesc& d = D[ch.pair];
        const int e = min(ch.start + kVch, d.n);
        if (ph == PH_RUN) {
            const double beta = st->beta;
            for (int i = ch.start + threadIdx.x; i < e; i += 256) d.p[i] = fma(beta, d.p[i], d.z[i]);
        } else {
            for (int i = ch.start + threadIdx.x; i < e; i += 256) d.p[i] = d.z[i];
            // the last chunk of an admitted slot moves it to the running phase
            reduce_slot(0.0, partials, c, d.vch0, d.vch1 - d.vch0, st, ctl, BF_START);
        }
    }
}

__global__ void __launch_bounds__(256) bk_true(const BDesc* __restrict__ D, BState* S, const BTile* __restrict__ T,
                                               BCtl* ctl, double* partials) {
    const int tid = threadIdx.x + kTX * threadIdx.y;   // launched as kTX x kTY
    const int nt = ctl->ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BTile tl = T[t];
        BState* st = S + tl.pair;
        if (st->phase != PH_FINISH) continue;
        const BDesc& d = D[tl.pair];
        StencilCoef<double> c;   // q = b - A x
        c.e0 = -d.c0;
        c.ex = d.cx;
        c.ey = d.cy;
        c.ez = d.cz;
        c.cb = 0.0;
        c.cc = 1.0;
        c.terms = kTermR;
        const int k0 = tl.bz * kZC, k1 = min(k0 + kZC, d.nz);
        const double dv = stencil_flat<double, double, 3>(d.nx, d.ny, d.nz, tl.f0, k0, k1, d.x, nullptr, d.b, d.q,
                                                          c, nullptr, tid);
        reduce_slot(dv, partials, t, d.tile0, d.tile1 - d.tile0, st, ctl, BF_TRUE);
    }
}

__global__ void bk_cond(BCtl* ctl, cudaGraphConditionalHandle h, int use_cond) {
    ctl->iters_this_call += 1;
    const int go = ctl->active > 0 && ctl->iters_this_call < ctl->iter_limit;
    if (use_cond) cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void bk_scale(int n, const double* __restrict__ in, double s, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[i] * s;
}

// out = s * d .* in (a Jacobi-scaled explicit matrix: d = d^{-1/2}; s = 0 for b = 0)
__global__ void bk_scale_vec(int n, const double* __restrict__ in, const double* __restrict__ d, double s,
                             double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = s * d[i] * in[i];
}

}  // namespace
}  // namespace nc

using namespace nc;

struct nc_batch_s {
    int flags = 0;
    int cap_slots = 0;
    int64_t cap_units = 0;        // unknowns the pools hold
    int kmax = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    // device
    BDesc* d_desc = nullptr;
    BState* d_state = nullptr;
    BCtl* d_ctl = nullptr;
    BTile* d_tiles = nullptr;
    BVch* d_vch = nullptr;
    BCoef* d_coef = nullptr;
    int* d_ntile_step = nullptr;  // tiles of slots with k >= j, j = 0..kmax
    BTile* d_stiles = nullptr;    // tiles of explicit-matrix slots
    int* d_sntile_step = nullptr; // and their counts with k >= j
    int cap_stiles = 0;
    BGDesc* d_gdesc = nullptr;    // groups
    BTile* d_gtiles = nullptr;    // tiles of groups
    int* d_gntile_step = nullptr; // and their counts with k >= j
    double* d_gpartials = nullptr;   // kGroupWidth rows of cap_gtiles
    int cap_gdesc = 0, cap_gtiles = 0;
    int gwidths = 0;              // group widths the captured iteration launches (bits 2 and 4)
    int graph_sell = 0;           // explicit-slot kernels the captured iteration launches:
                                  // bit 0 float32 / float64 values, bit 1 bfloat16 values;
                                  // bits 2 and 3 the same for groups
    double* d_partials = nullptr;
    double* pool64 = nullptr;
    float* pool32 = nullptr;
    int cap_tiles = 0, cap_vch = 0, cap_coef = 0;
    // host
    std::vector<BDesc> desc;
    std::vector<int> used;        // slot in use
    std::vector<int> kdeg;
    std::vector<double> dis;      // d^{-1/2} constant per slot
    std::vector<std::vector<BCoef>> coefs;
    std::vector<int64_t> off;     // pool offset (unknowns) per slot
    std::vector<int> gid;         // group of a slot (-1: none)
    std::vector<BGDesc> groups;   // host copies; live == 0: free
    std::vector<std::vector<BCoef>> gcoefs;
    std::map<int64_t, int64_t> free_list;   // offset -> length
    bool dirty = true;
    BState* h_state = nullptr;    // pinned
    std::vector<int> state_upload;   // slots whose host state goes to the device at the next run
    BCtl* h_ctl = nullptr;        // pinned
    int64_t stat_iters = 0;       // engine iterations run since creation
    int64_t stat_launches = 0;    // kernels launched since creation
};

namespace {

thread_local cudaError_t g_batch_err = cudaSuccess;

#define NB_CU(call)                                 \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) {                    \
            g_batch_err = e_;                       \
            return NC_ERR_CUDA;                     \
        }                                           \
    } while (0)

nc_status balloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return NC_ERR_OOM;
    }
    if (e != cudaSuccess) {
        g_batch_err = e;
        *p = nullptr;
        return NC_ERR_CUDA;
    }
    return NC_OK;
}

int64_t pool_alloc(nc_batch B, int64_t len) {   // first fit; -1 if none
    for (auto it = B->free_list.begin(); it != B->free_list.end(); ++it) {
        if (it->second >= len) {
            const int64_t o = it->first, rest = it->second - len;
            B->free_list.erase(it);
            if (rest > 0) B->free_list[o + len] = rest;
            return o;
        }
    }
    return -1;
}

void pool_free(nc_batch B, int64_t o, int64_t len) {
    auto it = B->free_list.emplace(o, len).first;
    auto nx = std::next(it);
    if (nx != B->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        B->free_list.erase(nx);
    }
    if (it != B->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            B->free_list.erase(it);
        }
    }
}

nc_status grow(void** p, int* cap, int need, size_t elem) {
    if (need <= *cap) return NC_OK;
    int nc_ = std::max(need, *cap * 2);
    if (nc_ < 64) nc_ = 64;
    if (*p) cudaFree(*p);
    *p = nullptr;
    nc_status s = balloc(p, elem * (size_t)nc_);
    if (s != NC_OK) {
        *cap = 0;
        return s;
    }
    *cap = nc_;
    return NC_OK;
}

// One PCG iteration of every slot (the graph body).
void enqueue_iteration(nc_batch B, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    const dim3 tb(kTX, kTY);
    // CTAs over the work lists of the stencil and vector kernels: four times
    // as many as the device holds at 8 per SM, so that each walks a few tiles
    // and the CTAs that finish early are replaced instead of waiting for the
    // slowest's statically assigned tiles (C4 batch: 1x 2502, 2x 2647, 4x 2718,
    // 8x 2704, 16x 2650 solves/s)
    const int grid = 4 * vec_grid_max();
    SellLaunch L;
    L.desc = B->d_desc;
    L.state = B->d_state;
    L.stiles = B->d_stiles;
    L.gdesc = B->d_gdesc;
    L.gtiles = B->d_gtiles;
    L.coef = B->d_coef;
    L.ctl = B->d_ctl;
    L.partials = B->d_partials;
    L.gpartials = B->d_gpartials;
    L.sntile_step = B->d_sntile_step;
    L.gntile_step = B->d_gntile_step;
    L.kmax = B->kmax;
    L.graph_sell = B->graph_sell;
    L.gwidths = B->gwidths;
    L.f64 = (B->flags & NC_BATCH_F64_APPLY) != 0;
    bk_opq<<<grid, tb, 0, st>>>(B->d_desc, B->d_state, B->d_tiles, B->d_ctl, B->d_partials);
    launch_sell_opq(L, st);
    bk_axpy<<<grid, 256, 0, st>>>(B->d_desc, B->d_state, B->d_vch, B->d_ctl, B->d_partials);
    for (int j = 1; j <= B->kmax; ++j) {
        if (L.f64)
            bk_cheb<true><<<grid, tb, 0, st>>>(B->d_desc, B->d_state, B->d_tiles, B->d_coef, B->d_ctl,
                                                     B->d_partials, j, B->d_ntile_step);
        else
            bk_cheb<false><<<grid, tb, 0, st>>>(B->d_desc, B->d_state, B->d_tiles, B->d_coef, B->d_ctl,
                                                      B->d_partials, j, B->d_ntile_step);
        launch_sell_cheb(L, j, st);
    }
    bk_pupd<<<grid, 256, 0, st>>>(B->d_desc, B->d_state, B->d_vch, B->d_ctl, B->d_partials);
    bk_true<<<grid, tb, 0, st>>>(B->d_desc, B->d_state, B->d_tiles, B->d_ctl, B->d_partials);
    launch_sell_true(L, st);
    bk_cond<<<1, 1, 0, st>>>(B->d_ctl, h, use_cond);
}

nc_status build_batch_graph(nc_batch B) {
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaGraphNode_t nw = nullptr;
    cudaGraphConditionalHandle h = 0;
    nc_status out = NC_ERR_CUDA;
    cudaError_t e;
    do {
        if ((e = cudaGraphCreate(&g, 0))) break;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&nw, g, nullptr, nullptr, 0, &cp))) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
            break;
        enqueue_iteration(B, h, 1, B->cap);
        cudaError_t e1 = cudaGetLastError();
        cudaGraph_t tmp = nullptr;
        e = cudaStreamEndCapture(B->cap, &tmp);
        if (e1) { e = e1; break; }
        if (e) break;
        if ((e = cudaGraphInstantiate(&B->exec, g, 0))) break;
        out = NC_OK;
    } while (0);
    if (out != NC_OK) {
        g_batch_err = e;
        cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
    return out;
}

// Rebuild the work lists and descriptors of all slots in use and upload them.
nc_status sync_tables(nc_batch B, cudaStream_t st) {
    std::vector<BTile> tiles, stiles;
    std::vector<BVch> vch;
    std::vector<BCoef> coef;
    std::vector<int> order;
    for (int s = 0; s < B->cap_slots; ++s)
        if (B->used[s]) order.push_back(s);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->kdeg[a] > B->kdeg[b]; });
    std::vector<int> nstep(B->kmax + 1, 0), snstep(B->kmax + 1, 0);
    for (int s : order) {
        BDesc& d = B->desc[s];
        if (d.kind == SLOT_SELL && B->gid[s] >= 0) {   // a group column: the group's tiles
            d.tile0 = d.tile1 = 0;
        } else if (d.kind == SLOT_SELL) {   // kSellTileRows-row tiles of the layout, in their own list
            d.tile0 = (int)stiles.size();
            for (int f0 = 0; f0 < d.n; f0 += kSellTileRows) stiles.push_back(BTile{s, f0, 0, 0});
            d.tile1 = (int)stiles.size();
            for (int j = 0; j <= std::min(d.k, B->kmax); ++j) snstep[j] = d.tile1;
        } else {
            d.tile0 = (int)tiles.size();
            const int nxy = d.nx * d.ny, tz = (d.nz + kZC - 1) / kZC;
            for (int bz = 0; bz < tz; ++bz)
                for (int f0 = 0; f0 < nxy; f0 += kFT) tiles.push_back(BTile{s, f0, 0, bz});
            d.tile1 = (int)tiles.size();
            for (int j = 0; j <= std::min(d.k, B->kmax); ++j) nstep[j] = d.tile1;   // prefix ends after this slot
        }
        d.vch0 = (int)vch.size();
        for (int i = 0; i < d.n; i += kVch) vch.push_back(BVch{s, i});
        d.vch1 = (int)vch.size();
        d.coef0 = (int)coef.size();
        coef.insert(coef.end(), B->coefs[s].begin(), B->coefs[s].end());
    }
    // groups: one segment of the list per width, each by degree as well
    std::vector<BTile> gtiles;
    std::vector<int> gorder, gnstep(2 * (B->kmax + 1), 0);
    for (int g = 0; g < (int)B->groups.size(); ++g)
        if (B->groups[g].live) gorder.push_back(g);
    std::stable_sort(gorder.begin(), gorder.end(), [&](int a, int b) {
        const BGDesc &x = B->groups[a], &y = B->groups[b];
        return x.M != y.M ? x.M < y.M : x.k > y.k;
    });
    int want_sell = 0, want_w = 0;
    int gseg[3] = {0, 0, 0};
    for (int g : gorder) {
        BGDesc& gd = B->groups[g];
        const int seg = gd.M == 2 ? 0 : 1;
        gd.tile0 = (int)gtiles.size();
        for (int f0 = 0; f0 < gd.n; f0 += kSellTileRows) gtiles.push_back(BTile{g, f0, 0, 0});
        gd.tile1 = (int)gtiles.size();
        for (int i = seg + 1; i < 3; ++i) gseg[i] = gd.tile1;   // later segments start at the end so far
        for (int j = 0; j <= std::min(gd.k, B->kmax); ++j) gnstep[seg * (B->kmax + 1) + j] = gd.tile1 - gseg[seg];
        gd.coef0 = (int)coef.size();
        coef.insert(coef.end(), B->gcoefs[g].begin(), B->gcoefs[g].end());
        want_sell |= gd.vdtP == NC_BF16 ? 8 : 4;
        want_w |= gd.M;
    }
    const int cap_t = B->cap_tiles, cap_v = B->cap_vch, cap_s = B->cap_stiles;
    const int cap_gd = B->cap_gdesc, cap_gt = B->cap_gtiles;
    nc_status s;
    if ((s = grow(reinterpret_cast<void**>(&B->d_tiles), &B->cap_tiles, (int)tiles.size(), sizeof(BTile)))) return s;
    if ((s = grow(reinterpret_cast<void**>(&B->d_stiles), &B->cap_stiles, (int)stiles.size(), sizeof(BTile))))
        return s;
    if ((s = grow(reinterpret_cast<void**>(&B->d_vch), &B->cap_vch, (int)vch.size(), sizeof(BVch)))) return s;
    int cap_c = B->cap_coef;
    if ((s = grow(reinterpret_cast<void**>(&B->d_coef), &B->cap_coef, (int)coef.size(), sizeof(BCoef)))) return s;
    if ((s = grow(reinterpret_cast<void**>(&B->d_gdesc), &B->cap_gdesc, (int)B->groups.size(), sizeof(BGDesc))))
        return s;
    if ((s = grow(reinterpret_cast<void**>(&B->d_gtiles), &B->cap_gtiles, (int)gtiles.size(), sizeof(BTile))))
        return s;
    for (const BTile& tl : stiles) want_sell |= B->desc[tl.pair].vdtP == NC_BF16 ? 2 : 1;
    const bool realloc_ = cap_t != B->cap_tiles || cap_v != B->cap_vch || cap_c != B->cap_coef ||
                          cap_s != B->cap_stiles || cap_gd != B->cap_gdesc || cap_gt != B->cap_gtiles ||
                          want_sell != B->graph_sell || want_w != B->gwidths;
    if (realloc_) {
        if (B->d_partials) cudaFree(B->d_partials);
        if (B->d_gpartials) cudaFree(B->d_gpartials);
        B->d_partials = nullptr;
        B->d_gpartials = nullptr;
        B->graph_sell = want_sell;
        B->gwidths = want_w;
        const int np = std::max(std::max(B->cap_tiles, B->cap_vch), B->cap_stiles);
        if ((s = balloc(reinterpret_cast<void**>(&B->d_partials), sizeof(double) * (size_t)np))) return s;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_gpartials),
                        sizeof(double) * kGroupWidth * (size_t)B->cap_gtiles)))
            return s;
        if ((s = build_batch_graph(B))) return s;
    }
    if (!tiles.empty())
        NB_CU(cudaMemcpyAsync(B->d_tiles, tiles.data(), sizeof(BTile) * tiles.size(), cudaMemcpyHostToDevice, st));
    if (!vch.empty())
        NB_CU(cudaMemcpyAsync(B->d_vch, vch.data(), sizeof(BVch) * vch.size(), cudaMemcpyHostToDevice, st));
    if (!coef.empty())
        NB_CU(cudaMemcpyAsync(B->d_coef, coef.data(), sizeof(BCoef) * coef.size(), cudaMemcpyHostToDevice, st));
    NB_CU(cudaMemcpyAsync(B->d_ntile_step, nstep.data(), sizeof(int) * nstep.size(), cudaMemcpyHostToDevice, st));
    if (!stiles.empty())
        NB_CU(cudaMemcpyAsync(B->d_stiles, stiles.data(), sizeof(BTile) * stiles.size(), cudaMemcpyHostToDevice, st));
    NB_CU(cudaMemcpyAsync(B->d_sntile_step, snstep.data(), sizeof(int) * snstep.size(), cudaMemcpyHostToDevice, st));
    if (!gtiles.empty())
        NB_CU(cudaMemcpyAsync(B->d_gtiles, gtiles.data(), sizeof(BTile) * gtiles.size(), cudaMemcpyHostToDevice, st));
    if (!B->groups.empty())
        NB_CU(cudaMemcpyAsync(B->d_gdesc, B->groups.data(), sizeof(BGDesc) * B->groups.size(),
                              cudaMemcpyHostToDevice, st));
    NB_CU(cudaMemcpyAsync(B->d_gntile_step, gnstep.data(), sizeof(int) * gnstep.size(), cudaMemcpyHostToDevice, st));
    // states of slots admitted or released since the last run (pinned source)
    for (int slot : B->state_upload)
        NB_CU(cudaMemcpyAsync(B->d_state + slot, &B->h_state[slot], sizeof(BState), cudaMemcpyHostToDevice, st));
    B->state_upload.clear();
    NB_CU(cudaMemcpyAsync(B->d_desc, B->desc.data(), sizeof(BDesc) * B->cap_slots, cudaMemcpyHostToDevice, st));
    B->h_ctl->ntiles = (int)tiles.size();
    B->h_ctl->nstiles = (int)stiles.size();
    for (int i = 0; i < 3; ++i) B->h_ctl->gseg[i] = gseg[i];
    B->h_ctl->gpstride = B->cap_gtiles;
    B->h_ctl->nvch = (int)vch.size();
    // the host vectors must outlive the copies
    NB_CU(cudaStreamSynchronize(st));
    B->dirty = false;
    return NC_OK;
}

}  // namespace

extern "C" {

const char* nc_batch_last_cuda_error(void) { return cudaGetErrorString(g_batch_err); }

nc_status pcg_batch_create(int max_slots, int64_t max_unknowns, int kmax, int flags, void* stream, nc_batch* out) {
    if (!out) return NC_ERR_ARG;
    *out = nullptr;
    if (max_slots < 1 || max_unknowns < 1 || kmax < 1 || kmax > 4096 ||
        (flags & ~(NC_BATCH_HOST_LOOP | NC_BATCH_F64_APPLY)))
        return NC_ERR_ARG;
    nc_batch B = new (std::nothrow) nc_batch_s();
    if (!B) return NC_ERR_OOM;
    B->flags = flags;
    B->cap_slots = max_slots;
    B->cap_units = max_unknowns;
    B->kmax = kmax;
    B->desc.assign(max_slots, BDesc{});
    B->used.assign(max_slots, 0);
    B->kdeg.assign(max_slots, 0);
    B->dis.assign(max_slots, 1.0);
    B->coefs.assign(max_slots, {});
    B->off.assign(max_slots, -1);
    B->gid.assign(max_slots, -1);
    B->free_list[0] = max_unknowns;
    nc_status s = NC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    do {
        if ((s = balloc(reinterpret_cast<void**>(&B->d_desc), sizeof(BDesc) * max_slots))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_state), sizeof(BState) * max_slots))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_ctl), sizeof(BCtl)))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_ntile_step), sizeof(int) * (kmax + 1)))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_sntile_step), sizeof(int) * (kmax + 1)))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->d_gntile_step), sizeof(int) * 2 * (kmax + 1)))) break;
        if ((s = balloc(reinterpret_cast<void**>(&B->pool64), sizeof(double) * 6 * (size_t)max_unknowns))) break;
        // apply vectors: 4 float32 per unknown (t0..t2, r32), or 3 float64 (+ slack
        // for the 16-byte rounding of the split below)
        if ((s = balloc(reinterpret_cast<void**>(&B->pool32),
                        (flags & NC_BATCH_F64_APPLY) ? sizeof(double) * 3 * (size_t)max_unknowns
                                                     : sizeof(float) * 4 * (size_t)max_unknowns)))
            break;
        cudaError_t e;
        if ((e = cudaMallocHost(&B->h_state, sizeof(BState) * max_slots)) ||
            (e = cudaMallocHost(&B->h_ctl, sizeof(BCtl))) ||
            (e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking)) ||
            (e = cudaMemsetAsync(B->d_state, 0, sizeof(BState) * max_slots, st)) ||
            (e = cudaMemsetAsync(B->d_ctl, 0, sizeof(BCtl), st)) || (e = cudaStreamSynchronize(st))) {
            g_batch_err = e;
            s = NC_ERR_CUDA;
            break;
        }
        std::memset(B->h_ctl, 0, sizeof(BCtl));
        if ((s = sync_tables(B, st))) break;   // allocates the tables and captures the graph
    } while (0);
    if (s != NC_OK) {
        pcg_batch_destroy(B);
        return s;
    }
    *out = B;
    return NC_OK;
}

nc_status pcg_batch_add(nc_batch B, int nx, int ny, int nz, double c0, double cx, double cy, double cz,
                        double lambda_min, double lambda_max, int degree_k, double theta_scale, const double* b_dev,
                        void* stream, int* slot) {
    if (!B || !slot || !b_dev) return NC_ERR_ARG;
    *slot = -1;
    if (nx < 1 || ny < 1 || nz < 1 || degree_k < 1 || degree_k > B->kmax || !(c0 > 0.0) ||
        !(lambda_min > 0.0) || !(lambda_max > lambda_min) || !(theta_scale > 0.0))
        return NC_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    if (n >= ((int64_t)1 << 31)) return NC_ERR_ARG;
    int s = -1;
    for (int i = 0; i < B->cap_slots; ++i)
        if (!B->used[i]) { s = i; break; }
    if (s < 0) return NC_ERR_ADMISSION;
    const int64_t o = pool_alloc(B, n);
    if (o < 0) return NC_ERR_ADMISSION;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // symmetric diagonal scaling of the constant stencil: c0 -> 1, c_a -> c_a/c0;
    // the bounds refer to the scaled operator
    const double dsc = 1.0 / std::sqrt(c0);
    BDesc d{};
    d.nx = nx; d.ny = ny; d.nz = nz; d.n = (int)n; d.k = degree_k;
    d.c0 = 1.0; d.cx = cx / c0; d.cy = cy / c0; d.cz = cz / c0;
    double* base64 = B->pool64 + 6 * o;
    d.b = base64; d.x = base64 + n; d.r = base64 + 2 * n; d.z = base64 + 3 * n; d.p = base64 + 4 * n;
    d.q = base64 + 5 * n;
    if (B->flags & NC_BATCH_F64_APPLY) {
        double* baseP = reinterpret_cast<double*>(B->pool32) + 3 * o;
        d.dt0 = baseP; d.dt1 = baseP + n; d.dt2 = baseP + 2 * n;
    } else {
        float* base32 = B->pool32 + 4 * o;
        d.t0 = base32; d.t1 = base32 + n; d.t2 = base32 + 2 * n; d.r32 = base32 + 3 * n;
    }
    // Chebyshev step coefficients (Eq. rhocheb, theta' = s theta) folded into
    // the stencil form: e0 = a_j + d_j c0, e_a = -d_j c_a
    const double theta = theta_scale * (lambda_max + lambda_min) / 2.0;
    const double delta = (lambda_max - lambda_min) / 2.0;
    const double sigma = theta / delta;
    std::vector<BCoef> cf(degree_k);
    double rho_prev = 1.0 / sigma;
    // float64 apply: iterates stored as y_j = x_j / g_j with g_j = d_j c_x g_{j-1},
    // which makes the x-coefficient exactly -1 (a kernel variant without the
    // centre multiply); g falls back to 1 outside [2^-64, 2^64], and the last
    // step stores z itself unless g_k > 0 (PCG does not change when z, and
    // with it p and q, are scaled by a positive constant: alpha and beta
    // compensate).  The float apply keeps the plain coefficients.
    std::vector<double> g(degree_k + 1, 1.0);
    for (int j = 1; j <= degree_k; ++j) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        double ca, cb, cc, cd;
        if (j == 1) {
            ca = 4.0 * rho / delta; cb = 0.0; cc = 0.0; cd = -2.0 * rho / (delta * theta);
        } else {
            ca = 2.0 * sigma * rho; cb = -rho * rho_prev; cc = 2.0 * rho / delta; cd = -2.0 * rho / delta;
            if (j == 2) { cc += cb / theta; cb = 0.0; }
        }
        BCoef c{};
        c.e0 = (float)(ca + cd * d.c0);
        c.ex = (float)(-cd * d.cx);
        c.ey = (float)(-cd * d.cy);
        c.ez = (float)(-cd * d.cz);
        c.cb = (float)cb;
        c.cc = (float)cc;
        c.terms = (cb != 0.0 ? kTermW : 0) | (cc != 0.0 ? kTermR : 0);
        const double gu = (j == 1) ? 1.0 : g[j - 1];   // scale of u (r at step 1)
        const double gw = (j >= 3) ? g[j - 2] : 1.0;   // scale of w = y_{j-2}
        const double t = cd * d.cx * gu;
        const bool unit = d.cx != 0.0 && (j < degree_k || t > 0.0) && std::fabs(t) >= 0x1p-64 &&
                          std::fabs(t) <= 0x1p64;
        g[j] = unit ? t : 1.0;
        c.xu = unit ? 1 : 0;
        c.e0d = (ca + cd * d.c0) * gu / g[j];
        c.exd = unit ? -1.0 : -cd * d.cx * gu;
        c.eyd = -cd * d.cy * gu / g[j];
        c.ezd = -cd * d.cz * gu / g[j];
        c.cbd = cb * gw / g[j];
        c.ccd = cc / g[j];
        cf[j - 1] = c;
        rho_prev = rho;
    }
    B->desc[s] = d;
    B->used[s] = 1;
    B->kdeg[s] = degree_k;
    B->dis[s] = dsc;
    B->coefs[s] = cf;
    B->off[s] = o;
    B->dirty = true;
    // b_s = D^{-1/2} b into the slot; state: admitted (prologue runs with the next iteration)
    bk_scale<<<std::min<int64_t>(4096, (n + 255) / 256), 256, 0, st>>>((int)n, b_dev, dsc, d.b);
    NB_CU(cudaGetLastError());
    BState init{};
    init.phase = PH_INIT;
    init.status = NC_ERR_MAXIT;
    B->h_state[s] = init;
    B->state_upload.push_back(s);   // uploaded (stream-ordered) by the next pcg_batch_run
    B->h_ctl->active += 1;
    B->stat_launches += 1;          // bk_scale
    *slot = s;
    return NC_OK;
}

nc_status pcg_batch_add_solver(nc_batch B, nc_solver S, const double* b_dev, void* stream, int* slot) {
    if (!slot) return NC_ERR_ARG;
    return pcg_batch_add_solver_multi(B, S, 1, b_dev, 0, stream, slot);
}

nc_status pcg_batch_add_solver_multi(nc_batch B, nc_solver S, int m, const double* B_dev, int64_t ldb,
                                     void* stream, int* slots) {
    if (!B || !S || !slots || !B_dev || m < 1 || m > kMaxGroup) return NC_ERR_ARG;
    for (int c = 0; c < m; ++c) slots[c] = -1;
    const bool f64 = (B->flags & NC_BATCH_F64_APPLY) != 0;
    // an explicit matrix in a sliced layout, the Chebyshev form, no residual
    // replacement, scalar (Jacobi) scaling only; the apply precision must be
    // the engine's
    if (S->op64.kind != OP_SELL || S->opP.kind != OP_SELL || S->nlev >= 0 || S->opt.rr_period > 0 ||
        S->A->wblk != nullptr || f64 == S->mixed)
        return NC_ERR_UNSUPPORTED;
    if (S->k < 1 || S->k > B->kmax || S->n < 1) return NC_ERR_ARG;
    const int64_t n = S->n;
    if (m > 1 && ldb < n) return NC_ERR_ARG;
    // the columns form groups of up to kGroupWidth (a last one of a single
    // column is a plain slot); the group kernels index column q by q times a
    // 32-bit stride (6 n at most), so larger systems are admitted as m
    // separate slots, which give the same results (bit for bit)
    const bool groupable = (int64_t)(kGroupWidth - 1) * 6 * n < ((int64_t)1 << 31);
    std::vector<int> ids;
    for (int i = 0; i < B->cap_slots && (int)ids.size() < m; ++i)
        if (!B->used[i]) ids.push_back(i);
    if ((int)ids.size() < m) return NC_ERR_ADMISSION;
    const int64_t o = pool_alloc(B, m * n);   // the columns side by side
    if (o < 0) return NC_ERR_ADMISSION;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the solver's own step coefficients, as its solves take them (the
    // float64 iterates scaled so that the product's coefficient is 1)
    // (a diagonal the layout leaves out enters through the u coefficient)
    const std::vector<StepC> sc = step_coefs(S, true);
    std::vector<BCoef> cf(S->k);
    for (int j = 1; j <= S->k; ++j) {
        BCoef c{};
        const double ca = sc[j].ca + sc[j].cd * S->opP.dfold;
        c.e0 = (float)ca;
        c.ex = (float)sc[j].cd;
        c.cb = (float)sc[j].cb;
        c.cc = (float)sc[j].cc;
        c.e0d = ca;
        c.exd = sc[j].cd;
        c.cbd = sc[j].cb;
        c.ccd = sc[j].cc;
        c.terms = (ca != 0.0 ? kTermU : 0) | (sc[j].cb != 0.0 ? kTermW : 0) | (sc[j].cc != 0.0 ? kTermR : 0) |
                  (sc[j].cd == 1.0 ? kUnitD : 0);
        c.xu = sc[j].cd == 1.0 ? 1 : 0;
        cf[j - 1] = c;
    }
    int g = -1, gc0 = 0, gw = 0;   // the current chunk's group, first column and width
    const int grid = (int)std::min<int64_t>(4096, (n + 255) / 256);
    for (int c = 0; c < m; ++c) {
        if (c % kGroupWidth == 0) {   // a new chunk of columns
            gc0 = c;
            gw = std::min(kGroupWidth, m - c);
            g = -1;
            if (groupable && gw > 1) {
                for (int i = 0; i < (int)B->groups.size(); ++i)
                    if (B->groups[i].live == 0) { g = i; break; }
                if (g < 0) {
                    g = (int)B->groups.size();
                    B->groups.push_back(BGDesc{});
                    B->gcoefs.emplace_back();
                }
            }
        }
        const int s = ids[c];
        const int64_t oc = o + c * n;
        BDesc d{};
        d.kind = SLOT_SELL;
        d.nx = (int)n; d.ny = 1; d.nz = 1; d.n = (int)n; d.k = S->k;
        d.sptr = S->op64.ptr;
        d.scol = S->op64.col;
        d.pat = S->op64.pat;
        d.val64 = static_cast<const double*>(S->op64.val);
        d.valP = S->opP.val;
        d.vdtP = S->opP.vdt;
        d.shift = S->shift + S->op64.dfold;   // the u term of q = A p and b - A x
        d.disv = S->A->scaled ? S->A->dis : nullptr;
        double* base64 = B->pool64 + 6 * oc;
        d.b = base64; d.x = base64 + n; d.r = base64 + 2 * n; d.z = base64 + 3 * n; d.p = base64 + 4 * n;
        d.q = base64 + 5 * n;
        if (f64) {
            double* baseP = reinterpret_cast<double*>(B->pool32) + 3 * oc;
            d.dt0 = baseP; d.dt1 = baseP + n; d.dt2 = baseP + 2 * n;
        } else {
            float* base32 = B->pool32 + 4 * oc;
            d.t0 = base32; d.t1 = base32 + n; d.t2 = base32 + 2 * n; d.r32 = base32 + 3 * n;
        }
        if (g >= 0 && c == gc0) {   // the group: its first column's vectors, the matrix, the strides
            BGDesc gd{};
            gd.M = gw <= 2 ? 2 : kGroupWidth;
            gd.n = (int)n;
            gd.k = S->k;
            gd.live = (1 << gw) - 1;
            gd.vdtP = d.vdtP;
            for (int q = 0; q < kGroupWidth; ++q) gd.slot[q] = ids[gc0 + (q < gw ? q : 0)];
            gd.shift = d.shift;
            gd.sptr = d.sptr; gd.scol = d.scol; gd.pat = d.pat; gd.val64 = d.val64; gd.valP = d.valP;
            gd.b = d.b; gd.x = d.x; gd.r = d.r; gd.z = d.z; gd.p = d.p; gd.q = d.q;
            gd.t0 = d.t0; gd.t1 = d.t1; gd.t2 = d.t2; gd.r32 = d.r32;
            gd.dt0 = d.dt0; gd.dt1 = d.dt1; gd.dt2 = d.dt2;
            gd.ld64 = (int)(6 * n);
            gd.ldP = (int)((f64 ? 3 : 4) * n);
            B->groups[g] = gd;
            B->gcoefs[g] = cf;
        }
        B->desc[s] = d;
        B->used[s] = 1;
        B->kdeg[s] = S->k;
        B->dis[s] = 1.0;   // the scaling is the vector d.disv
        B->gid[s] = g;
        if (g < 0) B->coefs[s] = cf;
        else B->coefs[s].clear();
        B->off[s] = oc;
        const double* bc = B_dev + (size_t)c * (size_t)ldb;
        if (d.disv != nullptr)
            bk_scale_vec<<<grid, 256, 0, st>>>((int)n, bc, d.disv, 1.0, d.b);
        else
            bk_scale<<<grid, 256, 0, st>>>((int)n, bc, 1.0, d.b);
        NB_CU(cudaGetLastError());
        BState init{};
        init.phase = PH_INIT;
        init.status = NC_ERR_MAXIT;
        B->h_state[s] = init;
        B->state_upload.push_back(s);
        B->h_ctl->active += 1;
        B->stat_launches += 1;
        slots[c] = s;
    }
    B->dirty = true;
    return NC_OK;
}

nc_status pcg_solve_batched(int nsys, const nc_solver* S, const int* nrhs, const double* const* B_dev,
                            double* const* X_dev, double tol, int maxit, void* stream, nc_result* res) {
    if (nsys < 1 || !S || !nrhs || !B_dev || !X_dev || !res || !(tol >= 0.0) || maxit < 0) return NC_ERR_ARG;
    int slots = 0, kmax = 1;
    int64_t units = 0;
    bool mixed = false;
    for (int i = 0; i < nsys; ++i) {
        if (!S[i] || nrhs[i] < 1 || !B_dev[i] || !X_dev[i]) return NC_ERR_ARG;
        if (i == 0) mixed = S[i]->mixed;
        else if (S[i]->mixed != mixed) return NC_ERR_UNSUPPORTED;   // one apply precision per batch
        slots += nrhs[i];
        units += S[i]->n * nrhs[i];
        kmax = std::max(kmax, S[i]->k);
    }
    nc_batch B = nullptr;
    nc_status st = pcg_batch_create(slots, units, kmax, mixed ? 0 : NC_BATCH_F64_APPLY, stream, &B);
    if (st != NC_OK) return st;
    std::vector<int> ids;
    ids.reserve(slots);
    // each system's right-hand sides, up to kMaxGroup per admission (groups of
    // up to kGroupWidth columns)
    for (int i = 0; i < nsys && st == NC_OK; ++i)
        for (int c0 = 0; c0 < nrhs[i] && st == NC_OK; c0 += kMaxGroup) {
            const int m = std::min(kMaxGroup, nrhs[i] - c0);
            int sl[kMaxGroup];
            st = pcg_batch_add_solver_multi(B, S[i], m, B_dev[i] + (size_t)c0 * S[i]->n, S[i]->n, stream, sl);
            ids.insert(ids.end(), sl, sl + m);
        }
    int left = 0;
    if (st == NC_OK) st = pcg_batch_run(B, tol, maxit, 0, stream, &left);
    nc_status first = NC_OK;
    int q = 0;
    for (int i = 0; i < nsys && st == NC_OK; ++i)
        for (int c = 0; c < nrhs[i] && st == NC_OK; ++c, ++q) {
            int done = 0;
            st = pcg_batch_status(B, ids[q], &done, &res[q]);
            if (st == NC_OK) st = pcg_batch_collect(B, ids[q], X_dev[i] + (size_t)c * S[i]->n, stream);
            if (st == NC_OK && first == NC_OK && res[q].status != NC_OK) first = (nc_status)res[q].status;
        }
    if (st == NC_OK) {
        const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) {
            g_batch_err = e;
            st = NC_ERR_CUDA;
        }
    }
    pcg_batch_destroy(B);
    return st != NC_OK ? st : first;
}

nc_status pcg_batch_run(nc_batch B, double tol, int maxit, int iter_limit, void* stream, int* active_left) {
    if (!B || !(tol >= 0.0) || maxit < 0) return NC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B->dirty) {
        nc_status s = sync_tables(B, st);
        if (s) return s;
    }
    if (B->h_ctl->active > 0) {
        BCtl* c = B->h_ctl;
        c->tol2 = tol * tol;
        c->maxit = maxit;
        c->iters_this_call = 0;
        c->iter_limit = iter_limit > 0 ? iter_limit : 0x7fffffff;
        NB_CU(cudaMemcpyAsync(B->d_ctl, c, sizeof(BCtl), cudaMemcpyHostToDevice, st));
        if (B->flags & NC_BATCH_HOST_LOOP) {
            // the same kernels driven from the host, one iteration at a time
            for (;;) {
                enqueue_iteration(B, 0, 0, st);
                NB_CU(cudaGetLastError());
                NB_CU(cudaMemcpyAsync(c, B->d_ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
                NB_CU(cudaStreamSynchronize(st));
                if (!(c->active > 0 && c->iters_this_call < c->iter_limit)) break;
            }
        } else {
            NB_CU(cudaGraphLaunch(B->exec, st));
        }
        NB_CU(cudaMemcpyAsync(c, B->d_ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
        NB_CU(cudaMemcpyAsync(B->h_state, B->d_state, sizeof(BState) * B->cap_slots, cudaMemcpyDeviceToHost, st));
        NB_CU(cudaStreamSynchronize(st));
        // one iteration: opq, axpy, kmax Chebyshev steps, pupd, true, cond
        B->stat_iters += c->iters_this_call;
        // explicit-slot and group Chebyshev kernels per step: 1 (float64), 2
        // per float value type; plus their opq and true kernels
        const int gs = B->graph_sell;
        const bool f64 = (B->flags & NC_BATCH_F64_APPLY) != 0;
        const int nsell = f64 ? ((gs & 3) ? 1 : 0) : 2 * ((gs & 1) + ((gs >> 1) & 1));
        const int nw = ((B->gwidths >> 1) & 1) + ((B->gwidths >> 2) & 1);
        const int ngrp = nw * (f64 ? ((gs & 12) ? 2 : 0) : 2 * (((gs >> 2) & 1) + ((gs >> 3) & 1)));
        B->stat_launches += (int64_t)c->iters_this_call *
                            (B->kmax + 5 + (nsell ? nsell * B->kmax + 2 : 0) + (ngrp ? ngrp * B->kmax + 2 * nw : 0));
    }
    if (active_left) *active_left = B->h_ctl->active;
    return NC_OK;
}

nc_status pcg_batch_status(nc_batch B, int slot, int* done, nc_result* res) {
    if (!B || slot < 0 || slot >= B->cap_slots || !B->used[slot]) return NC_ERR_ARG;
    const BState& s = B->h_state[slot];
    if (done) *done = s.phase == PH_DONE;
    if (res) {
        const double bn = std::sqrt(s.bb);
        res->iters = s.iter;
        res->status = s.status;
        res->relres = bn > 0 ? std::sqrt(s.rr) / bn : 0.0;
        res->true_relres = bn > 0 ? std::sqrt(s.rr_true) / bn : 0.0;
        res->n_dot = s.n_dot;
        res->n_spmv = (int64_t)s.iter + (int64_t)B->kdeg[slot] * s.n_prec;
        res->n_replace = 0;
    }
    return NC_OK;
}

nc_status pcg_batch_collect(nc_batch B, int slot, double* x_dev, void* stream) {
    if (!B || slot < 0 || slot >= B->cap_slots || !B->used[slot] || !x_dev) return NC_ERR_ARG;
    if (B->h_state[slot].phase != PH_DONE) return NC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const BDesc& d = B->desc[slot];
    const double scale = B->h_state[slot].bb == 0.0 ? 0.0 : B->dis[slot];
    const int grid = (int)std::min<int64_t>(4096, ((int64_t)d.n + 255) / 256);
    if (d.disv != nullptr)
        bk_scale_vec<<<grid, 256, 0, st>>>(d.n, d.x, d.disv, scale, x_dev);
    else
        bk_scale<<<grid, 256, 0, st>>>(d.n, d.x, scale, x_dev);
    NB_CU(cudaGetLastError());
    B->stat_launches += 1;
    return NC_OK;
}

nc_status pcg_batch_stats(nc_batch B, int64_t* iterations, int64_t* launches) {
    if (!B) return NC_ERR_ARG;
    if (iterations) *iterations = B->stat_iters;
    if (launches) *launches = B->stat_launches;
    return NC_OK;
}

nc_status pcg_batch_release(nc_batch B, int slot, void* stream) {
    if (!B || slot < 0 || slot >= B->cap_slots || !B->used[slot]) return NC_ERR_ARG;
    const int ph = B->h_state[slot].phase;
    if (ph != PH_DONE) return NC_ERR_ARG;   // only finished slots can be released
    // no synchronisation: collects already enqueued on the engine's stream
    // run before any later kernel that reuses this memory
    pool_free(B, B->off[slot], B->desc[slot].n);
    const int g = B->gid[slot];
    if (g >= 0) {   // the group no longer reads or writes this column; gone with its last
        BGDesc& gd = B->groups[g];
        for (int q = 0; q < kGroupWidth; ++q)
            if (((gd.live >> q) & 1) && gd.slot[q] == slot) gd.live &= ~(1 << q);
        if (gd.live == 0) B->gcoefs[g].clear();
        B->gid[slot] = -1;
    }
    B->used[slot] = 0;
    B->off[slot] = -1;
    B->desc[slot] = BDesc{};
    B->coefs[slot].clear();
    B->h_state[slot] = BState{};
    B->state_upload.push_back(slot);
    B->dirty = true;
    return NC_OK;
}

nc_status pcg_batch_free_units(nc_batch B, int64_t* largest, int64_t* total) {
    if (!B) return NC_ERR_ARG;
    int64_t lg = 0, tt = 0;
    for (auto& kv : B->free_list) {
        lg = std::max(lg, kv.second);
        tt += kv.second;
    }
    if (largest) *largest = lg;
    if (total) *total = tt;
    return NC_OK;
}

nc_status pcg_batch_destroy(nc_batch B) {
    if (!B) return NC_ERR_ARG;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    cudaFree(B->d_desc);
    cudaFree(B->d_state);
    cudaFree(B->d_ctl);
    cudaFree(B->d_tiles);
    cudaFree(B->d_vch);
    cudaFree(B->d_coef);
    cudaFree(B->d_ntile_step);
    cudaFree(B->d_stiles);
    cudaFree(B->d_sntile_step);
    cudaFree(B->d_gdesc);
    cudaFree(B->d_gtiles);
    cudaFree(B->d_gntile_step);
    cudaFree(B->d_gpartials);
    cudaFree(B->d_partials);
    cudaFree(B->pool64);
    cudaFree(B->pool32);
    if (B->h_state) cudaFreeHost(B->h_state);
    if (B->h_ctl) cudaFreeHost(B->h_ctl);
    delete B;
    return NC_OK;
}

}  // extern "C"
