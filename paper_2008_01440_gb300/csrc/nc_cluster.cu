// Whole PCG solve (Algorithm 1 with z = P_k(A) r by the recurrence of
// Algorithm 2) in one kernel on one thread-block cluster, for small systems.
//
// For a few thousand unknowns one PCG iteration is microseconds of work but
// k + 3 kernel launches, each a round trip through L2: launches and
// L2 latency set the time.  Here the system lives in the distributed shared
// memory of a cluster of up to 16 CTAs (one per SM):
//   - CTA c owns the rows [c R, (c+1) R) (R a multiple of the 32-row SELL
//     slice); its slices of the float64 SELL-32 operator A' = A - shift I
//     and its entries of the eight vectors r, t0, t1, t2, p, x, q, z are
//     copied into its shared memory once per solve;
//   - a product gathers u_j through the cluster window (ld.shared::cluster),
//     with each column's address in the owning CTA precomputed at load time;
//   - phases are separated by the hardware cluster barrier, and a dot
//     product is one CTA sum per CTA plus a barrier, after which every CTA
//     adds the cluster's partials in the same fixed order: identical,
//     deterministic scalars everywhere.
// There is no spin-wait: the cluster's CTAs are co-scheduled by the hardware
// and every CTA takes the same branches (same scalars), so every barrier is
// reached by all of them.
#include <type_traits>

#include "nc_common.cuh"

namespace nc {
namespace {

constexpr int kCT = 256;           // threads per CTA
constexpr int kMaxCluster = 16;    // non-portable cluster size on sm_100-class parts

// vector slots in shared memory, R doubles each; R, T0..T2, P and X are read
// by other CTAs, Q and Z only by their owner
enum : int { V_R = 0, V_T0 = 1, V_P = 4, V_X = 5, V_Q = 6, V_Z = 7, kNumVec = 8 };

struct ClusterArgs {
    int n, k, x0_zero, maxit;
    int rows;     // R
    int slots;    // capacity of the per-CTA matrix arrays (SELL entries)
    double tol2, shift;
    const int32_t* sptr;
    const int32_t* col;
    const double* val;
    const double* coef;   // 4*(k+1): (a, b, c, d) of step j at 4j (shifted operator, scaled iterates: d = 1
                          // takes the product as it is); coef[0] = 1/theta'
    const double* b;
    double* x;
    PcgScalars* S;
};

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// address in the cluster window of shared address `a` of CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// volatile: the value changes between phases although the address does not
__device__ __forceinline__ double ld_cluster(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

// Cluster sum s of v (every thread gets it) and, computed once per CTA by
// thread 0, a derived scalar q: `div` 1 gives num / s, 2 gives s / num.
// On GB300 a warp-wide float64 instruction costs about as much as a few
// dozen float32 ones, so the CTA stage is the shared-memory halving tree of
// block_sum (12 warp-wide adds for 256 threads) and only warp 0 finishes.
// The CTA's partial goes to one of two alternating slots: a CTA writes slot
// s again only two sums later, after a barrier that every reader of the
// previous use of s has passed.  The butterfly gives the same bits in every
// lane and every CTA (each level adds the same two values, in either order).
struct ClusterSum {
    double s, q;
};

__device__ __forceinline__ ClusterSum cluster_sum(double v, double num, int div, double* sh, double* red,
                                                  double* bc, int& slot) {
    const double c = block_sum<kCT>(v, sh, (int)threadIdx.x);   // valid in warp 0
    double* mine = red + (slot & 1);
    ++slot;
    if (threadIdx.x == 0) *mine = c;
    cluster_sync();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double t = 0.0;
        if (lane < (int)gridDim.x) t = ld_cluster(map_rank((uint32_t)__cvta_generic_to_shared(mine), (uint32_t)lane));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            bc[0] = t;
            bc[1] = div == 1 ? num / t : (div == 2 ? t / num : 0.0);
        }
    }
    __syncthreads();
    return ClusterSum{bc[0], bc[1]};
}

// acc + (A' u)_i for local row i; `uoff` is the byte offset of u's slot.
// On GB300 a float64 FMA is the scarce resource (about two per clock per
// SM): the loop adds nothing beyond the row's own FMAs.  (Measured on the
// 64 x 64 Laplacian: splitting the chain over two accumulators, or issuing
// all gathers of a row before its FMAs, made the solve 8-15% slower.)
__device__ __forceinline__ double row_product(int i, const int32_t* lptr, const double* mval, const uint32_t* maddr,
                                              uint32_t uoff, double acc) {
    const int s = i >> 5;
    const int end = lptr[s + 1];
#pragma unroll 4
    for (int e = lptr[s] + (i & 31); e < end; e += 32) acc = fma(mval[e], ld_cluster(maddr[e] + uoff), acc);
    return acc;
}

__global__ void __launch_bounds__(kCT) cluster_pcg_kernel(const ClusterArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = a.rows;
    double* vec = reinterpret_cast<double*>(smem);                      // kNumVec * R
    double* mval = vec + (size_t)kNumVec * R;                           // slots
    double* red = mval + a.slots;                                       // 2 partial slots
    double* bc = red + 2;                                               // 2 broadcast scalars
    double* sh = bc + 2;                                                // kCT, CTA sums
    uint32_t* maddr = reinterpret_cast<uint32_t*>(sh + kCT);            // slots
    int32_t* lptr = reinterpret_cast<int32_t*>(maddr + a.slots);        // R / 32 + 1
    const int C = (int)gridDim.x;   // the grid is one cluster
    const int rank = (int)blockIdx.x;
    const int n = a.n, k = a.k;
    const int row0 = rank * R;
    const int nloc = max(0, min(R, n - row0));
    const int s0 = row0 >> 5;
    const int nsl = (nloc + 31) >> 5;
    const uint32_t vbase = (uint32_t)__cvta_generic_to_shared(vec);
    const uint32_t vstride = 8u * (uint32_t)R;
    double* const Rv = vec + (size_t)V_R * R;
    double* const Pv = vec + (size_t)V_P * R;
    double* const Xv = vec + (size_t)V_X * R;
    double* const Qv = vec + (size_t)V_Q * R;
    double* const Zv = vec + (size_t)V_Z * R;

    // ---- load this CTA's slices, x0; zero the rest -------------------------------------
    const int gbeg = nsl > 0 ? a.sptr[s0] : 0;
    const int nslot = nsl > 0 ? a.sptr[s0 + nsl] - gbeg : 0;   // <= a.slots (checked by the planner)
    for (int s = threadIdx.x; s <= R / 32; s += kCT) lptr[s] = nsl > 0 ? a.sptr[s0 + min(s, nsl)] - gbeg : 0;
    for (int e = threadIdx.x; e < nslot; e += kCT) {
        mval[e] = a.val[gbeg + e];
        const int c = a.col[gbeg + e];
        int owner = c / R, off = c - owner * R;
        if (c < 0 || owner >= C) { owner = rank; off = 0; }   // padding of rows past n: never read
        maddr[e] = map_rank(vbase + 8u * (uint32_t)off, (uint32_t)owner);
    }
    for (int i = threadIdx.x; i < kNumVec * R; i += kCT) vec[i] = 0.0;
    __syncthreads();
    if (!a.x0_zero)
        for (int i = threadIdx.x; i < nloc; i += kCT) Xv[i] = a.x[row0 + i];
    cluster_sync();   // every CTA running and x0 visible

    // ---- prologue: r = b - A x0 = b - A' x0 - shift x0, ||b||^2, ||r0||^2 -------------
    int slot = 0;
    double pb = 0.0, pr = 0.0;
    for (int i = threadIdx.x; i < nloc; i += kCT) {
        const double bi = a.b[row0 + i];
        double ri = bi;
        if (!a.x0_zero) ri = bi - fma(a.shift, Xv[i], row_product(i, lptr, mval, maddr, V_X * vstride, 0.0));
        Rv[i] = ri;
        pb = fma(bi, bi, pb);
        pr = fma(ri, ri, pr);
    }
    const double bb = cluster_sum(pb, 0.0, 0, sh, red, bc, slot).s;
    double rr = cluster_sum(pr, 0.0, 0, sh, red, bc, slot).s;
    int status = NC_ERR_MAXIT, iter = 0, n_dot = 0, n_prec = 0;
    bool done = false;
    if (!isfinite(rr)) { status = NC_ERR_BREAKDOWN; done = true; }
    else if (bb == 0.0 || rr <= a.tol2 * bb) { status = NC_OK; done = true; }
    else if (a.maxit <= 0) { status = NC_ERR_MAXIT; done = true; }

    // z = P_k r: x_j in slot T0 + j % 3, the last into Z; returns (r, z) and
    // the derived scalar of `div` (see cluster_sum)
    auto apply_poly = [&](double num, int div) -> ClusterSum {
        double pz = 0.0;
        if (k == 0) {
            const double c0 = a.coef[0];
            for (int i = threadIdx.x; i < nloc; i += kCT) {
                const double zi = c0 * Rv[i];
                Zv[i] = zi;
                pz = fma(Rv[i], zi, pz);
            }
        }
        for (int j = 1; j <= k; ++j) {
            const int us = (j == 1) ? V_R : V_T0 + (j - 1) % 3;
            const int ws = V_T0 + (j + 1) % 3;   // x_{j-2}; read only when cb != 0 (j >= 3)
            const int ys = (j == k) ? V_Z : V_T0 + j % 3;
            const double ca = a.coef[4 * j], cb = a.coef[4 * j + 1], cc = a.coef[4 * j + 2], cd = a.coef[4 * j + 3];
            // which optional terms the step has, decided once (a float64
            // compare per row would occupy the float64 pipe)
            const bool ha = ca != 0.0, hb = cb != 0.0, hc = cc != 0.0, hd = cd != 1.0;
            const double* U = vec + (size_t)us * R;
            const double* Wv = vec + (size_t)ws * R;
            double* Y = vec + (size_t)ys * R;
            const uint32_t uoff = (uint32_t)us * vstride;
            // the test of the product's coefficient stays outside the row
            // loop: inside it the compiler issues the multiply either way
            auto rows = [&](auto scaled) {
                for (int i = threadIdx.x; i < nloc; i += kCT) {
                    double o = row_product(i, lptr, mval, maddr, uoff, 0.0);
                    if constexpr (decltype(scaled)::value) o *= cd;
                    if (hc) o = fma(cc, Rv[i], o);
                    if (hb) o = fma(cb, Wv[i], o);
                    if (ha) o = fma(ca, U[i], o);
                    Y[i] = o;
                    if (j == k) pz = fma(Rv[i], o, pz);
                }
            };
            if (hd) rows(std::true_type{});
            else rows(std::false_type{});
            if (j < k) cluster_sync();   // x_j visible before step j+1 gathers it
        }
        return cluster_sum(pz, num, div, sh, red, bc, slot);
    };

    double rz = 0.0;
    if (!done) {
        rz = apply_poly(0.0, 0).s;
        n_dot += 1;
        n_prec += 1;
        if (!(rz > 0.0)) { status = isfinite(rz) ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN; done = true; }
        for (int i = threadIdx.x; i < nloc; i += kCT) Pv[i] = Zv[i];
        cluster_sync();
    }
    while (!done) {
        // q = A p = A' p + shift p, (p, q), alpha = rz / (p, q)
        double pq = 0.0;
        for (int i = threadIdx.x; i < nloc; i += kCT) {
            const double qi = fma(a.shift, Pv[i], row_product(i, lptr, mval, maddr, V_P * vstride, 0.0));
            Qv[i] = qi;
            pq = fma(Pv[i], qi, pq);
        }
        const ClusterSum sq = cluster_sum(pq, rz, 1, sh, red, bc, slot);
        pq = sq.s;
        n_dot += 1;
        if (!(pq > 0.0) || !isfinite(pq)) { status = isfinite(pq) ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN; break; }
        const double alpha = sq.q;
        double prr = 0.0;
        for (int i = threadIdx.x; i < nloc; i += kCT) {
            Xv[i] = fma(alpha, Pv[i], Xv[i]);
            const double ri = fma(-alpha, Qv[i], Rv[i]);
            Rv[i] = ri;
            prr = fma(ri, ri, prr);
        }
        rr = cluster_sum(prr, 0.0, 0, sh, red, bc, slot).s;   // also publishes r for step 1
        n_dot += 1;
        iter += 1;
        if (!isfinite(rr)) { status = NC_ERR_BREAKDOWN; break; }
        if (rr <= a.tol2 * bb) { status = NC_OK; break; }
        if (iter >= a.maxit) { status = NC_ERR_MAXIT; break; }
        // new (r, z) and beta = (r, z)_new / (r, z)_old
        const ClusterSum sz = apply_poly(rz, 2);
        const double rz_new = sz.s;
        n_dot += 1;
        n_prec += 1;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) {
            status = isfinite(rz_new) ? NC_ERR_INDEFINITE : NC_ERR_BREAKDOWN;
            break;
        }
        const double beta = sz.q;
        rz = rz_new;
        for (int i = threadIdx.x; i < nloc; i += kCT) Pv[i] = fma(beta, Pv[i], Zv[i]);
        cluster_sync();   // p visible before the next product gathers it
    }
    for (int i = threadIdx.x; i < nloc; i += kCT) a.x[row0 + i] = Xv[i];
    if (rank == 0 && threadIdx.x == 0) {
        PcgScalars* S = a.S;
        S->iter = iter;
        S->status = status;
        S->rr = rr;
        S->bb = bb;
        S->rz = rz;
        S->n_dot = n_dot;
        S->n_prec = n_prec;
        S->done = 1;
    }
    cluster_sync();   // no CTA leaves while another may still read its shared memory
}

size_t cluster_smem(int R, int slots) {
    return (size_t)kNumVec * R * 8 + (size_t)slots * 8 + (4 + kCT) * 8 + (size_t)slots * 4 +
           (size_t)(R / 32 + 1) * 4;
}

}  // namespace

bool plan_cluster_pcg(int n, const int32_t* hsptr, ClusterPlan* plan) {
    *plan = ClusterPlan{};
    if (n <= 0 || hsptr == nullptr) return false;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(cluster_pcg_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(cluster_pcg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int nsl_total = (n + 31) / 32;
    int c0 = (n + kCT - 1) / kCT;   // about one row per thread
    if (c0 > kMaxCluster) c0 = kMaxCluster;
    for (int C = c0; C <= kMaxCluster; ++C) {
        const int R = ((n + C - 1) / C + 31) / 32 * 32;
        int slots = 0;
        for (int c = 0; c < C; ++c) {
            const int s0 = c * (R / 32);
            if (s0 >= nsl_total) break;
            const int s1 = s0 + R / 32 < nsl_total ? s0 + R / 32 : nsl_total;
            const int e = hsptr[s1] - hsptr[s0];
            if (e > slots) slots = e;
        }
        const size_t smem = cluster_smem(R, slots);
        if (smem > (size_t)optin) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kCT);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_pcg_kernel, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters < 1) continue;
        *plan = ClusterPlan{C, R, slots, smem};
        return true;
    }
    return false;
}

cudaError_t launch_cluster_pcg(const ClusterPlan& p, int n, int k, int x0_zero, int maxit, double tol2, double shift,
                               const int32_t* sptr, const int32_t* col, const double* val, const double* coef,
                               const double* b, double* x, PcgScalars* S, cudaStream_t st) {
    ClusterArgs a;
    a.n = n;
    a.k = k;
    a.x0_zero = x0_zero;
    a.maxit = maxit;
    a.rows = p.R;
    a.slots = p.slots;
    a.tol2 = tol2;
    a.shift = shift;
    a.sptr = sptr;
    a.col = col;
    a.val = val;
    a.coef = coef;
    a.b = b;
    a.x = x;
    a.S = S;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.C);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = p.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_pcg_kernel, a);
}

}  // namespace nc
