// Staged form of the fused SELL-32 step (offset-pattern layout): the same
// arithmetic as sell_step_kernel, with the streamed operands moved into
// shared memory ahead of use by the copy engine.
//
// Why: the direct kernel issues, per warp, the slot loads of its slice and
// then the gathers of x_{k-1} that need them; the DRAM stream and the L2
// gathers alternate, so only part of the time are enough bytes in flight to
// cover HBM latency (the float step of the 128^3 system reached 0.54 of the
// copy bandwidth at 25.6 us, the same time as the layout with column indices
// that moves 70 % more bytes).  Here persistent CTAs (a few per SM) walk the
// 256-row tiles t = blockIdx.x + i*gridDim.x.  For every tile one thread
// issues bulk asynchronous copies (cp.async.bulk, global -> shared, the 1-D
// form of the tensor-memory-accelerator path, completion counted in bytes on
// an mbarrier) of
//   * the tile's matrix slices: the entries of its 8 slices are contiguous
//     in the layout, [slice_ptr[8t], slice_ptr[8t+8]), 128-byte aligned;
//   * its rows of r and of x_{k-2} when the step uses them (whole tiles only,
//     and only when both vectors are 16-byte aligned);
// `stages` tiles ahead of the one being computed; warp 0 also puts the tile's
// slice offsets and pattern starts into shared memory, and every CTA holds
// the whole offset table (a few hundred bytes for a grid operator).  The HBM
// stream then runs in the copy engine, independent of the warps, and a
// warp's work on a tile has a single global-memory latency on its path: the
// gathers of x_{k-1} (L1/L2).  The stage capacity vcap covers the largest
// tile (else the variant does not apply); vectors that are not staged are
// read from global memory.
//
// The arithmetic is the direct kernel's, operation for operation (the same
// fma chain in slot order and the same epilogue), so both variants give
// identical bits.
//
// Waits are bounded: a wait that has not seen its tile's bytes within
// kWaitNs (0.2 s; a tile normally takes microseconds) sets PcgScalars::fault,
// waits (bounded again) for the copies this CTA still has in flight, adds a
// NaN to the dot product if there is one (so that the reduction completes and
// the solve ends with a breakdown status) and returns.
#include "nc_step.cuh"

namespace nc {
namespace {

constexpr int kSlices = kBlock / 32;      // slices per 256-row tile
constexpr int kMaxStages = 4;
constexpr int kVcapMax = kBlock * 16;     // stage capacity limit: 16 slots per row
constexpr unsigned long long kWaitNs = 200000000ull;
constexpr long long kWaitIters = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// arrive once and announce `bytes` of copies that will complete on the barrier
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase with this parity has completed; false after the limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < kWaitIters; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// bulk copy global -> this CTA's shared memory, completion on `bar`;
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// shared-memory loads by address (explicit, so that they are LDS)
__device__ __forceinline__ double lds(uint32_t a, double*) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds(uint32_t a, float*) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds(uint32_t a, __nv_bfloat16*) {
    unsigned short b;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(b) : "r"(a));
    return __uint_as_float(((unsigned int)b) << 16);
}

template <typename T>
__device__ __forceinline__ auto lds_as(uint32_t a) {
    return lds(a, static_cast<T*>(nullptr));
}

constexpr int kFlagR = 2, kFlagW = 4;

__host__ __device__ constexpr uint32_t align128(uint32_t b) { return (b + 127u) & ~127u; }

// RPT rows per thread: a tile is RPT * 256 rows (RPT * 8 slices); warp w
// takes slices w, w + 8, ... of it, and a thread issues the gathers of all
// its rows before their fma chains, so RPT slices' gathers are in flight per
// warp.  contig: CTA b takes the tiles [b T, (b+1) T) in order (neighbouring
// rows: the gathers at small offsets hit L1 lines of the previous tile),
// else tiles b, b + gridDim.x, ...
template <typename VT, typename XT, typename YT, int DOT, bool UNIT, int RPT>
__global__ void __launch_bounds__(kBlock)
sell_staged_kernel(const int n, const int32_t* __restrict__ slice_ptr, const SellPat pat, const int npoff,
                   const VT* __restrict__ val, const XT* __restrict__ u, const XT* __restrict__ w,
                   const XT* __restrict__ r, YT* __restrict__ y, const StepCoef<typename AccOf<XT>::type> c,
                   const double* __restrict__ rdot, const Reduce R, const int* __restrict__ done, const int vcap,
                   const int stages, const int stage_rw, const int contig) {
    using AT = typename AccOf<XT>::type;
    constexpr int kTS = kSlices * RPT;   // slices per tile
    constexpr int kTR = kBlock * RPT;    // rows per tile
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[kMaxStages];
    __shared__ int meta_sp[kMaxStages][kTS + 1];   // the tile's slice offsets
    __shared__ int meta_ps[kMaxStages][kTS];       // and its slices' pattern starts
    __shared__ int meta_fl[kMaxStages];
    if (done != nullptr && *done) return;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nslices = (n + 31) >> 5;
    const int ntiles = (n + kTR - 1) / kTR;
    const int per_cta = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    // this CTA's i-th tile, or -1
    auto tile_of = [&](int i) -> int {
        if (contig) {
            const int t = (int)blockIdx.x * per_cta + i;
            return (i < per_cta && t < ntiles) ? t : -1;
        }
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        return t < ntiles ? t : -1;
    };
    const uint32_t tbytes = align128((uint32_t)npoff * 4u);   // the offset table
    const uint32_t vbytes = align128((uint32_t)vcap * (uint32_t)sizeof(VT));
    const uint32_t vrow = kTR * (uint32_t)sizeof(XT);
    const uint32_t sbytes = vbytes + 2u * vrow;
    const bool need_r = (c.terms & kTermR) != 0, need_w = (c.terms & kTermW) != 0;
    int* s_pat = reinterpret_cast<int*>(smem);
    const uint32_t sm0 = smem_u32(smem) + tbytes;   // stage 0

    // the whole offset table into shared memory (a few hundred bytes for a grid)
    for (int q = tid; q < npoff; q += kBlock) s_pat[q] = __ldg(pat.poff + q);
    if (tid == 0) {
        for (int q = 0; q < stages; ++q) mbar_init(smem_u32(&bar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // producer (warp 0): the metadata of this CTA's i-th tile into stage i % stages,
    // then (lane 0) the bulk copies of its slices and rows
    uint64_t pol_stream = 0, pol_keep = 0;
    if (tid == 0) {
        pol_stream = policy_evict_first();
        pol_keep = policy_evict_normal();
    }
    auto issue = [&](int i) {   // all lanes of warp 0; warp-uniform control
        const int t = tile_of(i);
        if (t < 0) return;
        const int sidx = i % stages;
        const int s0 = t * kTS;
        const int ns = min(kTS, nslices - s0);
        int v = 0;
        if (lane <= ns) {
            v = slice_ptr[s0 + lane];
            meta_sp[sidx][lane] = v;
        }
        if (lane < ns) meta_ps[sidx][lane] = pat.pstart[s0 + lane];
        const int vb = __shfl_sync(0xffffffffu, v, 0), ve = __shfl_sync(0xffffffffu, v, ns);
        __syncwarp();
        if (lane == 0) {
            const uint32_t nvb = (uint32_t)(ve - vb) * (uint32_t)sizeof(VT);   // <= vbytes (vcap >= every tile)
            const bool full = (t + 1) * kTR <= n;
            const bool sr = need_r && stage_rw && full;
            const bool sw = need_w && stage_rw && full;
            meta_fl[sidx] = (sr ? kFlagR : 0) | (sw ? kFlagW : 0);
            const uint32_t bytes = nvb + (sr ? vrow : 0u) + (sw ? vrow : 0u);
            const uint32_t b = smem_u32(&bar[sidx]);
            const uint32_t dst = sm0 + (uint32_t)sidx * sbytes;
            // the stage was last read through the generic proxy (ordered
            // before this point by the CTA barrier); order those reads
            // before the async-proxy writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_tx(b, bytes);
            if (nvb > 0) bulk_g2s(dst, val + vb, nvb, b, pol_stream);
            if (sr) bulk_g2s(dst + vbytes, r + (size_t)t * kTR, vrow, b, pol_keep);
            if (sw) bulk_g2s(dst + vbytes + vrow, w + (size_t)t * kTR, vrow, b, pol_stream);
        }
    };
    if (warp == 0)
        for (int i = 0; i < stages; ++i) issue(i);

    double dv = 0.0;
    bool fault = false;
    int i = 0;
    for (;; ++i) {
        const int t = tile_of(i);
        if (t < 0) break;
        const int sidx = i % stages;
        const bool ok = mbar_wait(smem_u32(&bar[sidx]), (uint32_t)((i / stages) & 1));
        if (ok) {
            const int fl = meta_fl[sidx];
            const uint32_t stage = sm0 + (uint32_t)sidx * sbytes;
            const int vb = meta_sp[sidx][0];
            // this thread's rows: slice warp + 8q of the tile, q < RPT
            int row[RPT], len[RPT];
            const int* op[RPT];
            uint32_t va[RPT];
            int maxlen = 0;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int ls = warp + kSlices * q;      // slice within the tile
                row[q] = t * kTR + 32 * ls + lane;
                len[q] = 0;
                op[q] = s_pat;
                va[q] = stage;
                if (t * kTS + ls < nslices) {         // warp-uniform
                    const int beg = meta_sp[sidx][ls];
                    len[q] = (meta_sp[sidx][ls + 1] - beg) >> 5;
                    op[q] = s_pat + meta_ps[sidx][ls];
                    va[q] = stage + (uint32_t)(beg - vb + lane) * (uint32_t)sizeof(VT);
                    maxlen = max(maxlen, len[q]);
                }
            }
            auto vload = [&](int q, int j) -> AT {
                return (AT)lds_as<VT>(va[q] + (uint32_t)(32 * j) * (uint32_t)sizeof(VT));
            };
            auto colj = [&](int q, int j) -> int { return min(max(row[q] + op[q][j], 0), n - 1); };
            AT acc[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) acc[q] = AT(0);
            // float64: groups of 4 slots, float: 8; every gather of a group
            // (all RPT rows) before its fma chains
            constexpr int G = sizeof(AT) == 8 ? 4 : 8;
            for (int j0 = 0; j0 < maxlen; j0 += G) {
                AT xx[RPT][G];
#pragma unroll
                for (int q = 0; q < RPT; ++q)
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (j0 + g < len[q]) xx[q][g] = (AT)__ldg(u + colj(q, j0 + g));
#pragma unroll
                for (int q = 0; q < RPT; ++q)
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (j0 + g < len[q]) acc[q] = fma(vload(q, j0 + g), xx[q][g], acc[q]);
            }
            // epilogue, in the direct kernel's order
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int rw = row[q];
                if (rw >= n) continue;
                const uint32_t off = (uint32_t)(rw - t * kTR) * (uint32_t)sizeof(XT);
                AT o;
                if constexpr (UNIT) o = acc[q];
                else o = (c.terms & kUnitD) ? acc[q] : c.cd * acc[q];
                if (need_r) {
                    const AT rv = (fl & kFlagR) ? (AT)lds_as<XT>(stage + vbytes + off) : (AT)r[rw];
                    o = fma(c.cc, rv, o);
                }
                if (need_w) {
                    const AT wv = (fl & kFlagW) ? (AT)lds_as<XT>(stage + vbytes + vrow + off) : (AT)w[rw];
                    o = fma(c.cb, wv, o);
                }
                if (c.terms & kTermU) o = fma(c.ca, (AT)u[rw], o);
                const YT yo = (YT)o;
                y[rw] = yo;
                if (DOT == 1) dv += rdot[rw] * (double)yo;
                if (DOT == 2) dv += (double)u[rw] * (double)yo;
            }
        }
        if (__syncthreads_or(ok ? 0 : 1)) {
            fault = true;
            break;
        }
        if (warp == 0) issue(i + stages);
    }
    if (fault) {
        // tiles i .. i + stages - 1 of this CTA may still have copies in flight
        if (tid == 0) {
            if (R.S != nullptr) atomicExch(&R.S->fault, 1);
            for (int j = i; j < i + stages; ++j) {
                if (tile_of(j) < 0) break;
                mbar_wait(smem_u32(&bar[j % stages]), (uint32_t)((j / stages) & 1));
            }
        }
        __syncthreads();
        dv = __longlong_as_double(0x7ff8000000000000ll);   // NaN: the reduction reports a breakdown
    }
    if constexpr (DOT != 0) grid_reduce<kBlock>(dv, R);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Launch shape of one staged instantiation: stages, stage capacity, dynamic
// shared memory and resident CTAs per SM (at most tune.ctas_per_sm).
// cudaErrorNotSupported when it cannot run on this device.
struct StagedShape {
    int stages, vcap, per_sm;
    size_t smem;
};
constexpr int kPatSmemMax = 4096;   // offset-table entries held in shared memory

template <typename VT, typename XT, typename YT, int DOT, bool UNIT, int RPT>
cudaError_t staged_shape(const StepTune& tune, StagedShape* out) {
    StagedShape sh;
    const int stages = DOT == 0 ? tune.stages : tune.dot_stages;
    const int want = DOT == 0 ? tune.ctas_per_sm : tune.dot_ctas_per_sm;
    sh.stages = stages < 2 ? 2 : (stages > kMaxStages ? kMaxStages : stages);
    // every tile's slices must fit one stage, and the offset table the CTA
    sh.vcap = ((RPT == 1 ? tune.vcap : tune.vcap2) + 31) & ~31;
    if (sh.vcap <= 0 || sh.vcap > kVcapMax * RPT || tune.npoff <= 0 || tune.npoff > kPatSmemMax)
        return cudaErrorNotSupported;
    const uint32_t vbytes = align128((uint32_t)sh.vcap * (uint32_t)sizeof(VT));
    sh.smem = align128((uint32_t)tune.npoff * 4u) +
              (size_t)sh.stages * (vbytes + 2u * kBlock * RPT * (uint32_t)sizeof(XT));
    auto kern = sell_staged_kernel<VT, XT, YT, DOT, UNIT, RPT>;
    const size_t smem = sh.smem;
    // raise the kernel's dynamic shared-memory limit (once per device and size)
    static int raised[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    if ((int)smem > raised[dev]) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if ((int)smem > optin - 4096) return cudaErrorNotSupported;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        raised[dev] = (int)smem;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    const int cap = want > 0 ? want : 2;
    sh.per_sm = per_sm < cap ? per_sm : cap;
    *out = sh;
    return cudaSuccess;
}

template <typename VT, typename XT, typename YT, int DOT, bool UNIT, int RPT>
cudaError_t staged_launch(int n, const int32_t* sptr, const SellPat& pat, const void* val, const void* u,
                          const void* w, const void* r, void* y, double ca, double cb, double cc, double cd,
                          const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                          const StepTune& tune) {
    using AT = typename AccOf<XT>::type;
    StagedShape sh;
    const cudaError_t e = staged_shape<VT, XT, YT, DOT, UNIT, RPT>(tune, &sh);
    if (e != cudaSuccess) return e;
    const int tiles = (n + kBlock * RPT - 1) / (kBlock * RPT);
    const int grid = tiles < sh.per_sm * num_sms() ? tiles : sh.per_sm * num_sms();
    const StepCoef<AT> c = make_coef<AT>(ca, cb, cc, cd);
    const int stage_rw = aligned16(r) && aligned16(w) ? 1 : 0;
    const int contig = DOT == 0 ? tune.contig : tune.dot_contig;
    sell_staged_kernel<VT, XT, YT, DOT, UNIT, RPT><<<grid, kBlock, sh.smem, st>>>(
        n, sptr, pat, tune.npoff, static_cast<const VT*>(val), static_cast<const XT*>(u), static_cast<const XT*>(w),
        static_cast<const XT*>(r), static_cast<YT*>(y), c, rdot, R, done, sh.vcap, sh.stages, stage_rw, contig);
    return cudaGetLastError();
}

template <typename VT, typename XT, typename YT, bool UNIT>
cudaError_t staged_dot(int dot, int n, const int32_t* sptr, const SellPat& pat, const void* val, const void* u,
                       const void* w, const void* r, void* y, double ca, double cb, double cc, double cd,
                       const double* rdot, const Reduce& R, const int* done, cudaStream_t st, const StepTune& tune) {
#define NC_STG_ARGS n, sptr, pat, val, u, w, r, y, ca, cb, cc, cd, rdot, R, done, st, tune
    const int rpt = dot == 0 ? tune.rpt : tune.dot_rpt;
    if (rpt == 2) {
        if (dot == 0) return staged_launch<VT, XT, YT, 0, UNIT, 2>(NC_STG_ARGS);
        if (dot == 1) return staged_launch<VT, XT, YT, 1, UNIT, 2>(NC_STG_ARGS);
        return staged_launch<VT, XT, YT, 2, UNIT, 2>(NC_STG_ARGS);
    }
    if (dot == 0) return staged_launch<VT, XT, YT, 0, UNIT, 1>(NC_STG_ARGS);
    if (dot == 1) return staged_launch<VT, XT, YT, 1, UNIT, 1>(NC_STG_ARGS);
    return staged_launch<VT, XT, YT, 2, UNIT, 1>(NC_STG_ARGS);
#undef NC_STG_ARGS
}

}  // namespace

int sell_staged_ctas(int vdt, bool x_f32, bool y_f64, int dot, bool unit, const StepTune& tune) {
    StagedShape sh{0, 0, 0, 0};
    cudaError_t e = cudaErrorNotSupported;
    const int rpt = dot == 0 ? tune.rpt : tune.dot_rpt;
#define NC_SHAPE_R(VT, XT, YT, U, P)                                                       \
    (dot == 0 ? staged_shape<VT, XT, YT, 0, U, P>(tune, &sh)                               \
              : (dot == 1 ? staged_shape<VT, XT, YT, 1, U, P>(tune, &sh) : staged_shape<VT, XT, YT, 2, U, P>(tune, &sh)))
#define NC_SHAPE(VT, XT, YT, U) (rpt == 2 ? NC_SHAPE_R(VT, XT, YT, U, 2) : NC_SHAPE_R(VT, XT, YT, U, 1))
    if (!x_f32 && vdt == NC_F64)
        e = unit ? NC_SHAPE(double, double, double, true) : NC_SHAPE(double, double, double, false);
    else if (x_f32 && vdt == NC_F32)
        e = y_f64 ? NC_SHAPE(float, float, double, false) : NC_SHAPE(float, float, float, false);
    else if (x_f32 && vdt == NC_BF16)
        e = y_f64 ? NC_SHAPE(__nv_bfloat16, float, double, false) : NC_SHAPE(__nv_bfloat16, float, float, false);
#undef NC_SHAPE
#undef NC_SHAPE_R
    return e == cudaSuccess ? sh.per_sm : 0;
}

int sell_max_tile_entries(const int32_t* hsptr, int nslices, int per_tile) {
    int m = 0;
    for (int s0 = 0; s0 < nslices; s0 += per_tile) {
        const int s1 = s0 + per_tile < nslices ? s0 + per_tile : nslices;
        const int e = hsptr[s1] - hsptr[s0];
        if (e > m) m = e;
    }
    return m;
}

cudaError_t launch_sell_staged(int n, const int32_t* slice_ptr, const int32_t* col, const SellPat& pat,
                               const void* val, int vdt, bool x_f32, bool y_f64, const void* u, const void* w,
                               const void* r, void* y, double ca, double cb, double cc, double cd, int dot,
                               const double* rdot, const Reduce& R, const int* done, cudaStream_t st,
                               const StepTune& tune) {
    (void)col;
    // offset-pattern layout only; a scalar block must exist to report a
    // fault in; the values must be 16-byte aligned for the bulk copies
    if (n <= 0 || pat.pstart == nullptr || R.S == nullptr || !aligned16(val)) return cudaErrorNotSupported;
#define NC_STG_ARGS dot, n, slice_ptr, pat, val, u, w, r, y, ca, cb, cc, cd, rdot, R, done, st, tune
    if (!x_f32) {
        if (vdt != NC_F64) return cudaErrorInvalidValue;
        if (cd == 1.0) return staged_dot<double, double, double, true>(NC_STG_ARGS);
        return staged_dot<double, double, double, false>(NC_STG_ARGS);
    }
    if (vdt == NC_F32)
        return y_f64 ? staged_dot<float, float, double, false>(NC_STG_ARGS)
                     : staged_dot<float, float, float, false>(NC_STG_ARGS);
    if (vdt == NC_BF16)
        return y_f64 ? staged_dot<__nv_bfloat16, float, double, false>(NC_STG_ARGS)
                     : staged_dot<__nv_bfloat16, float, float, false>(NC_STG_ARGS);
#undef NC_STG_ARGS
    return cudaErrorInvalidValue;
}

}  // namespace nc
