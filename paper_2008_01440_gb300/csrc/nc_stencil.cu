// Matrix-free 7-point stencil: the fused Chebyshev step with no matrix in
// memory (Sec. 1: polynomial preconditioners need only v -> A v; Sec. 5.3's
// FD-3D Poisson operator).
//
//   (A u)_p = c0 u_p - cx (u_{p-ex} + u_{p+ex}) - cy (...) - cz (...),
//   zero Dirichlet halo, unknown (i, j, k) at i + nx (j + ny k).
//
// One Chebyshev step y = ca u + cb w + cc r + cd A u becomes
//   y = e0 u + ex (u_{i-1} + u_{i+1}) + ey (u_{j-1} + u_{j+1})
//            + ez (u_{k-1} + u_{k+1}) + cb w + cc r,
// e0 = ca + cd c0, e_a = -cd c_a (the x_{k-1} term folds into the centre
// coefficient for free).
//
// Layout: a CTA owns a 32 x 8 tile of an (x, y) plane and marches along z
// over a chunk of planes, keeping u at planes k-1, k, k+1 in registers, so
// every u value is read from memory once per chunk.  x-neighbours come from
// the adjacent lanes by warp shuffle (lane 0 and 31 read across the tile
// edge), y-neighbours through the read-only cache (the adjacent warps loaded
// them as their own centre values).  Each point reads u, w, r and writes y
// once: 4 vector accesses, the minimum.
#include "nc_stencil.cuh"

namespace nc {
namespace {

template <typename XT, typename YT, int DOT, bool XU, int PZ>
__global__ void __launch_bounds__(kTX * kTY)
stencil7_step_kernel(const int nx, const int ny, const int nz, const int zchunk, const XT* __restrict__ u,
                     const XT* __restrict__ w, const XT* __restrict__ r, YT* __restrict__ y,
                     const StencilCoef<typename AccOf<XT>::type> c, const double* __restrict__ rdot,
                     const Reduce R, const int* __restrict__ done) {
    if (done != nullptr && *done) return;
    const int k0 = blockIdx.z * zchunk;
    const int k1 = min(k0 + zchunk, nz);
    const double dv = stencil_tile<XT, YT, DOT, XU, PZ>(nx, ny, nz, blockIdx.x, blockIdx.y, k0, k1, u, w, r, y, c, rdot,
                                                threadIdx.x, threadIdx.y);
    if (DOT != 0) {
        const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        grid_reduce_ex<kTX * kTY>(dv, R, bid, nb);
    }
}

constexpr int kDeepChunk = 128;   // float z-chunks at least this long take 4-plane batches

template <typename XT, typename YT>
cudaError_t stencil_dispatch(const StencilGeom& g, const double* c4, const void* u, const void* w, const void* r,
                             void* y, double ca, double cb, double cc, double cd, int dot, const double* rdot,
                             const Reduce& R, const int* done, cudaStream_t st) {
    using AT = typename AccOf<XT>::type;
    StencilCoef<AT> c;
    c.e0 = (AT)(ca + cd * c4[0]);
    c.ex = (AT)(-cd * c4[1]);
    c.ey = (AT)(-cd * c4[2]);
    c.ez = (AT)(-cd * c4[3]);
    c.cb = (AT)cb;
    c.cc = (AT)cc;
    c.terms = (cb != 0.0 ? kTermW : 0) | (cc != 0.0 ? kTermR : 0);
    // plain steps take the tuned chunking; dot-product steps the policy's
    StencilGeom gg = g;
    if (dot != 0) gg.zc = gg.pz = 0;
    const dim3 grid = stencil_grid(gg);
    const dim3 block(kTX, kTY);
    const int zc = stencil_zchunk(gg);
    const XT* uu = static_cast<const XT*>(u);
    const XT* ww = static_cast<const XT*>(w);
    const XT* rr = static_cast<const XT*>(r);
    YT* yy = static_cast<YT*>(y);
#define NC_ST_ARGS g.nx, g.ny, g.nz, zc, uu, ww, rr, yy, c, rdot, R, done
    if constexpr (sizeof(AT) == 8) {
        // float64 with ex == -1 exactly (a normalised operator with scaled
        // iterates, or cx = 1 with cd = 1): the kernel without the centre
        // multiply
        if (c.ex == -1.0) {
            switch (dot) {
            case 0: stencil7_step_kernel<XT, YT, 0, true, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            case 1: stencil7_step_kernel<XT, YT, 1, true, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            default: stencil7_step_kernel<XT, YT, 2, true, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            }
            return cudaGetLastError();
        }
    } else {
        // float: 4-plane batches for long z-chunks (or as tuned)
        if (gg.pz == 4 || (gg.pz == 0 && zc >= kDeepChunk)) {
            switch (dot) {
            case 0: stencil7_step_kernel<XT, YT, 0, false, 4><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            case 1: stencil7_step_kernel<XT, YT, 1, false, 4><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            default: stencil7_step_kernel<XT, YT, 2, false, 4><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
            }
            return cudaGetLastError();
        }
    }
    switch (dot) {
    case 0: stencil7_step_kernel<XT, YT, 0, false, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
    case 1: stencil7_step_kernel<XT, YT, 1, false, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
    default: stencil7_step_kernel<XT, YT, 2, false, 2><<<grid, block, 0, st>>>(NC_ST_ARGS); break;
    }
#undef NC_ST_ARGS
    return cudaGetLastError();
}

}  // namespace

// z-chunk length.  Large systems: about eight waves of the 8 resident
// 256-thread CTAs per SM, so a partial last wave of long z-marches costs
// little (1023^3: 3 chunks of 341 planes, float step 4545 -> 3481 us against
// one 1023-plane chunk; 511^3: 10 chunks of 52, float 412 -> 389 us), with
// chunks of at least 32 planes so the two extra plane loads at a chunk's
// start stay a few percent of the traffic.  Where 32-plane chunks would not
// give two waves (small and mid-size systems, up to about 255^3), about two
// waves with chunks of at least 4 planes, so that the GPU is filled.
int stencil_zchunk(const StencilGeom& g) {
    if (g.zc > 0) return g.zc < g.nz ? g.zc : (g.nz > 0 ? g.nz : 1);
    return stencil_zchunk_policy(g);
}

int stencil_zchunk_policy(const StencilGeom& g) {
    const long long tiles = (long long)((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY);
    const long long wave = (long long)vec_grid_max();
    const long long c8 = (8 * wave + tiles - 1) / tiles;
    long long zc = (g.nz + c8 - 1) / c8;
    if (zc < 32) {
        if (tiles * ((g.nz + 31) / 32) >= 2 * wave) {
            zc = 32;
        } else {
            const long long c2 = (2 * wave + tiles - 1) / tiles;
            zc = (g.nz + c2 - 1) / c2;
            if (zc < 4) zc = 4;
        }
    }
    if (zc > g.nz) zc = g.nz > 0 ? g.nz : 1;
    return (int)zc;
}

dim3 stencil_grid(const StencilGeom& g) {
    const int zc = stencil_zchunk(g);
    return dim3((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + zc - 1) / zc);
}

long long stencil_nblocks(const StencilGeom& g) {
    const dim3 d = stencil_grid(g);
    return (long long)d.x * d.y * d.z;
}

cudaError_t launch_stencil_step(const StencilGeom& g, const double* c4, bool x_f32, bool y_f64, const void* u,
                                const void* w, const void* r, void* y, double ca, double cb, double cc, double cd,
                                int dot, const double* rdot, const Reduce& R, const int* done, cudaStream_t st) {
    if ((long long)g.nx * g.ny * g.nz <= 0) return cudaSuccess;
    if (!x_f32) return stencil_dispatch<double, double>(g, c4, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done, st);
    if (y_f64) return stencil_dispatch<float, double>(g, c4, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done, st);
    return stencil_dispatch<float, float>(g, c4, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done, st);
}

}  // namespace nc
