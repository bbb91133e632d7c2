// z = P_k(A) v for a CSR matrix without any device allocation.
//
// Who this is for: code that must not call cudaMalloc/cudaFree at the time
// it applies the preconditioner -- for example a Krylov solver embedded in
// a host application that hands out all device memory from its own fixed
// arena, a real-time loop where an allocation (and the implicit device
// synchronisation cudaFree can cause) is not allowed, or a plugin running
// inside a framework that owns the device heap.  pcg_setup/pcg_apply_poly
// allocate their work vectors per solver; this entry point instead works in
// one fixed, file-scope device array and only uses memory the caller passes.
//
// The three-term recurrence needs x_{j-1} (gathered by the product, so it
// cannot be overwritten in the same step), x_{j-2} and the new x_j.  Two of
// the three rotating vectors live in the static array below; the caller's
// output z serves as the third, arranged so that the last step (j = k)
// writes into z.  Nothing in the array has to start at zero: every slot is
// written before it is read, so leftovers of an earlier call are harmless.
// Calls that overlap on the GPU (two streams, or two host threads on one
// device) share the array and race; serialise them.
#include "nc_common.cuh"

namespace {

constexpr int64_t kNoAllocMaxN = (int64_t)1 << 20;   // 1,048,576 unknowns

// 2 vectors x 2^20 float64 = 16 MiB on every device that loads the library,
// held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxN];

// Device address of the array for the current device.  The host-side name
// g_noalloc_scratch is only a stand-in for the symbol; its device address
// must come from cudaGetSymbolAddress with the device current.  It is looked
// up on every call (no cache), so a context torn down and re-created by the
// caller (cudaDeviceReset) never leaves a stale address behind.  The first
// lookup on a device may load the library's module there (lazy loading),
// which is when the array's memory is taken.
nc_status noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return NC_ERR_CUDA;
    }
    *out = static_cast<double*>(p);
    return NC_OK;
}

}  // namespace

extern "C" {

int64_t nc_apply_poly_noalloc_max_n(void) { return kNoAllocMaxN; }

nc_status nc_apply_poly_csr_noalloc(int64_t n, const int32_t* rowptr_dev, const int32_t* col_dev,
                                    const double* val_dev, double lambda_min, double lambda_max,
                                    int degree_k, double theta_scale, const double* v_dev,
                                    double* z_dev, void* stream) {
    if (n < 0 || degree_k < 0 || degree_k > 4096 || !(lambda_min > 0.0) ||
        !(lambda_max > lambda_min) || !(theta_scale > 0.0))
        return NC_ERR_ARG;
    if (n > kNoAllocMaxN) return NC_ERR_SCRATCH_LIMIT;
    if (n == 0) return NC_OK;
    if (!rowptr_dev || !col_dev || !val_dev || !v_dev || !z_dev || v_dev == z_dev) return NC_ERR_ARG;
    double* scratch = nullptr;
    const nc_status s = noalloc_scratch(&scratch);
    if (s != NC_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ni = (int)n;
    // interval parameters and rho_j (Eq. rhocheb) with theta' = s theta
    const double theta = theta_scale * (lambda_max + lambda_min) / 2.0;
    const double delta = (lambda_max - lambda_min) / 2.0;
    const double sigma = theta / delta;
    nc::Reduce none;
    none.partials = nullptr;
    none.counter = nullptr;
    none.S = nullptr;
    none.out = nullptr;
    none.fin = nc::FIN_NONE;
    if (degree_k == 0) {   // P_0 = 1/theta: the step kernel with u = v, a = 1/theta, d = 0
        const cudaError_t e = nc::launch_csr_step(ni, rowptr_dev, col_dev, val_dev, NC_F64, false, true, v_dev,
                                                  nullptr, nullptr, z_dev, 1.0 / theta, 0.0, 0.0, 0.0, 0,
                                                  nullptr, none, nullptr, st);
        return e == cudaSuccess ? NC_OK : NC_ERR_CUDA;
    }
    // x_j lives in slot (k - j) mod 3 of {z, scratch[0:n], scratch[n:2n]}
    double* slot[3] = {z_dev, scratch, scratch + kNoAllocMaxN};
    auto buf = [&](int j) { return slot[(degree_k - j) % 3]; };
    double rho_prev = 1.0 / sigma;   // rho_0
    for (int j = 1; j <= degree_k; ++j) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        double ca, cb, cc, cd;
        const double* u;
        const double* w = nullptr;
        if (j == 1) {   // x_1 = (2 rho_1/delta)(2 v - A v/theta)
            ca = 4.0 * rho / delta;
            cb = 0.0;
            cc = 0.0;
            cd = -2.0 * rho / (delta * theta);
            u = v_dev;
        } else {
            ca = 2.0 * sigma * rho;
            cb = -rho * rho_prev;
            cc = 2.0 * rho / delta;
            cd = -2.0 * rho / delta;
            u = buf(j - 1);
            if (j == 2) {   // x_0 = v/theta folded into the v term
                cc += cb / theta;
                cb = 0.0;
            } else {
                w = buf(j - 2);
            }
        }
        const cudaError_t e = nc::launch_csr_step(ni, rowptr_dev, col_dev, val_dev, NC_F64, false, true, u, w,
                                                  v_dev, buf(j), ca, cb, cc, cd, 0, nullptr, none, nullptr, st);
        if (e != cudaSuccess) return NC_ERR_CUDA;
        rho_prev = rho;
    }
    return NC_OK;
}

}  // extern "C"
