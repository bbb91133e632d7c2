// Matrix handles (CSR, 3x3 BSR, matrix-free 7-point stencil), the symmetric
// diagonal scaling of Sec. 2 / Sec. 5 and its block form (Sec. 6), products,
// Gershgorin bounds, and the extreme-eigenvalue estimates (Lanczos, and the
// power method of Sec. 5.1).
#include "nc_internal.h"

using namespace nc;

namespace {

// Cyclic Jacobi eigen-decomposition of a small symmetric matrix (row-major),
// eigenvectors in the columns of V.  Used only for the Lanczos tridiagonal.
void sym_eig(int m, std::vector<double>& a, std::vector<double>& V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double v = a[(size_t)i * m + j] * a[(size_t)i * m + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = a[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
                const double th = (aqq - app) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {   // columns p, q
                    const double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
                    a[(size_t)k * m + p] = c * akp - s * akq;
                    a[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {   // rows p, q
                    const double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
                    a[(size_t)p * m + k] = c * apk - s * aqk;
                    a[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
}

}  // namespace

extern "C" {

nc_status nc_matrix_csr(int64_t n, int64_t nnz, const int32_t* rowptr_dev, const int32_t* col_dev,
                        const double* val_dev, nc_matrix* out) {
    if (!out) return NC_ERR_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || nnz >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31)) return NC_ERR_ARG;
    if (n > 0 && (!rowptr_dev || (nnz > 0 && (!col_dev || !val_dev)))) return NC_ERR_ARG;
    nc_matrix A = new (std::nothrow) nc_matrix_s();
    if (!A) return NC_ERR_OOM;
    A->kind = MAT_CSR;
    A->n = n;
    A->nnz = nnz;
    A->rowptr = rowptr_dev;
    A->col = col_dev;
    A->val = val_dev;
    *out = A;
    return NC_OK;
}

nc_status nc_matrix_bsr3(int64_t nb, int64_t nnzb, const int32_t* browptr_dev, const int32_t* bcol_dev,
                         const double* val_dev, nc_matrix* out) {
    if (!out) return NC_ERR_ARG;
    *out = nullptr;
    if (nb < 0 || nnzb < 0 || 3 * nb >= ((int64_t)1 << 31) || nnzb >= ((int64_t)1 << 31)) return NC_ERR_ARG;
    if (nb > 0 && (!browptr_dev || (nnzb > 0 && (!bcol_dev || !val_dev)))) return NC_ERR_ARG;
    nc_matrix A = new (std::nothrow) nc_matrix_s();
    if (!A) return NC_ERR_OOM;
    A->kind = MAT_BSR3;
    A->n = 3 * nb;
    A->nnz = nnzb;
    A->rowptr = browptr_dev;
    A->col = bcol_dev;
    A->val = val_dev;
    *out = A;
    return NC_OK;
}

nc_status nc_matrix_stencil7(int nx, int ny, int nz, double c0, double cx, double cy, double cz, nc_matrix* out) {
    if (!out) return NC_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return NC_ERR_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    if (n >= ((int64_t)1 << 31)) return NC_ERR_ARG;
    if (!std::isfinite(c0) || !std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(cz)) return NC_ERR_ARG;
    nc_matrix A = new (std::nothrow) nc_matrix_s();
    if (!A) return NC_ERR_OOM;
    A->kind = MAT_STENCIL7;
    A->n = n;
    A->nnz = 0;
    A->geom = StencilGeom{nx, ny, nz};
    A->c4[0] = c0;
    A->c4[1] = cx;
    A->c4[2] = cy;
    A->c4[3] = cz;
    *out = A;
    return NC_OK;
}

nc_status nc_matrix_jacobi(nc_matrix A, void* stream, nc_matrix* out) {
    if (!A || !out) return NC_ERR_ARG;
    *out = nullptr;
    if (A->scaled) return NC_ERR_ARG;   // already scaled
    if (A->kind == MAT_STENCIL7) {      // constant diagonal c0: D^{-1/2} = c0^{-1/2} I
        if (!(A->c4[0] > 0.0)) return NC_ERR_ARG;
        nc_matrix B = new (std::nothrow) nc_matrix_s(*A);
        if (!B) return NC_ERR_OOM;
        const double d = std::sqrt(A->c4[0]);
        B->c4[0] = 1.0;
        for (int i = 1; i < 4; ++i) B->c4[i] = A->c4[i] / A->c4[0];
        B->dis_scalar = 1.0 / d;
        B->scaled = true;
        *out = B;
        return NC_OK;
    }
    cudaStream_t st = as_stream(stream);
    nc_matrix B = new (std::nothrow) nc_matrix_s(*A);
    if (!B) return NC_ERR_OOM;
    B->owned_val = nullptr;
    B->dis = nullptr;
    int* bad = nullptr;
    int h_bad = 0;
    nc_status s = NC_OK;
    const bool bsr = A->kind == MAT_BSR3;
    const int nb = (int)(A->n / 3);
    do {
        if ((s = dev_alloc_n(&B->dis, A->n)) != NC_OK) break;
        if ((s = dev_alloc_n(&B->owned_val, (bsr ? 9 : 1) * A->nnz)) != NC_OK) break;
        if ((s = dev_alloc_n(&bad, 1)) != NC_OK) break;
        cudaError_t e;
        if ((e = cudaMemsetAsync(bad, 0, sizeof(int), st)) ||
            (e = bsr ? launch_bsr3_diag(nb, A->rowptr, A->col, A->val, B->dis, bad, st)
                     : launch_csr_diag((int)A->n, A->rowptr, A->col, A->val, B->dis, bad, st)) ||
            (e = bsr ? launch_bsr3_scale(nb, A->rowptr, A->col, A->val, B->dis, B->owned_val, st)
                     : launch_csr_scale((int)A->n, A->rowptr, A->col, A->val, B->dis, B->owned_val, st)) ||
            (e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            s = NC_ERR_CUDA;
            break;
        }
        if (h_bad) s = NC_ERR_ARG;
    } while (0);
    dev_free(bad);
    if (s != NC_OK) {
        dev_free(B->dis);
        dev_free(B->owned_val);
        delete B;
        return s;
    }
    B->val = B->owned_val;
    B->scaled = true;
    *out = B;
    return NC_OK;
}

nc_status nc_matrix_block_jacobi(nc_matrix A, void* stream, nc_matrix* out) {
    if (!A || !out) return NC_ERR_ARG;
    *out = nullptr;
    if (A->scaled || A->kind != MAT_BSR3) return NC_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    const int nb = (int)(A->n / 3);
    nc_matrix B = new (std::nothrow) nc_matrix_s(*A);
    if (!B) return NC_ERR_OOM;
    B->owned_val = nullptr;
    B->dis = nullptr;
    B->wblk = B->lblk = nullptr;
    int* bad = nullptr;
    int h_bad = 0;
    nc_status s = NC_OK;
    do {
        if ((s = dev_alloc_n(&B->owned_val, 9 * (A->nnz > 0 ? A->nnz : 1))) || (s = dev_alloc_n(&B->wblk, 9 * (int64_t)(nb > 0 ? nb : 1))) ||
            (s = dev_alloc_n(&B->lblk, 9 * (int64_t)(nb > 0 ? nb : 1))) || (s = dev_alloc_n(&bad, 1)))
            break;
        cudaError_t e;
        if ((e = cudaMemsetAsync(bad, 0, sizeof(int), st)) ||
            (e = launch_bsr3_block_factor(nb, A->rowptr, A->col, A->val, B->wblk, B->lblk, bad, st)) ||
            (e = launch_bsr3_block_scale(nb, A->rowptr, A->col, A->val, B->wblk, B->owned_val, st)) ||
            (e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            s = NC_ERR_CUDA;
            break;
        }
        if (h_bad) s = NC_ERR_ARG;
    } while (0);
    dev_free(bad);
    if (s != NC_OK) {
        dev_free(B->owned_val);
        dev_free(B->wblk);
        dev_free(B->lblk);
        delete B;
        return s;
    }
    B->val = B->owned_val;
    B->scaled = true;
    *out = B;
    return NC_OK;
}

nc_status nc_matvec(nc_matrix A, const double* x_dev, double* y_dev, void* stream) {
    if (!A || (A->n > 0 && (!x_dev || !y_dev)) || x_dev == y_dev) return NC_ERR_ARG;
    const Reduce none = make_reduce(nullptr, nullptr, nullptr, nullptr, FIN_NONE);
    NC_CU(op_step_f64(A, x_dev, nullptr, nullptr, y_dev, 0.0, 0.0, 0.0, 1.0, 0, nullptr, none, nullptr,
                      as_stream(stream)));
    return NC_OK;
}

nc_status nc_gershgorin(nc_matrix A, void* stream, double* bound) {
    if (!A || !bound) return NC_ERR_ARG;
    if (A->kind == MAT_STENCIL7) {   // the fullest row: |c0| + sum_a (neighbours along a) |c_a|
        const int dims[3] = {A->geom.nx, A->geom.ny, A->geom.nz};
        double g = std::fabs(A->c4[0]);
        for (int a = 0; a < 3; ++a) g += (dims[a] >= 3 ? 2.0 : (dims[a] == 2 ? 1.0 : 0.0)) * std::fabs(A->c4[1 + a]);
        *bound = g;
        return NC_OK;
    }
    cudaStream_t st = as_stream(stream);
    unsigned long long* d = nullptr;
    unsigned long long h = 0;
    NC_TRY(dev_alloc_n(&d, 1));
    cudaError_t e;
    if ((e = cudaMemsetAsync(d, 0, sizeof(*d), st)) ||
        (e = A->kind == MAT_BSR3 ? launch_bsr3_gershgorin((int)(A->n / 3), A->rowptr, A->val, d, st)
                                 : launch_csr_gershgorin((int)A->n, A->rowptr, A->val, d, st)) ||
        (e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st))) {
        g_last_cuda = e;
        dev_free(d);
        return NC_ERR_CUDA;
    }
    dev_free(d);
    double v;
    std::memcpy(&v, &h, sizeof(v));
    *bound = v;
    return NC_OK;
}

nc_status nc_bounds_power(nc_matrix A, int iters, const double* v0_dev, void* stream, double* lmax) {
    if (!A || !v0_dev || !lmax || iters < 1 || iters > 100000 || A->n < 1) return NC_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    const int n = (int)A->n;
    double *v = nullptr, *w = nullptr, *part = nullptr, *sc = nullptr;
    unsigned int* cnt = nullptr;
    nc_status s = NC_OK;
    double lam = 0.0;
    do {
        if ((s = dev_alloc_n(&v, n)) || (s = dev_alloc_n(&w, n)) || (s = dev_alloc_n(&part, partials_for(A))) ||
            (s = dev_alloc_n(&sc, 1)) || (s = dev_alloc_n(&cnt, 1)))
            break;
        cudaError_t e = cudaSuccess;
        auto fetch = [&](double* out) -> cudaError_t {
            cudaError_t ee = cudaMemcpyAsync(out, sc, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ee) return ee;
            return cudaStreamSynchronize(st);
        };
        const Reduce Rs = make_reduce(part, cnt, nullptr, sc, FIN_STORE);
        double h = 0.0;
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st)) ||
            (e = launch_dot(n, v0_dev, v0_dev, Rs, nullptr, st)) || (e = fetch(&h))) {
            g_last_cuda = e; s = NC_ERR_CUDA; break;
        }
        if (!(h > 0.0) || !std::isfinite(h)) { s = NC_ERR_ARG; break; }
        if ((e = launch_div(n, v0_dev, std::sqrt(h), v, st))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
        for (int it = 0; it < iters; ++it) {
            double ww = 0.0;
            // w = A v with lambda = (v, w); then v = w / ||w||
            if ((e = op_step_f64(A, v, nullptr, nullptr, w, 0.0, 0.0, 0.0, 1.0, 2, nullptr, Rs, nullptr, st)) ||
                (e = fetch(&lam)) || (e = launch_dot(n, w, w, Rs, nullptr, st)) || (e = fetch(&ww))) {
                g_last_cuda = e; s = NC_ERR_CUDA; break;
            }
            if (!(ww > 0.0) || !std::isfinite(ww)) { s = NC_ERR_BREAKDOWN; break; }
            if ((e = launch_div(n, w, std::sqrt(ww), v, st))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
        }
    } while (0);
    dev_free(v); dev_free(w); dev_free(part); dev_free(sc); dev_free(cnt);
    if (s != NC_OK) return s;
    if (!std::isfinite(lam)) return NC_ERR_BREAKDOWN;
    *lmax = lam;
    return NC_OK;
}

nc_status nc_bounds_lanczos(nc_matrix A, int steps, const double* v0_dev, void* stream, double* lmin,
                            double* lmax, double* ritz_min, double* ritz_max) {
    if (!A || !v0_dev || !lmin || !lmax || steps < 1 || steps > 256 || A->n < 1) return NC_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    const int n = (int)A->n;
    double *vp = nullptr, *v = nullptr, *w = nullptr, *part = nullptr, *sc = nullptr;
    unsigned int* cnt = nullptr;
    nc_status s = NC_OK;
    std::vector<double> al, be;
    do {
        if ((s = dev_alloc_n(&vp, n)) || (s = dev_alloc_n(&v, n)) || (s = dev_alloc_n(&w, n)) ||
            (s = dev_alloc_n(&part, partials_for(A))) || (s = dev_alloc_n(&sc, 4)) ||
            (s = dev_alloc_n(&cnt, 1)))
            break;
        cudaError_t e = cudaSuccess;
        double h = 0.0;
        auto fetch = [&](double* out) -> cudaError_t {
            cudaError_t ee = cudaMemcpyAsync(out, sc, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ee) return ee;
            return cudaStreamSynchronize(st);
        };
        const Reduce Rs = make_reduce(part, cnt, nullptr, sc, FIN_STORE);
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st)) ||
            (e = cudaMemsetAsync(vp, 0, sizeof(double) * n, st)) ||
            (e = launch_dot(n, v0_dev, v0_dev, Rs, nullptr, st)) || (e = fetch(&h))) {
            g_last_cuda = e;
            s = NC_ERR_CUDA;
            break;
        }
        if (!(h > 0.0) || !std::isfinite(h)) { s = NC_ERR_ARG; break; }
        if ((e = launch_div(n, v0_dev, std::sqrt(h), v, st))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
        double b_prev = 0.0;
        for (int j = 0; j < steps; ++j) {
            double a = 0.0, ww = 0.0;
            // w = A v - b_prev v_prev, a = (w, v)
            if ((e = op_step_f64(A, v, vp, nullptr, w, 0.0, -b_prev, 0.0, 1.0, 2, nullptr, Rs, nullptr, st)) ||
                (e = fetch(&a)) ||
                // w = w - a v, ||w||^2
                (e = launch_axpy_dot(n, -a, v, w, Rs, st)) || (e = fetch(&ww))) {
                g_last_cuda = e;
                s = NC_ERR_CUDA;
                break;
            }
            const double b = std::sqrt(ww);
            al.push_back(a);
            be.push_back(b);
            if (b == 0.0 || !std::isfinite(b)) break;
            // v_prev <- v, v <- w / b
            if ((e = launch_div(n, w, b, vp, st))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
            std::swap(vp, v);
            b_prev = b;
        }
    } while (0);
    dev_free(vp); dev_free(v); dev_free(w); dev_free(part); dev_free(sc); dev_free(cnt);
    if (s != NC_OK) return s;
    const int m = (int)al.size();
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(al[i])) return NC_ERR_BREAKDOWN;
    std::vector<double> T((size_t)m * m, 0.0), V;
    for (int i = 0; i < m; ++i) {
        T[(size_t)i * m + i] = al[i];
        if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = be[i];
    }
    sym_eig(m, T, V);
    int imin = 0, imax = 0;
    for (int i = 1; i < m; ++i) {
        if (T[(size_t)i * m + i] < T[(size_t)imin * m + imin]) imin = i;
        if (T[(size_t)i * m + i] > T[(size_t)imax * m + imax]) imax = i;
    }
    const double rmin = T[(size_t)imin * m + imin], rmax = T[(size_t)imax * m + imax];
    const double resid = std::fabs(be[m - 1] * V[(size_t)(m - 1) * m + imax]);
    double upper = std::fmax(rmax + resid, 1.01 * rmax);
    double g = 0.0;
    NC_TRY(nc_gershgorin(A, stream, &g));
    if (rmax <= g && g < upper) upper = g;
    *lmin = rmin;
    *lmax = upper;
    if (ritz_min) *ritz_min = rmin;
    if (ritz_max) *ritz_max = rmax;
    return NC_OK;
}

nc_status nc_matrix_destroy(nc_matrix A) {
    if (!A) return NC_ERR_ARG;
    dev_free(A->owned_val);
    dev_free(A->dis);
    dev_free(A->wblk);
    dev_free(A->lblk);
    delete A;
    return NC_OK;
}

}  // extern "C"
