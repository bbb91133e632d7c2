// Layouts the fused step kernels read, built once by pcg_setup from the
// matrix handle (SELL-32, its offset-pattern form, BSELL-32 for 3x3 blocks,
// or the handle's own CSR arrays), and the measurements that choose between
// layouts (NC_FORMAT_TUNE) and between step-kernel variants (NC_STEP_TUNE).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <unordered_map>

#include "nc_internal.h"

namespace nc {

// of a Chebyshev step after the first) with operator view `op`, in the
// solver's apply precision, on the zero-filled rotating buffers.
nc_status time_step(nc_solver S, const OpView& op, bool shifted, cudaStream_t st, double* us) {
    const size_t vb = S->mixed ? sizeof(float) : sizeof(double);
    for (int i = 0; i < 3; ++i) NC_CU(cudaMemsetAsync(S->buf[i], 0, vb * (size_t)S->n, st));
    const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
    const double ca = shifted ? 0.0 : 0.5;
    auto launch = [&]() {
        return op_step(op, S->mixed, !S->mixed, S->buf[0], S->buf[1], S->buf[0], S->buf[2], ca, -0.25, 0.1, -1.0, 0,
                       nullptr, none, nullptr, st);
    };
    for (int i = 0; i < 3; ++i) NC_CU(launch());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NC_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e) { cudaEventDestroy(e0); g_last_cuda = e; return NC_ERR_CUDA; }
    const int reps = 10;
    e = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) { g_last_cuda = e; return NC_ERR_CUDA; }
    *us = 1e3 * (double)ms / reps;
    return NC_OK;
}

// Choose and build the layout the step kernels read.  SELL-32 when its
// padding is at most kSellMaxPadding (or when forced), else the CSR arrays.
constexpr double kSellMaxPadding = 1.5;
constexpr double kSellTunePadding = 4.0;   // TUNE times SELL only below this padding

// Block counterpart of the SELL setup: BSELL-32 over block rows when its
// padding is at most kSellMaxPadding (or forced), else the plain block CSR.
nc_status setup_operator_bsr3(nc_solver S, cudaStream_t st, size_t eb) {
    nc_matrix A = S->A;
    const int nb = (int)(A->n / 3);
    const int n = (int)A->n;
    bool sliced = S->opt.spmv_format != NC_FORMAT_CSR && nb > 0;
    std::vector<int64_t> hptr;
    if (sliced) {
        const int nslices = (nb + 31) / 32;
        int32_t* dlen = nullptr;
        NC_TRY(dev_alloc_n(&dlen, nslices));
        std::vector<int32_t> hlen(nslices);
        cudaError_t e;
        if ((e = launch_bsell3_lengths(nb, A->rowptr, dlen, st)) ||
            (e = cudaMemcpyAsync(hlen.data(), dlen, sizeof(int32_t) * nslices, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            dev_free(dlen);
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
        dev_free(dlen);
        hptr.resize(nslices + 1);
        hptr[0] = 0;
        for (int i = 0; i < nslices; ++i) hptr[i + 1] = hptr[i] + 32 * (int64_t)hlen[i];
        S->padding = A->nnz > 0 ? (double)hptr[nslices] / (double)A->nnz : 1.0;
        if (hptr[nslices] >= ((int64_t)1 << 31)) sliced = false;
        if (S->opt.spmv_format == NC_FORMAT_AUTO && S->padding > kSellMaxPadding) sliced = false;
        if (S->opt.spmv_format == NC_FORMAT_TUNE && S->padding > kSellTunePadding) sliced = false;
    }
    OpView bsr64{OP_BSR3, n, A->rowptr, A->col, A->val, NC_F64};
    OpView bsrP = bsr64;
    if (S->mixed && (!sliced || S->opt.spmv_format == NC_FORMAT_TUNE)) {
        NC_TRY(dev_alloc(&S->lval, eb * 9 * (size_t)(A->nnz > 0 ? A->nnz : 1)));
        cudaError_t e = launch_convert(9 * A->nnz, A->val, S->vdt, S->lval, st);
        if (e) { g_last_cuda = e; return NC_ERR_CUDA; }
        bsrP = OpView{OP_BSR3, n, A->rowptr, A->col, S->lval, S->vdt};
    }
    if (!sliced) {
        S->padding = 1.0;
        S->shift = 0.0;
        S->op64 = bsr64;
        S->opP = bsrP;
        return NC_OK;
    }
    const int nslices = (nb + 31) / 32;
    const int64_t total = hptr[nslices];
    std::vector<int32_t> hp32(nslices + 1);
    for (int i = 0; i <= nslices; ++i) hp32[i] = (int32_t)hptr[i];
    NC_TRY(dev_alloc_n(&S->sell_ptr, nslices + 1));
    NC_TRY(dev_alloc_n(&S->sell_col, total));
    NC_TRY(dev_alloc_n(&S->sell_val64, 9 * total));
    int* nodiag = nullptr;
    NC_TRY(dev_alloc_n(&nodiag, 1));
    int h_nodiag = 0;
    S->shift = S->k >= 1 ? S->theta : 0.0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(nodiag, 0, sizeof(int), st)) ||
        (e = cudaMemcpyAsync(S->sell_ptr, hp32.data(), sizeof(int32_t) * (nslices + 1), cudaMemcpyHostToDevice, st)) ||
        (e = launch_bsell3_fill(nb, A->rowptr, A->col, A->val, S->sell_ptr, NC_F64, S->shift, S->sell_col,
                                S->sell_val64, nodiag, st)) ||
        (e = cudaMemcpyAsync(&h_nodiag, nodiag, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st))) {
        dev_free(nodiag);
        g_last_cuda = e;
        return NC_ERR_CUDA;
    }
    dev_free(nodiag);
    if (h_nodiag) {
        S->shift = 0.0;
        if ((e = launch_bsell3_fill(nb, A->rowptr, A->col, A->val, S->sell_ptr, NC_F64, 0.0, S->sell_col,
                                    S->sell_val64, nullptr, st))) {
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
    }
    S->op64 = OpView{OP_BSELL3, n, S->sell_ptr, S->sell_col, S->sell_val64, NC_F64};
    S->opP = S->op64;
    if (S->mixed) {
        NC_TRY(dev_alloc(&S->sell_valP, eb * 9 * (size_t)total));
        if ((e = launch_bsell3_fill(nb, A->rowptr, A->col, A->val, S->sell_ptr, S->vdt, S->shift, S->sell_col,
                                    S->sell_valP, nullptr, st))) {
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
        S->opP = OpView{OP_BSELL3, n, S->sell_ptr, S->sell_col, S->sell_valP, S->vdt};
    }
    if ((e = cudaStreamSynchronize(st))) { g_last_cuda = e; return NC_ERR_CUDA; }
    if (S->opt.spmv_format == NC_FORMAT_TUNE) {
        NC_TRY(time_step(S, bsrP, false, st, &S->tune_us[0]));
        NC_TRY(time_step(S, S->opP, S->shift != 0.0, st, &S->tune_us[1]));
        if (S->tune_us[0] < S->tune_us[1]) {
            dev_free(S->sell_ptr); dev_free(S->sell_col); dev_free(S->sell_val64); dev_free(S->sell_valP);
            S->sell_ptr = nullptr; S->sell_col = nullptr; S->sell_val64 = nullptr; S->sell_valP = nullptr;
            S->padding = 1.0;
            S->shift = 0.0;
            S->op64 = bsr64;
            S->opP = bsrP;
        } else if (S->lval) {
            dev_free(S->lval);
            S->lval = nullptr;
        }
    }
    return NC_OK;
}

// Offset-pattern layout (NC_FORMAT_PSELL) from the CSR arrays.  Returns
// NC_ERR_UNSUPPORTED, with nothing left allocated, when the matrix does not
// qualify: a row whose columns do not increase, a slice with more than 64
// offsets, padding above kSellMaxPadding, distinct offset sets holding more
// than kPatMaxTable offsets in all, or more than 2^30 rows (the kernels form
// row + offset in 32 bits, which stays in range for |offset| < n <= 2^30).
constexpr int64_t kPatMaxTable = 16384;

nc_status setup_psell(nc_solver S, cudaStream_t st, size_t eb) {
    nc_matrix A = S->A;
    if (S->n > ((int64_t)1 << 30)) return NC_ERR_UNSUPPORTED;
    const int n = (int)S->n;
    const int nslices = (n + 31) / 32;
    int32_t *dcnt = nullptr, *dopos = nullptr, *doff = nullptr;
    int* dbad = nullptr;
    nc_status ret = NC_ERR_UNSUPPORTED;
    std::vector<int32_t> hp32;
    do {
        if ((ret = dev_alloc_n(&dcnt, nslices)) != NC_OK || (ret = dev_alloc_n(&dbad, 1)) != NC_OK) break;
        ret = NC_ERR_UNSUPPORTED;
        std::vector<int32_t> cnt(nslices);
        int bad = 0;
        cudaError_t e;
        // a constant diagonal (every row's a_ii bitwise equal) stays out of the
        // layout: the steps apply it through their u coefficient
        int fold = 0;
        double d0 = 0.0;
        if (!S->opt.keep_diagonal && n > 0) {
            int flags = 0, r0[2] = {0, 0};
            if ((e = cudaMemsetAsync(dbad, 0, sizeof(int), st)) ||
                (e = launch_csr_diag_const(n, A->rowptr, A->col, A->val, dbad, st)) ||
                (e = cudaMemcpyAsync(&flags, dbad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaMemcpyAsync(r0, A->rowptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st))) {
                g_last_cuda = e;
                ret = NC_ERR_CUDA;
                break;
            }
            if (flags == 0) {   // row 0 has its diagonal: find its value
                std::vector<int32_t> c0(r0[1] - r0[0]);
                std::vector<double> v0(c0.size());
                if (!c0.empty() &&
                    ((e = cudaMemcpyAsync(c0.data(), A->col + r0[0], sizeof(int32_t) * c0.size(),
                                          cudaMemcpyDeviceToHost, st)) ||
                     (e = cudaMemcpyAsync(v0.data(), A->val + r0[0], sizeof(double) * v0.size(),
                                          cudaMemcpyDeviceToHost, st)) ||
                     (e = cudaStreamSynchronize(st)))) {
                    g_last_cuda = e;
                    ret = NC_ERR_CUDA;
                    break;
                }
                for (size_t i = 0; i < c0.size(); ++i)
                    if (c0[i] == 0) {
                        d0 = v0[i];
                        fold = 1;
                    }
            }
        }
        if ((e = cudaMemsetAsync(dbad, 0, sizeof(int), st)) ||
            (e = launch_psell_merge(n, A->rowptr, A->col, nullptr, dcnt, nullptr, dbad, fold, st)) ||
            (e = cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int32_t) * nslices, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            ret = NC_ERR_CUDA;
            break;
        }
        if (bad) break;
        std::vector<int32_t> opos(nslices + 1);
        hp32.assign(nslices + 1, 0);
        int64_t noff = 0, total = 0;
        for (int i = 0; i < nslices; ++i) {
            opos[i] = (int32_t)noff;
            hp32[i] = (int32_t)total;
            noff += cnt[i];
            total += 32 * (int64_t)cnt[i];
            if (total >= ((int64_t)1 << 31)) break;
        }
        if (total >= ((int64_t)1 << 31)) break;
        opos[nslices] = (int32_t)noff;
        hp32[nslices] = (int32_t)total;
        const double padding = A->nnz > 0 ? (double)total / (double)A->nnz : 1.0;
        if (padding > kSellMaxPadding) break;
        // the sets themselves, then each distinct set stored once
        if ((ret = dev_alloc_n(&dopos, nslices + 1)) != NC_OK || (ret = dev_alloc_n(&doff, noff)) != NC_OK) break;
        ret = NC_ERR_UNSUPPORTED;
        std::vector<int32_t> off((size_t)noff);
        if ((e = cudaMemcpyAsync(dopos, opos.data(), sizeof(int32_t) * (nslices + 1), cudaMemcpyHostToDevice, st)) ||
            (e = launch_psell_merge(n, A->rowptr, A->col, dopos, nullptr, doff, dbad, fold, st)) ||
            (e = cudaMemcpyAsync(off.data(), doff, sizeof(int32_t) * (size_t)noff, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            ret = NC_ERR_CUDA;
            break;
        }
        std::unordered_map<std::string, int32_t> seen;
        std::vector<int32_t> table, pstart(nslices);
        bool fits = true;
        for (int i = 0; i < nslices && fits; ++i) {
            std::string key(sizeof(int32_t) * (size_t)cnt[i], '\0');
            if (cnt[i] > 0) std::memcpy(&key[0], off.data() + opos[i], key.size());
            auto it = seen.find(key);
            if (it == seen.end()) {
                if ((int64_t)table.size() + cnt[i] > kPatMaxTable) {
                    fits = false;
                    break;
                }
                it = seen.emplace(std::move(key), (int32_t)table.size()).first;
                table.insert(table.end(), off.begin() + opos[i], off.begin() + opos[i] + cnt[i]);
            }
            pstart[i] = it->second;
        }
        if (!fits) break;
        // the layout itself (solver-owned)
        if ((ret = dev_alloc_n(&S->sell_ptr, nslices + 1)) != NC_OK ||
            (ret = dev_alloc_n(&S->psell_start, nslices)) != NC_OK ||
            (ret = dev_alloc_n(&S->psell_off, (int64_t)table.size())) != NC_OK ||
            (ret = dev_alloc_n(&S->sell_val64, total)) != NC_OK)
            break;
        int h_nodiag = 0;
        S->shift = S->k >= 1 ? S->theta : 0.0;
        if ((e = cudaMemsetAsync(dbad, 0, sizeof(int), st)) ||
            (e = cudaMemcpyAsync(S->sell_ptr, hp32.data(), sizeof(int32_t) * (nslices + 1), cudaMemcpyHostToDevice,
                                 st)) ||
            (e = cudaMemcpyAsync(S->psell_start, pstart.data(), sizeof(int32_t) * nslices, cudaMemcpyHostToDevice,
                                 st)) ||
            (!table.empty() && (e = cudaMemcpyAsync(S->psell_off, table.data(), sizeof(int32_t) * table.size(),
                                                    cudaMemcpyHostToDevice, st))) ||
            (e = launch_psell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->psell_start, S->psell_off, NC_F64,
                                   S->shift, S->sell_val64, dbad, fold, st)) ||
            (e = cudaMemcpyAsync(&h_nodiag, dbad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            ret = NC_ERR_CUDA;
            break;
        }
        if (h_nodiag) {   // a row without a diagonal entry: store A itself
            S->shift = 0.0;
            if ((e = launch_psell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->psell_start, S->psell_off,
                                       NC_F64, 0.0, S->sell_val64, nullptr, fold, st))) {
                g_last_cuda = e;
                ret = NC_ERR_CUDA;
                break;
            }
        }
        S->op64 = OpView{OP_SELL, n, S->sell_ptr, nullptr, S->sell_val64, NC_F64};
        S->op64.pat = SellPat{S->psell_start, S->psell_off};
        S->op64.dfold = fold ? d0 - S->shift : 0.0;   // the stored operator's diagonal, a_ii - shift
        S->op64.dfolded = fold;
        S->opP = S->op64;
        if (S->mixed) {
            if ((ret = dev_alloc(&S->sell_valP, eb * (size_t)(total > 0 ? total : 1))) != NC_OK) break;
            if ((e = launch_psell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->psell_start, S->psell_off,
                                       S->vdt, S->shift, S->sell_valP, nullptr, fold, st))) {
                g_last_cuda = e;
                ret = NC_ERR_CUDA;
                break;
            }
            S->opP.val = S->sell_valP;
            S->opP.vdt = S->vdt;
        }
        if ((e = cudaStreamSynchronize(st))) {   // the host arrays must outlive the copies
            g_last_cuda = e;
            ret = NC_ERR_CUDA;
            break;
        }
        S->padding = padding;
        S->npatterns = (int64_t)seen.size();
        S->h_sell_ptr = hp32;
        // stage capacity of the staged step kernels: the largest tile
        S->op64.tune.vcap = sell_max_tile_entries(hp32.data(), nslices, 8);
        S->op64.tune.vcap2 = sell_max_tile_entries(hp32.data(), nslices, 16);
        S->op64.tune.npoff = (int)table.size();
        S->opP.tune.vcap = S->op64.tune.vcap;
        S->opP.tune.vcap2 = S->op64.tune.vcap2;
        S->opP.tune.npoff = S->op64.tune.npoff;
        ret = NC_OK;
    } while (0);
    if (ret != NC_OK) cudaStreamSynchronize(st);   // no copy may still read a host vector
    dev_free(dcnt);
    dev_free(dopos);
    dev_free(doff);
    dev_free(dbad);
    if (ret != NC_OK) {
        dev_free(S->sell_ptr); dev_free(S->psell_start); dev_free(S->psell_off);
        dev_free(S->sell_val64); dev_free(S->sell_valP);
        S->sell_ptr = nullptr; S->psell_start = nullptr; S->psell_off = nullptr;
        S->sell_val64 = nullptr; S->sell_valP = nullptr;
        S->op64 = OpView{};
        S->opP = OpView{};
        S->shift = 0.0;
        S->npatterns = 0;
    }
    return ret;
}

nc_status setup_operator(nc_solver S, cudaStream_t st) {
    nc_matrix A = S->A;
    const int n = (int)S->n;
    if (A->kind == MAT_STENCIL7) {   // matrix-free: nothing to build
        S->op64 = mat_view(A);
        S->opP = S->op64;
        S->opP.vdt = S->vdt;
        S->padding = 1.0;
        S->shift = 0.0;
        // inside P the stencil is taken divided by its x-weight, which then
        // is exactly 1: with the scaled float64 iterates the step's
        // x-coefficient is exactly -1 and the kernel skips a multiply
        const double kap = S->op64.c4[1];
        if (kap != 0.0 && std::isfinite(kap) && std::isfinite(1.0 / kap)) {
            S->pscale = kap;
            S->opP.c4[0] = S->op64.c4[0] / kap;
            S->opP.c4[1] = 1.0;
            S->opP.c4[2] = S->op64.c4[2] / kap;
            S->opP.c4[3] = S->op64.c4[3] / kap;
        }
        return NC_OK;
    }
    const size_t eb = S->vdt == NC_F64 ? 8 : (S->vdt == NC_F32 ? 4 : 2);
    if (A->kind == MAT_BSR3) return setup_operator_bsr3(S, st, eb);
    if (n > 0 && (S->opt.spmv_format == NC_FORMAT_PSELL ||
                  (S->opt.spmv_format == NC_FORMAT_AUTO && S->opt.use_graph != 2))) {
        const nc_status ps = setup_psell(S, st, eb);
        if (ps != NC_ERR_UNSUPPORTED) return ps;   // built, or a CUDA / memory error
    }
    bool sell = S->opt.spmv_format != NC_FORMAT_CSR && n > 0;
    std::vector<int64_t> hptr;
    if (sell) {
        const int nslices = (n + 31) / 32;
        int32_t* dlen = nullptr;
        NC_TRY(dev_alloc_n(&dlen, nslices));
        std::vector<int32_t> hlen(nslices);
        cudaError_t e;
        if ((e = launch_sell_lengths(n, A->rowptr, dlen, st)) ||
            (e = cudaMemcpyAsync(hlen.data(), dlen, sizeof(int32_t) * nslices, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            dev_free(dlen);
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
        dev_free(dlen);
        hptr.resize(nslices + 1);
        hptr[0] = 0;
        for (int i = 0; i < nslices; ++i) hptr[i + 1] = hptr[i] + 32 * (int64_t)hlen[i];
        const int64_t total = hptr[nslices];
        S->padding = A->nnz > 0 ? (double)total / (double)A->nnz : 1.0;
        if (total >= ((int64_t)1 << 31)) sell = false;
        if (S->opt.spmv_format == NC_FORMAT_AUTO && S->padding > kSellMaxPadding) sell = false;
        if (S->opt.spmv_format == NC_FORMAT_TUNE && S->padding > kSellTunePadding) sell = false;
    }
    // the plain CSR view (always available: the handle's arrays)
    OpView csr64{OP_CSR, n, A->rowptr, A->col, A->val, NC_F64};
    OpView csrP = csr64;
    if (S->mixed && (!sell || S->opt.spmv_format == NC_FORMAT_TUNE)) {
        NC_TRY(dev_alloc(&S->lval, eb * (size_t)(A->nnz > 0 ? A->nnz : 1)));
        cudaError_t e = launch_convert(A->nnz, A->val, S->vdt, S->lval, st);
        if (e) { g_last_cuda = e; return NC_ERR_CUDA; }
        csrP = OpView{OP_CSR, n, A->rowptr, A->col, S->lval, S->vdt};
    }
    if (!sell) {
        S->padding = 1.0;
        S->op64 = csr64;
        S->opP = csrP;
        return NC_OK;
    }
    const int nslices = (n + 31) / 32;
    const int64_t total = hptr[nslices];
    std::vector<int32_t> hp32(nslices + 1);
    for (int i = 0; i <= nslices; ++i) hp32[i] = (int32_t)hptr[i];
    NC_TRY(dev_alloc_n(&S->sell_ptr, nslices + 1));
    NC_TRY(dev_alloc_n(&S->sell_col, total));
    NC_TRY(dev_alloc_n(&S->sell_val64, total));
    int* nodiag = nullptr;
    NC_TRY(dev_alloc_n(&nodiag, 1));
    int h_nodiag = 0;
    // the shifted operator A - theta' I needs every row's diagonal entry;
    // without one, store A itself (shift 0)
    S->shift = S->k >= 1 ? S->theta : 0.0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(nodiag, 0, sizeof(int), st)) ||
        (e = cudaMemcpyAsync(S->sell_ptr, hp32.data(), sizeof(int32_t) * (nslices + 1), cudaMemcpyHostToDevice, st)) ||
        (e = launch_sell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, NC_F64, S->shift, S->sell_col,
                              S->sell_val64, nodiag, st)) ||
        (e = cudaMemcpyAsync(&h_nodiag, nodiag, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st))) {
        dev_free(nodiag);
        g_last_cuda = e;
        return NC_ERR_CUDA;
    }
    dev_free(nodiag);
    if (h_nodiag) {
        S->shift = 0.0;
        if ((e = launch_sell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, NC_F64, 0.0, S->sell_col,
                                  S->sell_val64, nullptr, st))) {
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
    }
    S->op64 = OpView{OP_SELL, n, S->sell_ptr, S->sell_col, S->sell_val64, NC_F64};
    S->opP = S->op64;
    S->h_sell_ptr = hp32;
    if (S->mixed) {
        NC_TRY(dev_alloc(&S->sell_valP, eb * (size_t)total));
        if ((e = launch_sell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->vdt, S->shift, S->sell_col,
                                  S->sell_valP, nullptr, st))) {
            g_last_cuda = e;
            return NC_ERR_CUDA;
        }
        S->opP = OpView{OP_SELL, n, S->sell_ptr, S->sell_col, S->sell_valP, S->vdt};
    }
    // the host vector hp32 must outlive the copy
    if ((e = cudaStreamSynchronize(st))) { g_last_cuda = e; return NC_ERR_CUDA; }
    if (S->opt.spmv_format == NC_FORMAT_TUNE) {
        // measure both layouts on this matrix and keep the faster
        NC_TRY(time_step(S, csrP, false, st, &S->tune_us[0]));
        NC_TRY(time_step(S, S->opP, S->shift != 0.0, st, &S->tune_us[1]));
        if (S->tune_us[0] < S->tune_us[1]) {
            dev_free(S->sell_ptr); dev_free(S->sell_col); dev_free(S->sell_val64); dev_free(S->sell_valP);
            S->sell_ptr = nullptr; S->sell_col = nullptr; S->sell_val64 = nullptr; S->sell_valP = nullptr;
            S->padding = 1.0;
            S->shift = 0.0;
            S->op64 = csr64;
            S->opP = csrP;
        } else if (S->lval) {
            dev_free(S->lval);
            S->lval = nullptr;
        }
    }
    return NC_OK;
}

// ---- step-kernel variant and launch shape ----------------------------------
// The fused step of the offset-pattern layout has two variants (direct loads,
// or tiles staged in shared memory by bulk copies) and launch parameters
// whose best values depend on the operator's size, row length and value
// type.  NC_STEP_TUNE (and AUTO on large PSELL operators) measures a small
// candidate set on the solver's own operator and buffers and keeps the
// fastest; every measurement is kept for pcg_tune_candidate.

namespace {

constexpr int64_t kTuneMinRows = (int64_t)1 << 16;   // AUTO tunes PSELL operators of at least this many rows

// Mean duration (us) of `reps` launches after two warm-up launches.
template <typename F>
nc_status time_launches(cudaStream_t st, F launch, double* us) {
    for (int i = 0; i < 2; ++i) NC_CU(launch());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NC_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e) { cudaEventDestroy(e0); g_last_cuda = e; return NC_ERR_CUDA; }
    const int reps = 20;
    e = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) { g_last_cuda = e; return NC_ERR_CUDA; }
    *us = 1e3 * (double)ms / reps;
    return NC_OK;
}

// One launch of the step kind the solve runs: 0 = a Chebyshev step inside
// P_k (x_{k-1}, x_{k-2} and r terms; in float64 the unit product coefficient
// of the scaled iterates), 1 = the last step with (r, z), 2 = q = A p with
// (p, q) on the float64 operator.
cudaError_t launch_kind(nc_solver S, const OpView& op, int kind, cudaStream_t st) {
    const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
    const double cd = S->mixed ? -1.0 : 1.0;
    const void* rx = S->mixed ? static_cast<const void*>(S->r32) : static_cast<const void*>(S->r);
    if (kind == 0)
        return op_step(op, S->mixed, !S->mixed, S->buf[0], S->buf[1], rx, S->buf[2], 0.0, -0.25, 0.1, cd, 0, nullptr,
                       none, nullptr, st);
    if (kind == 1)
        return op_step(op, S->mixed, true, S->buf[0], S->buf[1], rx, S->z, 0.0, -0.25, 0.1, cd, 1, S->r, none, nullptr,
                       st);
    return op_step(op, false, true, S->p, nullptr, nullptr, S->q, S->shift, 0.0, 0.0, 1.0, 2, nullptr, none, nullptr,
                   st);
}

nc_status tune_kind(nc_solver S, OpView& op, int kind, cudaStream_t st) {
    const bool x_f32 = S->mixed && kind != 2;
    const bool y_f64 = !x_f32 || kind == 1;
    const int vdt = kind == 2 ? NC_F64 : op.vdt;
    const int dot = kind == 0 ? 0 : (kind == 1 ? 1 : 2);
    const bool unit = !x_f32;
    std::vector<StepTune> cands;
    StepTune base = op.tune;
    auto with_variant = [&](StepTune t, int v) {
        if (kind == 0) t.variant = v;
        else t.dot_variant = v;
        return t;
    };
    {   // direct loads: L2 prefetch distance (float) and rows per thread
        // for the plain step, persistent CTAs per SM for the dot steps
        StepTune t = with_variant(base, STEP_DIRECT);
        t.lookahead = -1;
        t.red_ctas_per_sm = kCtasPerSm;
        if (kind == 0) {
            for (int rpt = 1; rpt <= 2; ++rpt) {
                t.rpt = rpt;
                t.lookahead = -1;
                cands.push_back(t);
                if (x_f32) {
                    t.lookahead = 0;
                    cands.push_back(t);
                }
            }
        } else {
            // persistent grids of 4 to 8 CTAs per SM (the float64 dot
            // kernels hold 6 per SM: 8 leaves a second, partial wave), or
            // one 256-row tile per CTA (a grid as large as the tile count)
            for (int red : {4, 5, 6, 8, kRedOneTile}) {
                t.red_ctas_per_sm = red;
                cands.push_back(t);
            }
            // or the plain step (as chosen for it) and a separate dot product
            StepTune s = with_variant(base, STEP_SPLIT);
            cands.push_back(s);
        }
    }
    // staged: (stages, CTAs per SM, rows per thread, tile order); a shape the
    // device cannot hold or that repeats another after the occupancy cap is skipped
    std::vector<std::array<int, 4>> seen;
    // (the contiguous tile order measured slower on every operator tried: not a candidate)
    for (int rpt = 1; rpt <= 2; ++rpt)
        for (int contig = 0; contig <= 0; ++contig)
            for (int stages = 2; stages <= 3; ++stages)
                for (int ctas : {4, 6, 8}) {
                    StepTune t = with_variant(base, STEP_STAGED);
                    if (kind == 0) {
                        t.stages = stages;
                        t.ctas_per_sm = ctas;
                        t.rpt = rpt;
                        t.contig = contig;
                    } else {
                        t.dot_stages = stages;
                        t.dot_ctas_per_sm = ctas;
                        t.dot_rpt = rpt;
                        t.dot_contig = contig;
                    }
                    const int got = sell_staged_ctas(vdt, x_f32, y_f64, dot, unit, t);
                    const std::array<int, 4> key{stages, got, rpt, contig};
                    if (got <= 0 || std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
                    seen.push_back(key);
                    if (kind == 0) t.ctas_per_sm = got;
                    else t.dot_ctas_per_sm = got;
                    cands.push_back(t);
                }
    double best = 0.0;
    int ibest = -1;
    const size_t first = S->tune.size();
    // two passes over the candidates, the second in reverse order; each keeps
    // the lower of its two means (a transient slowdown during one
    // measurement does not decide the choice)
    std::vector<double> tus(cands.size(), 0.0);
    for (int pass = 0; pass < 2; ++pass)
        for (size_t ii = 0; ii < cands.size(); ++ii) {
            const size_t ci = pass == 0 ? ii : cands.size() - 1 - ii;
            OpView v = op;
            v.tune = cands[ci];
            double us = 0.0;
            NC_TRY(time_launches(st, [&]() { return launch_kind(S, v, kind, st); }, &us));
            tus[ci] = pass == 0 ? us : std::min(tus[ci], us);
        }
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const StepTune& t = cands[ci];
        const double us = tus[ci];
        const int var = kind == 0 ? t.variant : t.dot_variant;
        S->tune.push_back(TuneRec{kind, var, kind == 0 ? t.stages : t.dot_stages,
                                  kind == 0 ? t.ctas_per_sm : t.dot_ctas_per_sm, kind == 0 ? t.rpt : t.dot_rpt,
                                  kind == 0 ? t.contig : t.dot_contig, t.lookahead, t.red_ctas_per_sm, us, 0});
        if (ibest < 0 || us < best) {
            best = us;
            ibest = (int)(S->tune.size() - 1);
        }
    }
    // a staged kernel whose wait ran out during the measurements is not kept
    int fault = 0;
    NC_CU(cudaMemcpyAsync(&fault, &S->S->fault, sizeof(int), cudaMemcpyDeviceToHost, st));
    NC_CU(cudaStreamSynchronize(st));
    if (fault) {
        NC_CU(cudaMemsetAsync(&S->S->fault, 0, sizeof(int), st));
        ibest = (int)first;   // the direct default
    }
    if (ibest < 0) return NC_OK;
    TuneRec& b = S->tune[(size_t)ibest];
    b.chosen = 1;
    if (kind == 0) {
        op.tune.variant = b.variant;
        op.tune.rpt = b.rpt;
        if (b.variant == STEP_DIRECT) op.tune.lookahead = b.lookahead;
        else {
            op.tune.stages = b.stages;
            op.tune.ctas_per_sm = b.ctas_per_sm;
            op.tune.rpt = b.rpt;
            op.tune.contig = b.contig;
        }
    } else {
        op.tune.dot_variant = b.variant;
        if (b.variant == STEP_DIRECT) op.tune.red_ctas_per_sm = b.red_ctas_per_sm;
        else {
            op.tune.dot_stages = b.stages;
            op.tune.dot_ctas_per_sm = b.ctas_per_sm;
            op.tune.dot_rpt = b.rpt;
            op.tune.dot_contig = b.contig;
        }
    }
    return NC_OK;
}

constexpr int64_t kStencilTuneMinPoints = (int64_t)1 << 20;   // AUTO tunes stencils of at least this size

// Matrix-free stencil: the z-chunk of the plain steps (planes per CTA; more
// chunks fill the GPU, longer ones read fewer extra planes) and, in float,
// the planes per z-march batch.  Candidates around the size policy.
nc_status tune_stencil(nc_solver S, OpView& op, cudaStream_t st) {
    const int nz = op.geom.nz;
    const int pol = stencil_zchunk_policy(op.geom);
    std::vector<int> zcs;
    for (int z : {pol, pol / 2, 2 * pol, 32, 64, 128, 256}) {
        z = std::min(z, nz);
        if (z >= 4 && std::find(zcs.begin(), zcs.end(), z) == zcs.end()) zcs.push_back(z);
    }
    if (zcs.empty()) return NC_OK;
    std::vector<int> pzs = S->mixed ? std::vector<int>{2, 4} : std::vector<int>{2};
    double best = 0.0;
    int ibest = -1;
    for (int zc : zcs)
        for (int pz : pzs) {
            OpView v = op;
            v.geom.zc = zc;
            v.geom.pz = pz;
            double us = 0.0;
            NC_TRY(time_launches(st, [&]() { return launch_kind(S, v, 0, st); }, &us));
            TuneRec rec{0, STEP_DIRECT, 0, 0, 1, 0, 0, 0, us, 0};
            rec.zchunk = zc;
            rec.pz = pz;
            S->tune.push_back(rec);
            if (ibest < 0 || us < best) {
                best = us;
                ibest = (int)S->tune.size() - 1;
            }
        }
    TuneRec& b = S->tune[(size_t)ibest];
    b.chosen = 1;
    op.geom.zc = b.zchunk;
    op.geom.pz = b.pz;
    return NC_OK;
}

}  // namespace

// Persistent tuner choices.  When the environment variable NC_TUNE_CACHE
// names a text file, a solver that would be tuned first looks for its
// operator's signature there (rows, stored entries, offset sets, table
// size, apply precision, SM count and compute capability) and takes the
// recorded choices without measuring; otherwise it measures and appends one
// line.  Each line is written by one append, so processes sharing the file
// do not interleave lines.  (Timings taken under a profiler mislead the
// tuner; a cache written by an unprofiled run makes the profiled process
// run what the unprofiled one ran.)
constexpr int kTuneFields = 12;

void tune_to_ints(const StepTune& t, int* v) {
    const int f[kTuneFields] = {t.variant,     t.rpt,         t.stages,    t.ctas_per_sm,     t.contig,
                                t.lookahead,   t.dot_variant, t.dot_rpt,   t.dot_stages,      t.dot_ctas_per_sm,
                                t.dot_contig,  t.red_ctas_per_sm};
    for (int i = 0; i < kTuneFields; ++i) v[i] = f[i];
}

void tune_from_ints(const int* v, StepTune& t) {
    t.variant = v[0];
    t.rpt = v[1];
    t.stages = v[2];
    t.ctas_per_sm = v[3];
    t.contig = v[4];
    t.lookahead = v[5];
    t.dot_variant = v[6];
    t.dot_rpt = v[7];
    t.dot_stages = v[8];
    t.dot_ctas_per_sm = v[9];
    t.dot_contig = v[10];
    t.red_ctas_per_sm = v[11];
}

bool tune_ints_valid(const int* v) {
    auto var = [](int x) { return x == STEP_DIRECT || x == STEP_STAGED; };
    return var(v[0]) && v[1] >= 1 && v[1] <= 2 && v[2] >= 2 && v[2] <= 4 && v[3] >= 1 && v[3] <= 8 &&
           (v[4] == 0 || v[4] == 1) && v[5] >= -1 && (var(v[6]) || v[6] == STEP_SPLIT) && v[7] >= 1 && v[7] <= 2 && v[8] >= 2 &&
           v[8] <= 4 && v[9] >= 1 && v[9] <= 8 && (v[10] == 0 || v[10] == 1) && v[11] >= 1 &&
           v[11] <= kRedOneTile;
}

std::string tune_key(nc_solver S) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaGetLastError();
    char buf[256];
    std::snprintf(buf, sizeof(buf), "ncpcg-tune-v1 n=%lld e=%lld p=%lld o=%d dt=%d sm=%d cc=%d%d", (long long)S->n,
                  (long long)(S->h_sell_ptr.empty() ? 0 : S->h_sell_ptr.back()), (long long)S->npatterns,
                  S->opP.tune.npoff, S->vdt, S->num_sms, major, minor);
    return std::string(buf);
}

// true when the cache held this operator's choices (applied to opP, op64)
bool tune_cache_load(nc_solver S, const char* path) {
    std::FILE* f = std::fopen(path, "r");
    if (!f) return false;
    const std::string key = tune_key(S) + " |";
    char line[1024];
    bool found = false;
    while (!found && std::fgets(line, sizeof(line), f)) {
        if (std::strncmp(line, key.c_str(), key.size()) != 0) continue;
        int a[kTuneFields], b[kTuneFields];
        const char* q = line + key.size();
        int used = 0;
        bool ok = std::sscanf(q, " P%n", &used) >= 0 && used > 0;
        q += used;
        for (int i = 0; ok && i < kTuneFields; ++i) {
            ok = std::sscanf(q, "%d%n", &a[i], &used) == 1;
            q += used;
        }
        used = 0;
        ok = ok && std::sscanf(q, " | D%n", &used) >= 0 && used > 0;
        q += used;
        for (int i = 0; ok && i < kTuneFields; ++i) {
            ok = std::sscanf(q, "%d%n", &b[i], &used) == 1;
            q += used;
        }
        if (ok && tune_ints_valid(a) && tune_ints_valid(b)) {
            tune_from_ints(a, S->opP.tune);
            tune_from_ints(b, S->op64.tune);
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(nc_solver S, const char* path) {
    int a[kTuneFields], b[kTuneFields];
    tune_to_ints(S->opP.tune, a);
    tune_to_ints(S->op64.tune, b);
    std::string line = tune_key(S) + " | P";
    for (int v : a) line += " " + std::to_string(v);
    line += " | D";
    for (int v : b) line += " " + std::to_string(v);
    line += "\n";
    std::FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fputs(line.c_str(), f);
    std::fclose(f);
}

nc_status setup_step_kernels(nc_solver S, cudaStream_t st) {
    const nc_options& o = S->opt;
    StepTune t;
    t.lookahead = o.prefetch_tiles == 0 ? -1 : (o.prefetch_tiles < 0 ? 0 : o.prefetch_tiles);
    t.red_ctas_per_sm = o.red_ctas_per_sm > 0 ? o.red_ctas_per_sm : kCtasPerSm;
    t.stages = t.dot_stages = o.step_stages > 0 ? o.step_stages : 2;
    t.ctas_per_sm = t.dot_ctas_per_sm = o.step_ctas_per_sm > 0 ? o.step_ctas_per_sm : 6;
    t.rpt = t.dot_rpt = o.step_rows_per_thread > 0 ? o.step_rows_per_thread : 1;
    t.contig = t.dot_contig = o.step_tile_order == 1 ? 1 : 0;
    const bool psell = S->opP.kind == OP_SELL && S->opP.pat.pstart != nullptr;
    const int mode = o.step_kernel;
    if (mode == NC_STEP_STAGED) t.variant = t.dot_variant = STEP_STAGED;
    if (mode == NC_STEP_SPLIT) t.dot_variant = STEP_SPLIT;
    for (OpView* op : {&S->op64, &S->opP}) {
        const int vcap = op->tune.vcap, vcap2 = op->tune.vcap2, npoff = op->tune.npoff;
        op->tune = t;
        op->tune.vcap = vcap;
        op->tune.vcap2 = vcap2;
        op->tune.npoff = npoff;
    }
    if (S->opP.kind == OP_STENCIL &&
        (mode == NC_STEP_TUNE || (mode == NC_STEP_AUTO && S->n >= kStencilTuneMinPoints))) {
        const size_t vb = S->mixed ? sizeof(float) : sizeof(double);
        for (int i = 0; i < 3; ++i) NC_CU(cudaMemsetAsync(S->buf[i], 0, vb * (size_t)S->n, st));
        NC_CU(cudaMemsetAsync(S->r, 0, sizeof(double) * (size_t)S->n, st));
        if (S->mixed) NC_CU(cudaMemsetAsync(S->r32, 0, sizeof(float) * (size_t)S->n, st));
        return tune_stencil(S, S->opP, st);
    }
    const bool tune = psell && (mode == NC_STEP_TUNE || (mode == NC_STEP_AUTO && S->n >= kTuneMinRows));
    if (!tune) return NC_OK;
    const char* cache = std::getenv("NC_TUNE_CACHE");
    if (cache != nullptr && cache[0] != '\0' && tune_cache_load(S, cache)) {
        S->tune_cached = true;
        return NC_OK;
    }
    // the buffers the measured launches read and write start at zero
    const size_t vb = S->mixed ? sizeof(float) : sizeof(double);
    const size_t n = (size_t)S->n;
    for (int i = 0; i < 3; ++i) NC_CU(cudaMemsetAsync(S->buf[i], 0, vb * n, st));
    for (double* p : {S->r, S->z, S->p, S->q}) NC_CU(cudaMemsetAsync(p, 0, sizeof(double) * n, st));
    if (S->mixed) NC_CU(cudaMemsetAsync(S->r32, 0, sizeof(float) * n, st));
    NC_TRY(tune_kind(S, S->opP, 0, st));
    NC_TRY(tune_kind(S, S->opP, 1, st));
    if (S->mixed) {
        NC_TRY(tune_kind(S, S->op64, 2, st));
    } else {
        S->op64.tune = S->opP.tune;   // the same operator: q = A p takes the dot-step choice
    }
    if (cache != nullptr && cache[0] != '\0') tune_cache_store(S, cache);
    return NC_OK;
}

}  // namespace nc
