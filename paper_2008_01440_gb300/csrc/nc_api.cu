// C ABI of libncpcg: options, status strings and the pcg_* entry points
// (declarations and contracts in include/nc_pcg.h).  The solver machinery
// lives in nc_solve.cu, nc_solve_multi.cu and nc_setup.cu, the matrix
// handles in nc_matrix.cu.
#include "nc_internal.h"

using namespace nc;

extern "C" {

void nc_options_default(nc_options* opt) {
    if (!opt) return;
    opt->apply_dtype = NC_F64;
    opt->rr_period = 0;
    opt->x0_is_zero = 0;
    opt->use_graph = 1;
    opt->spmv_format = NC_FORMAT_AUTO;
    opt->poly_form = NC_POLY_CHEBYSHEV;
    opt->step_kernel = NC_STEP_AUTO;
    opt->step_stages = 0;
    opt->step_ctas_per_sm = 0;
    opt->step_rows_per_thread = 0;
    opt->step_tile_order = 0;
    opt->prefetch_tiles = 0;
    opt->red_ctas_per_sm = 0;
    opt->keep_diagonal = 0;
}

const char* nc_strerror(nc_status s) {
    switch (s) {
    case NC_OK: return "ok";
    case NC_ERR_ARG: return "invalid argument";
    case NC_ERR_CUDA: return "CUDA runtime error";
    case NC_ERR_OOM: return "device out of memory";
    case NC_ERR_INDEFINITE: return "indefinite operator or preconditioner ((p,Ap) or (r,z) <= 0)";
    case NC_ERR_MAXIT: return "maximum iterations reached";
    case NC_ERR_BREAKDOWN: return "NaN or Inf in a reduction";
    case NC_ERR_UNSUPPORTED: return "unsupported option for this matrix format";
    case NC_ERR_SCRATCH_LIMIT: return "n exceeds the fixed scratch array of the no-allocation apply";
    case NC_ERR_ADMISSION: return "batch engine: no free slot or not enough pooled memory";
    case NC_ERR_TIMEOUT: return "a staged step kernel's bounded wait for its copies ran out (results invalid)";
    }
    return "unknown status";
}

const char* nc_version(void) { return "ncpcg 0.1 (sm_103a)"; }

const char* nc_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }


nc_status pcg_destroy(nc_solver S);

nc_status pcg_setup(nc_matrix A, double lambda_min, double lambda_max, int degree_k, double theta_scale,
                    const nc_options* opt, void* stream, nc_solver* out) {
    if (!out) return NC_ERR_ARG;
    *out = nullptr;
    if (!A || !(lambda_min > 0.0) || !(lambda_max > lambda_min) || !std::isfinite(lambda_max) ||
        degree_k < 0 || degree_k > 4096 || !(theta_scale > 0.0) || !std::isfinite(theta_scale))
        return NC_ERR_ARG;
    nc_options o;
    nc_options_default(&o);
    if (opt) o = *opt;
    if (o.apply_dtype != NC_F64 && o.apply_dtype != NC_F32 && o.apply_dtype != NC_BF16) return NC_ERR_ARG;
    if (o.rr_period < 0) return NC_ERR_ARG;
    if (o.spmv_format < NC_FORMAT_AUTO || o.spmv_format > NC_FORMAT_PSELL) return NC_ERR_ARG;
    if (o.step_kernel < NC_STEP_AUTO || o.step_kernel > NC_STEP_SPLIT || o.step_stages < 0 || o.step_stages > 4 ||
        o.step_stages == 1 || o.step_ctas_per_sm < 0 || o.step_ctas_per_sm > 8 || o.red_ctas_per_sm < 0 ||
        o.red_ctas_per_sm > 64 || o.step_rows_per_thread < 0 || o.step_rows_per_thread > 2 ||
        o.step_tile_order < 0 || o.step_tile_order > 1)
        return NC_ERR_ARG;
    int nlev = -1;
    if (o.poly_form == NC_POLY_NEWTON) {
        // Algorithm 1 builds P of degree 2^nlev - 1 only; float64 only
        for (int L = 0; L <= 12; ++L)
            if ((1 << L) - 1 == degree_k) nlev = L;
        if (nlev < 0) return NC_ERR_ARG;
        if (o.apply_dtype != NC_F64) return NC_ERR_UNSUPPORTED;
    } else if (o.poly_form != NC_POLY_CHEBYSHEV) {
        return NC_ERR_ARG;
    }
    cudaStream_t st = as_stream(stream);
    nc_solver S = new (std::nothrow) nc_solver_s();
    if (!S) return NC_ERR_OOM;
    S->A = A;
    S->n = A->n;
    S->k = degree_k;
    S->s = theta_scale;
    S->lmin = lambda_min;
    S->lmax = lambda_max;
    S->opt = o;
    S->num_sms = num_sms();
    S->mixed = o.apply_dtype != NC_F64;
    S->vdt = o.apply_dtype;
    setup_coefficients(S);
    if (nlev >= 0) {
        // zeta_0..zeta_nlev (Eq. zetaNewt) on the interval of the scaled
        // Chebyshev polynomial, [theta' - delta, theta' + delta] (Sec. 4)
        S->nlev = nlev;
        S->zeta.assign(nlev + 1, 0.0);
        const double a0 = S->theta - S->delta, b0 = S->theta + S->delta;
        S->zeta[0] = 2.0 / (a0 + b0);
        if (nlev >= 1) {
            const double a = a0 * S->zeta[0];
            S->zeta[1] = 2.0 / (1.0 + 2.0 * a - a * a);
        }
        for (int i = 2; i <= nlev; ++i) S->zeta[i] = 2.0 / (1.0 + 2.0 * S->zeta[i - 1] - S->zeta[i - 1] * S->zeta[i - 1]);
    }
    const int64_t n = S->n;
    nc_status s = NC_OK;
    do {
        if ((s = dev_alloc_n(&S->b, n)) || (s = dev_alloc_n(&S->x, n)) || (s = dev_alloc_n(&S->r, n)) ||
            (s = dev_alloc_n(&S->z, n)) || (s = dev_alloc_n(&S->p, n)) || (s = dev_alloc_n(&S->q, n)) ||
            (s = dev_alloc_n(&S->partials, partials_for(A))) || (s = dev_alloc_n(&S->counter, 1)) ||
            (s = dev_alloc_n(&S->S, 1)))
            break;
        const size_t vb = S->mixed ? sizeof(float) : sizeof(double);
        for (int i = 0; i < 3 && s == NC_OK; ++i) s = dev_alloc(&S->buf[i], vb * (size_t)(n > 0 ? n : 1));
        if (s) break;
        if (S->mixed && (s = dev_alloc_n(&S->r32, n))) break;
        if (S->nlev >= 2) {
            S->nbuf.assign(2 * (S->nlev - 1), nullptr);
            for (auto& bp : S->nbuf)
                if ((s = dev_alloc_n(&bp, n > 0 ? n : 1))) break;
            if (s) break;
        }
        if ((s = setup_operator(S, st)) != NC_OK) break;
        cudaError_t e;
        if ((e = cudaMemsetAsync(S->counter, 0, sizeof(unsigned int), st)) ||
            (e = cudaMemsetAsync(S->S, 0, sizeof(PcgScalars), st))) {
            g_last_cuda = e; s = NC_ERR_CUDA; break;
        }
        if ((e = cudaMallocHost(&S->h_io, sizeof(PcgScalars)))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
        if ((s = setup_step_kernels(S, st)) != NC_OK) break;
        if ((e = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
        if (o.use_graph == 2 && S->op64.kind == OP_SELL && S->op64.pat.pstart == nullptr && !S->mixed &&
            o.rr_period == 0 && S->nlev < 0 &&
            plan_cluster_pcg(n, S->h_sell_ptr.data(), &S->plan)) {
            // one-cluster solve: per-step coefficients of the shifted operator
            std::vector<double> cf(4 * (size_t)(S->k + 1), 0.0);
            if (S->k == 0) cf[0] = 1.0 / S->theta;
            const std::vector<StepC> sc = step_coefs(S, true);
            for (int j = 1; j <= S->k; ++j) {
                cf[4 * j] = sc[j].ca;
                cf[4 * j + 1] = sc[j].cb;
                cf[4 * j + 2] = sc[j].cc;
                cf[4 * j + 3] = sc[j].cd;
            }
            if ((s = dev_alloc_n(&S->pcoef, (int64_t)cf.size()))) break;
            if ((e = cudaMemcpyAsync(S->pcoef, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice, st)) ||
                (e = cudaStreamSynchronize(st))) {
                g_last_cuda = e; s = NC_ERR_CUDA; break;
            }
            S->persistent = true;
        }
        if ((e = cudaStreamSynchronize(st))) { g_last_cuda = e; s = NC_ERR_CUDA; break; }
    } while (0);
    if (s != NC_OK) {
        pcg_destroy(S);
        return s;
    }
    *out = S;
    return NC_OK;
}

nc_status pcg_apply_poly(nc_solver S, const double* v_dev, double* z_dev, void* stream) {
    if (!S || (S->n > 0 && (!v_dev || !z_dev)) || v_dev == z_dev) return NC_ERR_ARG;
    if (S->n == 0) return NC_OK;
    cudaStream_t st = as_stream(stream);
    if (S->mixed) NC_CU(launch_convert(S->n, v_dev, NC_F32, S->r32, st));
    NC_CU(enqueue_poly(S, v_dev, z_dev, FIN_NONE, nullptr, st));
    return NC_OK;
}

nc_status pcg_solve(nc_solver S, const double* b_dev, double* x_dev, double tol, int maxit, void* stream,
                    nc_result* res) {
    if (!S || !(tol >= 0.0) || maxit < 0) return NC_ERR_ARG;
    if (S->n == 0) {
        if (res) *res = nc_result{0, NC_OK, 0.0, 0.0, 0, 0, 0};
        return NC_OK;
    }
    if (!b_dev || !x_dev || b_dev == x_dev) return NC_ERR_ARG;
    return run_solve(S, b_dev, x_dev, tol, maxit, as_stream(stream), res);
}

nc_status pcg_solve_multi(nc_solver S, int m, const double* B_dev, double* X_dev, double tol, int maxit,
                          void* stream, nc_result* res) {
    if (!S || !(tol >= 0.0) || maxit < 0 || m < 1 || m > max_rhs() || !res) return NC_ERR_ARG;
    if (S->n == 0) {
        for (int c = 0; c < m; ++c) res[c] = nc_result{0, NC_OK, 0.0, 0.0, 0, 0, 0};
        return NC_OK;
    }
    if (!B_dev || !X_dev || B_dev == X_dev) return NC_ERR_ARG;
    if (S->op64.kind != OP_SELL || S->opP.kind != OP_SELL || S->opt.rr_period > 0 || S->nlev >= 0)
        return NC_ERR_UNSUPPORTED;
    NC_TRY(mreserve(S, m));
    cudaStream_t st = as_stream(stream);
    const int n = (int)S->n;
    const size_t cn = (size_t)n;
    for (int c = 0; c < m; ++c) {
        PcgScalars init;
        std::memset(&init, 0, sizeof(init));
        init.tol2 = tol * tol;
        init.maxit = maxit;
        init.status = NC_ERR_MAXIT;
        init.rr_skip = 1;
        S->mh[c] = init;
    }
    NC_CU(cudaMemcpyAsync(S->mS, S->mh, sizeof(PcgScalars) * m, cudaMemcpyHostToDevice, st));
    for (int c = 0; c < m; ++c)
        NC_CU(mat_copy_in(S->A, B_dev + c * cn, X_dev + c * cn, S->opt.x0_is_zero,
                             S->mb + c * cn, S->mx + c * cn, st));
    bool graph = S->opt.use_graph && !S->mgraph_failed;
    if (graph && (S->mexec == nullptr || S->mexec_m != m) && mbuild_graph(S, m) != NC_OK) {
        S->mgraph_failed = true;
        graph = false;
    }
    if (graph) {
        NC_CU(cudaGraphLaunch(S->mexec, st));
    } else {
        int* active = reinterpret_cast<int*>(&S->mS[0].pad1);   // scratch word of column 0's block
        int h_active = 1;
        NC_CU(menqueue_prologue(S, m, st));
        for (;;) {
            NC_CU(menqueue_body(S, m, 0, 0, active, st));
            NC_CU(cudaMemcpyAsync(&h_active, active, sizeof(int), cudaMemcpyDeviceToHost, st));
            NC_CU(cudaStreamSynchronize(st));
            if (!h_active) break;
        }
    }
    const Reduce none = make_reduce(S->partials, S->counter, S->mS, nullptr, FIN_NONE);
    for (int c = 0; c < m; ++c) {
        NC_CU(op64_apply(S, S->mx + c * cn, S->mb + c * cn, S->mq + c * cn, 1.0, -1.0, 0, none, nullptr, st));
        NC_CU(launch_dot(n, S->mq + c * cn, S->mq + c * cn,
                         make_reduce(S->partials, S->counter, S->mS + c, nullptr, FIN_TRUE), nullptr, st));
        NC_CU(mat_copy_out(S->A, S->mx + c * cn, S->mS + c, X_dev + c * cn, st));
    }
    NC_CU(cudaMemcpyAsync(S->mh, S->mS, sizeof(PcgScalars) * m, cudaMemcpyDeviceToHost, st));
    NC_CU(cudaStreamSynchronize(st));
    nc_status first = NC_OK;
    for (int c = 0; c < m; ++c) {
        const PcgScalars& o = S->mh[c];
        const double bn = std::sqrt(o.bb);
        res[c].iters = o.iter;
        res[c].status = o.status;
        res[c].relres = bn > 0 ? std::sqrt(o.rr) / bn : 0.0;
        res[c].true_relres = bn > 0 ? std::sqrt(o.rr_true) / bn : 0.0;
        res[c].n_dot = o.n_dot;
        res[c].n_spmv = (int64_t)o.iter + (int64_t)S->k * o.n_prec;
        res[c].n_replace = 0;
        if (first == NC_OK && o.status != NC_OK) first = (nc_status)o.status;
    }
    return first;
}

nc_status pcg_solve_host(nc_solver S, const double* b_host, double* x_host, double tol, int maxit,
                         void* stream, nc_result* res) {
    if (!S || !(tol >= 0.0) || maxit < 0) return NC_ERR_ARG;
    if (S->n == 0) {
        if (res) *res = nc_result{0, NC_OK, 0.0, 0.0, 0, 0, 0};
        return NC_OK;
    }
    if (!b_host || !x_host) return NC_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    const size_t bytes = sizeof(double) * (size_t)S->n;
    // stage b in q and x0 in z (both are rewritten by the solve before use)
    NC_CU(cudaMemcpyAsync(S->q, b_host, bytes, cudaMemcpyHostToDevice, st));
    if (!S->opt.x0_is_zero) NC_CU(cudaMemcpyAsync(S->z, x_host, bytes, cudaMemcpyHostToDevice, st));
    // copy_in reads the staged vectors before any kernel of the solve writes q or z
    nc_status s = run_solve(S, S->q, S->z, tol, maxit, st, res);
    if (s == NC_ERR_CUDA || s == NC_ERR_ARG) return s;
    NC_CU(cudaMemcpyAsync(x_host, S->z, bytes, cudaMemcpyDeviceToHost, st));
    NC_CU(cudaStreamSynchronize(st));
    return s;
}

nc_status pcg_get_info(nc_solver S, nc_solver_info* info) {
    if (!S || !info) return NC_ERR_ARG;
    info->n = S->n;
    info->degree_k = S->k;
    info->spmv_format = (S->op64.kind == OP_SELL || S->op64.kind == OP_BSELL3) ? NC_FORMAT_SELL : NC_FORMAT_CSR;
    if (S->op64.pat.pstart != nullptr) info->spmv_format = NC_FORMAT_PSELL;
    info->patterns = S->npatterns;
    info->apply_dtype = S->vdt;
    info->persistent = S->persistent ? 1 : 0;
    info->padding = S->padding;
    info->theta = S->theta;
    info->delta = S->delta;
    info->sigma = S->sigma;
    info->shift = S->shift;
    info->tune_us_plain = S->tune_us[0];
    info->tune_us_sliced = S->tune_us[1];
    const StepTune& tp = S->opP.tune;
    info->step_kernel = tp.variant == STEP_STAGED ? NC_STEP_STAGED : NC_STEP_DIRECT;
    info->dot_step_kernel = tp.dot_variant == STEP_STAGED ? NC_STEP_STAGED
                          : (tp.dot_variant == STEP_SPLIT ? NC_STEP_SPLIT : NC_STEP_DIRECT);
    info->step_stages = tp.stages;
    info->step_ctas_per_sm = tp.ctas_per_sm;
    info->step_rows_per_thread = tp.rpt;
    info->step_tile_order = tp.contig;
    info->dot_step_stages = tp.dot_stages;
    info->dot_step_ctas_per_sm = tp.dot_ctas_per_sm;
    info->dot_step_rows_per_thread = tp.dot_rpt;
    info->dot_step_tile_order = tp.dot_contig;
    info->prefetch_tiles = tp.lookahead < 0 ? 2 * S->num_sms : tp.lookahead;
    info->red_ctas_per_sm = tp.red_ctas_per_sm;
    info->tune_candidates = (int32_t)S->tune.size();
    info->num_sms = S->num_sms;
    info->faults = 0;
    info->tune_from_cache = S->tune_cached ? 1 : 0;
    info->stencil_zchunk = S->opP.kind == OP_STENCIL ? stencil_zchunk(S->opP.geom) : 0;
    info->stencil_planes_per_batch = S->opP.geom.pz;
    info->diag_folded = S->op64.dfolded;
    info->diag_value = S->op64.dfold;
    if (S->S) {
        int f = 0;
        if (cudaMemcpy(&f, &S->S->fault, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            g_last_cuda = cudaGetLastError();
            return NC_ERR_CUDA;
        }
        info->faults = f;
    }
    return NC_OK;
}

nc_status pcg_tune_candidate(nc_solver S, int i, nc_tune_candidate* out) {
    if (!S || !out || i < 0 || i >= (int)S->tune.size()) return NC_ERR_ARG;
    const TuneRec& t = S->tune[(size_t)i];
    out->op = t.op;
    out->step_kernel = t.variant == STEP_STAGED ? NC_STEP_STAGED
                     : (t.variant == STEP_SPLIT ? NC_STEP_SPLIT : NC_STEP_DIRECT);
    out->stages = t.stages;
    out->ctas_per_sm = t.ctas_per_sm;
    out->rows_per_thread = t.rpt;
    out->tile_order = t.contig;
    out->zchunk = t.zchunk;
    out->planes_per_batch = t.pz;
    out->prefetch_tiles = t.lookahead;
    out->red_ctas_per_sm = t.red_ctas_per_sm;
    out->us = t.us;
    out->chosen = t.chosen;
    out->reserved0 = 0;
    return NC_OK;
}

nc_status pcg_destroy(nc_solver S) {
    if (!S) return NC_ERR_ARG;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->cap) cudaStreamDestroy(S->cap);
    dev_free(S->b); dev_free(S->x); dev_free(S->r); dev_free(S->z); dev_free(S->p); dev_free(S->q);
    for (int i = 0; i < 3; ++i) dev_free(S->buf[i]);
    dev_free(S->r32); dev_free(S->lval); dev_free(S->partials); dev_free(S->counter); dev_free(S->S);
    dev_free(S->sell_ptr); dev_free(S->sell_col); dev_free(S->sell_val64); dev_free(S->sell_valP);
    dev_free(S->psell_start); dev_free(S->psell_off);
    dev_free(S->pcoef);
    for (double* bp : S->nbuf) dev_free(bp);
    if (S->mexec) cudaGraphExecDestroy(S->mexec);
    dev_free(S->mb); dev_free(S->mx); dev_free(S->mr); dev_free(S->mz); dev_free(S->mp); dev_free(S->mq);
    for (void* bp : S->mbuf) dev_free(bp);
    dev_free(S->mr32); dev_free(S->mS);
    if (S->mh) cudaFreeHost(S->mh);
    if (S->h_io) cudaFreeHost(S->h_io);
    delete S;
    return NC_OK;
}

}  // extern "C"

