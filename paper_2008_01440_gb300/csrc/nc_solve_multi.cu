// Several right-hand sides sharing one solver's matrix (pcg_solve_multi).
#include "nc_internal.h"

namespace nc {

// ---- several right-hand sides sharing the matrix ----------------------------
// m PCG recurrences (Algorithm 1's outer loop, one per column) whose products
// with A are one block kernel per step (launch_sell_mstep: the matrix read
// once for all columns); dot products, updates and the stopping test run
// per column in the single-vector kernels, each on its own scalar block, so
// a column that stops is frozen while the others go on.

cudaError_t menqueue_poly(nc_solver S, int m, int fin, cudaStream_t st) {
    const int n = (int)S->n;
    const size_t cn = (size_t)n;
    if (S->k == 0) {
        for (int c = 0; c < m; ++c) {
            cudaError_t e = launch_scale_dot(n, S->mr + c * cn, 1.0 / S->theta, S->mz + c * cn,
                                             make_reduce(S->partials, S->counter, S->mS + c, nullptr, fin),
                                             &S->mS[c].done, st);
            if (e) return e;
        }
        return cudaSuccess;
    }
    const void* rx = S->mixed ? static_cast<const void*>(S->mr32) : static_cast<const void*>(S->mr);
    const std::vector<StepC> cf = step_coefs(S, fin != FIN_NONE);
    for (int j = 1; j <= S->k; ++j) {
        const void* u = (j == 1) ? rx : S->mbuf[(j - 1) % 3];
        const void* w = (j >= 3) ? S->mbuf[(j - 2) % 3] : nullptr;
        const bool last = (j == S->k);
        void* y = last ? static_cast<void*>(S->mz) : S->mbuf[j % 3];
        cudaError_t e = launch_sell_mstep(n, m, n, S->opP.ptr, S->opP.col, S->opP.pat, S->opP.val, S->opP.vdt,
                                          S->mixed, last || !S->mixed, u, w, rx, y,
                                          cf[j].ca + cf[j].cd * S->opP.dfold, cf[j].cb, cf[j].cc, cf[j].cd, S->mS,
                                          st);
        if (e) return e;
    }
    if (fin == FIN_NONE) return cudaSuccess;
    for (int c = 0; c < m; ++c) {
        cudaError_t e = launch_dot(n, S->mr + c * cn, S->mz + c * cn,
                                   make_reduce(S->partials, S->counter, S->mS + c, nullptr, fin), &S->mS[c].done, st);
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t menqueue_prologue(nc_solver S, int m, cudaStream_t st) {
    const int n = (int)S->n;
    const size_t cn = (size_t)n;
    cudaError_t e;
    for (int c = 0; c < m; ++c) {
        double* b = S->mb + c * cn;
        double* x = S->mx + c * cn;
        double* r = S->mr + c * cn;
        PcgScalars* Sc = S->mS + c;
        const Reduce none = make_reduce(S->partials, S->counter, Sc, nullptr, FIN_NONE);
        if ((e = launch_dot(n, b, b, make_reduce(S->partials, S->counter, Sc, nullptr, FIN_BB), nullptr, st))) return e;
        e = S->opt.x0_is_zero ? launch_copy(n, b, r, nullptr, st) : op64_apply(S, x, b, r, 1.0, -1.0, 0, none, nullptr, st);
        if (e) return e;
        if ((e = launch_dot(n, r, r, make_reduce(S->partials, S->counter, Sc, nullptr, FIN_RR0), nullptr, st))) return e;
        if (S->mixed && (e = launch_convert(n, r, NC_F32, S->mr32 + c * cn, st))) return e;
    }
    if ((e = menqueue_poly(S, m, FIN_RZ0, st))) return e;
    for (int c = 0; c < m; ++c)
        if ((e = launch_copy(n, S->mz + c * cn, S->mp + c * cn, &S->mS[c].done, st))) return e;
    return cudaSuccess;
}

cudaError_t menqueue_body(nc_solver S, int m, cudaGraphConditionalHandle h, int use_cond, int* active,
                          cudaStream_t st) {
    const int n = (int)S->n;
    const size_t cn = (size_t)n;
    cudaError_t e;
    // q = A p for all columns (A' p + shift p with the shifted operator)
    if ((e = launch_sell_mstep(n, m, n, S->op64.ptr, S->op64.col, S->op64.pat, S->op64.val, NC_F64, false, true,
                               S->mp, nullptr, nullptr, S->mq, S->shift + S->op64.dfold, 0.0, 0.0, 1.0, S->mS,
                               st)))
        return e;
    for (int c = 0; c < m; ++c) {
        PcgScalars* Sc = S->mS + c;
        if ((e = launch_dot(n, S->mp + c * cn, S->mq + c * cn,
                            make_reduce(S->partials, S->counter, Sc, nullptr, FIN_ALPHA), &Sc->done, st)))
            return e;
        if ((e = launch_axpy2_rr(n, S->mx + c * cn, S->mr + c * cn, S->mp + c * cn, S->mq + c * cn,
                                 S->mixed ? S->mr32 + c * cn : nullptr,
                                 make_reduce(S->partials, S->counter, Sc, nullptr, FIN_RR), st)))
            return e;
    }
    if ((e = menqueue_poly(S, m, FIN_BETA, st))) return e;
    for (int c = 0; c < m; ++c)
        if ((e = launch_p_update(n, S->mp + c * cn, S->mz + c * cn, S->mS + c, h, 0, st))) return e;
    return launch_any_active(S->mS, m, h, use_cond, active, st);
}

nc_status mbuild_graph(nc_solver S, int m) {
    if (S->mexec) {
        cudaGraphExecDestroy(S->mexec);
        S->mexec = nullptr;
    }
    cudaGraph_t g = nullptr, gp = nullptr;
    cudaGraphNode_t np = nullptr, nw = nullptr;
    cudaGraphConditionalHandle h = 0;
    nc_status st = NC_ERR_CUDA;
    cudaError_t e;
    do {
        if ((e = cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal))) break;
        cudaError_t e1 = menqueue_prologue(S, m, S->cap);
        e = cudaStreamEndCapture(S->cap, &gp);
        if (e1) { e = e1; break; }
        if (e) break;
        if ((e = cudaGraphCreate(&g, 0))) break;
        if ((e = cudaGraphAddChildGraphNode(&np, g, nullptr, 0, gp))) break;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&nw, g, &np, nullptr, 1, &cp))) break;
        cudaGraph_t gb = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(S->cap, gb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
            break;
        e1 = menqueue_body(S, m, h, 1, nullptr, S->cap);
        cudaGraph_t gb_out = nullptr;
        e = cudaStreamEndCapture(S->cap, &gb_out);
        if (e1) { e = e1; break; }
        if (e) break;
        if ((e = cudaGraphInstantiate(&S->mexec, g, 0))) break;
        S->mexec_m = m;
        st = NC_OK;
    } while (0);
    if (st != NC_OK) {
        g_last_cuda = e;
        cudaGetLastError();
        S->mexec = nullptr;
    }
    if (gp) cudaGraphDestroy(gp);
    if (g) cudaGraphDestroy(g);
    return st;
}

nc_status mreserve(nc_solver S, int m) {
    if (m <= S->mcap) return NC_OK;
    if (S->mexec) {
        cudaGraphExecDestroy(S->mexec);
        S->mexec = nullptr;
    }
    dev_free(S->mb); dev_free(S->mx); dev_free(S->mr); dev_free(S->mz); dev_free(S->mp); dev_free(S->mq);
    for (auto& bp : S->mbuf) { dev_free(bp); bp = nullptr; }
    dev_free(S->mr32); dev_free(S->mS);
    if (S->mh) cudaFreeHost(S->mh);
    S->mb = S->mx = S->mr = S->mz = S->mp = S->mq = nullptr;
    S->mr32 = nullptr; S->mS = nullptr; S->mh = nullptr; S->mcap = 0;
    const int64_t len = (int64_t)m * S->n;
    const size_t vb = S->mixed ? sizeof(float) : sizeof(double);
    NC_TRY(dev_alloc_n(&S->mb, len)); NC_TRY(dev_alloc_n(&S->mx, len)); NC_TRY(dev_alloc_n(&S->mr, len));
    NC_TRY(dev_alloc_n(&S->mz, len)); NC_TRY(dev_alloc_n(&S->mp, len)); NC_TRY(dev_alloc_n(&S->mq, len));
    for (auto& bp : S->mbuf) NC_TRY(dev_alloc(&bp, vb * (size_t)len));
    if (S->mixed) NC_TRY(dev_alloc_n(&S->mr32, len));
    NC_TRY(dev_alloc_n(&S->mS, m));
    cudaError_t e = cudaMallocHost(&S->mh, sizeof(PcgScalars) * m);
    if (e) { g_last_cuda = e; return NC_ERR_CUDA; }
    S->mcap = m;
    return NC_OK;
}

// Average time of one representative fused step (DOT-free, all four terms

}  // namespace nc
