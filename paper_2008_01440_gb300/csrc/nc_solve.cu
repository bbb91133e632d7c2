// The solve machinery of libncpcg: coefficients of the fused Chebyshev steps
// (Sec. 3, Eq. rhocheb, with theta' = s theta of Sec. 4), z = P_k(A) r by
// Algorithm 2 (or Algorithm 1's Newton recursion), and PCG as one CUDA graph.
//
// A solve is one CUDA graph: a prologue (||b||, r0, z0 = P_k r0, p0 = z0)
// followed by a conditional WHILE node whose body is one PCG iteration
//   q = A p, (p,q) -> alpha;  x += alpha p, r -= alpha q, (r,r) -> stop?;
//   z = P_k(A) r (k fused steps, the last with (r,z) -> beta);  p = z + beta p
// and whose condition is written on the device by the p-update kernel, so
// the host waits once per solve.  Every kernel of the body returns at once
// after the stopping test has fired, so the final iteration does not apply
// the preconditioner (the counts of Table 4: (k+1) products with A and 3 dot
// products per iteration).
#include "nc_internal.h"

namespace nc {

thread_local cudaError_t g_last_cuda = cudaSuccess;



nc_status dev_alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return NC_ERR_OOM;
    }
    if (e != cudaSuccess) {
        g_last_cuda = e;
        *p = nullptr;
        return NC_ERR_CUDA;
    }
    return NC_OK;
}


void dev_free(void* p) {
    if (p) cudaFree(p);
}


int64_t max_partials(int64_t n) {
    const int64_t rows = (n + kBlock - 1) / kBlock;
    return (rows > kMaxGrid ? rows : kMaxGrid) + 1;
}

// partial-sum slots any reduction kernel on this matrix may need
int64_t partials_for(nc_matrix A) {
    int64_t p = max_partials(A->n);
    if (A->kind == MAT_STENCIL7) {
        const int64_t sb = stencil_nblocks(A->geom) + 1;
        if (sb > p) p = sb;
    }
    return p;
}

// float64 operator view of a matrix handle
OpView mat_view(nc_matrix A) {
    OpView v;
    v.n = (int)A->n;
    if (A->kind == MAT_STENCIL7) {
        v.kind = OP_STENCIL;
        v.geom = A->geom;
        for (int i = 0; i < 4; ++i) v.c4[i] = A->c4[i];
    } else if (A->kind == MAT_BSR3) {
        v.kind = OP_BSR3;
        v.ptr = A->rowptr;
        v.col = A->col;
        v.val = A->val;
    } else {
        v.kind = OP_CSR;
        v.ptr = A->rowptr;
        v.col = A->col;
        v.val = A->val;
    }
    v.vdt = NC_F64;
    return v;
}


cudaError_t op_step(const OpView& op, bool x_f32, bool y_f64, const void* u, const void* w, const void* r,
                    void* y, double ca, double cb, double cc, double cd, int dot, const double* rdot,
                    const Reduce& R, const int* done, cudaStream_t st) {
    if (op.kind == OP_SELL)   // a diagonal left out of the layout enters through the u term
        return launch_sell_step(op.n, op.ptr, op.col, op.pat, op.val, op.vdt, x_f32, y_f64, u, w, r, y,
                                ca + cd * op.dfold, cb, cc, cd, dot, rdot, R, done, st, op.tune);
    if (op.kind == OP_STENCIL)
        return launch_stencil_step(op.geom, op.c4, x_f32, y_f64, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done,
                                   st);
    if (op.kind == OP_BSR3 || op.kind == OP_BSELL3)
        return launch_bsr3_step(op.kind == OP_BSELL3, op.n / 3, op.ptr, op.col, op.val, op.vdt, x_f32, y_f64, u, w,
                                r, y, ca, cb, cc, cd, dot, rdot, R, done, st);
    return launch_csr_step(op.n, op.ptr, op.col, op.val, op.vdt, x_f32, y_f64, u, w, r, y, ca, cb, cc, cd, dot,
                           rdot, R, done, st);
}

// y = ca u + cb w + cc r + cd (A u) with the handle's float64 operator
cudaError_t op_step_f64(nc_matrix A, const double* u, const double* w, const double* r, double* y,
                        double ca, double cb, double cc, double cd, int dot, const double* rdot,
                        const Reduce& R, const int* done, cudaStream_t st) {
    return op_step(mat_view(A), false, true, u, w, r, y, ca, cb, cc, cd, dot, rdot, R, done, st);
}

// ---- solver internals -------------------------------------------------------

// y = cc*r + cd*(A u) with the solver's float64 operator.  When the stored
// values are A' = A - shift*I, A u = A' u + shift*u: the u term carries it.
cudaError_t op64_apply(nc_solver S, const double* u, const double* r, double* y, double cc, double cd, int dot,
                       const Reduce& R, const int* done, cudaStream_t st) {
    return op_step(S->op64, false, true, u, nullptr, r, y, cd * S->shift, 0.0, cc, cd, dot, nullptr, R, done, st);
}

// Coefficients of the fused steps from rho_k (Eq. rhocheb), theta' = s theta.
void setup_coefficients(nc_solver S) {
    const double theta = S->s * (S->lmax + S->lmin) / 2.0;
    const double delta = (S->lmax - S->lmin) / 2.0;
    const double sigma = theta / delta;
    S->theta = theta;
    S->delta = delta;
    S->sigma = sigma;
    const int k = S->k;
    std::vector<double> rho(k + 1);
    rho[0] = 1.0 / sigma;
    for (int j = 1; j <= k; ++j) rho[j] = 1.0 / (2.0 * sigma - rho[j - 1]);
    S->ca.assign(k + 1, 0.0);
    S->cb.assign(k + 1, 0.0);
    S->cc.assign(k + 1, 0.0);
    S->cd.assign(k + 1, 0.0);
    if (k >= 1) {   // x_1 = (2 rho_1/delta)(2 r - A r/theta), product applied to u = r
        S->ca[1] = 4.0 * rho[1] / delta;
        S->cd[1] = -2.0 * rho[1] / (delta * theta);
        S->ca1_shifted = 2.0 * rho[1] / delta;
    }
    for (int j = 2; j <= k; ++j) {
        S->ca[j] = 2.0 * sigma * rho[j];
        S->cb[j] = -rho[j] * rho[j - 1];
        S->cc[j] = 2.0 * rho[j] / delta;
        S->cd[j] = -2.0 * rho[j] / delta;
    }
    if (k >= 2) {   // x_0 = r/theta: fold the x_{k-2} term of step 2 into its r term
        S->cc[2] += S->cb[2] / theta;
        S->cb[2] = 0.0;
    }
}

// Coefficients of the fused steps as the kernels take them, for the stored
// iterates y_j = x_j / g_j.  In float64 the scale g_j = cd_j g_{j-1} makes the
// coefficient of the product exactly 1, so the step kernels drop one float64
// multiply per row (their bound is the float64 pipe); g falls back to 1 at
// any step where it would leave [2^-64, 2^64].  The last step keeps g_k = 1,
// so z itself is stored, unless `in_solve`: PCG's iterates do not change when
// P is multiplied by a positive constant (z, p and q scale alike, alpha and
// beta compensate), so inside a solve the last step also stores z / g_k when
// g_k > 0.  The mixed-precision path stores x_j itself.  Entry j = step j
// (index 0 unused); the x_{k-1} term is dropped for the shifted operator
// (see enqueue_poly).
std::vector<StepC> step_coefs(const nc_solver S, bool in_solve) {
    const int k = S->k;
    std::vector<StepC> out(k + 1, StepC{0.0, 0.0, 0.0, 0.0});
    std::vector<double> g(k + 1, 1.0);
    // a stencil inside P is stored divided by its x-weight kap (A = kap A^),
    // so the coefficient of its product is cd kap
    const double kap = S->pscale;
    for (int j = 1; j <= k; ++j) {
        double ca = S->ca[j];
        if (S->shift != 0.0) ca = (j == 1) ? S->ca1_shifted : 0.0;
        const double gu = (j == 1) ? 1.0 : g[j - 1];   // scale of u (r at step 1)
        const double gw = (j >= 3) ? g[j - 2] : 1.0;   // scale of w = y_{j-2}
        const double t = S->cd[j] * kap * gu;
        const bool unit = !S->mixed && (j < k || (in_solve && t > 0.0)) && std::fabs(t) >= 0x1p-64 &&
                          std::fabs(t) <= 0x1p64;
        g[j] = unit ? t : 1.0;
        out[j].ca = ca * gu / g[j];
        out[j].cb = S->cb[j] * gw / g[j];
        out[j].cc = S->cc[j] / g[j];
        out[j].cd = unit ? 1.0 : t;
    }
    return out;
}

// z = P_k(A) r.  r64: float64 residual; the mixed path reads S->r32 (which
// must already hold (float) r64).  fin: reduction of (r, z) or FIN_NONE.
// out = g P_j v (+ w_coef w when w is non-null) by the recursion of
// Algorithm 1, P_0 = zeta_0 I, P_{j+1} v = zeta_{j+1} (2 P_j v - P_j A P_j v),
// depth first: 2^j - 1 products.  A level-1 application is one fused step,
// g zeta_1 zeta_0 (2 v - zeta_0 A v); a level j >= 2 computes t1 = P_{j-1} v
// and p = A t1 into its own two vectors, then P_{j-1} p into `out`, and
// combines out = g zeta_j (2 t1 - out) -- for j = 2 inside the last fused
// step (its x_{k-2} slot carries t1).  With rdot, the last kernel also forms
// (rdot, out) for the PCG scalars.
cudaError_t enqueue_newton(nc_solver S, int j, const double* v, double* out, double g, const double* w,
                           double w_coef, const double* rdot, const Reduce& R, const int* done, cudaStream_t st) {
    const int n = (int)S->n;
    const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
    const std::vector<double>& z = S->zeta;
    const int dot = rdot != nullptr ? 1 : 0;
    if (j == 0) {   // only as the whole preconditioner (k = 0): out = zeta_0 v
        return launch_scale_dot(n, v, g * z[0], out, R, done, st);
    }
    if (j == 1) {
        // g zeta_1 zeta_0 (2 v - zeta_0 A v) (+ w_coef w); A v = A' v + shift v
        const double cd = -g * z[1] * z[0] * z[0];
        const double ca = 2.0 * g * z[1] * z[0] + cd * S->shift;
        return op_step(S->op64, false, true, v, w, nullptr, out, ca, w != nullptr ? w_coef : 0.0, 0.0, cd, dot,
                       rdot, dot ? R : none, done, st);
    }
    double* t1 = S->nbuf[2 * (j - 2)];
    double* pv = S->nbuf[2 * (j - 2) + 1];
    cudaError_t e = enqueue_newton(S, j - 1, v, t1, 1.0, nullptr, 0.0, nullptr, none, done, st);
    if (e) return e;
    e = op64_apply(S, t1, nullptr, pv, 0.0, 1.0, 0, none, done, st);   // p = A t1
    if (e) return e;
    if (j == 2 && w == nullptr) {
        // out = g zeta_2 (2 t1 - P_1 p): the fused level-1 step with t1 in its w slot
        return enqueue_newton(S, 1, pv, out, -g * z[2], t1, 2.0 * g * z[2], rdot, R, done, st);
    }
    e = enqueue_newton(S, j - 1, pv, out, 1.0, nullptr, 0.0, nullptr, none, done, st);
    if (e) return e;
    // out = g zeta_j (2 t1 - out) (+ w_coef w, folded by one more pass)
    e = launch_axpby_dot(n, 2.0 * g * z[j], t1, -g * z[j], out, out, w != nullptr ? nullptr : rdot,
                         w != nullptr ? none : R, done, st);
    if (e || w == nullptr) return e;
    return launch_axpby_dot(n, 1.0, out, w_coef, w, out, rdot, rdot ? R : none, done, st);
}

cudaError_t enqueue_poly(nc_solver S, const double* r64, double* z, int fin, const int* done,
                         cudaStream_t st) {
    const int n = (int)S->n;
    const Reduce R = make_reduce(S->partials, S->counter, S->S, nullptr, fin);
    if (S->k == 0) return launch_scale_dot(n, r64, 1.0 / S->theta, z, R, done, st);
    if (S->nlev >= 1)
        return enqueue_newton(S, S->nlev, r64, z, 1.0, nullptr, 0.0, fin != FIN_NONE ? r64 : nullptr, R, done, st);
    const void* rx = S->mixed ? static_cast<const void*>(S->r32) : static_cast<const void*>(r64);
    // with the shifted operator A' = A - theta' I the x_{k-1} term of every
    // step k >= 2 vanishes (a_k + d_k theta' = 0 exactly) and step 1 keeps
    // (4 rho_1 - 2 rho_1)/delta = 2 rho_1/delta on r
    const std::vector<StepC> cf = step_coefs(S, fin != FIN_NONE);
    for (int j = 1; j <= S->k; ++j) {
        const void* u = (j == 1) ? rx : S->buf[(j - 1) % 3];
        const void* w = (j >= 3) ? S->buf[(j - 2) % 3] : nullptr;
        const bool last = (j == S->k);
        void* y = last ? static_cast<void*>(z) : S->buf[j % 3];
        const int dot = (last && fin != FIN_NONE) ? 1 : 0;
        cudaError_t e = op_step(S->opP, S->mixed, last || !S->mixed, u, w, rx, y, cf[j].ca, cf[j].cb, cf[j].cc,
                                cf[j].cd, dot, r64, R, done, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_prologue(nc_solver S, cudaStream_t st) {
    const int n = (int)S->n;
    const int* done = &S->S->done;
    cudaError_t e;
    e = launch_dot(n, S->b, S->b, make_reduce(S->partials, S->counter, S->S, nullptr, FIN_BB), nullptr, st);
    if (e) return e;
    if (S->opt.x0_is_zero) {
        e = launch_copy(n, S->b, S->r, nullptr, st);
    } else {
        const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
        e = op64_apply(S, S->x, S->b, S->r, 1.0, -1.0, 0, none, nullptr, st);
    }
    if (e) return e;
    if (S->mixed) {
        e = launch_convert(S->n, S->r, NC_F32, S->r32, st);
        if (e) return e;
    }
    e = launch_dot(n, S->r, S->r, make_reduce(S->partials, S->counter, S->S, nullptr, FIN_RR0), nullptr, st);
    if (e) return e;
    e = enqueue_poly(S, S->r, S->z, FIN_RZ0, done, st);
    if (e) return e;
    return launch_copy(n, S->z, S->p, done, st);
}

cudaError_t enqueue_body(nc_solver S, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
    const int n = (int)S->n;
    const int* done = &S->S->done;
    cudaError_t e;
    e = op64_apply(S, S->p, nullptr, S->q, 0.0, 1.0, 2, make_reduce(S->partials, S->counter, S->S, nullptr, FIN_ALPHA),
                   done, st);
    if (e) return e;
    e = launch_axpy2_rr(n, S->x, S->r, S->p, S->q, S->mixed ? S->r32 : nullptr,
                        make_reduce(S->partials, S->counter, S->S, nullptr, FIN_RR), st);
    if (e) return e;
    if (S->opt.rr_period > 0) {
        // residual replacement: r = b - A x in float64 (kernels skip unless
        // this iteration is a multiple of rr_period and the solve goes on)
        const int* skip = &S->S->rr_skip;
        const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
        e = op64_apply(S, S->x, S->b, S->r, 1.0, -1.0, 0, none, skip, st);
        if (e) return e;
        if (S->mixed) {
            e = launch_refresh_r32(n, S->r, S->r32, skip, st);
            if (e) return e;
        }
    }
    e = enqueue_poly(S, S->r, S->z, FIN_BETA, done, st);
    if (e) return e;
    return launch_p_update(n, S->p, S->z, S->S, h, use_cond, st);
}

nc_status build_graph(nc_solver S) {
    cudaGraph_t g = nullptr, gp = nullptr, gb = nullptr;
    cudaGraphNode_t np = nullptr, nw = nullptr;
    cudaGraphConditionalHandle h = 0;
    nc_status st = NC_ERR_CUDA;
    cudaError_t e;
    do {
        if ((e = cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal))) break;
        cudaError_t e1 = enqueue_prologue(S, S->cap);
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
        gb = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(S->cap, gb, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)))
            break;
        e1 = enqueue_body(S, h, 1, S->cap);
        cudaGraph_t gb_out = nullptr;
        e = cudaStreamEndCapture(S->cap, &gb_out);
        if (e1) { e = e1; break; }
        if (e) break;
        if ((e = cudaGraphInstantiate(&S->exec, g, 0))) break;
        st = NC_OK;
    } while (0);
    if (st != NC_OK) {
        g_last_cuda = e;
        cudaGetLastError();
        S->exec = nullptr;
    }
    if (gp) cudaGraphDestroy(gp);
    if (g) cudaGraphDestroy(g);
    return st;
}

// Into the scaled system: bs = W^T b, xs = W^{-1} x (or 0) -- a diagonal W
// (Jacobi, or none) or the block W of the two-level variant.
cudaError_t mat_copy_in(nc_matrix A, const double* b, const double* x, int zero, double* bs, double* xs,
                        cudaStream_t st) {
    if (A->wblk) return launch_bsr3_block_copy_in((int)(A->n / 3), b, x, A->wblk, A->lblk, zero, bs, xs, st);
    return launch_copy_in((int)A->n, b, x, A->dis, A->dis_scalar, zero, bs, xs, st);
}

// Back to the original system: x = W ys (0 when b = 0)
cudaError_t mat_copy_out(nc_matrix A, const double* ys, const PcgScalars* S, double* x, cudaStream_t st) {
    if (A->wblk) return launch_bsr3_block_copy_out((int)(A->n / 3), ys, A->wblk, S, x, st);
    return launch_copy_out((int)A->n, ys, A->dis, A->dis_scalar, S, x, st);
}

nc_status run_solve(nc_solver S, const double* b_dev, double* x_dev, double tol, int maxit,
                    cudaStream_t st, nc_result* res) {
    const int n = (int)S->n;
    PcgScalars init;
    std::memset(&init, 0, sizeof(init));
    init.tol2 = tol * tol;
    init.maxit = maxit;
    init.status = NC_ERR_MAXIT;
    init.rr_period = S->opt.rr_period;
    init.rr_skip = 1;
    // the pinned staging block is reused by every solve; the previous solve
    // synchronised the stream, so it is free
    *S->h_io = init;
    NC_CU(cudaMemcpyAsync(S->S, S->h_io, sizeof(PcgScalars), cudaMemcpyHostToDevice, st));
    NC_CU(mat_copy_in(S->A, b_dev, x_dev, S->opt.x0_is_zero, S->b, S->x, st));
    if (S->persistent) {
        NC_CU(launch_cluster_pcg(S->plan, n, S->k, S->opt.x0_is_zero, maxit, tol * tol, S->shift, S->op64.ptr,
                                 S->op64.col, static_cast<const double*>(S->op64.val), S->pcoef, S->b, S->x, S->S,
                                 st));
    } else {
        bool graph = S->opt.use_graph && !S->graph_failed;
        if (graph && S->exec == nullptr && build_graph(S) != NC_OK) {
            S->graph_failed = true;
            graph = false;
        }
        if (graph) {
            NC_CU(cudaGraphLaunch(S->exec, st));
        } else {
            NC_CU(enqueue_prologue(S, st));
            for (;;) {
                NC_CU(cudaMemcpyAsync(S->h_io, S->S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
                NC_CU(cudaStreamSynchronize(st));
                if (S->h_io->done) break;
                NC_CU(enqueue_body(S, 0, 0, st));
            }
        }
    }
    // true residual of the (scaled) system at exit
    const Reduce none = make_reduce(S->partials, S->counter, S->S, nullptr, FIN_NONE);
    NC_CU(op64_apply(S, S->x, S->b, S->q, 1.0, -1.0, 0, none, nullptr, st));
    NC_CU(launch_dot(n, S->q, S->q, make_reduce(S->partials, S->counter, S->S, nullptr, FIN_TRUE), nullptr, st));
    NC_CU(mat_copy_out(S->A, S->x, S->S, x_dev, st));
    NC_CU(cudaMemcpyAsync(S->h_io, S->S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
    NC_CU(cudaStreamSynchronize(st));
    const PcgScalars& o = *S->h_io;
    const double bnorm = std::sqrt(o.bb);
    nc_result rr;
    rr.iters = o.iter;
    rr.status = o.fault ? NC_ERR_TIMEOUT : o.status;
    rr.relres = bnorm > 0 ? std::sqrt(o.rr) / bnorm : 0.0;
    rr.true_relres = bnorm > 0 ? std::sqrt(o.rr_true) / bnorm : 0.0;
    rr.n_dot = o.n_dot;
    rr.n_spmv = (int64_t)o.iter + (int64_t)S->k * o.n_prec + o.n_replace;
    rr.n_replace = o.n_replace;
    if (res) *res = rr;
    return (nc_status)rr.status;
}

}  // namespace nc
