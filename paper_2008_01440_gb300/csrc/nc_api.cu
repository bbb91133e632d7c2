// C ABI of libncpcg: matrix handles, the polynomial setup, Lanczos bounds
// and the PCG solve (declarations and contracts in include/nc_pcg.h).
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
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "nc_common.cuh"

using namespace nc;

enum MatKind : int { MAT_CSR = 0, MAT_STENCIL7 = 1, MAT_BSR3 = 2 };

struct nc_matrix_s {
    int kind = MAT_CSR;
    int64_t n = 0, nnz = 0;
    const int32_t* rowptr = nullptr;   // CSR row pointers, or BSR3 block-row pointers
    const int32_t* col = nullptr;      // CSR columns, or BSR3 block columns
    const double* val = nullptr;    // values used by products (borrowed or owned_val); BSR3: 9 per block
    double* owned_val = nullptr;    // scaled copy (nc_matrix_jacobi)
    double* dis = nullptr;          // d^{-1/2} of the scaling, owned (CSR)
    bool scaled = false;            // built by nc_matrix_jacobi
    double dis_scalar = 1.0;        // constant d^{-1/2} (stencil)
    double* wblk = nullptr;         // two-level first level (BSR3): W_i = L_i^{-T}, owned
    double* lblk = nullptr;         // and L_i (A_ii = L_i L_i^T), owned
    StencilGeom geom{0, 0, 0};      // stencil grid
    double c4[4] = {0, 0, 0, 0};    // stencil coefficients c0, cx, cy, cz
};

// A matrix as the step kernels see it: CSR (the handle's arrays) or the
// solver-owned SELL-32 layout, with float64 or low-precision values.
enum OpKind : int { OP_CSR = 0, OP_SELL = 1, OP_STENCIL = 2, OP_BSR3 = 3, OP_BSELL3 = 4 };
struct OpView {
    int kind = OP_CSR;
    int n = 0;
    const int32_t* ptr = nullptr;   // row pointers (CSR) or slice pointers (SELL)
    const int32_t* col = nullptr;
    const void* val = nullptr;
    int vdt = NC_F64;
    StencilGeom geom{0, 0, 0};      // OP_STENCIL
    double c4[4] = {0, 0, 0, 0};
    SellPat pat;                    // OP_SELL with offset patterns (pat.pstart set): col unused
};

struct nc_solver_s {
    nc_matrix A = nullptr;
    int64_t n = 0;
    int k = 0;
    double s = 1.0, lmin = 0.0, lmax = 0.0;
    nc_options opt{};
    double theta = 0.0, delta = 0.0, sigma = 0.0;
    std::vector<double> ca, cb, cc, cd;   // per Chebyshev step 1..k (index 0 unused)
    double ca1_shifted = 0.0;             // step-1 coefficient of u = r for the shifted operator
    // Newton form (Algorithm 1): k = 2^nlev - 1, zeta_0..zeta_nlev, and two
    // float64 work vectors per level >= 2 (t1 = P_{j-1} v and p = A t1)
    int nlev = -1;
    std::vector<double> zeta;
    std::vector<double*> nbuf;
    // multi-right-hand-side workspace (pcg_solve_multi), allocated on first
    // use for up to mcap columns: column c of each block at offset c * n
    int mcap = 0;
    double *mb = nullptr, *mx = nullptr, *mr = nullptr, *mz = nullptr, *mp = nullptr, *mq = nullptr;
    void* mbuf[3] = {nullptr, nullptr, nullptr};
    float* mr32 = nullptr;
    PcgScalars* mS = nullptr;          // device, one per column
    PcgScalars* mh = nullptr;          // pinned host copy
    cudaGraphExec_t mexec = nullptr;   // graph of the last column count
    int mexec_m = 0;
    bool mgraph_failed = false;
    bool mixed = false;
    int vdt = NC_F64;
    OpView op64;                          // float64 operator (outer CG, true residual)
    OpView opP;                           // operator inside P_k (apply precision)
    double padding = 1.0;                 // SELL stored entries / nnz
    double tune_us[2] = {0.0, 0.0};       // measured step time, plain / sliced layout (TUNE)
    double shift = 0.0;                   // op values hold A - shift*I (theta' for SELL, else 0)
    double pscale = 1.0;                  // opP holds A / pscale (a stencil: its x-weight), else 1
    void* lval = nullptr;                 // converted CSR values (F32/BF16), owned
    int32_t* sell_ptr = nullptr;          // SELL-32 arrays, owned
    int32_t* sell_col = nullptr;
    int32_t* psell_start = nullptr;       // offset-pattern layout: per-slice start in psell_off, owned
    int32_t* psell_off = nullptr;         // the distinct offset sets, owned
    int64_t npatterns = 0;
    double* sell_val64 = nullptr;
    void* sell_valP = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    void* buf[3] = {nullptr, nullptr, nullptr};
    float* r32 = nullptr;
    PcgScalars* S = nullptr;
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    PcgScalars* h_io = nullptr;           // pinned host copy of the scalars
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    // one-cluster solve (use_graph == 2)
    bool persistent = false;
    ClusterPlan plan{};
    double* pcoef = nullptr;          // 4*(k+1) step coefficients, shifted-operator form
    std::vector<int32_t> h_sell_ptr;  // host copy of the scalar SELL slice offsets
};

namespace {

thread_local cudaError_t g_last_cuda = cudaSuccess;

#define NC_CU(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            g_last_cuda = e_;                         \
            return NC_ERR_CUDA;                       \
        }                                             \
    } while (0)

#define NC_TRY(call)                     \
    do {                                 \
        nc_status s_ = (call);           \
        if (s_ != NC_OK) return s_;      \
    } while (0)

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

template <typename T>
nc_status dev_alloc_n(T** p, int64_t count) {
    return dev_alloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

int64_t max_partials(int64_t n) {
    const int64_t rows = (n + kBlock - 1) / kBlock;
    return (rows > kVecGrid ? rows : kVecGrid) + 1;
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

Reduce make_reduce(double* partials, unsigned int* counter, PcgScalars* S, double* out, int fin) {
    Reduce R;
    R.partials = partials;
    R.counter = counter;
    R.S = S;
    R.out = out;
    R.fin = fin;
    return R;
}

cudaError_t op_step(const OpView& op, bool x_f32, bool y_f64, const void* u, const void* w, const void* r,
                    void* y, double ca, double cb, double cc, double cd, int dot, const double* rdot,
                    const Reduce& R, const int* done, cudaStream_t st) {
    if (op.kind == OP_SELL)
        return launch_sell_step(op.n, op.ptr, op.col, op.pat, op.val, op.vdt, x_f32, y_f64, u, w, r, y, ca, cb, cc,
                                cd, dot, rdot, R, done, st);
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
struct StepC {
    double ca, cb, cc, cd;
};

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
    rr.status = o.status;
    rr.relres = bnorm > 0 ? std::sqrt(o.rr) / bnorm : 0.0;
    rr.true_relres = bnorm > 0 ? std::sqrt(o.rr_true) / bnorm : 0.0;
    rr.n_dot = o.n_dot;
    rr.n_spmv = (int64_t)o.iter + (int64_t)S->k * o.n_prec + o.n_replace;
    rr.n_replace = o.n_replace;
    if (res) *res = rr;
    return (nc_status)o.status;
}

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
                                          S->mixed, last || !S->mixed, u, w, rx, y, cf[j].ca, cf[j].cb, cf[j].cc,
                                          cf[j].cd, S->mS, st);
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
                               S->mp, nullptr, nullptr, S->mq, S->shift, 0.0, 0.0, 1.0, S->mS, st)))
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
        if ((e = cudaMemsetAsync(dbad, 0, sizeof(int), st)) ||
            (e = launch_psell_merge(n, A->rowptr, A->col, nullptr, dcnt, nullptr, dbad, st)) ||
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
            (e = launch_psell_merge(n, A->rowptr, A->col, dopos, nullptr, doff, dbad, st)) ||
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
                                   S->shift, S->sell_val64, dbad, st)) ||
            (e = cudaMemcpyAsync(&h_nodiag, dbad, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            g_last_cuda = e;
            ret = NC_ERR_CUDA;
            break;
        }
        if (h_nodiag) {   // a row without a diagonal entry: store A itself
            S->shift = 0.0;
            if ((e = launch_psell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->psell_start, S->psell_off,
                                       NC_F64, 0.0, S->sell_val64, nullptr, st))) {
                g_last_cuda = e;
                ret = NC_ERR_CUDA;
                break;
            }
        }
        S->op64 = OpView{OP_SELL, n, S->sell_ptr, nullptr, S->sell_val64, NC_F64};
        S->op64.pat = SellPat{S->psell_start, S->psell_off};
        S->opP = S->op64;
        if (S->mixed) {
            if ((ret = dev_alloc(&S->sell_valP, eb * (size_t)(total > 0 ? total : 1))) != NC_OK) break;
            if ((e = launch_psell_fill(n, A->rowptr, A->col, A->val, S->sell_ptr, S->psell_start, S->psell_off,
                                       S->vdt, S->shift, S->sell_valP, nullptr, st))) {
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

}  // namespace

// =============================================================================
extern "C" {

void nc_options_default(nc_options* opt) {
    if (!opt) return;
    opt->apply_dtype = NC_F64;
    opt->rr_period = 0;
    opt->x0_is_zero = 0;
    opt->use_graph = 1;
    opt->spmv_format = NC_FORMAT_AUTO;
    opt->poly_form = NC_POLY_CHEBYSHEV;
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
    }
    return "unknown status";
}

const char* nc_version(void) { return "ncpcg 0.1 (sm_103a)"; }

const char* nc_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

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
