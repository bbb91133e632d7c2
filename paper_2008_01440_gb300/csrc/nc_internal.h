// Internal declarations shared by the host-side translation units of
// libncpcg: the matrix and solver handles, the operator view the step
// kernels read, and the solver machinery split across
//   nc_matrix.cu       matrix handles, scaling, Gershgorin, Lanczos, power method
//   nc_setup.cu        layouts the step kernels read, and the step-kernel tuner
//   nc_solve.cu        Chebyshev coefficients, P_k(A) r, the PCG graph and solve
//   nc_solve_multi.cu  several right-hand sides sharing the matrix
//   nc_api.cu          the pcg_* entry points
#pragma once

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nc_common.cuh"

namespace nc {

enum MatKind : int { MAT_CSR = 0, MAT_STENCIL7 = 1, MAT_BSR3 = 2 };

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
    StepTune tune;                  // OP_SELL: kernel variant and launch shape
    // OP_SELL whose layout leaves out a constant diagonal: its value in the
    // stored operator (a_ii - shift), applied through the step's u term
    // (op_step adds cd * dfold to ca); 0 when the diagonal is stored
    double dfold = 0.0;
    int dfolded = 0;                // 1: the layout leaves the diagonal out
};


// Coefficients of one fused step as the kernels take them
struct StepC {
    double ca, cb, cc, cd;
};

// One measured launch configuration of the tuner
struct TuneRec {
    int op, variant, stages, ctas_per_sm, rpt, contig, lookahead, red_ctas_per_sm;
    double us;
    int chosen;
    int zchunk = 0, pz = 0;   // matrix-free stencil: z-chunk and planes per batch
};

}  // namespace nc

using nc::MatKind;
using nc::MAT_CSR;
using nc::MAT_STENCIL7;
using nc::MAT_BSR3;
using nc::OpView;
using nc::ClusterPlan;
using nc::PcgScalars;
using nc::StencilGeom;


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
    std::vector<nc::TuneRec> tune;    // tuner measurements (pcg_tune_candidate)
    bool tune_cached = false;         // choices taken from the NC_TUNE_CACHE file
    int num_sms = 0;                  // SM count of the device at setup
};

namespace nc {

// last CUDA error seen by a host entry point of this thread (nc_last_cuda_error)
extern thread_local cudaError_t g_last_cuda;

#define NC_CU(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            ::nc::g_last_cuda = e_;                   \
            return NC_ERR_CUDA;                       \
        }                                             \
    } while (0)

#define NC_TRY(call)                     \
    do {                                 \
        nc_status s_ = (call);           \
        if (s_ != NC_OK) return s_;      \
    } while (0)

nc_status dev_alloc(void** p, size_t bytes);
template <typename T>
nc_status dev_alloc_n(T** p, int64_t count) {
    return dev_alloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
}
void dev_free(void* p);
inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
int64_t max_partials(int64_t n);
int64_t partials_for(nc_matrix A);
OpView mat_view(nc_matrix A);
inline Reduce make_reduce(double* partials, unsigned int* counter, PcgScalars* S, double* out, int fin) {
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
                    const Reduce& R, const int* done, cudaStream_t st);
cudaError_t op_step_f64(nc_matrix A, const double* u, const double* w, const double* r, double* y,
                        double ca, double cb, double cc, double cd, int dot, const double* rdot,
                        const Reduce& R, const int* done, cudaStream_t st);

// nc_solve.cu
cudaError_t op64_apply(nc_solver S, const double* u, const double* r, double* y, double cc, double cd, int dot,
                       const Reduce& R, const int* done, cudaStream_t st);
void setup_coefficients(nc_solver S);
std::vector<StepC> step_coefs(const nc_solver S, bool in_solve);
cudaError_t enqueue_poly(nc_solver S, const double* r64, double* z, int fin, const int* done, cudaStream_t st);
nc_status run_solve(nc_solver S, const double* b_dev, double* x_dev, double tol, int maxit, cudaStream_t st,
                    nc_result* res);
cudaError_t mat_copy_in(nc_matrix A, const double* b, const double* x, int zero, double* bs, double* xs,
                        cudaStream_t st);
cudaError_t mat_copy_out(nc_matrix A, const double* ys, const PcgScalars* S, double* x, cudaStream_t st);

// nc_solve_multi.cu
nc_status mreserve(nc_solver S, int m);
nc_status mbuild_graph(nc_solver S, int m);
cudaError_t menqueue_prologue(nc_solver S, int m, cudaStream_t st);
cudaError_t menqueue_body(nc_solver S, int m, cudaGraphConditionalHandle h, int use_cond, int* active,
                          cudaStream_t st);

// nc_setup.cu
nc_status setup_operator(nc_solver S, cudaStream_t st);
// variant and launch shape of the SELL step kernels (after the solver's
// buffers and scalar block exist): the options' fixed choice, or the tuner's
nc_status setup_step_kernels(nc_solver S, cudaStream_t st);

}  // namespace nc
